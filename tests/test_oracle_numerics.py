"""Oracle pins: quadrature rules, K0, analytic potentials, Green's functions (each against an
independent reference: exact monomial integrals, scipy's Bessel routine, brute-force
subdivision, and two exact series representations of the stripline Green's function)."""
import math

import numpy as np
import pytest
import scipy.special as sp

import pmom_inputs as PI
from oracle import oracle as O


@pytest.mark.parametrize("n,deg", [(7, 5), (13, 7)])
def test_triangle_rules_exact_for_polynomials(n, deg):
    b, w = O.tri_rule(n)
    assert abs(w.sum() - 1.0) < 1e-14
    for a in range(deg + 1):
        for c in range(deg + 1 - a):
            num = 0.5 * np.sum(w * b[:, 1] ** a * b[:, 2] ** c)
            exact = math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
            assert abs(num - exact) < 1e-14
    # degree + 1 is no longer exact (the rule is not over-claimed)
    a = deg + 1
    num = 0.5 * np.sum(w * b[:, 1] ** a)
    assert abs(num - math.factorial(a) / math.factorial(a + 2)) > 1e-8


@pytest.mark.parametrize("w", [0.5, 1.6 + 0.01j, 3.0 - 0.2j, 10 + 0.5j, 0.05 + 0.001j, 25 + 3j])
def test_bessel_k0_matches_scipy(w):
    assert abs(O.bessel_k0(w) - sp.kv(0, w)) <= 1e-13 * abs(sp.kv(0, w)) + 1e-300


def _brute_potentials(tri, r, n=500):
    A = 0.5 * np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[0]))
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m1, m2 = i + j < n, i + j < n - 1
    u = np.concatenate([(i[m1] + 1 / 3), (i[m2] + 2 / 3)]) / n
    v = np.concatenate([(j[m1] + 1 / 3), (j[m2] + 2 / 3)]) / n
    P = tri[0] + u[:, None] * (tri[1] - tri[0]) + v[:, None] * (tri[2] - tri[0])
    R = np.linalg.norm(P - r, axis=1)
    wa = A / n ** 2
    return wa * np.sum(1 / R), wa * np.sum((P - r) / R[:, None], axis=0)


@pytest.mark.parametrize("r", [[0.4, 0.3, 0.5], [2.0, 1.0, 0.0], [0.5, -0.3, 0.2], [0.45, 0.35, 0.05],
                               [1.2, 0.12, 0.0]])
def test_analytic_potentials_vs_subdivision(r):
    tri = np.array([[0, 0, 0], [1.0, 0.1, 0], [0.3, 0.9, 0]])
    r = np.array(r, float)
    I1, Iv = O.tri_potentials(tri, r)
    b1, bv = _brute_potentials(tri, r)
    assert abs(I1 - b1) < 2e-6 * abs(b1)
    # Iv is the in-plane part of int (r' - r)/R
    assert np.allclose(Iv[:2], bv[:2], rtol=0, atol=3e-6 * np.abs(bv).max())
    assert Iv[2] == 0.0


def test_stripline_green_two_representations_agree():
    g = PI.grid_stripline_16x16x2()
    G = O.Grid(g)
    H = g.h_total_m
    for f in (1e9, 7e9):
        for lp, lq in ((0, 0), (0, 1), (1, 1)):
            for rho in (0.01 * H, 0.2 * H, 0.45 * H, 0.8 * H, 2 * H):
                hyb = O.green(G, f, lp, lq, rho)
                mod = O.green(G, f, lp, lq, rho, "modal")
                assert abs(hyb - mod) <= 1e-10 * abs(mod)
                assert abs(O.green(G, f, lq, lp, rho) - hyb) <= 1e-13 * abs(hyb)
    # at 7 GHz the plain image series (oscillating tail) converges; it must approach the same value
    for rho in (0.05 * H, 0.3 * H):
        ref = O.green(G, 7e9, 0, 0, rho)
        e1 = abs(O.green(G, 7e9, 0, 0, rho, "images", 2000) - ref)
        e2 = abs(O.green(G, 7e9, 0, 0, rho, "images", 8000) - ref)
        assert e2 < e1 and e2 < 1e-7 * abs(ref)


def test_microstrip_green_is_direct_minus_image():
    g = PI.grid_plain_8x8()
    G = O.Grid(g)
    f, h, rho = 2e9, g.layer_z_m[0], 1.3e-3
    k = 2 * np.pi * f / 299792458.0 * np.sqrt(O.eps_eff(G))
    R1, R2 = rho, np.hypot(rho, 2 * h)
    ref = np.exp(-1j * k * R1) / (4 * np.pi * R1) - np.exp(-1j * k * R2) / (4 * np.pi * R2)
    assert abs(O.green(G, f, 0, 0, rho) - ref) < 1e-12 * abs(ref)


def test_hammerstad_jensen_eps_eff():
    # u = w/h = 4, eps_r = 3.5: the HJ formula gives about 2.887
    G = O.Grid(PI.grid_plain_8x8())
    assert abs(O.eps_eff(G) - 2.8874) < 1e-3
