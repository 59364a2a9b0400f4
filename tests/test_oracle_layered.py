"""Oracle pins for the grounded-slab (microstrip) Green's functions by Sommerfeld integrals: the
scalar-potential kernel G_phi and the horizontal vector-potential kernel G_A of a PEC ground, a
dielectric slab up to the highest metal layer and a half-space above.

Closed forms they must reduce to: with air in the slab, the PEC image pair of free space; with the
slab's material also above, the image pair of that homogeneous medium (G_phi scaled by 1/eps_r);
in the static limit on the interface of a real microstrip (eps_r = 3.5, air above), G_A is the
magnetostatic image pair and G_phi the charge-image series
(2 / (eps_r + 1)) (1 / 4 pi) sum_n (-K)^n (1 / R_n - 1 / R_{n+1}), K = (eps_r - 1) / (eps_r + 1),
R_n = sqrt(rho^2 + (2 n d)^2), which follows from the static transmission-line kernel
1 / (k (eps_r coth(k d) + 1)).  And both kernels are reciprocal between heights."""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O

C0 = 299792458.0
D = 0.5e-3


def _g(k, R):
    return np.exp(-1j * k * R) / (4 * np.pi * R)


def _slab(er, tan_d=0.0):
    return O.Grid(PI.Grid("slab", 2, 3, 3, 1e-3, PI.MEDIUM_MICROSTRIP, (0.3e-3, D), D, er, tan_d, 2, ()))


@pytest.mark.parametrize("er", [1.0, 3.5])
def test_homogeneous_limits_are_image_pairs(er):
    """er = 1: air slab under air; er = 3.5 with eps_top = er: one homogeneous dielectric."""
    G = _slab(er)
    for f in (1e6, 1e9, 5e9):
        k = 2 * np.pi * f / C0 * np.sqrt(er)
        for kind in (0, 1):
            for z, zp in ((D, D), (0.3e-3, D), (0.3e-3, 0.3e-3)):
                for rho in (0.0, 0.2e-3, 2e-3, 10e-3):
                    if rho == 0.0 and z == zp:
                        continue
                    R, Ri = np.hypot(rho, z - zp), np.hypot(rho, z + zp)
                    ref = (_g(k, R) - _g(k, Ri)) * (1.0 if kind == 1 else 1.0 / er)
                    val, _ = O.slab_green(G, f, kind, z, zp, rho, er_top=er)
                    assert abs(val - ref) <= 1e-7 * abs(ref), (f, kind, z, zp, rho)


def test_static_limit_on_the_microstrip_interface():
    er = 3.5
    G = _slab(er)
    K = (er - 1) / (er + 1)
    for rho in (0.1e-3, 0.5e-3, 2e-3, 10e-3):
        n = np.arange(0, 2000)
        Rn, Rn1 = np.hypot(rho, 2 * n * D), np.hypot(rho, 2 * (n + 1) * D)
        phi = 2 / (er + 1) / (4 * np.pi) * np.sum((-K) ** n * (1 / Rn - 1 / Rn1))
        a_ref = (1 / rho - 1 / np.hypot(rho, 2 * D)) / (4 * np.pi)
        v, c = O.slab_green(G, 1e6, 0, D, D, rho)
        va, ca = O.slab_green(G, 1e6, 1, D, D, rho)
        assert abs(v - phi) <= 1e-6 * abs(phi) and abs(va - a_ref) <= 1e-6 * abs(a_ref)
        assert c == pytest.approx(2 / (er + 1)) and ca == 1.0


def test_reciprocity_between_heights():
    G = _slab(3.66, 0.004)
    for kind in (0, 1):
        for f in (1e9, 6e9):
            a, _ = O.slab_green(G, f, kind, 0.3e-3, D, 1.3e-3)
            b, _ = O.slab_green(G, f, kind, D, 0.3e-3, 1.3e-3)
            assert abs(a - b) <= 1e-12 * abs(a)


def test_layered_fill_with_an_air_slab_is_the_image_fill():
    """medium 2 (kernels by Sommerfeld integrals, tabulated in rho) with eps_r = 1 against medium 0
    (closed-form image pair): same Z to interpolation accuracy."""
    import dataclasses
    g0 = dataclasses.replace(PI.grid_tiny(3), eps_r=1.0, tan_d=0.0)
    f = [2.4e9, 5.2e9]
    Z0, _ = O.fill(O.Grid(g0), f)
    Z2, _ = O.fill(O.Grid(dataclasses.replace(g0, medium=2)), f)
    assert np.abs(Z2 - Z0).max() <= 1e-7 * np.abs(Z0).max()


def test_layered_fill_reciprocal_and_passive():
    import dataclasses
    g = dataclasses.replace(PI.grid_tiny(3), medium=2, eps_r=3.66, tan_d=0.004)
    Z, asym = O.fill(O.Grid(g), [2.4e9, 5.2e9])
    assert asym < 1e-4
    for Zf in Z:
        herm = 0.5 * (Zf + Zf.conj().T)
        assert np.linalg.eigvalsh(herm).min() >= -1e-10 * np.abs(Zf).max()


@pytest.mark.slow
def test_layered_microstrip_line_matches_line_theory():
    """A one-pixel-wide microstrip through line (eps_r = 3.5, h = 0.5 mm, w = 2 mm) with the
    layered kernels: Z12 = Zc / sinh(gamma l) over six lengths fits a TEM-like line whose beta / k0
    is within 1 % of Hammerstad-Jensen's sqrt(eps_eff) at 2 GHz -- predicted here from the slab's
    permittivity, not put in as with the effective-medium reading."""
    from scipy.optimize import least_squares
    a, h, er, f = 2e-3, 0.5e-3, 3.5, 2e9
    z12 = []
    lengths = range(4, 16, 2)
    for L in lengths:
        g = PI.Grid("line", 1, L, 1, a, 2, (h,), h, er, 0.0, 2, (PI.Port(0, PI.SIDE_LEFT, 0), PI.Port(0, PI.SIDE_RIGHT, 0)))
        G = O.Grid(g)
        Z, _ = O.fill(G, [f], threads=1)
        S, _ = O.eval_map(G, Z, np.ones((1, 1, L), np.uint8))
        Y = np.linalg.solve(np.eye(2) + S[0], np.eye(2) - S[0]) / 50.0
        z12.append(np.linalg.inv(Y)[0, 1])
    ls, z12 = np.array([(L + 2) * a for L in lengths]), np.array(z12)
    k0 = 2 * np.pi * f / C0
    ee = O.eps_eff(O.Grid(PI.Grid("hj", 1, 4, 1, a, 0, (h,), h, er, 0.0, 2, ())))

    def res(p):
        r = ((p[0] + 1j * p[1]) / np.sinh((p[2] + 1j * p[3]) * (ls + p[4])) - z12) / np.abs(z12)
        return np.concatenate([r.real, r.imag])
    sol = least_squares(res, [40, 0, 0, 1.6 * k0, 0], x_scale="jac")
    assert sol.cost < 1e-6
    assert abs(sol.x[3] / k0 / np.sqrt(ee) - 1) < 0.01
