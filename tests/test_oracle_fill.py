"""Oracle pins for the EFIE fill (Eq. 1-2): translation invariance, reciprocity, passivity, the
static capacitance of a strip against closed-form line theory, the propagation constant of a
TEM line, and the textbook half-wave dipole."""
import numpy as np
import pytest
from scipy.optimize import least_squares
from scipy.special import ellipk

import pmom_inputs as PI
from oracle import oracle as O

C0 = 299792458.0
ETA0 = 376.730313668
EPS0 = 8.8541878128e-12


@pytest.fixture(scope="module")
def c1_fill():
    w = PI.workload_plain()
    G = O.Grid(w.grid)
    Z, asym = O.fill(G, w.freqs())
    return w, G, Z, asym


@pytest.mark.parametrize("g", [PI.grid_plain_8x8(), PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2)])
def test_lattice_table_fill_equals_direct_fill(g):
    G = O.Grid(g)
    f = [1.3e9, 6.1e9]
    Zd, _ = O.fill(G, f, mode=0)
    Zt, _ = O.fill(G, f, mode=1)
    assert np.abs(Zd - Zt).max() <= 1e-12 * np.abs(Zd).max()


def test_reciprocity_and_passivity(c1_fill):
    w, G, Z, asym = c1_fill
    assert asym < 1e-4                     # quadrature-level asymmetry before symmetrisation
    for Zf in Z:
        assert np.abs(Zf - Zf.T).max() == 0.0
        herm = 0.5 * (Zf + Zf.conj().T)
        assert np.linalg.eigvalsh(herm).min() >= -1e-10 * np.abs(Zf).max()


def test_stripline_passivity():
    g = PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2)
    G = O.Grid(g)
    Z, asym = O.fill(G, [1e9, 5e9, 9e9])
    assert asym < 1e-4
    for Zf in Z:
        herm = 0.5 * (Zf + Zf.conj().T)
        assert np.linalg.eigvalsh(herm).min() >= -1e-10 * np.abs(Zf).max()


def _static_cap(g):
    G = O.Grid(g)
    keys = sorted(set(G.table[:, 4]).union(set(G.table[:, 5])))
    tris = [O.triangle(G, k) for k in keys]
    areas = np.array([0.5 * np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0])) for t in tris])
    P = np.array([[O.pair_integrals(G, 1.0, kp, kq)[0].real for kq in keys] for kp in keys])
    P /= EPS0 * areas[:, None] * areas[None, :]
    return np.linalg.solve(P, np.ones(len(keys))).sum()


def _strip(L, a, medium, z, H, ports=()):
    return PI.Grid("strip", 1, L, 1, a, medium, (z,), H, 1.0, 0.0, 2, ports)


@pytest.mark.slow
def test_static_line_capacitance_matches_line_theory():
    """Per-unit-length capacitance of a long strip (difference of two lengths) gives the air-line
    impedance 1/(c C') within 8 % of Hammerstad-Jensen (microstrip) and Cohn (stripline)."""
    a, h = 2e-3, 0.5e-3
    cp = (_static_cap(_strip(24, a, 0, h, h)) - _static_cap(_strip(12, a, 0, h, h))) / (12 * a)
    u = a / h
    F1 = 6 + (2 * np.pi - 6) * np.exp(-(30.666 / u) ** 0.7528)
    z_hj = ETA0 / (2 * np.pi) * np.log(F1 / u + np.sqrt(1 + (2 / u) ** 2))
    assert abs(1 / (C0 * cp) - z_hj) < 0.08 * z_hj
    a, H = 0.5e-3, 0.9732e-3
    cp = (_static_cap(_strip(24, a, 1, H / 2, H)) - _static_cap(_strip(12, a, 1, H / 2, H))) / (12 * a)
    k = 1 / np.cosh(np.pi * a / (2 * H))
    z_cohn = ETA0 / 4 * ellipk(k ** 2) / ellipk(1 - k ** 2)
    assert abs(1 / (C0 * cp) - z_cohn) < 0.08 * z_cohn


def _line_beta(medium, a, z, H, er, f, lengths):
    z12 = []
    for L in lengths:
        g = PI.Grid("line", 1, L, 1, a, medium, (z,), H, er, 0.0, 2,
                    (PI.Port(0, PI.SIDE_LEFT, 0), PI.Port(0, PI.SIDE_RIGHT, 0)))
        G = O.Grid(g)
        Z, _ = O.fill(G, [f], threads=1)
        S, _ = O.eval_map(G, Z, np.ones((1, 1, L), np.uint8))
        Y = np.linalg.solve(np.eye(2) + S[0], np.eye(2) - S[0]) / 50.0
        z12.append(np.linalg.inv(Y)[0, 1])
    ls, z12 = np.array([(L + 2) * a for L in lengths]), np.array(z12)
    ee = O.eps_eff(G)
    beta0 = 2 * np.pi * f / C0 * np.sqrt(ee)

    def res(p):
        r = ((p[0] + 1j * p[1]) / np.sinh((p[2] + 1j * p[3]) * (ls + p[4])) - z12) / np.abs(z12)
        return np.concatenate([r.real, r.imag])
    sol = least_squares(res, [40, 0, 0, beta0, 0], x_scale="jac")
    return sol.x[3] / beta0, sol.cost


def test_tem_line_propagation_constant():
    """Transfer impedance Z12 = Zc / sinh(gamma l) of a through line: beta within 1 % of the
    dielectric wavenumber (stripline, exact TEM) and within 2 % of k0 sqrt(eps_eff) (microstrip)."""
    ratio, cost = _line_beta(1, 0.5e-3, 0.4866e-3, 0.9732e-3, 3.66, 6e9, range(6, 30, 4))
    assert cost < 1e-8 and abs(ratio - 1) < 0.01
    ratio, cost = _line_beta(0, 2e-3, 0.5e-3, 0.5e-3, 3.5, 3e9, range(4, 16, 2))
    assert cost < 1e-4 and abs(ratio - 1) < 0.02


def test_half_wave_strip_dipole():
    """A strip dipole far above the ground image behaves as in free space: series resonance near
    0.47-0.48 lambda with a radiation resistance of about 70 ohm."""
    f, a = 1e9, 2e-3
    zin = []
    for L in (69, 71, 73, 75):
        g = PI.Grid("dipole", 1, L, 1, a, 0, (10.0,), 10.0, 1.0, 0.0, 2, (PI.Port(0, PI.SIDE_LEFT, 0),))
        G = O.Grid(g)
        Z, _ = O.fill(G, [f], threads=1)
        t = G.table
        c = L // 2
        m = [i for i in range(G.M) if t[i, 0] == 2 and t[i, 1] == c and t[i, 2] == c + 1][0]
        keep = [i for i in range(G.M) if t[i, 0] in (1, 2)]
        V = np.zeros(len(keep), complex)
        V[keep.index(m)] = a
        x = np.linalg.solve(Z[0][np.ix_(keep, keep)], V)
        zin.append(1 / (a * x[keep.index(m)]))
    zin = np.array(zin)
    assert np.all(np.diff(zin.imag) > 0)
    i = int(np.argmin(np.abs(zin.imag)))
    assert abs(zin[i].imag) < 15 and 60 < zin[i].real < 85
    assert 0.46 < (69 + 2 * i) * a / (C0 / f) < 0.49


@pytest.mark.parametrize("pattern", [1, 2])
def test_other_orientations_fill(pattern):
    """Uniform and random diagonals (Fig. mesh_orientation a, c): the lattice-table fill, whose
    classes carry both triangles' orientations, equals the direct fill; reciprocity and passivity
    hold as for the alternating mesh."""
    import dataclasses
    g = dataclasses.replace(PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2), diag_pattern=pattern, diag_seed=3)
    G = O.Grid(g)
    f = [1.3e9, 6.1e9]
    Zd, _ = O.fill(G, f, mode=0)
    Zt, asym = O.fill(G, f, mode=1)
    assert np.abs(Zd - Zt).max() <= 1e-12 * np.abs(Zd).max()
    assert asym < 1e-4
    for Zf in Zt:
        herm = 0.5 * (Zf + Zf.conj().T)
        assert np.linalg.eigvalsh(herm).min() >= -1e-10 * np.abs(Zf).max()


@pytest.mark.parametrize("case", ["microstrip", "vias"])
def test_substructure_premise(case):
    """Eq. (4)-(5): the interaction matrix of a candidate's own mesh, filled directly with only its
    active BFs, is bit for bit the parent's rows and columns of those BFs (same per-pair code), so a
    database of the all-metal parent serves every candidate."""
    import dataclasses
    if case == "microstrip":
        g = PI.grid_tiny(3)
        maps = PI.all_maps(g)[[5, 200, 511]]
    else:
        g = dataclasses.replace(PI.grid_tiny(3, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5e-3), n_states=3)
        maps = PI.state_changes(PI.seed_map_vias(g, 0.6, 0.5, 1), 1, 3, 2)
        assert (maps == 2).any()
    G = O.Grid(g)
    f = [2.4e9, 5.2e9]
    Z, _ = O.fill(G, f, mode=0)
    for m in maps:
        idx = O.active_set(G, m)
        Zs = O.fill_subset(G, f, idx, mode=0)
        assert np.array_equal(Zs.view(np.uint64), np.ascontiguousarray(Z[:, idx][:, :, idx]).view(np.uint64))


@pytest.mark.parametrize("medium", [PI.MEDIUM_MICROSTRIP, PI.MEDIUM_STRIPLINE])
def test_low_frequency_limit(medium):
    """As f -> 0, f Z(f) tends to the static capacitive term (the scalar potential of Eq. 1 over
    j 2 pi eps) and the first correction is quadratic in f: the O(k) terms of each source and its
    image cancel, and the Dirichlet mode sum is analytic in k^2.  Doubling f quadruples the
    departure from the static limit (to 1e-4 here); an unbalanced image or a wrong k would leave
    a linear term."""
    g = PI.grid_tiny(3) if medium == PI.MEDIUM_MICROSTRIP else PI.grid_tiny(3, PI.MEDIUM_STRIPLINE, 2)
    G = O.Grid(g)
    fs = [1e3, 2e7, 4e7, 8e7]
    Z, _ = O.fill(G, fs)
    X = np.array([f * Z[i] for i, f in enumerate(fs)])
    d = [np.abs(X[i] - X[0]).max() for i in (1, 2, 3)]
    assert d[0] < 1e-5 * np.abs(X[0]).max()
    assert abs(d[1] / d[0] - 4.0) < 1e-4 and abs(d[2] / d[1] - 4.0) < 1e-4


@pytest.mark.parametrize("g", [PI.grid_plain_8x8(), PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2)])
def test_pair_integrals_reciprocal_per_triangle_pair(g):
    """Reciprocity below the level of Z: the integrals of a triangle pair (the scalar
    int int G and the vector moments int int (r - v_a) . G (r' - v_b)) taken with the two triangles
    swapped.  Far pairs (centroids at least two longest edges apart, ties near) use one product
    Gauss rule on both triangles, so the swap reproduces them -- the moment matrix transposed -- to
    rounding (measured 8.5e-16 relative over 3000 sampled pairs of each grid); near pairs integrate
    the 1/R part analytically over one triangle only, so they agree to quadrature level (measured up
    to 1.1e-3 on the microstrip grid, 2.3e-3 on the two-layer stripline; on Z the sums of such terms
    leave 3e-5).  A height or a vertex taken from the wrong triangle breaks the first."""
    G = O.Grid(g)
    t = O.bf_table(G)
    keys = sorted(set(t[:, 4]).union(set(t[:, 5])))
    tris = {k: O.triangle(G, k) for k in keys}
    cen = {k: tris[k].mean(axis=0) for k in keys}
    lmax = {k: max(np.linalg.norm(tris[k][i] - tris[k][(i + 1) % 3]) for i in range(3)) for k in keys}
    rng = np.random.default_rng(7)
    far, near = [], []
    for _ in range(4000):
        p, q = rng.choice(keys, 2, replace=False)
        d = np.linalg.norm(cen[p] - cen[q])
        (near if d < 2.0 * max(lmax[p], lmax[q]) * (1.0 + 1e-9) else far).append((p, q))
        if len(far) >= 200 and len(near) >= 100:
            break
    assert len(far) >= 200 and len(near) >= 100
    f = 3.7e9
    for group, tol in ((far[:200], 1e-13), (near[:100], 5e-3)):
        for p, q in group:
            a = O.pair_integrals(G, f, p, q)
            b = O.pair_integrals(G, f, q, p)
            scale = np.abs(a).max()
            assert abs(a[0] - b[0]) <= tol * abs(a[0]), (p, q)
            Ma, Mb = a[1:].reshape(3, 3), b[1:].reshape(3, 3)
            assert np.abs(Ma - Mb.T).max() <= tol * scale, (p, q)
