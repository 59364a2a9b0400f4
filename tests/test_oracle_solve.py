"""Oracle pins for the candidate evaluation: dense solve vs LAPACK, S-parameter forms
(Eq. 6-7) against each other, reciprocity and passivity, FoM closed forms (Eq. 8-9), band
assignment, complex64 promotion, and brute force over every map of a 3x3 grid."""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O


@pytest.fixture(scope="module")
def c1():
    w = PI.workload_plain()
    G = O.Grid(w.grid)
    Z, _ = O.fill(G, w.freqs())
    return w, G, Z


def test_lu_solve_matches_lapack(c1):
    w, G, Z = c1
    rng = np.random.default_rng(1)
    idx = O.active_set(G, PI.seed_map(w.grid, 0.5, 0))
    for A in (Z[0][np.ix_(idx, idx)], rng.standard_normal((57, 57)) + 1j * rng.standard_normal((57, 57))):
        B = rng.standard_normal((A.shape[0], 3)) + 1j * rng.standard_normal((A.shape[0], 3))
        LU, piv, sing = O.lu(A)
        assert sing == 0
        X = O.lu_solve(LU, piv, B)
        Xr = np.linalg.solve(A, B)
        assert np.abs(X - Xr).max() <= 1e-12 * np.linalg.cond(A) * np.abs(Xr).max() / 1e3 + 1e-10 * np.abs(Xr).max()
        bw = np.abs(B - A @ X).max() / (np.abs(A).max() * np.abs(X).max())
        assert bw <= 1e-15 * A.shape[0]


def test_pivot_ties_take_lowest_row():
    A = np.array([[1, 2, 0], [1j, 1, 0], [-1, 0, 1]], dtype=complex)   # |a_i0| = 1 for every row
    LU, piv, _ = O.lu(A)
    assert piv[0] == 0
    A2 = np.array([[0.5, 1], [1j, 0], [-1, 2]], dtype=complex)[:2]
    LU, piv, _ = O.lu(np.array([[0.5, 1], [1j, 0]], dtype=complex))
    assert piv[0] == 1


def test_singular_flag():
    _, _, sing = O.lu(np.zeros((3, 3), complex))
    assert sing == 1


def test_s_forms_agree_reciprocal_passive(c1):
    w, G, Z = c1
    for seed in range(4):
        m = PI.seed_map(w.grid, 0.5, seed)
        S0, st = O.eval_map(G, Z, m, form=0)
        S1, _ = O.eval_map(G, Z, m, form=1)
        assert st == 0
        assert np.abs(S0 - S1).max() <= 1e-12
        for s in S0:
            assert np.abs(s - s.T).max() <= 1e-12
            assert np.linalg.norm(s, 2) <= 1 + 1e-9
            assert (np.abs(s) ** 2).sum(0).max() <= 1 + 1e-9


def test_one_port_reflection_closed_form(c1):
    """S11 of the solved network equals (Zin - Z0)/(Zin + Z0) with Zin = V / (l i) at port 1 with
    the other ports shorted (their gaps carry no source and no load)."""
    w, G, Z = c1
    m = PI.seed_map(w.grid, 0.5, 2)
    idx = O.active_set(G, m)
    A = Z[3][np.ix_(idx, idx)]
    l = w.grid.pitch_m
    V = np.zeros(len(idx), complex)
    V[1] = l
    x = np.linalg.solve(A, V)
    y11 = l * x[1]
    S, _ = O.eval_map(G, Z[3:4], m)
    Y = np.linalg.solve(np.eye(3) + S[0], np.eye(3) - S[0]) / 50.0
    assert abs(Y[0, 0] - y11) <= 1e-10 * abs(y11)


def test_complex64_database_is_promoted_exactly(c1):
    w, G, Z = c1
    m = PI.seed_map(w.grid, 0.5, 1)
    Z64 = Z[:2].astype(np.complex64)
    Sa, _ = O.eval_map(G, Z64, m)
    Sb, _ = O.eval_map(G, Z64.astype(np.complex128), m)
    assert np.array_equal(Sa, Sb)


def _s_from_db(s11, s21, s31, s32):
    S = np.zeros((3, 3), complex)
    S[0, 0] = 10 ** (s11 / 20)
    S[1, 0] = S[0, 1] = 10 ** (s21 / 20)
    S[2, 0] = S[0, 2] = 10 ** (s31 / 20)
    S[2, 1] = S[1, 2] = 10 ** (s32 / 20) * 1j
    return S


def test_fom_closed_forms():
    # p1: 1/rw_p1 (S21 = -1 dB) + 1/rw_m1 (S11 = -15 dB) + 1/rw_s2 (S31 = -35 dB) = 3
    assert abs(O.fom(_s_from_db(-15, -1, -35, -60)[None], np.array([0], np.uint8)) - 3) < 1e-12
    # p2: 1/rw_p2 (S31 = -1) + 1/rw_m2 (S11 = -15) + 1/rw_s1 (S21 = -35) = 3
    assert abs(O.fom(_s_from_db(-15, -35, -1, -60)[None], np.array([1], np.uint8)) - 3) < 1e-12
    # i: 1/rw_oi (S32 = -20) = 1 ; s: 1/rw_s3 + 1/rw_s4 (S21 = S31 = -20) = 2 ; none: 0
    assert abs(O.fom(_s_from_db(0, 0, 0, -20)[None], np.array([2], np.uint8)) - 1) < 1e-12
    assert abs(O.fom(_s_from_db(0, -20, -20, 0)[None], np.array([3], np.uint8)) - 2) < 1e-12
    assert O.fom(_s_from_db(0, -20, -20, 0)[None], np.array([255], np.uint8)) == 0.0
    # exponents: 10 dB worse insertion loss in p1 multiplies that term by 10
    assert abs(O.fom(_s_from_db(-15, -11, -35, -60)[None], np.array([0], np.uint8)) - 12) < 1e-12
    # the dB floor keeps an exact zero finite
    S = _s_from_db(-15, -1, -35, -60)
    S[2, 0] = S[0, 2] = 0
    assert np.isfinite(O.fom(S[None], np.array([0], np.uint8)))
    # frequencies add in order
    S2 = np.stack([_s_from_db(-15, -1, -35, -60), _s_from_db(0, 0, 0, -20)])
    assert abs(O.fom(S2, np.array([0, 2], np.uint8)) - 4) < 1e-12


def test_band_assignment():
    w = PI.workload_plain()
    assert O.bands(w.freqs(), w.bands).tolist() == [3, 3, 0, 0, 2, 2, 2, 2, 1, 1, 3]
    w = PI.workload_precision()
    b = O.bands(w.freqs(), w.bands)
    f = w.freqs()
    for fi, bi in zip(f, b):
        if 5.15e9 <= fi <= 5.925e9:
            assert bi == 0
        elif 6.425e9 <= fi <= 7.125e9:
            assert bi == 1
        elif 5.925e9 < fi < 6.425e9:
            assert bi == 2
        elif 3e9 <= fi <= 9e9:
            assert bi == 3
        else:
            assert bi == 255


@pytest.mark.slow
def test_brute_force_every_3x3_map():
    g = PI.grid_tiny(3)
    G = O.Grid(g)
    f = [2.5e9, 5.0e9]
    Z, _ = O.fill(G, f)
    maps = PI.all_maps(g)
    S, status = O.eval_batch(G, Z, maps)
    assert np.all(status == 0)
    assert np.abs(S - np.swapaxes(S, 2, 3)).max() <= 1e-12
    assert max(np.linalg.norm(s, 2) for s in S.reshape(-1, 3, 3)) <= 1 + 1e-9
    # batch evaluation equals the single-map route, map by map
    for b in (0, 77, 300, 511):
        Sb, _ = O.eval_map(G, Z, maps[b])
        assert np.array_equal(Sb, S[b])
    # the empty map leaves each port with its own stub only: nearly total reflection and only
    # weak stub-to-stub coupling through the medium
    off = S[0] * (1 - np.eye(3))
    assert np.abs(off).max() < 1e-2
    assert np.abs(np.diagonal(S[0], axis1=1, axis2=2)).min() > 0.99


def test_lapack_solve_route_matches_c_oracle(c1):
    """The LAPACK-backed evaluation (used for support sets of thousands of BFs) follows the same
    definition as the plain C path: agreement to 1e-12 on the 8x8 microstrip and a 4x4x2
    stripline, both storage precisions; port edges are one pixel side (R2 stub geometry)."""
    w, OG, Z = c1
    g = w.grid
    maps = PI.random_maps(g, 3, 0.5, 11)
    assert np.allclose(O.port_lengths(OG), g.pitch_m, rtol=1e-14)
    for m in maps:
        S_c, st = O.eval_map(OG, Z, m)
        assert st == 0
        assert np.abs(O.eval_map_lapack(OG, Z, m) - S_c).max() <= 1e-12
    gs = PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2)
    OGs = O.Grid(gs)
    Zs, _ = O.fill(OGs, [2.0e9, 6.5e9])
    Zs64 = Zs.astype(np.complex64)
    for m in PI.random_maps(gs, 3, 0.6, 12):
        S_c, st = O.eval_map(OGs, Zs64, m)
        assert st == 0
        assert np.abs(O.eval_map_lapack(OGs, Zs64, m) - S_c).max() <= 1e-12


def test_condition_numbers_support_the_precision_policy():
    """cond_2(Z_sub) of sampled candidates at five frequencies of the plain and precision
    workloads (complex64 storage promoted exactly).  Mixed-precision refinement converges when
    u_32 cond < 1 with a contraction of about u_32 cond per correction, and the forward error of
    the refined solution is about cond times its backward error (1e-12), so cond <= 1e5 keeps
    |dS| far inside 1e-6.  A report with a loose bound, not a tight pin."""
    import pmom_inputs as PI
    for w, bound in ((PI.workload_plain(), 1e5), (PI.workload_precision(), 2e5)):
        OG = O.Grid(w.grid)
        fr = w.freqs()
        fs = fr[np.linspace(0, len(fr) - 1, 5).round().astype(int)]
        Z, _ = O.fill(OG, fs)
        maps = PI.workload_maps(w)[[0, 7, w.batch - 1]]
        cs = []
        for m in maps:
            idx = O.active_set(OG, m)
            for f in range(len(fs)):
                A = Z[f][np.ix_(idx, idx)]
                if w.z_dtype == "c64":
                    A = A.astype(np.complex64).astype(np.complex128)
                cs.append(np.linalg.cond(A))
        print(w.name, "cond_2(Z_sub) min / median / max: %.3g / %.3g / %.3g" % (min(cs), np.median(cs), max(cs)))
        assert max(cs) <= bound
        assert max(cs) * 2.0 ** -24 < 1e-2
