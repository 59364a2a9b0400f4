"""Oracle pins for the finer pixel meshes of the paper's mesh study (Section V-A): s x s
sub-squares per pixel, 8 (s = 2) or 18 (s = 3) triangles, and ports whose delta gap is the s edges
between the two stub pixels.

Closed-form BF counts; every BF's triangles share exactly its edge and every shared edge carries
one BF; the gap edges tile the stub side; the support set of every sampled map against a counting
formula; lattice fill = direct fill, reciprocity and passivity; the two S forms with multi-edge
ports (unloaded Y -> S and the Z0-loaded gap of Eq. 6) agree, S is reciprocal and passive, the
LAPACK route agrees; and the static line capacitance converges toward Cohn's stripline formula as
the mesh is refined (6.0 %, 4.4 %, 3.0 % for 2, 8, 18 triangles)."""
import dataclasses
import sys
import os

import numpy as np
import pytest
from scipy.special import ellipk

import pmom_inputs as PI
from oracle import oracle as O

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_oracle_fill import C0, ETA0, _static_cap   # noqa: E402


def _sub(g, s):
    return dataclasses.replace(g, name=f"{g.name}_s{s}", sub=s)


def _m_closed_form(g, s):
    ni = s * s + 2 * s * (s - 1)
    per_layer = g.nx * g.ny * ni + s * ((g.nx - 1) * g.ny + g.nx * (g.ny - 1))
    return g.n_ports * (2 * ni + s) + g.n_ports * s + g.layers * per_layer


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("g", [PI.grid_tiny(3), PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2)])
def test_bf_count_and_triangles_per_pixel(g, s):
    G = O.Grid(_sub(g, s))
    assert G.M == _m_closed_form(g, s)
    # the inner BFs of one grid pixel touch exactly 2 s^2 triangles
    rows = G.table[(G.table[:, 0] == 1) & (G.table[:, 1] == 0)]
    assert len(set(rows[:, 4]) | set(rows[:, 5])) == 2 * s * s


def _r(p):
    return tuple(np.round(p, 12))


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("pattern", [0, 2])
def test_rwg_geometry_and_edge_census(s, pattern):
    g = dataclasses.replace(PI.grid_tiny(3, PI.MEDIUM_STRIPLINE, 2), sub=s, diag_pattern=pattern, diag_seed=4)
    G = O.Grid(g)
    a = g.pitch_m / s
    tris = {int(k): O.triangle(G, k) for row in G.table for k in (row[4], row[5])}
    bf_edges = []
    for row in G.table:
        vp, vm = tris[int(row[4])], tris[int(row[5])]
        shared = {_r(p) for p in vp} & {_r(p) for p in vm}
        assert len(shared) == 2
        assert _r(vp[row[6]]) not in shared and _r(vm[row[7]]) not in shared
        e = np.array(sorted(shared))
        L = np.linalg.norm(e[0] - e[1])
        assert np.isclose(L, a) or np.isclose(L, a * np.sqrt(2))
        bf_edges.append(frozenset(shared))
    assert len(set(bf_edges)) == len(bf_edges)
    count = {}
    for v in tris.values():
        for i in range(3):
            e = frozenset([_r(v[i]), _r(v[(i + 1) % 3])])
            count[e] = count.get(e, 0) + 1
    assert max(count.values()) == 2
    assert {e for e, c in count.items() if c == 2} == set(bf_edges)
    # each port's gap: s collinear edges of length a/s tiling the side between the stub pixels
    for bf, lens in O.port_gaps(G):
        assert len(bf) == s and np.allclose(lens, a)
        pts = set()
        for m in bf:
            r = G.table[int(m)]
            v = tris[int(r[4])]
            pts |= {_r(v[(int(r[6]) + 1) % 3]), _r(v[(int(r[6]) + 2) % 3])}
        P = np.array(sorted(pts))
        assert len(P) == s + 1 and np.isclose(np.linalg.norm(P[-1] - P[0]), g.pitch_m)
        assert np.linalg.matrix_rank(P[1:] - P[0], tol=1e-12) == 1


@pytest.mark.parametrize("s", [2, 3])
def test_activation_counts(s):
    """N = P K + n_inner #metal + s #edge-adjacent metal pairs + s #ports whose grid pixel is
    metal, with n_inner = s^2 + 2 s (s - 1) and K = 2 n_inner + s always-present stub BFs."""
    g = _sub(PI.grid_tiny(3), s)
    G = O.Grid(g)
    ni = s * s + 2 * s * (s - 1)
    gp = {0: (g.nx - 1, None), 1: (None, g.ny - 1), 2: (0, None), 3: (None, 0)}
    for m in PI.all_maps(PI.grid_tiny(3))[::5]:
        a = m[0]
        pairs = int(np.sum(a[:, :-1] & a[:, 1:]) + np.sum(a[:-1, :] & a[1:, :]))
        nport = 0
        for p in g.ports:
            x, y = gp[p.side]
            nport += int(a[p.pos if y is None else y, p.pos if x is None else x])
        idx = O.active_set(G, m)
        assert len(idx) == g.n_ports * (2 * ni + s) + ni * int(a.sum()) + s * pairs + s * nport
        assert np.array_equal(idx[: g.n_ports * (2 * ni + s)], np.arange(g.n_ports * (2 * ni + s)))


@pytest.mark.parametrize("s", [2, 3])
def test_fill_and_both_s_forms(s):
    g = _sub(PI.grid_tiny(3), s)
    G = O.Grid(g)
    f = [2.4e9, 5.2e9]
    Zd, _ = O.fill(G, f, mode=0)
    Z, asym = O.fill(G, f, mode=1)
    assert np.abs(Zd - Z).max() <= 1e-12 * np.abs(Zd).max()
    assert asym < 1e-4
    for Zf in Z:
        herm = 0.5 * (Zf + Zf.conj().T)
        assert np.linalg.eigvalsh(herm).min() >= -1e-10 * np.abs(Zf).max()
    for m in PI.all_maps(PI.grid_tiny(3))[::41]:
        S0, st = O.eval_map(G, Z, m)
        S1, _ = O.eval_map(G, Z, m, form=1)
        assert st == 0
        assert np.abs(S0 - S1).max() <= 1e-12
        assert np.abs(S0 - np.swapaxes(S0, 1, 2)).max() <= 1e-12
        assert np.abs(O.eval_map_lapack(G, Z, m) - S0).max() <= 1e-12
        for Sf in S0:
            assert np.linalg.svd(Sf, compute_uv=False).max() <= 1 + 1e-9


@pytest.mark.slow
def test_refinement_converges_toward_line_theory():
    """Air-line impedance 1 / (c C') of a stripline strip from the static capacitance of two
    lengths: the error against Cohn's closed form falls with every refinement of the pixel mesh."""
    a, H = 0.5e-3, 0.9732e-3
    k = 1 / np.cosh(np.pi * a / (2 * H))
    z_cohn = ETA0 / 4 * ellipk(k ** 2) / ellipk(1 - k ** 2)
    err = []
    for s in (1, 2, 3):
        strip = lambda L: PI.Grid("strip", 1, L, 1, a, 1, (H / 2,), H, 1.0, 0.0, 2, (), sub=s)
        cp = (_static_cap(strip(12)) - _static_cap(strip(6))) / (6 * a)
        err.append(abs(1 / (C0 * cp) - z_cohn) / z_cohn)
    assert err[0] > err[1] > err[2]
    assert err[2] < 0.04
