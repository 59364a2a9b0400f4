"""Oracle pins: mesh, basis-function classes and support set (Section II-C, Eq. 3, Section VI-A)."""
import itertools

import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O


def _m_closed_form(g):
    n, m = g.nx, g.ny
    return 4 * g.n_ports + g.layers * (n * m + (n - 1) * m + n * (m - 1))


@pytest.mark.parametrize("g", [PI.grid_plain_8x8(), PI.grid_stripline_16x16x2(), PI.grid_tiny(3),
                               PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2), PI.grid_microstrip_24x24x3()])
def test_bf_count_closed_form(g):
    G = O.Grid(g)
    assert G.M == _m_closed_form(g)
    if g.name == "microstrip_24x24x3":
        assert G.M == 5052
    if g.name == "plain_8x8_microstrip":
        assert G.M == 188
    if g.name == "stripline_16x16x2":
        assert G.M == 1484


def _edges_of(v):
    return [frozenset([tuple(np.round(v[i], 12)), tuple(np.round(v[(i + 1) % 3], 12))]) for i in range(3)]


@pytest.mark.parametrize("g", [PI.grid_tiny(3), PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2)])
def test_rwg_geometry_and_edge_census(g):
    """Each BF's two triangles share exactly its edge; the free vertices are off that edge; every
    edge shared by two triangles carries exactly one BF; each layer's sheet is a disk (V - E + F = 1
    per connected sheet of grid + stubs)."""
    G = O.Grid(g)
    tris = {}
    for row in G.table:
        for k in (row[4], row[5]):
            tris[int(k)] = O.triangle(G, k)
    bf_edges = []
    for row in G.table:
        vp, vm = tris[int(row[4])], tris[int(row[5])]
        shared = set(map(tuple, np.round(vp, 12))) & set(map(tuple, np.round(vm, 12)))
        assert len(shared) == 2
        fp, fm = tuple(np.round(vp[row[6]], 12)), tuple(np.round(vm[row[7]], 12))
        assert fp not in shared and fm not in shared
        L = np.linalg.norm(np.array(list(shared))[0] - np.array(list(shared))[1])
        assert np.isclose(L, g.pitch_m) or np.isclose(L, g.pitch_m * np.sqrt(2))
        bf_edges.append(frozenset(shared))
    assert len(set(bf_edges)) == len(bf_edges)
    count = {}
    for v in tris.values():
        for e in _edges_of(v):
            count[e] = count.get(e, 0) + 1
    interior = {e for e, c in count.items() if c == 2}
    assert max(count.values()) == 2
    assert interior == set(bf_edges)
    for layer in range(g.layers):
        vs = [v for v in tris.values() if np.isclose(v[0][2], g.layer_z_m[layer])]
        V = {tuple(np.round(p, 12)) for v in vs for p in v}
        E = {e for v in vs for e in _edges_of(v)}
        assert len(V) - len(E) + len(vs) == 1


def test_activation_brute_force_3x3():
    """All 512 maps: N = 3P (stub) + #metal + #edge-adjacent metal pairs + #ports whose grid pixel is
    metal.  Pixels touching only at a corner add nothing (Section VI-A)."""
    g = PI.grid_tiny(3)
    G = O.Grid(g)
    maps = PI.all_maps(g)
    assert maps.shape[0] == 512
    for m in maps:
        a = m[0]
        pairs = int(np.sum(a[:, :-1] & a[:, 1:]) + np.sum(a[:-1, :] & a[1:, :]))
        gp = {0: (g.nx - 1, None), 1: (None, g.ny - 1), 2: (0, None), 3: (None, 0)}
        nport = 0
        for p in g.ports:
            x, y = gp[p.side]
            x = p.pos if x is None else x
            y = p.pos if y is None else y
            nport += int(a[y, x])
        idx = O.active_set(G, m)
        assert len(idx) == 3 * g.n_ports + int(a.sum()) + pairs + nport
        assert np.all(np.diff(idx) > 0)
        assert np.all(idx[: 3 * g.n_ports] == np.arange(3 * g.n_ports))


def test_diagonal_contact_is_not_a_connection():
    g = PI.grid_tiny(3)
    G = O.Grid(g)
    diag = np.array([[[1, 0, 0], [0, 1, 0], [0, 0, 0]]], np.uint8)
    single = np.array([[[1, 0, 0], [0, 0, 0], [0, 0, 0]]], np.uint8)
    both = O.active_set(G, diag)
    one = O.active_set(G, single)
    # two isolated pixels: exactly one more inner BF than a single pixel (plus none between them)
    assert len(both) == len(one) + 1


def test_single_flip_changes_at_most_five_bfs():
    g = PI.grid_plain_8x8()
    G = O.Grid(g)
    seed = PI.seed_map(g, 0.5, 3)
    base = set(O.active_set(G, seed).tolist())
    for c in PI.single_flip_batch(seed):
        d = base.symmetric_difference(O.active_set(G, c).tolist())
        assert 1 <= len(d) <= 5


def test_bad_state_rejected():
    g = PI.grid_tiny(3)
    G = O.Grid(g)
    m = np.zeros((1, 3, 3), np.uint8)
    m[0, 1, 1] = 2
    with pytest.raises(ValueError):
        O.active_set(G, m)


def _patterned(g, pattern, seed=0):
    import dataclasses
    return dataclasses.replace(g, name=f"{g.name}_diag{pattern}", diag_pattern=pattern, diag_seed=seed)


def test_diagonal_orientation_patterns():
    """Section V-A / Fig. mesh_orientation (a)-(c): alternating = (x + y) mod 2, uniform = 0,
    random = the top bit of SplitMix64 chained over (seed, position), checked against the search
    module's own SplitMix64; about half of the random diagonals take each orientation and two
    seeds give different patterns."""
    from oracle import search as OS
    g = PI.grid_tiny(8)
    G0, G1 = O.Grid(g), O.Grid(_patterned(g, 1))
    G2, G2b = O.Grid(_patterned(g, 2, 17)), O.Grid(_patterned(g, 2, 18))
    pos = [(x, y) for y in range(-2, 10) for x in range(-2, 10)]
    assert all(O.orient(G0, x, y) == (x + y) % 2 for x, y in pos)
    assert all(O.orient(G1, x, y) == 0 for x, y in pos)
    r = [O.orient(G2, x, y) for x, y in pos]
    assert r == [OS.key(17, (y + 4) * 128 + x + 4) >> 63 for x, y in pos]
    assert 0.35 < np.mean(r) < 0.65
    assert r != [O.orient(G2b, x, y) for x, y in pos]


@pytest.mark.parametrize("pattern", [1, 2])
def test_rwg_geometry_other_orientations(pattern):
    g = _patterned(PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2), pattern, 5)
    test_rwg_geometry_and_edge_census(g)


@pytest.mark.parametrize("pattern", [1, 2])
def test_activation_does_not_depend_on_orientation(pattern):
    g = PI.grid_tiny(3)
    G0, G = O.Grid(g), O.Grid(_patterned(g, pattern, 9))
    assert G.M == G0.M and np.array_equal(G.table[:, :4], G0.table[:, :4])
    for m in PI.all_maps(g)[::7]:
        assert np.array_equal(O.active_set(G, m), O.active_set(G0, m))
