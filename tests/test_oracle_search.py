"""Oracle pins for the tree search (Algorithm 1): the generator against SplitMix64's published
output sequence, and the search against brute force over every map of a small grid."""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O
from oracle import search as OS


def test_splitmix64_reference_sequence():
    # first outputs of SplitMix64 started from state 0 (Steele, Lea and Flood 2014)
    state, outs = 0, []
    for _ in range(3):
        outs.append(OS.splitmix64(state))
        state = (state + OS.GOLDEN) & OS.MASK
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _tiny_problem():
    g = PI.grid_tiny(3)
    OG = O.Grid(g)
    freqs = np.array([2.0e9, 2.5e9, 3.5e9, 5.0e9])
    Z, _ = O.fill(OG, freqs)
    band = O.bands(freqs, PI.PLAIN_BANDS)

    def evaluate(maps):
        S, _ = O.eval_batch(OG, Z, maps)
        return O.fom_batch(S, band)
    return g, evaluate


@pytest.mark.slow
def test_search_reaches_brute_force_optimum():
    g, evaluate = _tiny_problem()
    allf = evaluate(PI.all_maps(g))
    gmin = float(allf.min())
    init = PI.seed_map(g, 0.5, 11)
    best_map, best_F, evals, trace = OS.tree_search(evaluate, init, seed=7, d_max=2, m_of_d=(10, 3), max_evals=600)
    assert evals >= 600
    assert best_F == pytest.approx(gmin, rel=1e-12)
    assert float(evaluate(best_map[None])[0]) == pytest.approx(best_F, rel=1e-12)
    # the current FoM never increases between restarts, and the best is monotone
    assert min(trace) >= gmin


def test_search_bookkeeping_small_budget():
    g, evaluate = _tiny_problem()
    init = PI.seed_map(g, 0.5, 3)
    f0 = float(evaluate(init[None])[0])
    best_map, best_F, evals, trace = OS.tree_search(evaluate, init, seed=1, d_max=2, m_of_d=(2, 1), max_evals=20)
    assert best_F <= f0
    assert evals >= 20
    # a 1-layer grid has two states per column: one child per node, D children per tree
    assert len(trace) >= 5


def _via_problem():
    import dataclasses
    g = dataclasses.replace(PI.grid_tiny(2, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5625e-3), name="via_2x2x2", n_states=3)
    OG = O.Grid(g)
    freqs = np.array([5.5e9, 6.2e9, 6.8e9, 8.0e9])
    Z, _ = O.fill(OG, freqs)
    band = O.bands(freqs, PI.UNII_BANDS)

    def evaluate(maps):
        S, _ = O.eval_batch(OG, Z, maps)
        return O.fom_batch(S, band)
    return g, evaluate


def test_three_state_column_states():
    """Mixed-radix column states of a three-layer grid with vias: 3 x 3 x 2 = 18 states, each
    set/read back exactly, together exactly the valid layer patterns (no via on the last layer);
    the restart map keeps about half the pixels metal and puts vias only below the last layer."""
    m = np.zeros((3, 2, 2), np.uint8)
    assert OS.radices(3, 3) == [3, 3, 2] and OS.radices(3, 2) == [2, 2, 2]
    seen = set()
    for s in range(18):
        c = OS.set_column(m, 3, s, 3)
        assert OS.column_state(c, 3, 3) == s
        seen.add(tuple(int(v) for v in c[:, 1, 1]))
        assert np.array_equal(np.delete(c.reshape(3, -1), 3, axis=1), np.zeros((3, 3), np.uint8))
    assert seen == {(a, b, t) for a in range(3) for b in range(3) for t in range(2)}
    r = OS.random_map(5, 1, (3, 20, 20), 3)
    assert (r[2] <= 1).all() and (r[:2] == 2).any()
    assert abs((r >= 1).mean() - 0.5) < 0.05
    assert np.array_equal(OS.random_map(5, 1, (2, 4, 4), 2), OS.random_map(5, 1, (2, 4, 4)))


@pytest.mark.slow
def test_search_with_vias_reaches_brute_force_optimum():
    g, evaluate = _via_problem()
    allm = np.stack([np.array([lo, hi], np.uint8).reshape(2, 2, 2)
                     for lo in __import__("itertools").product(range(3), repeat=4)
                     for hi in __import__("itertools").product(range(2), repeat=4)])
    allf = evaluate(allm)
    gmin = float(allf.min())
    init = PI.seed_map(g, 0.5, 11)
    best_map, best_F, evals, trace = OS.tree_search(evaluate, init, seed=7, d_max=2, m_of_d=(6, 2), max_evals=900,
                                                    n_states=3)
    assert best_F == pytest.approx(gmin, rel=1e-12)
    assert (best_map == 2).any() == (allm[int(np.argmin(allf))] == 2).any()


@pytest.mark.parametrize("n_states", [2, 3])
def test_depth1_neighbourhood_equals_brute_force(n_states):
    """The children the search evaluates at depth 1 are exactly the maps that differ from the node
    in the chosen column only (every other valid state of that column), checked against a filter
    over every map of a 2 x 2 two-layer grid, in the search's order (column states ascending)."""
    import itertools
    L, ny, nx = 2, 2, 2
    top = 3 if n_states == 3 else 2
    allm = np.stack([np.array([lo, hi], np.uint8).reshape(L, ny, nx)
                     for lo in itertools.product(range(top), repeat=4) for hi in itertools.product(range(2), repeat=4)])
    init = allm[37].copy()
    seen = []

    def evaluate(maps):
        seen.append(np.array(maps))
        return np.arange(len(maps), 0, -1, dtype=float)   # the last child is best: it is accepted
    OS.tree_search(evaluate, init, seed=3, d_max=1, m_of_d=(1,), max_evals=2, n_states=n_states)
    kids = seen[1]
    j = OS.key(3, 0, 0, 0, 0) % (ny * nx)
    y, x = divmod(j, nx)
    mask = np.ones((L, ny, nx), bool)
    mask[:, y, x] = False
    brute = [m for m in allm if np.array_equal(m[mask], init[mask]) and not np.array_equal(m, init)]
    assert len(kids) == len(brute) == int(np.prod(OS.radices(L, n_states))) - 1
    order = sorted(brute, key=lambda m: OS.column_state(m, j, n_states))
    assert all(np.array_equal(a, b) for a, b in zip(kids, order))


@pytest.mark.parametrize("split", [60, 151, 290])
def test_resumed_search_equals_uninterrupted(split):
    """Checkpoint / resume: a search stopped after `split` evaluations and continued from its state
    makes the same decisions as one uninterrupted run (same trace, best map, best FoM and
    evaluation count), including across restarts."""
    g, evaluate = _tiny_problem()
    init = PI.seed_map(g, 0.5, 2)
    args = dict(seed=5, d_max=2, m_of_d=(3, 1))
    full = OS.tree_search(evaluate, init, max_evals=400, **args)
    a = OS.tree_search(evaluate, init, max_evals=split, return_state=True, **args)
    b = OS.tree_search(evaluate, init, max_evals=400, state=a[4], **args)
    assert np.array_equal(b[0], full[0]) and b[1] == full[1] and b[2] == full[2]
    assert a[3] + b[3] == full[3]
    assert a[4]["restart"] >= 0 and (split < 100 or a[4]["restart"] >= 1 or a[4]["iteration"] > 10)


def test_depth_beyond_the_column_count_is_rejected():
    """A depth-D tree changes D distinct columns: on a 2 x 2 grid (four columns) d_max = 8 has no
    node to draw at depth 5, so the search refuses it instead of drawing from an empty list."""
    g = PI.grid_tiny(2)
    init = PI.seed_map(g, 0.5, 1)
    with pytest.raises(ValueError):
        OS.tree_search(lambda m: np.zeros(len(m)), init, seed=1, d_max=8, m_of_d=(1,) * 8, max_evals=10)
    with pytest.raises(ValueError):
        OS.tree_search(lambda m: np.zeros(len(m)), init, seed=1, d_max=0, m_of_d=(1,), max_evals=10)
