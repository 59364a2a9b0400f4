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
