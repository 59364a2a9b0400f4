"""Decision parity of the native tree search (Algorithm 1 on the GPU evaluator) with the oracle's."""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O
from oracle import search as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import pmom
    return pmom


def _problem(g, freqs, bands):
    OG = O.Grid(g)
    Z, _ = O.fill(OG, freqs)
    band = O.bands(freqs, bands)

    def evaluate(maps):
        S, _ = O.eval_batch(OG, Z, maps)
        return O.fom_batch(S, band)
    return Z, band, evaluate


@pytest.mark.parametrize("case", ["tiny_3x3", "plain_8x8", "stripline_4x4x2", "via_3x3x2"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_search_decisions_match_oracle(built, case, prec):
    if case == "tiny_3x3":
        g, freqs, bands, budget = PI.grid_tiny(3), np.array([2.0e9, 2.5e9, 3.5e9, 5.0e9]), PI.PLAIN_BANDS, 300
    elif case == "plain_8x8":
        g, freqs, bands, budget = PI.grid_plain_8x8(), np.array([2.0e9, 3.0e9, 5.0e9]), PI.PLAIN_BANDS, 120
    elif case == "stripline_4x4x2":
        g = PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5625e-3)
        freqs, bands, budget = np.array([5.5e9, 6.2e9, 6.8e9, 8.0e9]), PI.UNII_BANDS, 150
    else:   # three pixel states: columns of 3 x 2 mixed-radix states, vias placed by the search
        import dataclasses
        g = dataclasses.replace(PI.grid_tiny(3, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5625e-3), name="via_3x3x2", n_states=3)
        freqs, bands, budget = np.array([5.5e9, 6.2e9, 6.8e9, 8.0e9]), PI.UNII_BANDS, 200
    Z, band, evaluate = _problem(g, freqs, bands)
    ev = built.Evaluator(g)
    ev.load_Z(freqs, torch.from_numpy(Z).cuda())
    ev.set_fom(band)
    init = PI.seed_map(g, 0.5, 5)
    m_ref, f_ref, e_ref, t_ref = OS.tree_search(evaluate, init, seed=42, d_max=2, m_of_d=(10, 3), max_evals=budget,
                                                n_states=g.n_states)
    m_gpu, f_gpu, e_gpu, t_gpu = ev.search(init, seed=42, d_max=2, m_of_d=(10, 3), max_evals=budget, precision=prec)
    ev.close()
    tol = 1e-6 if prec == "mixed" else 1e-10
    assert e_gpu == e_ref
    assert len(t_gpu) == len(t_ref)
    assert np.allclose(t_gpu, t_ref, rtol=tol, atol=0)      # identical decisions, same FoM path
    assert np.array_equal(m_gpu, m_ref)
    assert f_gpu == pytest.approx(f_ref, rel=tol)


def test_native_search_resume_matches_uninterrupted_and_oracle(built):
    """Checkpoint / resume on the GPU evaluator: a search stopped after 120 evaluations and resumed
    to 300 makes the decisions of the uninterrupted native run and of the oracle's search."""
    g, freqs, bands = PI.grid_tiny(3), np.array([2.0e9, 2.5e9, 3.5e9, 5.0e9]), PI.PLAIN_BANDS
    Z, band, evaluate = _problem(g, freqs, bands)
    ev = built.Evaluator(g)
    ev.load_Z(freqs, torch.from_numpy(Z).cuda())
    ev.set_fom(band)
    init = PI.seed_map(g, 0.5, 5)
    args = dict(seed=42, d_max=2, m_of_d=(10, 3))
    full = ev.search(init, max_evals=300, precision="fp64", **args)
    a = ev.search_resume(init, max_evals=120, precision="fp64", **args)
    b = ev.search_resume(init, max_evals=300, precision="fp64", state=a[4], **args)
    ev.close()
    assert b[2] == full[2] and np.array_equal(b[0], full[0]) and b[1] == pytest.approx(full[1], rel=1e-10)
    assert np.allclose(np.concatenate([a[3], b[3]]), full[3], rtol=1e-10, atol=0)
    ref = OS.tree_search(evaluate, init, max_evals=300, **args)
    assert ref[2] == b[2] and np.array_equal(ref[0], b[0])
