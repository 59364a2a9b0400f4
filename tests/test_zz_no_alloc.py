"""The allocation-free entry point (pmom_eval_candidates_noalloc) gives the same results as
pmom_eval_candidates.

Callers that may not allocate device memory during a call (graph capture, memory pools owned by
another framework, real-time loops) use this entry point; its temporaries live in a fixed device
array owned by the library.  This file is collected last so that a run stopping at the first
failure has run every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import pmom
    w = PI.workload_plain()
    OG = O.Grid(w.grid)
    Z, _ = O.fill(OG, w.freqs())
    ev = pmom.Evaluator(w.grid)
    ev.load_Z(w.freqs(), torch.from_numpy(Z).cuda())
    ev.set_fom(pmom.band_codes(w.freqs(), w.bands))
    maps = torch.from_numpy(PI.workload_maps(w, seed=3)).cuda()
    yield pmom, w, ev, maps
    ev.close()


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-6), ("fp64", 1e-10)])
def test_noalloc_matches_allocating_entry_point(setup, prec, tol):
    pmom, w, ev, maps = setup
    S_ref, fom_ref, st_ref = ev.eval(maps, prec)
    torch.cuda.synchronize()
    S_ref, fom_ref, st_ref = S_ref.cpu().numpy(), fom_ref.cpu().numpy(), st_ref.cpu().numpy()
    for _ in range(2):   # two calls in a row: the shared array keeps the previous contents
        S, fom, st = ev.eval_noalloc(maps, prec)
        torch.cuda.synchronize()
        S, fom, st = S.cpu().numpy(), fom.cpu().numpy(), st.cpu().numpy()
        assert np.array_equal(st, st_ref)
        assert np.abs(S - S_ref).max() <= tol
        assert (np.abs(fom - fom_ref) <= tol * np.abs(fom_ref)).all()


def test_noalloc_without_S_output_and_oversize_rejection(setup):
    pmom, w, ev, maps = setup
    fom = torch.empty((maps.shape[0],), dtype=torch.float64, device="cuda")
    st = torch.empty((maps.shape[0],), dtype=torch.int32, device="cuda")
    _, fom_ref, _ = ev.eval(maps, "mixed")
    ev.eval_noalloc(maps, "mixed", out=(None, fom, st))
    torch.cuda.synchronize()
    assert torch.allclose(fom, fom_ref, rtol=1e-6, atol=0)
    # a grid whose single-task FP64 workspace exceeds the fixed array is refused, not run
    big = pmom.Evaluator(PI.grid_stripline_16x16x2())
    big.fill_Z([3e9], "c64")
    big.set_fom(np.array([3], np.uint8))
    m = torch.zeros((2, 2, 16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(pmom.PmomError) as e:
        big.eval_noalloc(m, "mixed")
    assert e.value.status == 1 and "scratch" in str(e.value)
    big.close()
