"""The allocation-free entry point (pmom_eval_candidates_noalloc) gives the same results as
pmom_eval_candidates, bit for bit, and both agree with the oracle.

Some callers cannot let a library call cudaMalloc or cudaFree while they run: a host that hands
all device memory to another framework's caching pool at start-up, or a real-time loop that cannot
take the allocator's latency and the device synchronization of cudaFree.  They use this entry
point, whose temporaries live in a fixed device array owned by the library.  It launches the same
kernels on the same inputs as the allocating entry point (only the workspaces' addresses and
leading dimension differ), so S, FoM and status must be identical, on two calls in a row (the
array keeps the previous call's contents).  This file is collected last so that a run stopping at
the first failure has run every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# tolerances against the oracle (the mixed path's |dS| <= 1e-6, the FP64 path's 1e-10 max(1, |S|))
TOL = {"mixed": 1e-6, "fp64": 1e-10}


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
    maps_np = PI.workload_maps(w, seed=3)
    # the oracle on a sample of the batch: every eighth candidate
    sample = np.arange(0, maps_np.shape[0], 8)
    S_or, st_or = O.eval_batch(OG, Z, maps_np[sample])
    assert (st_or == 0).all()
    fom_or = O.fom_batch(S_or, O.bands(w.freqs(), w.bands))
    yield pmom, w, ev, torch.from_numpy(maps_np).cuda(), (sample, S_or, fom_or)
    ev.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_matches_allocating_entry_point(setup, prec):
    pmom, w, ev, maps, (sample, S_or, fom_or) = setup
    S_ref, fom_ref, st_ref = ev.eval(maps, prec)
    torch.cuda.synchronize()
    S_ref, fom_ref, st_ref = S_ref.cpu().numpy(), fom_ref.cpu().numpy(), st_ref.cpu().numpy()
    assert (st_ref == 0).all()
    tol = TOL[prec]
    assert np.abs(S_ref[sample] - S_or).max() <= tol * max(1.0, np.abs(S_or).max())
    assert (np.abs(fom_ref[sample] - fom_or) <= tol * np.abs(fom_or)).all()
    for _ in range(2):   # two calls in a row: the shared array keeps the previous contents
        S, fom, st = ev.eval_noalloc(maps, prec)
        torch.cuda.synchronize()
        S, fom, st = S.cpu().numpy(), fom.cpu().numpy(), st.cpu().numpy()
        assert np.array_equal(st, st_ref)
        assert np.array_equal(S.view(np.float64), S_ref.view(np.float64))
        assert np.array_equal(fom.view(np.uint64), fom_ref.view(np.uint64))


def test_noalloc_without_S_output_and_oversize_rejection(setup):
    pmom, w, ev, maps, _ = setup
    fom = torch.empty((maps.shape[0],), dtype=torch.float64, device="cuda")
    st = torch.empty((maps.shape[0],), dtype=torch.int32, device="cuda")
    _, fom_ref, _ = ev.eval(maps, "mixed")
    ev.eval_noalloc(maps, "mixed", out=(None, fom, st))
    torch.cuda.synchronize()
    assert torch.equal(fom, fom_ref)
    # a grid whose single-task FP64 workspace exceeds the fixed array is refused, not run
    big = pmom.Evaluator(PI.grid_stripline_16x16x2())
    big.fill_Z([3e9], "c64")
    big.set_fom(np.array([3], np.uint8))
    m = torch.zeros((2, 2, 16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(pmom.PmomError) as e:
        big.eval_noalloc(m, "mixed")
    assert e.value.status == 1 and "scratch" in str(e.value)
    big.close()
