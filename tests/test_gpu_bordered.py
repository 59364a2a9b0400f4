"""GPU parity of the bordered low-rank evaluation (single-pixel changes of a reference map):
against the oracle's direct solve of every candidate, and against the library's own full FP64
path on the same batch.

Two precisions: "fp64" (reference LU, inverse and products in FP64) is held to the FP64 path's
1e-10 per S entry (relative to max(1, |S|)) and per FoM (its results follow from the reference
inverse by exact block-inverse identities);
"mixed" (tensor-core reference LU, inverse refined with float-float residuals, float-float
products) to the mixed path's 1e-6.  Decisions must equal the oracle's in both.
"""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-10), "mixed": (1e-6, 1e-6)}


@pytest.fixture(scope="module")
def pm():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import pmom
    return pmom


def _check(S, fom, S_ref, fom_ref, prec):
    ts, tf = TOL[prec]
    err = np.abs(S - S_ref)
    assert err.max() <= ts * max(1.0, np.abs(S_ref).max()), float(err.max())
    rel = np.abs(fom - fom_ref) / np.abs(fom_ref)
    assert rel.max() <= tf, float(rel.max())


def test_plain_all_flips(pm):
    """8x8 microstrip, complex128 database (which always takes the FP64 route), all 64 single
    flips of the seed (removals and additions of up to five BFs)."""
    w = PI.workload_plain()
    OG = O.Grid(w.grid)
    Z, _ = O.fill(OG, w.freqs())
    seed = PI.seed_map(w.grid, w.fill, 0)
    maps = PI.workload_maps(w, seed=0)
    S_ref, st = O.eval_batch(OG, Z, maps)
    assert (st == 0).all()
    fom_ref = O.fom_batch(S_ref, O.bands(w.freqs(), w.bands))
    ev = pm.Evaluator(w.grid)
    ev.load_Z(w.freqs(), torch.from_numpy(Z).cuda())
    ev.set_fom(pm.band_codes(w.freqs(), w.bands))
    S, fom, status = ev.eval_bordered(torch.from_numpy(seed).cuda(), torch.from_numpy(maps).cuda())
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    _check(S.cpu().numpy(), fom.cpu().numpy(), S_ref, fom_ref, "fp64")
    assert int(np.argmin(fom.cpu().numpy())) == int(np.argmin(fom_ref))
    # the reference itself (no change) and a two-pixel change come out right too
    two = seed.copy()
    two[0, 0, 0] ^= 1
    two[0, 5, 6] ^= 1
    extra = np.ascontiguousarray(np.stack([seed, two]))
    S2, f2, s2 = ev.eval_bordered(torch.from_numpy(seed).cuda(), torch.from_numpy(extra).cuda())
    S2_ref, _ = O.eval_batch(OG, Z, extra)
    assert (s2.cpu().numpy() == 0).all()
    _check(S2.cpu().numpy(), f2.cpu().numpy(), S2_ref, O.fom_batch(S2_ref, O.bands(w.freqs(), w.bands)), "fp64")
    ev.close()


@pytest.fixture(scope="module")
def precision_case(pm):
    w = PI.workload_precision()
    OG = O.Grid(w.grid)
    Z, _ = O.fill(OG, w.freqs())
    Z64 = Z.astype(np.complex64)
    del Z
    seed = PI.seed_map(w.grid, w.fill, 0)
    maps = PI.workload_maps(w, seed=0)
    ev = pm.Evaluator(w.grid)
    ev.load_Z(w.freqs(), torch.from_numpy(Z64).cuda())
    ev.set_fom(pm.band_codes(w.freqs(), w.bands))
    sample = np.array([0, 3, 97, 142, 200, 255, 256, 300, 411, 480, 511])
    S_ref, st = O.eval_batch(OG, Z64, maps[sample])
    assert (st == 0).all()
    fom_ref = O.fom_batch(S_ref, O.bands(w.freqs(), w.bands))
    # the library's full FP64 path on the whole batch (checked against the oracle in
    # test_gpu_parity) as the reference for every candidate
    S64, f64, s64 = ev.eval(torch.from_numpy(maps).cuda(), "fp64")
    torch.cuda.synchronize()
    assert (s64.cpu().numpy() == 0).all()
    ref64 = (S64.cpu().numpy(), f64.cpu().numpy())
    yield w, seed, maps, ev, sample, S_ref, fom_ref, ref64
    ev.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_precision_workload_full_batch(precision_case, prec):
    """16x16x2 stripline, complex64 database, 41 frequencies, all 512 single-bit flips in one call
    (the benchmark's configuration); sampled candidates against the oracle (candidate 142 is a
    failed design with |S21| ~ 3e-5, whose FoM amplifies relative |S| errors), every candidate
    against the library's full FP64 path."""
    w, seed, maps, ev, sample, S_ref, fom_ref, ref64 = precision_case
    dm = torch.from_numpy(maps).cuda()
    S, fom, status = ev.eval_bordered(torch.from_numpy(seed).cuda(), dm, prec)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    Sn, fn = S.cpu().numpy(), fom.cpu().numpy()
    _check(Sn[sample], fn[sample], S_ref, fom_ref, prec)
    assert int(np.argmin(fn[sample])) == int(np.argmin(fom_ref))
    _check(Sn, fn, ref64[0], ref64[1], prec)
    assert int(np.argmin(fn)) == int(np.argmin(ref64[1]))


def test_far_and_bad_state(precision_case):
    """Candidates that change too many BFs report FAR; a bad pixel state reports BAD_STATE; both
    leave the other candidates of the batch untouched.  A bad reference is a call error."""
    w, seed, maps, ev, sample, S_ref, fom_ref, ref64 = precision_case
    far = PI.random_maps(w.grid, 1, 0.5, 3)
    bad = maps[:1].copy()
    bad[0, 1, 2, 3] = 7
    batch = np.ascontiguousarray(np.concatenate([maps[:2], far, bad, maps[2:3]]))
    S, fom, status = ev.eval_bordered(torch.from_numpy(seed).cuda(), torch.from_numpy(batch).cuda())
    torch.cuda.synchronize()
    codes = status.cpu().numpy()
    assert codes.tolist() == [0, 0, 7, 5, 0], codes
    keep = [0, 1, 4]
    Sn = S.cpu().numpy()
    # same numbers as the clean batch
    S0, f0, _ = ev.eval_bordered(torch.from_numpy(seed).cuda(), torch.from_numpy(np.ascontiguousarray(maps[:3])).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(Sn[keep], S0.cpu().numpy())
    badref = seed.copy()
    badref[0, 0, 0] = 9
    with pytest.raises(Exception):
        ev.eval_bordered(torch.from_numpy(badref).cuda(), torch.from_numpy(batch).cuda())
