"""GPU checks of the via state (three pixel states): the support set of every map of a small
two-layer grid bit-exact against the oracle (including the rejected via on the last layer), and
the GPU fill of a grid with via strips (vertical triangles, Neumann kernel for vertical currents)
against the oracle's fill entry by entry."""
import dataclasses
import itertools

import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import pmom
    return pmom


def via_grid(n, pitch=0.5e-3):
    g = PI.grid_tiny(n, PI.MEDIUM_STRIPLINE, 2, pitch_m=pitch)
    return dataclasses.replace(g, name=f"via_{n}x{n}x2", n_states=3)


def test_via_active_set_bit_exact(pm):
    g = via_grid(2)
    OG = O.Grid(g)
    maps = [np.array([lo, hi], np.uint8).reshape(2, 2, 2)
            for lo in itertools.product(range(3), repeat=4) for hi in itertools.product(range(2), repeat=4)]
    bad = np.zeros((2, 2, 2), np.uint8)
    bad[1, 0, 1] = 2                      # a via on the last layer
    allm = np.ascontiguousarray(np.stack(maps + [bad]))
    ev = pm.Evaluator(g)
    idx, n = ev.active_set(torch.from_numpy(allm).cuda())
    idx, n = idx.cpu().numpy(), n.cpu().numpy()
    for b in range(len(maps)):
        ref = O.active_set(OG, allm[b])
        assert n[b] == len(ref)
        assert np.array_equal(idx[b, : n[b]], ref)
    assert n[-1] == -1
    ev.close()


def test_gpu_fill_with_vias_matches_oracle_fill(pm):
    g = via_grid(4)
    freqs = [1.3e9, 6.1e9]
    OG = O.Grid(g)
    Zr, _ = O.fill(OG, freqs)
    ev = pm.Evaluator(g)
    ev.fill_Z(freqs, "c128")
    Zg = ev.copy_Z().cpu().numpy()
    for f in range(len(freqs)):
        assert np.abs(Zg[f] - Zr[f]).max() <= 1e-9 * np.abs(Zr[f]).max()
    ev.close()


def test_via_grid_eval_and_bordered_update_match_oracle(pm):
    """A 6 x 6 two-layer stripline with vias, complex128 database: every single-pixel change of a
    reference map that holds vias (to each other valid state), evaluated by the full solve in both
    precisions and by the bordered update (FP64 route), against the oracle's direct solve."""
    g = dataclasses.replace(PI.grid_tiny(6, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5625e-3), name="via_6x6x2", n_states=3)
    OG = O.Grid(g)
    freqs = np.array([5.5e9, 6.5e9, 7.5e9])
    Z, _ = O.fill(OG, freqs)
    band = O.bands(freqs, PI.UNII_BANDS)
    ref = PI.seed_map_vias(g, 0.6, 0.3, 3)
    assert (ref == 2).any()
    kids = []
    for l in range(2):
        for y in range(6):
            for x in range(6):
                for s in range(3 if l == 0 else 2):
                    if s != ref[l, y, x]:
                        c = ref.copy()
                        c[l, y, x] = s
                        kids.append(c)
    kids = np.ascontiguousarray(np.stack(kids))
    S_ref, st = O.eval_batch(OG, Z, kids)
    assert (st == 0).all()
    fom_ref = O.fom_batch(S_ref, band)
    ev = pm.Evaluator(g)
    ev.load_Z(freqs, torch.from_numpy(Z).cuda())
    ev.set_fom(band)
    dk = torch.from_numpy(kids).cuda()
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        S, fom, status = ev.eval(dk, prec)
        torch.cuda.synchronize()
        assert np.isin(status.cpu().numpy(), [0, 3]).all()
        assert np.abs(S.cpu().numpy() - S_ref).max() <= tol * max(1.0, np.abs(S_ref).max())
        assert (np.abs(fom.cpu().numpy() - fom_ref) / np.abs(fom_ref)).max() <= tol
    Sb, fb, sb = ev.eval_bordered(torch.from_numpy(ref).cuda(), dk, "fp64")
    torch.cuda.synchronize()
    codes = sb.cpu().numpy()
    near = codes == 0
    # changes of more than 8 BFs report FAR (7); every other candidate is solved
    nchg = np.array([len(set(O.active_set(OG, ref).tolist()) ^ set(O.active_set(OG, c).tolist())) for c in kids])
    assert np.array_equal(codes == 7, nchg > 8) and np.isin(codes, [0, 7]).all()
    assert np.abs(Sb.cpu().numpy()[near] - S_ref[near]).max() <= 1e-8 * max(1.0, np.abs(S_ref).max())
    assert (np.abs(fb.cpu().numpy()[near] - fom_ref[near]) / np.abs(fom_ref[near])).max() <= 1e-8
    ev.close()
