"""GPU parity for pixels of 8 and 18 triangles (s x s sub-squares, Section V-A) with multi-edge
port gaps: the GPU fill against the oracle's, and both precisions of the evaluation against the
oracle's solve; the bordered update, whose port rows assume one gap BF, refuses these grids."""
import dataclasses

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


@pytest.mark.parametrize("s,pattern", [(2, 0), (3, 2)])
def test_submesh_fill_and_eval(pm, s, pattern):
    g = dataclasses.replace(PI.grid_tiny(3, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5625e-3), name=f"sub{s}", sub=s,
                            diag_pattern=pattern, diag_seed=7)
    freqs = [5.5e9, 7.0e9]
    OG = O.Grid(g)
    Zr, _ = O.fill(OG, freqs)
    ev = pm.Evaluator(g)
    assert ev.M == OG.M
    ev.fill_Z(freqs, "c128")
    Zg = ev.copy_Z().cpu().numpy()
    for f in range(len(freqs)):
        assert np.abs(Zg[f] - Zr[f]).max() <= 1e-9 * np.abs(Zr[f]).max()
    maps = PI.random_maps(g, 8, 0.6, 3)
    S_ref, st = O.eval_batch(OG, Zr, maps)
    assert (st == 0).all()
    ev.set_fom(pm.band_codes(freqs, PI.UNII_BANDS))
    dm = torch.from_numpy(maps).cuda()
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        S, fom, status = ev.eval(dm, prec)
        torch.cuda.synchronize()
        assert np.isin(status.cpu().numpy(), [0, 3]).all()
        assert np.abs(S.cpu().numpy() - S_ref).max() <= tol * max(1.0, np.abs(S_ref).max())
    with pytest.raises(pm.PmomError) as e:
        ev.eval_bordered(dm[0:1].clone(), dm)
    assert e.value.status == 7
    ev.close()
