"""CUDA-graph replay, the support-set capacity guard and the autotuner, through the C ABI."""
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
    yield pmom, w, OG, Z, ev
    ev.close()


def test_graph_replay_matches_direct_and_follows_map_contents(setup):
    pmom, w, OG, Z, ev = setup
    a = torch.from_numpy(PI.workload_maps(w, seed=1)).cuda()
    b = torch.from_numpy(PI.workload_maps(w, seed=2)).cuda()
    maps = a.clone()
    S, fom, st = ev.graph_capture(maps, "mixed")
    for src in (a, b, a):
        maps.copy_(src)
        ev.graph_launch()
        torch.cuda.synchronize()
        Sd, fd, sd = ev.eval(src, "mixed")
        torch.cuda.synchronize()
        assert torch.equal(st, sd)
        assert (S - Sd).abs().max().item() <= 1e-12
        assert torch.allclose(fom, fd, rtol=1e-12, atol=0)
    # and against the oracle for the last contents
    S_ref, _ = O.eval_batch(OG, Z, a.cpu().numpy())
    assert np.abs(S.cpu().numpy() - S_ref).max() <= 1e-6


def test_capacity_guard(setup):
    pmom, w, OG, Z, ev = setup
    maps = torch.from_numpy(PI.workload_maps(w, seed=1)).cuda()
    n = ev.active_set(maps)[1].cpu().numpy()
    cap = int(np.median(n))
    S, fom, st = ev.graph_capture(maps, "mixed", ncap=cap)
    ev.graph_launch()
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    over = n > cap
    assert over.any() and (~over).any()
    assert (st[over] == pmom.CAND_CAPACITY).all()
    assert np.isnan(fom.cpu().numpy()[over]).all()
    Sd, fd, sd = ev.eval(maps, "mixed")
    torch.cuda.synchronize()
    assert (st[~over] == 0).all()
    assert np.allclose(fom.cpu().numpy()[~over], fd.cpu().numpy()[~over], rtol=1e-12, atol=0)


def test_autotune_keeps_results(setup):
    pmom, w, OG, Z, ev = setup
    maps = torch.from_numpy(PI.workload_maps(w, seed=4)).cuda()
    choice = ev.autotune(maps, "mixed")
    assert choice in (0, 1)
    S, fom, st = ev.eval(maps, "mixed")
    torch.cuda.synchronize()
    S_ref, _ = O.eval_batch(OG, Z, maps.cpu().numpy())
    assert (st.cpu().numpy() == 0).all()
    assert np.abs(S.cpu().numpy() - S_ref).max() <= 1e-6
    for tc in (0, 1):   # both variants meet the tolerance
        ev.set_tensor_cores(bool(tc))
        S, fom, st = ev.eval(maps, "mixed")
        torch.cuda.synchronize()
        assert np.abs(S.cpu().numpy() - S_ref).max() <= 1e-6
    ev.set_tensor_cores(bool(choice))
