"""Failure detection on the GPU without a fault: the bounded completion wait that the tensor-core
paths use gives up on an mbarrier that nothing arrives at and reports it (instead of hanging), sees
the phase complete when the arrival happens, and the device evaluates normally afterwards."""
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


def test_bounded_wait_reports_a_missing_arrival(pm):
    timed_out, ms = pm.selftest_wait(4096, arrive=False)
    assert timed_out is True and 0.0 <= ms < 5000.0
    timed_out, ms = pm.selftest_wait(4096, arrive=True)
    assert timed_out is False
    # the context is usable after the timeout: a small evaluation matches the oracle
    g = PI.grid_tiny(3)
    freqs = np.array([2.4e9, 5.2e9])
    OG = O.Grid(g)
    Z, _ = O.fill(OG, freqs)
    maps = PI.all_maps(g)[::64]
    S_ref, _ = O.eval_batch(OG, Z, maps)
    ev = pm.Evaluator(g)
    ev.load_Z(freqs, torch.from_numpy(Z).cuda())
    ev.set_fom(pm.band_codes(freqs, PI.PLAIN_BANDS))
    S, fom, status = ev.eval(torch.from_numpy(maps).cuda(), "mixed")
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    assert np.abs(S.cpu().numpy() - S_ref).max() <= 1e-6
    assert ev.stats()["tc_wait_timeouts"] == 0
    ev.close()
    with pytest.raises(pm.PmomError):
        pm.selftest_wait(0, arrive=False)
