"""Database files on the GPU: save and load are bit-exact, the library writes exactly the
documented layout (byte-identical to an independent writer), an oracle database written by that
writer loads and evaluates like the oracle, and a corrupted file is rejected."""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O
from test_zfile_host import write_db

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import pmom
    return pmom


def test_database_file_round_trip(pm, tmp_path):
    g = PI.grid_tiny(4, PI.MEDIUM_STRIPLINE, 2, pitch_m=0.5625e-3)
    freqs = [5.5e9, 7.0e9]
    ev = pm.Evaluator(g)
    ev.fill_Z(freqs, "c64")
    Z0 = ev.copy_Z().cpu().numpy()
    p = tmp_path / "db.zdb"
    ev.save_Z(str(p))
    q = tmp_path / "ref.zdb"
    write_db(q, ev.bf_table(), freqs, Z0)
    assert p.read_bytes() == q.read_bytes()
    ev2 = pm.Evaluator(g)
    ev2.load_Z_file(str(p))
    Z1 = ev2.copy_Z().cpu().numpy()
    assert Z1.dtype == np.complex64 and np.array_equal(Z0.view(np.uint64), Z1.view(np.uint64))
    # an oracle database written independently: loads bit-exactly, evaluates like the oracle
    OG = O.Grid(g)
    Zr, _ = O.fill(OG, freqs)
    write_db(q, ev.bf_table(), freqs, Zr)
    ev2.load_Z_file(str(q))
    assert np.array_equal(ev2.copy_Z().cpu().numpy().view(np.uint64), Zr.view(np.uint64))
    ev2.set_fom(pm.band_codes(freqs, PI.UNII_BANDS))
    maps = PI.random_maps(g, 6, 0.6, 4)
    S_ref, _ = O.eval_batch(OG, Zr, maps)
    S, fom, status = ev2.eval(torch.from_numpy(maps).cuda(), "fp64")
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    assert np.abs(S.cpu().numpy() - S_ref).max() <= 1e-10 * max(1.0, np.abs(S_ref).max())
    # one flipped byte of the data: checksum mismatch, the database is dropped
    b = bytearray(q.read_bytes())
    b[len(b) // 2] ^= 0x40
    q.write_bytes(bytes(b))
    with pytest.raises(pm.PmomError) as e:
        ev2.load_Z_file(str(q))
    assert e.value.status == 8
    with pytest.raises(pm.PmomError):
        ev2.save_Z(str(tmp_path / "after.zdb"))
    ev.close()
    ev2.close()
