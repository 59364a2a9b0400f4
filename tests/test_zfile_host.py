"""Database files on the host (no GPU): an independent writer of the documented layout, and the
loader's checks that run before any device work (not a database file, another grid, a truncated
file)."""
import struct

import numpy as np
import pytest

import pmom_inputs as PI
from paper_2412_17617_gb300 import build as B
from paper_2412_17617_gb300 import pmom

MASK = (1 << 64) - 1


def fnv1a_bytes(b: bytes, h: int = 0xCBF29CE484222325) -> int:
    for x in b:
        h = ((h ^ x) * 0x100000001B3) & MASK
    return h


def fnv1a_words(b: bytes, h: int = 0xCBF29CE484222325) -> int:
    for (w,) in struct.iter_unpack("<Q", b):
        h = ((h ^ w) * 0x100000001B3) & MASK
    return h


def write_db(path, table: np.ndarray, freqs, Z: np.ndarray, magic=b"PMOMZDB1", M=None, thash=None, cut=0):
    """The documented layout, written independently of the library."""
    dtype = 1 if Z.dtype == np.complex128 else 0
    M = Z.shape[1] if M is None else M
    th = fnv1a_bytes(np.ascontiguousarray(table, dtype=np.int32).tobytes()) if thash is None else thash
    data = np.ascontiguousarray(Z).tobytes()
    blob = (magic + struct.pack("<IIiiQ", 1, dtype, M, len(freqs), th) +
            np.asarray(freqs, np.float64).tobytes() + data + struct.pack("<Q", fnv1a_words(data)))
    with open(path, "wb") as fh:
        fh.write(blob[: len(blob) - cut])


@pytest.fixture(scope="module")
def ev():
    B.build()
    e = pmom.Evaluator(PI.grid_tiny(3))
    yield e
    e.close()


def test_loader_rejects_bad_files_before_device_work(ev, tmp_path):
    freqs = [1e9, 2e9]
    Z = (np.arange(2 * ev.M * ev.M) * (1 + 2j)).astype(np.complex64).reshape(2, ev.M, ev.M)
    table = ev.bf_table()
    cases = {"magic": (dict(magic=b"NOTADB!!"), 8), "grid_M": (dict(M=ev.M + 1), 4),
             "grid_table": (dict(thash=12345), 4), "truncated": (dict(cut=9), 8)}
    for name, (kw, status) in cases.items():
        p = tmp_path / f"{name}.zdb"
        write_db(p, table, freqs, Z, **kw)
        with pytest.raises(pmom.PmomError) as e:
            ev.load_Z_file(str(p))
        assert e.value.status == status, (name, e.value)
    with pytest.raises(pmom.PmomError) as e:
        ev.load_Z_file(str(tmp_path / "missing.zdb"))
    assert e.value.status == 8
    with pytest.raises(pmom.PmomError) as e:
        ev.save_Z(str(tmp_path / "nothing.zdb"))
    assert e.value.status == 6                 # no database yet


def test_table_hash_follows_the_grid():
    """Two grids that differ only in the diagonal orientation have different BF tables, hence
    different hashes: a database cannot be loaded into the wrong mesh."""
    import dataclasses
    B.build()
    g = PI.grid_tiny(3)
    a = pmom.Evaluator(g)
    b = pmom.Evaluator(dataclasses.replace(g, diag_pattern=1))
    ta, tb = a.bf_table(), b.bf_table()
    assert ta.shape == tb.shape and not np.array_equal(ta, tb)
    assert fnv1a_bytes(ta.astype(np.int32).tobytes()) != fnv1a_bytes(tb.astype(np.int32).tobytes())
    a.close()
    b.close()
