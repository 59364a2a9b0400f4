"""The multi-GPU path's host logic on CPU ranks (gloo, world size 2): every rank evaluates its own
batch (distinct maps, same shape, each a set of single flips of that rank's seed), the step time is
the slowest rank's (all-reduce MAX), and the job rate counts every rank's batch.  No GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import pmom_inputs as PI
    w = PI.workload_plain()
    maps = bench.rank_batch(w, rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    rate = bench.aggregate_rate(world, maps.shape[0], ms)
    np.save(os.path.join(out_dir, f"maps{rank}.npy"), maps)
    np.save(os.path.join(out_dir, f"res{rank}.npy"), np.array([ms, rate]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks(tmp_path):
    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    m0, m1 = np.load(tmp_path / "maps0.npy"), np.load(tmp_path / "maps1.npy")
    assert m0.shape == m1.shape and not np.array_equal(m0, m1)
    import pmom_inputs as PI
    w = PI.workload_plain()
    for r, m in enumerate((m0, m1)):
        seed = PI.seed_map(w.grid, w.fill, r)
        diff = (m != seed[None]).reshape(m.shape[0], -1).sum(axis=1)
        assert (diff == 1).all()
    r0, r1 = np.load(tmp_path / "res0.npy"), np.load(tmp_path / "res1.npy")
    assert r0[0] == r1[0] == 15.0
    assert r0[1] == r1[1] == 2 * m0.shape[0] / 15.0e-3
