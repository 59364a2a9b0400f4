"""The benchmark's reference arm on the host (no GPU): the CPU-oracle baseline on a bounded sample,
and the JSON line the reference arm prints (the keys and units the measurement contract asks for)."""
import io
import json
import sys
import types
from contextlib import redirect_stdout

import numpy as np

import bench


def test_cpu_baseline_sample():
    w = bench.workload("plain")
    info, (smp, nb, S) = bench.cpu_baseline(w, seconds_target=0.5)
    assert info["kind"] == "oracle" and info["unit"] == "candidate evals/s"
    assert info["value"] > 0 and info["cores"] >= 1 and "frequencies" in info["sample"]
    assert S.shape == (nb, 4, 3, 3) and nb >= 1


def test_reference_line(monkeypatch):
    """The reference arm times what it runs: ms_per_step is the measured time of one step's sample,
    so steps x ms_per_step fits the run, and its config is the GPU arm's (same function, same N)."""
    args = types.SimpleNamespace(workload="plain", steps=2, warmup=1, gpus=1, batch=8)
    out = io.StringIO()
    import time
    t0 = time.perf_counter()
    with redirect_stdout(out):
        bench.run_reference(args)
    wall = time.perf_counter() - t0
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["steps"] * line["ms_per_step"] <= 1000.0 * wall
    assert line["e2e"] == {"value": line["value"], "unit": "candidate evals/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    w = bench.workload("plain")
    from oracle import oracle as O
    OG = O.Grid(w.grid)
    maps = bench.rank_batch(w, 0, 8)
    N = np.array([len(O.active_set(OG, m)) for m in maps])
    assert line["config"] == json.loads(json.dumps(bench.workload_config(w, N, OG.M, 8, 1)))
    assert line["config"]["workload"] == "plain_8x8_f11_b64" and line["config"]["global_batch"] == 8
