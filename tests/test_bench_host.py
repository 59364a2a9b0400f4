"""The benchmark's reference arm on the host (no GPU): the CPU-oracle baseline on a bounded sample,
and the JSON line the reference arm prints (the keys and units the measurement contract asks for)."""
import io
import json
import sys
import types
from contextlib import redirect_stdout

import bench


def test_cpu_baseline_sample():
    w = bench.workload("plain")
    info = bench.cpu_baseline(w, seconds_target=0.5)
    assert info["kind"] == "oracle" and info["unit"] == "candidate evals/s"
    assert info["value"] > 0 and info["cores"] >= 1 and "frequencies" in info["sample"]


def test_reference_line(monkeypatch):
    fake = {"value": 2.0, "unit": "candidate evals/s", "cores": 3, "kind": "oracle", "sample": "s", "seconds": 0.1}
    monkeypatch.setattr(bench, "cpu_baseline", lambda w, seconds_target=15.0: dict(fake))
    args = types.SimpleNamespace(workload="precision", steps=2, warmup=1, gpus=1)
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(args)
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] == 2.0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["cores"] == 3 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": 2.0, "unit": "candidate evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "stripline_16x16x2_f41_b512"
