"""Benchmark of the candidate evaluator: candidate evaluations per second (all frequencies of a
candidate = one evaluation) of the mixed-precision refined path, with the plain FP64 GPU path and
the CPU oracle timed in the same run.

Default workload: 2-layer 16x16 stripline (M = 1484 BFs), 41 frequencies 1-7 GHz, complex64
parent database filled on the GPU, all 512 single-bit flips of a seeded map (about 700 active BFs
each).  One step = one evaluation of the whole batch through the C ABI (activation, gather,
LU + solves + refinement, S-parameters, FoM).  The database (0.72 GB) is larger than L2, so no
L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload precision|plain|profile|batching|scale] [--batch B] [--no-cpu] [--no-bordered]

The batching (3-layer 20x20 stripline with vias, 101 frequencies, support sets of about 800 to 2500)
and scale (4-layer 32x32 stripline, 117 GB database, support sets of about 4100) workloads are
opt-in legs; bound them with --batch.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pmom_inputs as PI  # noqa: E402

METRIC = "candidate evals/sec (all freqs) vs plain FP64 GPU path at |dS|<=1e-6"
FP32_LANES_PER_SM = 128          # Blackwell SM: 4 partitions x 32 FP32 lanes
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


# DRAM bytes (read + write) per task of the tensor-core evaluation kernel, from one ncu capture
# of a graph-replayed launch on the first 64 candidates x 41 frequencies of the 16x16x2 stripline
# batch (2624 tasks, 110.26 GB read + 35.03 GB written; profiles/
# eval_kernel_stripline16x16x2_b64_full.md gives the command).  Every task of the 512-candidate
# batch has the same structure (support sets of 683-693 BFs, one workspace slot each), so a
# launch over B x F tasks moves this figure times B x F bytes.
TRAFFIC_PER_TASK = {("stripline_16x16x2_f41_b512", "tc"): (110.260378e9 + 35.028002e9) / 2624}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(name: str):
    return {"precision": PI.workload_precision, "plain": PI.workload_plain, "profile": PI.workload_profile,
            "batching": PI.workload_batching, "scale": PI.workload_scale}[name]()


def lu_flops(N: np.ndarray, F: int, P: int) -> float:
    """Algorithmic flops of one batch: complex LU (8/3 N^3) + P-RHS solve (8 N^2 P) per task."""
    N = N.astype(np.float64)
    return float(F * np.sum(8.0 / 3.0 * N ** 3 + 8.0 * N ** 2 * P))


class OracleSample:
    """The oracle (plain C, complex128) on a bounded sample of a workload: the first candidates of
    rank 0's batch at four of its frequencies, on the oracle's own fill of the database at those
    frequencies (rounded to complex64 and promoted exactly when the workload stores complex64, as
    the library's input is)."""

    def __init__(self, w, batch: int = 0):
        from oracle import oracle as O
        self.O, self.w = O, w
        self.fsel = np.linspace(0, w.n_freq - 1, 4).round().astype(int)
        self.freqs = w.freqs()[self.fsel]
        self.OG = O.Grid(w.grid)
        Z, _ = O.fill(self.OG, self.freqs)
        self.Z = Z.astype(np.complex64) if w.z_dtype == "c64" else Z
        self.maps = rank_batch(w, 0, batch)
        self.cores = os.cpu_count() or 1

    def run(self, nb: int):
        """Evaluates the first nb candidates at the sampled frequencies; returns (S, seconds)."""
        t0 = time.perf_counter()
        S, _ = self.O.eval_batch(self.OG, self.Z, self.maps[:nb], threads=self.cores)
        return S, time.perf_counter() - t0

    def rate(self, nb: int, seconds: float) -> float:
        """Candidate evaluations (all frequencies of a candidate = one) per second."""
        return nb * len(self.fsel) / self.w.n_freq / seconds

    def describe(self, nb: int) -> str:
        return (f"{nb} candidates x {len(self.fsel)} of {self.w.n_freq} frequencies (scaled), complex128 LU, "
                f"{self.cores} host threads")

    def calibrate(self, seconds_target: float) -> int:
        """The sample size whose evaluation takes about seconds_target."""
        nb = max(1, min(self.maps.shape[0], self.cores))
        _, dt = self.run(nb)
        if dt < seconds_target / 2:
            nb = min(self.maps.shape[0], max(nb, int(nb * seconds_target / max(dt, 1e-3))))
        return nb


def cpu_baseline(w, seconds_target: float = 15.0, sample: "OracleSample" = None):
    """The oracle on the host cores, on a bounded sample of the workload, scaled to candidate
    evaluations per second.  Also returns (sample, candidates, S) for the accuracy check of the GPU
    paths against the oracle."""
    smp = sample or OracleSample(w)
    nb = smp.calibrate(seconds_target / 2)
    S, dt = smp.run(nb)
    return {"value": smp.rate(nb, dt), "unit": "candidate evals/s", "cores": smp.cores, "kind": "oracle",
            "sample": smp.describe(nb), "seconds": dt}, (smp, nb, S)


def workload_config(w, N: np.ndarray, M: int, batch: int, world: int) -> dict:
    """The `config` object of the JSON line (the same in both arms)."""
    h = np.histogram(N, bins=6)
    return {"workload": w.name, "global_batch": batch * world, "freqs": w.n_freq, "M": int(M),
            "N_mean": float(N.mean()), "N_min": int(N.min()), "N_max": int(N.max()),
            "N_hist": [[int(e) for e in h[1]], [int(c) for c in h[0]]],
            "l2": "inputs larger than L2 (Z database %.2f GB)" % (
                w.n_freq * M * M * (8 if w.z_dtype == "c64" else 16) / 1e9),
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The reference arm: the oracle as it stands, on the host cores.  Each step evaluates one
    fixed bounded sample of the workload (sized during the first warm-up step so that the whole
    run stays within about two minutes); ms_per_step is the measured time of that sample."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    w = workload(args.workload)
    smp = OracleSample(w, args.batch)
    N = np.array([len(smp.O.active_set(smp.OG, m)) for m in smp.maps])
    per_step = min(15.0, max(0.5, 120.0 / max(1, args.steps + args.warmup)))
    nb = smp.calibrate(per_step) if args.warmup > 0 else max(1, min(smp.maps.shape[0], smp.cores))
    for _ in range(max(0, args.warmup - 1)):
        smp.run(nb)
    secs = [smp.run(nb)[1] for _ in range(max(1, args.steps))]
    ms = 1000.0 * float(np.mean(secs))
    v = smp.rate(nb, ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "candidate evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": workload_config(w, N, smp.OG.M, smp.maps.shape[0], world),
            "cpu_baseline": {"kind": "oracle", "cores": smp.cores, "sample": "per step: " + smp.describe(nb),
                             "value": v, "unit": "candidate evals/s"},
            "e2e": {"value": v, "unit": "candidate evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def rank_batch(w, rank: int, batch: int = 0) -> np.ndarray:
    """The candidates one rank evaluates: every single flip of that rank's own seeded map, so ranks
    share no data and need no collective on the data path (weak scaling)."""
    maps = PI.workload_maps(w, seed=rank)
    if batch > 0:
        maps = np.ascontiguousarray(maps[:batch])
    return maps


def max_over_ranks(ms: float, dist, device) -> float:
    """The job's time for a step: the slowest rank's (all-reduce MAX of one scalar)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, batch: int, ms: float) -> float:
    """Whole-job candidate evaluations per second: every rank's batch over the slowest rank's time."""
    return world * batch / (ms * 1e-3)


def accuracy_vs_oracle(smp: "OracleSample", nb: int, S_or: np.ndarray) -> dict:
    """Both GPU paths against the oracle on the oracle's bounded sample: S per entry and the FoM of
    the sampled frequencies (Eq. 8-9 over the four-frequency sweep, on both sides)."""
    import torch
    from paper_2412_17617_gb300 import Evaluator, band_codes
    w = smp.w
    ev = Evaluator(w.grid)
    ev.load_Z(smp.freqs, torch.from_numpy(np.ascontiguousarray(smp.Z)).cuda())
    ev.set_fom(band_codes(smp.freqs, w.bands), w.z0_ohm)
    fom_or = smp.O.fom_batch(S_or, smp.O.bands(smp.freqs, w.bands))
    out = {"candidates": nb, "frequencies": [int(f) for f in smp.fsel]}
    maps = torch.from_numpy(np.ascontiguousarray(smp.maps[:nb])).cuda()
    for prec in ("mixed", "fp64"):
        S, fom, st = ev.eval(maps, prec)
        torch.cuda.synchronize()
        S, fom, st = S.cpu().numpy(), fom.cpu().numpy(), st.cpu().numpy()
        out[prec] = {"max_abs_dS": float(np.abs(S - S_or).max()),
                     "max_rel_fom": float((np.abs(fom - fom_or) / np.abs(fom_or)).max()),
                     "status_ok": int((st == 0).sum())}
    ev.close()
    return out


def run_ours(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2412_17617_gb300 import Evaluator, band_codes, build as B
    B.build()
    w = workload(args.workload)
    ev = Evaluator(w.grid)
    freqs = w.freqs()
    ev.fill_Z(freqs, w.z_dtype)
    ev.set_fom(band_codes(freqs, w.bands), w.z0_ohm)
    # each rank evaluates its own batch (independent candidates): weak scaling, no collective
    maps_np = rank_batch(w, rank, args.batch)
    maps = torch.from_numpy(maps_np).cuda()
    Bsz = maps.shape[0]
    idx, n = ev.active_set(maps)
    N = n.cpu().numpy()
    S = torch.empty((Bsz, w.n_freq, ev.P, ev.P), dtype=torch.complex128, device="cuda")
    fom = torch.empty((Bsz,), dtype=torch.float64, device="cuda")
    status = torch.empty((Bsz,), dtype=torch.int32, device="cuda")
    out = (S, fom, status)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- mixed refined path (the headline): autotuned variant, whole pipeline replayed from one
    #      CUDA graph per step (activation, ordering, persistent evaluation, repair, Y->S, FoM)
    tc_choice = ev.autotune(maps, "mixed")
    ev.set_timing(True)
    ev.eval(maps, "mixed", out=out)
    kern_ms = [ev.kernel_times()["eval"]]     # dominant kernel, CUDA events on the launch stream
    ev.set_timing(False)
    ncap = int(N.max())
    ev.graph_capture(maps, "mixed", out=out, ncap=ncap)
    for _ in range(args.warmup):
        ev.graph_launch()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            ev.graph_launch()
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    clocks = clk.summary()
    st = ev.stats()
    status_np = status.cpu().numpy()
    value = aggregate_rate(world, Bsz, ms)
    # ---- plain FP64 path on a subset of the same batch (its cost is ~25-50x higher), replayed
    #      from a CUDA graph like the headline: one warm-up, then the median of three replays
    three_state = w.grid.n_states == 3
    huge = int(N.max()) > 3000          # FP64 LU of N ~ 4000 at 101 frequencies: ~20 s per candidate
    nfp = min(Bsz, 2 if huge else 8 if three_state else 128)
    reps = 1 if huge else 3
    sub = maps[:nfp]
    S_mixed, fom_mixed = S[:nfp].clone(), fom[:nfp].clone()
    sub_out = (S[:nfp], fom[:nfp], status[:nfp])
    ev.graph_capture(sub, "fp64", out=sub_out, ncap=int(N[:nfp].max()))
    ev.graph_launch()
    barrier()
    fp64_runs = []
    for _ in range(reps):
        e0.record(stream)
        ev.graph_launch()
        e1.record(stream)
        barrier()
        fp64_runs.append(e0.elapsed_time(e1))
    fp64_ms = float(np.median(fp64_runs))
    fp64_value = world * nfp / (fp64_ms * 1e-3)
    S_ref64, fom_ref64 = S[:nfp].clone(), fom[:nfp].clone()
    fp64_status_ok = int((status[:nfp] == 0).sum().item())

    def accuracy(Sx, fx):
        return {"max_abs_dS_vs_fp64": float((Sx - S_ref64).abs().max().item()),
                "max_rel_fom_vs_fp64": float(((fx - fom_ref64).abs() / fom_ref64.abs()).max().item()),
                "candidates": nfp}
    # ---- bordered update of the same batch (every candidate is one pixel change of the seed map):
    #      reference factors and inverse per frequency, k x k updates per candidate, recomputed
    #      every step
    bordered = None
    # the three-state batch changes several seeds, not one reference; at N ~ 4000 the reference
    # inverse leaves the shared-memory route
    if args.bordered and not three_state and not huge:
        seed_d = torch.from_numpy(PI.seed_map(w.grid, w.fill, rank)).cuda()
        Sb, fb, sb = torch.empty_like(S), torch.empty_like(fom), torch.empty_like(status)
        for _ in range(args.warmup):
            ev.eval_bordered(seed_d, maps, "mixed", out=(Sb, fb, sb))
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            ev.eval_bordered(seed_d, maps, "mixed", out=(Sb, fb, sb))
        e1.record(stream)
        barrier()
        b_ms = e0.elapsed_time(e1) / args.steps
        ev.set_timing(True)
        ev.eval_bordered(seed_d, maps, "mixed", out=(Sb, fb, sb))
        phases = {k: float(v) for k, v in ev.kernel_times().items()}
        ev.set_timing(False)
        torch.cuda.synchronize()
        bordered = {"value": world * Bsz / (b_ms * 1e-3), "unit": "candidate evals/s", "ms_per_step": b_ms,
                    "precision": "mixed (tensor-core reference LU, float-float refined inverse)",
                    "speedup_over_full_solve": (world * Bsz / (b_ms * 1e-3)) / value,
                    "status_ok": int((sb == 0).sum().item()), "phases_ms": phases,
                    "accuracy": accuracy(Sb[:nfp], fb[:nfp])}
    # ---- the gather step as a launch of its own (batched, bulk-staged rows): every candidate's
    #      Z_sub at the middle frequency; algorithmic bytes = the Z_sub entries written (8 or 16 N^2)
    #      plus the same entries read (from the L2-resident Z(f)) and the index lists (4 N)
    gather = None
    if Bsz * ncap * ncap * (16 if w.z_dtype == "c128" else 8) < 8e9:
        fm = w.n_freq // 2
        gbuf = ev.gather_batch(idx, n, fm, ncap)
        g_runs = []
        for rep in range(7):
            e0.record(stream)
            ev.gather_batch(idx, n, fm, ncap, out=gbuf)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= 2:
                g_runs.append(e0.elapsed_time(e1))
        g_ms = float(np.median(g_runs))
        esz = 16 if w.z_dtype == "c128" else 8
        wbytes = float(np.sum(esz * N.astype(np.float64) ** 2))
        hbm = float(_peaks().get("hbm_gbs") or 6800.0)
        gather = {"kernel": "gather_batch_kernel", "candidates": Bsz, "ms": g_ms,
                  "written_GB_per_s": wbytes / (g_ms * 1e-3) / 1e9,
                  "algorithmic_GB_per_s": (2 * wbytes + float(np.sum(4.0 * N))) / (g_ms * 1e-3) / 1e9,
                  "frac_of_hbm_written": wbytes / (g_ms * 1e-3) / 1e9 / hbm,
                  "hbm_peak_GB_per_s": hbm}
        del gbuf
    # ---- end to end through the host-buffer entry point (pinned host memory)
    maps_h = torch.from_numpy(maps_np).pin_memory()
    S_h = torch.empty((Bsz, w.n_freq, ev.P, ev.P), dtype=torch.complex128).pin_memory()
    fom_h = torch.empty((Bsz,), dtype=torch.float64).pin_memory()
    st_h = torch.empty((Bsz,), dtype=torch.int32).pin_memory()
    e2e_val = None
    if args.e2e:
        ev.eval_host(maps_h.numpy(), "mixed", S=S_h.numpy(), fom=fom_h.numpy(), status=st_h.numpy())
        n_e2e = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            ev.eval_host(maps_h.numpy(), "mixed", S=S_h.numpy(), fom=fom_h.numpy(), status=st_h.numpy())
        e2e_s = (time.perf_counter() - t0) / n_e2e
        e2e_val = world * Bsz / e2e_s
    # ---- roofline of the dominant kernel (the evaluation kernel)
    peaks = _peaks()
    eval_ms = float(np.median(kern_ms)) if kern_ms else ms
    flops = lu_flops(N, w.n_freq, ev.P)
    large = int(N.max()) > ev.capacity("mixed")[0]
    achieved = flops / (eval_ms * 1e-3) / 1e12
    alu_peak = FP32_LANES_PER_SM * 2 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
    if tc_choice:
        # the LU's contraction runs on the tensor cores in TF32: measured dense BF16 burst peak x the
        # nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s); three TF32 products per useful product
        bf16 = float(peaks.get("bf16_tflops") or 1900.0)
        peak = bf16 * 1.1 / 2.25
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (TRAFFIC_PER_TASK[(w.name, "tc")] * Bsz * w.n_freq
                            if (w.name, "tc") in TRAFFIC_PER_TASK and not large else None),
                "traffic_note": "dram read + write bytes per launch: the per-task figure of a 64-candidate "
                                "capture of this kernel times the launch's tasks",
                "kernel": "eval_kernel<float2,float2,mixed,tc%s>" % (",large" if large else ""),
                "peak_source": "measured bf16 %.1f TFLOP/s x 1.1/2.25 (TF32 dense); %s" % (
                    bf16, "of measured" if peaks.get("bf16_tflops") else "of fallback"),
                "frac_of_3xtf32_peak": achieved / (peak / 3.0), "frac_of_fp32_alu": achieved / alu_peak}
    else:
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": None, "kernel": "eval_kernel<float2,float2,mixed,simt>",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (unit counts and max clock)"}
    line = {
        "metric": METRIC, "value": value, "unit": "candidate evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 (fp32/3xTF32 LU and solves, float-float refinement residual, f64 corrections, Y, S, FoM)",
        "data": "synthetic",
        "config": workload_config(w, N, ev.M, Bsz, world),
        "fp64_path": {"value": fp64_value, "unit": "candidate evals/s", "candidates": nfp,
                      "ms_per_step": fp64_ms, "runs_ms": fp64_runs, "status_ok": fp64_status_ok,
                      "timing": "CUDA-graph replay of the FP64 pipeline on the first %d candidates, "
                                "median of %d after one warm-up" % (nfp, reps),
                      "speedup_mixed_over_fp64": value / fp64_value},
        "accuracy": accuracy(S_mixed, fom_mixed),
        "bordered_update": bordered,
        "gather": gather,
        "refinement": {"iters_total": st["refine_iters"], "iters_max": st["refine_max"],
                       "repaired_tasks": st["repaired_tasks"], "tasks": st["tasks"],
                       "bad_status": int((status_np != 0).sum())},
        "kernel_ms": {"eval": eval_ms},
        "autotune": {"tensor_cores": bool(tc_choice), "table": ev.autotune_table()},
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "candidate evals/s", "h2d_bytes_per_step": int(maps_np.nbytes),
                "d2h_bytes_per_step": int(S_h.numel() * 16 + fom_h.numel() * 8 + st_h.numel() * 4)},
        "gpu_launches": 6 * args.steps,   # per graph replay: activate, order, eval, repair, Y->S, FoM
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
    }
    if rank == 0 and not args.no_cpu:
        # the oracle on a bounded sample (timed), and both GPU paths on the same sample: the
        # oracle's own database at the sampled frequencies, loaded into a second evaluator
        info, (smp, nb, S_or) = cpu_baseline(w, sample=OracleSample(w, args.batch))
        line["cpu_baseline"] = info
        line["accuracy_vs_oracle"] = accuracy_vs_oracle(smp, nb, S_or)
    if rank == 0:
        print(json.dumps(line))
    ev.close()
    if dist is not None:
        dist.destroy_process_group()


def column_pool(cur: np.ndarray, rng, size: int) -> np.ndarray:
    """Candidate pool of one search step on an on/off multilayer grid: every single-column change
    (each (x, y) column takes each of its other 2^layers - 1 layer patterns), then random changes of
    two distinct columns up to `size` maps (size 0: the single-column changes only)."""
    L, ny, nx = cur.shape
    K = 1 << L
    cols = cur.reshape(L, -1)
    code = sum(cols[l].astype(np.int64) << l for l in range(L))
    out = []
    for j in range(ny * nx):
        for v in range(K):
            if v != code[j]:
                m = cols.copy()
                for l in range(L):
                    m[l, j] = (v >> l) & 1
                out.append(m)
    while len(out) < size:
        j1, j2 = rng.choice(ny * nx, 2, replace=False)
        m = cols.copy()
        for j in (j1, j2):
            v = int(rng.integers(1, K))
            nv = int(code[j]) ^ v
            for l in range(L):
                m[l, j] = (nv >> l) & 1
        out.append(m)
    return np.ascontiguousarray(np.stack(out[:size] if size > 0 else out).reshape(-1, L, ny, nx).astype(np.uint8))


def run_learned(args):
    """The learned pre-ranker at the 3-layer 24x24 microstrip configuration (64 frequencies 3-9 GHz,
    complex64 database from the library's GPU fill): training data from exact solves the method
    makes anyway (a greedy walk whose steps evaluate a random 512 of the pool exactly), an MLP on
    the 3 x 24 x 24 occupancy trained on the GPU (BF16 tensor-core kernels), then on held-out steps
    the FoM regret of its top-k against exhaustive exact evaluation of every single-column change,
    and best-neighbour walks that exact-evaluate the network's top-k of a 10k pool against walks
    that evaluate a uniformly random k of it, at equal exact-evaluation budgets."""
    import torch
    from paper_2412_17617_gb300 import Evaluator, band_codes, build as B
    from paper_2412_17617_gb300 import surrogate as SG
    B.build()
    w = PI.workload_learned()
    ev = Evaluator(w.grid)
    freqs = w.freqs()
    t0 = time.perf_counter()
    ev.fill_Z(freqs, w.z_dtype)
    codes = band_codes(freqs, w.bands)
    ev.set_fom(codes, w.z0_ohm)
    bands = torch.from_numpy(np.ascontiguousarray(codes)).cuda()
    fill_s = time.perf_counter() - t0
    pool_size, per_step, steps_train = 10000, 512, args.learned_steps
    rng = np.random.default_rng(5)

    def exact(maps):
        out_f, out_t, out_x = [], [], []
        for i in range(0, maps.shape[0], 1024):
            dm = torch.from_numpy(np.ascontiguousarray(maps[i:i + 1024])).cuda()
            S, fom, st = ev.eval(dm, "mixed")
            f = fom.cpu().numpy()
            out_f.append(np.where(st.cpu().numpy() == 0, f, np.inf))
            out_t.append(SG.targets(S))
            out_x.append(dm.reshape(dm.shape[0], -1))
        return np.concatenate(out_f), torch.cat(out_t), torch.cat(out_x)

    # ---- training data: a greedy walk, each step a random 512 of the pool solved exactly
    cur = PI.seed_map(w.grid, w.fill, 0)
    xs, ts = [], []
    t0 = time.perf_counter()
    n_exact = 0
    for _ in range(steps_train):
        pool = column_pool(cur, rng, pool_size)
        sel = pool[rng.choice(pool.shape[0], per_step, replace=False)]
        f, t, x = exact(sel)
        n_exact += sel.shape[0]
        xs.append(x)
        ts.append(t)
        cur = sel[int(np.argmin(f))]
    torch.cuda.synchronize()
    exact_s = time.perf_counter() - t0
    X, T = torch.cat(xs).contiguous(), torch.cat(ts).contiguous()
    net = SG.MLP([X.shape[1], 1024, 1024, 4 * w.n_freq], seed=7)
    t0 = time.perf_counter()
    hist = SG.train(net, X, T, epochs=args.learned_epochs, batch=256, lr=5e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    def rank(pool):
        x = torch.from_numpy(pool).cuda().reshape(pool.shape[0], -1)
        return net.predict_fom(x, bands, w.n_freq).cpu().numpy()

    # ---- held-out steps: exhaustive exact evaluation of every single-column change
    regret, spearman = [], []
    start = cur.copy()
    for step in range(args.learned_heldout):
        singles = column_pool(cur, rng, 0)
        f, _, _ = exact(singles)
        pred = rank(singles)
        order = np.argsort(pred, kind="stable")
        best = float(f.min())
        row = {"children": int(singles.shape[0]), "best_exact_fom": best}
        for k in (64, 256):
            from math import lgamma
            srt = np.sort(f)
            n = len(srt)

            def lcomb(a, b):
                return lgamma(a + 1) - lgamma(b + 1) - lgamma(a - b + 1) if 0 <= b <= a else -np.inf
            # probability that the i-th smallest of n is the minimum of a uniform k-subset
            pk = np.exp(np.array([lcomb(n - i, k - 1) for i in range(1, n + 1)]) - lcomb(n, k))
            row[f"top{k}_regret"] = (float(f[order[:k]].min()) - best) / abs(best)
            row[f"random{k}_expected_regret"] = (float(np.dot(pk, srt)) - best) / abs(best)
        ra, rb = np.argsort(np.argsort(pred)), np.argsort(np.argsort(f))
        spearman.append(float(np.corrcoef(ra, rb)[0, 1]))
        regret.append(row)
        cur = singles[int(np.argmin(f))]
    # ---- network throughput on a 10k pool (the per-step ranking)
    pool = column_pool(cur, rng, pool_size)
    x = torch.from_numpy(pool).cuda().reshape(pool.shape[0], -1)
    net.predict_fom(x, bands, w.n_freq)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        net.predict_fom(x, bands, w.n_freq)
    torch.cuda.synchronize()
    rank_ms = (time.perf_counter() - t0) / 5 * 1e3

    # ---- walks at equal exact budgets: the network's top-k of a 10k pool vs a random k of it
    def walk(seed, k, budget, use_net):
        r = np.random.default_rng(100 + seed)
        c = start.copy()
        best, used = np.inf, 0
        while used < budget:
            pool = column_pool(c, r, pool_size)
            if use_net:
                sel = np.argsort(rank(pool), kind="stable")[:k]
            else:
                sel = r.choice(pool.shape[0], k, replace=False)
            f, _, _ = exact(pool[sel])
            used += k
            j = int(np.argmin(f))
            best = min(best, float(f[j]))
            c = pool[sel[j]]
        return best
    walks = []
    for seed in range(args.learned_walk_seeds):
        walks.append({"seed": seed, "k": args.learned_k, "budget": args.learned_budget,
                      "preranked_best_fom": walk(seed, args.learned_k, args.learned_budget, True),
                      "random_k_best_fom": walk(seed, args.learned_k, args.learned_budget, False)})
    line = {"metric": "learned pre-ranker (NEXT-2) at the 3-layer 24x24 microstrip configuration",
            "config": {"workload": w.name, "M": ev.M, "freqs": w.n_freq, "pool_per_step": pool_size,
                       "network": [int(X.shape[1]), 1024, 1024, 4 * w.n_freq], "training_solves": n_exact,
                       "epochs": args.learned_epochs},
            "fill_s": fill_s, "exact_solves_per_s": n_exact / exact_s, "train_s": train_s,
            "loss_first_last": [hist[0], hist[-1]], "rank_10k_ms": rank_ms,
            "heldout": {"spearman": spearman, "regret": regret}, "walks": walks}
    print(json.dumps(line))
    net.close()
    ev.close()


def run_peaks():
    """Measured throughput ceilings of this GPU for the roofline denominators that the measured
    peaks file does not carry: dense TF32, FP32 and FP64 matrix products through torch.matmul
    (cuBLAS) and, for comparison, BF16 and a device-to-device copy.  Best of ten, CUDA events."""
    import torch
    torch.cuda.init()
    dev = torch.cuda.get_device_properties(0)
    res = {"gpu": dev.name, "sms": dev.multi_processor_count, "torch": torch.__version__}

    def best(fn, reps=10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        return min(t)

    for name, dt, n, tf32 in (("bf16_tflops", torch.bfloat16, 8192, False), ("tf32_tflops", torch.float32, 8192, True),
                              ("fp32_tflops", torch.float32, 8192, False), ("fp64_tflops", torch.float64, 4096, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda").to(dt)
        b = torch.randn(n, n, device="cuda").to(dt)
        ms = best(lambda: torch.matmul(a, b))
        res[name] = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
        res[name.replace("_tflops", "_shape")] = f"{n}^3"
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    x = torch.empty(1 << 30, dtype=torch.bfloat16, device="cuda")
    y = torch.empty_like(x)
    ms = best(lambda: y.copy_(x))
    res["hbm_copy_gbs"] = 2.0 * x.numel() * 2 / (ms * 1e-3) / 1e9
    res["how"] = "torch.matmul n^3 (2 n^3 flop), best of 10 after one warm-up, CUDA events; copy of 1 Gi bf16 (read + write)"
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision", choices=["precision", "plain", "profile", "batching", "scale"],
                    help="profile: a smaller grid running the same kernels, for counter captures; batching: "
                         "the 3-layer 20x20 three-state stripline, 101 frequencies, uneven support sets; scale: "
                         "the 4-layer 32x32 stripline (M = 12048, N about 4000, 117 GB database); bound both "
                         "with --batch")
    ap.add_argument("--batch", type=int, default=0, help="evaluate only the first B candidates")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-bordered", dest="bordered", action="store_false",
                    help="skip the bordered-update measurement of the same batch")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false",
                    help="skip the end-to-end host-buffer measurement (long legs)")
    ap.add_argument("--learned", action="store_true",
                    help="the learned pre-ranker at the 24x24x3 microstrip configuration (training, held-out "
                         "regret against exhaustive evaluation, walks against a random-k control)")
    ap.add_argument("--learned-steps", type=int, default=12, help="training walk steps (512 exact solves each)")
    ap.add_argument("--learned-epochs", type=int, default=60)
    ap.add_argument("--learned-heldout", type=int, default=2)
    ap.add_argument("--learned-k", type=int, default=64)
    ap.add_argument("--learned-budget", type=int, default=1024)
    ap.add_argument("--learned-walk-seeds", type=int, default=2)
    ap.add_argument("--peaks", action="store_true", help="measure TF32 / FP32 / FP64 / BF16 matmul and copy "
                                                           "throughput of this GPU and print them as JSON")
    args = ap.parse_args()
    if args.peaks:
        run_peaks()
    elif args.learned:
        run_learned(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
