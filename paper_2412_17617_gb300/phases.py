"""Phase-clock profile of the evaluation kernel (profiling build, GB300).

    python -m paper_2412_17617_gb300.phases [--workload precision|plain|profile] [--batch B]

Builds the profiling variant of the library (`-DPMOM_PHASES`: thread 0 of each task group adds the
clock64 cycles of every phase of a task to a device counter, sub-phases lapped into local
accumulators), evaluates the workload once to warm up and once measured (mixed path, autotuned),
and prints the cycles per task per phase.  The counters cover the default-layout evaluation kernels
(support sets that fit one CTA, which includes every task of the three workloads offered here).
The phase marks add about 10 % to the launch; the cycles are per task group, two groups sharing an
SM.  This module runs the library; it is not part of the evaluation path.
"""
from __future__ import annotations

import argparse
import ctypes

# phase slots of the kernel (their order in the kernel's enum); slot 15 counts tasks, slots 16 and
# up split phases further and are also counted in the phase that encloses them
NAMES = ["gather", "lu", "solve0", "resid", "solvecorr", "other", "panelload", "panelfactor", "colgemm",
         "panelstore", "swap", "innerU", "innerupd", "rowgemm", "trsm", "tasks", "solveperm", "solvestage",
         "solveoff", "solvediag", "panelwork", "panelwait", "g_copywait", "g_stagewait", "g_sync", "g_mma",
         "g_epi", "g_issue", "g_conv"]
TASKS = 15


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="precision", choices=["precision", "plain", "profile"])
    ap.add_argument("--batch", type=int, default=0, help="first B candidates only (0: all)")
    args = ap.parse_args(argv)

    from . import build as B
    from . import pmom
    lib = pmom.load_library(B.build(phases=True))   # must be the process's first load of the library
    if not hasattr(lib, "pmom_phase_read"):
        raise RuntimeError("the loaded library has no phase counters (not a profiling build)")
    lib.pmom_phase_slots.restype = ctypes.c_int
    lib.pmom_phase_read.argtypes = [ctypes.c_void_p]
    lib.pmom_phase_read.restype = ctypes.c_int
    lib.pmom_phase_reset.restype = ctypes.c_int

    import torch
    import pmom_inputs as PI
    from .pmom import Evaluator, band_codes

    w = {"precision": PI.workload_precision, "plain": PI.workload_plain, "profile": PI.workload_profile}[args.workload]()
    torch.cuda.set_device(0)
    ev = Evaluator(w.grid)
    freqs = w.freqs()
    ev.fill_Z(freqs, w.z_dtype)
    ev.set_fom(band_codes(freqs, w.bands), w.z0_ohm)
    maps_np = PI.workload_maps(w, seed=0)
    if args.batch > 0:
        maps_np = maps_np[:args.batch]
    maps = torch.from_numpy(maps_np.copy()).cuda()
    ev.autotune(maps, "mixed")
    ev.eval(maps, "mixed")
    torch.cuda.synchronize()
    if lib.pmom_phase_reset() != 0:
        raise RuntimeError("phase counters: reset failed")
    ev.set_timing(True)
    ev.eval(maps, "mixed")
    torch.cuda.synchronize()
    ms = ev.kernel_times()["eval"]
    n = lib.pmom_phase_slots()
    buf = (ctypes.c_ulonglong * n)()
    if lib.pmom_phase_read(ctypes.addressof(buf)) != 0:
        raise RuntimeError("phase counters: read failed")
    v = [float(x) for x in buf]
    tasks = v[TASKS]
    if tasks <= 0:
        raise RuntimeError("no task reached the default-layout kernels")
    print(f"{args.workload}: {maps_np.shape[0]} candidates x {len(freqs)} frequencies, {tasks:.0f} tasks, "
          f"evaluation launch {ms:.1f} ms (profiling build), stats {ev.stats()}")
    print("Mcycles per task per group:")
    for i, name in enumerate(NAMES):
        if i != TASKS and v[i] > 0:
            print(f"  {name:12s} {v[i] / tasks / 1e6:8.3f}")
    print(f"  {'total':12s} {sum(v[:6]) / tasks / 1e6:8.3f}  (phases 0-5)")
    ev.close()


if __name__ == "__main__":
    main()
