"""Compile the CUDA library (sm_103a) in-tree: paper_2412_17617_gb300/_build/libpmom.so."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpmom.so")
SOURCES = ["pmom_api.cu", "pmom_eval.cu", "pmom_eval_large.cu", "pmom_border.cu", "pmom_mlp.cu", "pmom_fill.cu", "pmom_mesh.cpp", "pmom_search.cpp"]
PUBLIC_HEADER = os.path.join(os.path.dirname(HERE), "include", "pmom.h")
HEADERS = [os.path.join(CSRC, h) for h in ("pmom_internal.h", "pmom_eval_kernels.cuh", "pmom_tc.cuh")] + [PUBLIC_HEADER]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "177"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


PHASES_LIB = os.path.join(BUILD, "libpmom_phases.so")


def build(force: bool = False, verbose: bool = False, phases: bool = False) -> str:
    """Builds libpmom.so; with phases=True the profiling variant libpmom_phases.so instead (phase
    clocks compiled in with -DPMOM_PHASES, read by paper_2412_17617_gb300/phases.py)."""
    lib = PHASES_LIB if phases else LIB
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs + HEADERS)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    os.makedirs(BUILD, exist_ok=True)
    objs, procs = [], []
    extra = ["-DPMOM_PHASES"] if phases else []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + f".{os.getpid()}{'.ph' if phases else ''}.o")
        objs.append(o)
        cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", s, "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose:
            sys.stdout.write(out.decode(errors="replace"))
    if failed:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        msg = "\n".join(" ".join(c) + "\n" + out for c, out in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
