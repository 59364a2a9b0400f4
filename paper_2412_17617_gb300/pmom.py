"""Python binding of the C ABI in include/pmom.h (argument marshalling only).

Every computation runs in libpmom.so's CUDA kernels; this module only converts arguments.
Device buffers are torch CUDA tensors (torch provides device memory and streams).  If the
library is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import struct
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpmom.so")

PMOM_OK = 0
PMOM_C64, PMOM_C128 = 0, 1
PMOM_MEM_HOST, PMOM_MEM_DEVICE = 0, 1
PMOM_FP64, PMOM_MIXED_REFINED = 0, 1
CAND_OK, CAND_SINGULAR, CAND_NONFINITE, CAND_REPAIRED, CAND_BAD_STATE, CAND_CAPACITY, CAND_FAR = 0, 1, 2, 3, 5, 6, 7
BORDER_K = 8   # basis functions a candidate may remove from / add to the reference (pmom_eval_bordered)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "BAD_STATE_VALUE", 4: "Z_SHAPE_MISMATCH", 5: "CUDA",
                6: "NOT_READY", 7: "UNSUPPORTED", 8: "IO"}
# names exported by libpmom.so, one per declaration in include/pmom.h
EXPORTS = ("pmom_create", "pmom_destroy", "pmom_last_error", "pmom_num_bfs", "pmom_bf_table", "pmom_load_Z",
           "pmom_copy_Z", "pmom_fill_Z", "pmom_set_fom", "pmom_active_set", "pmom_gather", "pmom_gather_batch",
           "pmom_eval_candidates",
           "pmom_eval_candidates_host", "pmom_stats", "pmom_set_timing", "pmom_kernel_times", "pmom_sync",
           "pmom_eval_candidates_noalloc", "pmom_set_tensor_cores", "pmom_capacity", "pmom_graph_capture", "pmom_graph_launch",
           "pmom_autotune", "pmom_autotune_table", "pmom_search", "pmom_eval_bordered",
           "pmom_mlp_create", "pmom_mlp_destroy", "pmom_mlp_last_error", "pmom_mlp_num_params", "pmom_mlp_get_params",
           "pmom_mlp_set_params", "pmom_mlp_forward", "pmom_mlp_backward", "pmom_mlp_adam", "pmom_mlp_predict_fom",
           "pmom_mlp_targets", "pmom_mlp_errors", "pmom_selftest_wait", "pmom_save_Z", "pmom_load_Z_file",
           "pmom_search_resume")


class PmomError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Port(ctypes.Structure):
    _fields_ = [("layer", ctypes.c_int32), ("side", ctypes.c_int32), ("pos", ctypes.c_int32)]


class _GridDesc(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("pitch_m", ctypes.c_double), ("medium", ctypes.c_int32),
                ("layer_z_m", ctypes.POINTER(ctypes.c_double)), ("h_total_m", ctypes.c_double),
                ("eps_r", ctypes.c_double), ("tan_d", ctypes.c_double), ("n_states", ctypes.c_int32),
                ("n_ports", ctypes.c_int32), ("ports", ctypes.POINTER(_Port)),
                ("diag_pattern", ctypes.c_int32), ("diag_seed", ctypes.c_uint64), ("sub", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpmom.so (build it first with paper_2412_17617_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpmom.so not found at {path}; run paper_2412_17617_gb300.build.build() "
                           "(the evaluator has no CPU fallback)")
    L = ctypes.CDLL(path)
    V, I32, P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
    sig = {
        "pmom_create": [P, P],
        "pmom_destroy": [V],
        "pmom_last_error": [V],
        "pmom_num_bfs": [V, P, P],
        "pmom_bf_table": [V, P],
        "pmom_load_Z": [V, P, I32, P, I32, I32, V],
        "pmom_copy_Z": [V, P, I32, V],
        "pmom_fill_Z": [V, P, I32, I32, V],
        "pmom_set_fom": [V, P, I32, ctypes.c_double],
        "pmom_active_set": [V, P, I32, P, P, V],
        "pmom_gather": [V, P, I32, I32, P, V],
        "pmom_gather_batch": [V, P, P, I32, I32, I32, P, V],
        "pmom_eval_candidates": [V, P, I32, I32, P, P, P, V],
        "pmom_eval_candidates_host": [V, P, I32, I32, P, P, P, V],
        "pmom_stats": [V, P],
        "pmom_set_timing": [V, I32],
        "pmom_kernel_times": [V, P],
        "pmom_sync": [V, V],
        "pmom_eval_candidates_noalloc": [V, P, I32, I32, P, P, P, V],
        "pmom_set_tensor_cores": [V, I32],
        "pmom_capacity": [V, I32, P, P],
        "pmom_selftest_wait": [ctypes.c_int64, I32, P, P, V],
        "pmom_save_Z": [V, ctypes.c_char_p, V],
        "pmom_search_resume": [V, P, P, P, P, I32, P, V],
        "pmom_load_Z_file": [V, ctypes.c_char_p, V],
        "pmom_eval_bordered": [V, P, P, I32, I32, P, P, P, V],
        "pmom_graph_capture": [V, P, I32, I32, P, P, P, I32, V],
        "pmom_graph_launch": [V, V],
        "pmom_autotune": [V, P, I32, I32, P, V],
        "pmom_autotune_table": [V, P],
        "pmom_search": [V, P, P, P, P, P, P, I32, P, V],
        "pmom_mlp_create": [I32, P, ctypes.c_uint64, P],
        "pmom_mlp_destroy": [V],
        "pmom_mlp_num_params": [V, P],
        "pmom_mlp_get_params": [V, P, P],
        "pmom_mlp_set_params": [V, P],
        "pmom_mlp_forward": [V, P, I32, P, V],
        "pmom_mlp_backward": [V, P, P, I32, P, V],
        "pmom_mlp_adam": [V, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, V],
        "pmom_mlp_predict_fom": [V, P, I32, P, I32, ctypes.c_float, P, V],
        "pmom_mlp_targets": [P, I32, I32, I32, ctypes.c_float, P, V],
        "pmom_mlp_errors": [V, P],
        "pmom_mlp_last_error": [V],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int32
    L.pmom_last_error.restype = ctypes.c_char_p
    L.pmom_mlp_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        if not torch.cuda.is_available():   # host-only calls (argument and file checks) on a machine without a GPU
            return 0
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def band_codes(freqs, bands) -> np.ndarray:
    """Band of each frequency for the FoM (Eq. 8-9): p1 and p2 inclusive, then the open interval
    between the channels, then the rest of the scored range, else 255."""
    out = np.full(len(freqs), 255, dtype=np.uint8)
    for i, f in enumerate(np.asarray(freqs, dtype=np.float64)):
        if bands.p1[0] <= f <= bands.p1[1]:
            out[i] = 0
        elif bands.p2[0] <= f <= bands.p2[1]:
            out[i] = 1
        elif bands.i[0] < f < bands.i[1]:
            out[i] = 2
        elif bands.s[0] <= f <= bands.s[1]:
            out[i] = 3
    return out


class _SearchParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("d_max", ctypes.c_int32), ("m_of_d", ctypes.c_int32 * 8),
                ("max_evals", ctypes.c_int64), ("precision", ctypes.c_int32)]


def selftest_wait(polls: int, arrive: bool, stream=None):
    """Failure-detection self-test of the bounded completion wait (pmom_selftest_wait): returns
    (timed_out, kernel milliseconds)."""
    L = load_library()
    to, ms = ctypes.c_int32(-1), ctypes.c_double(0.0)
    st = L.pmom_selftest_wait(int(polls), 1 if arrive else 0, ctypes.byref(to), ctypes.byref(ms),
                              ctypes.c_void_p(_stream_ptr(stream)))
    if st != PMOM_OK:
        raise PmomError(st, "pmom_selftest_wait")
    return bool(to.value), ms.value


class _SearchState(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int32), ("depth", ctypes.c_int32), ("counter", ctypes.c_int32),
                ("evals", ctypes.c_int64), ("restart", ctypes.c_uint64), ("iteration", ctypes.c_uint64),
                ("fom", ctypes.c_double), ("best_fom", ctypes.c_double),
                ("map", ctypes.c_void_p), ("best_map", ctypes.c_void_p)]


class Evaluator:
    """One pmom context (one grid) on the current CUDA device."""

    def __init__(self, grid):
        self.L = load_library()
        self.grid = grid
        self._last_kind = "eval"
        self._z = (ctypes.c_double * grid.layers)(*grid.layer_z_m)
        self._ports = (_Port * len(grid.ports))(*[_Port(p.layer, p.side, p.pos) for p in grid.ports])
        desc = _GridDesc(grid.layers, grid.nx, grid.ny, grid.pitch_m, grid.medium, self._z, grid.h_total_m,
                         grid.eps_r, grid.tan_d, grid.n_states, len(grid.ports), self._ports,
                         getattr(grid, "diag_pattern", 0), getattr(grid, "diag_seed", 0), getattr(grid, "sub", 1))
        h = ctypes.c_void_p()
        st = self.L.pmom_create(ctypes.byref(desc), ctypes.byref(h))
        if st != PMOM_OK:
            raise PmomError(st, "pmom_create")
        self.h = h
        M, P = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.L.pmom_num_bfs(self.h, ctypes.byref(M), ctypes.byref(P)))
        self.M, self.P = M.value, P.value
        self.F = 0

    def _check(self, st: int):
        if st != PMOM_OK:
            raise PmomError(st, self.L.pmom_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.pmom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bf_table(self) -> np.ndarray:
        t = np.zeros((self.M, 8), dtype=np.int32)
        self._check(self.L.pmom_bf_table(self.h, t.ctypes.data_as(ctypes.c_void_p)))
        return t

    def load_Z(self, freqs, Z, stream=None):
        """Z: torch CUDA tensor or numpy array [F][M][M], complex64 or complex128."""
        import torch
        f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
        if isinstance(Z, torch.Tensor):
            Z = Z.contiguous()
            dtype = PMOM_C128 if Z.dtype == torch.complex128 else PMOM_C64
            mem = PMOM_MEM_DEVICE if Z.is_cuda else PMOM_MEM_HOST
            ptr = Z.data_ptr()
        else:
            Z = np.ascontiguousarray(Z)
            dtype = PMOM_C128 if Z.dtype == np.complex128 else PMOM_C64
            mem, ptr = PMOM_MEM_HOST, Z.ctypes.data
        if Z.shape != (len(f), self.M, self.M):
            raise ValueError(f"Z shape {tuple(Z.shape)} != {(len(f), self.M, self.M)}")
        self._check(self.L.pmom_load_Z(self.h, f.ctypes.data_as(ctypes.c_void_p), len(f), ctypes.c_void_p(ptr), dtype,
                                       mem, ctypes.c_void_p(_stream_ptr(stream))))
        self._check(self.L.pmom_sync(self.h, ctypes.c_void_p(_stream_ptr(stream))))
        self.F, self.dtype = len(f), dtype

    def fill_Z(self, freqs, dtype: str = "c64", stream=None):
        f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
        code = PMOM_C128 if dtype == "c128" else PMOM_C64
        self._check(self.L.pmom_fill_Z(self.h, f.ctypes.data_as(ctypes.c_void_p), len(f), code,
                                       ctypes.c_void_p(_stream_ptr(stream))))
        self.F, self.dtype = len(f), code

    def save_Z(self, path: str, stream=None):
        """Write the database to a file (pmom_save_Z)."""
        self._check(self.L.pmom_save_Z(self.h, os.fsencode(path), ctypes.c_void_p(_stream_ptr(stream))))

    def load_Z_file(self, path: str, stream=None):
        """Load a database file written by save_Z for this grid (pmom_load_Z_file)."""
        self._check(self.L.pmom_load_Z_file(self.h, os.fsencode(path), ctypes.c_void_p(_stream_ptr(stream))))
        with open(path, "rb") as fh:
            _, _, dtype, _, F = struct.unpack("<8sIIii", fh.read(24))
        self.F, self.dtype = F, dtype

    def copy_Z(self):
        import torch
        dt = torch.complex128 if self.dtype == PMOM_C128 else torch.complex64
        out = torch.empty((self.F, self.M, self.M), dtype=dt, device="cuda")
        self._check(self.L.pmom_copy_Z(self.h, ctypes.c_void_p(out.data_ptr()), PMOM_MEM_DEVICE,
                                       ctypes.c_void_p(_stream_ptr(None))))
        self._check(self.L.pmom_sync(self.h, ctypes.c_void_p(_stream_ptr(None))))
        return out

    def set_fom(self, band_of_freq, Z0: float = 50.0):
        b = np.ascontiguousarray(np.asarray(band_of_freq, dtype=np.uint8))
        self._check(self.L.pmom_set_fom(self.h, b.ctypes.data_as(ctypes.c_void_p), len(b), float(Z0)))

    def active_set(self, maps, stream=None):
        import torch
        B = maps.shape[0]
        idx = torch.empty((B, self.M), dtype=torch.int32, device="cuda")
        n = torch.empty((B,), dtype=torch.int32, device="cuda")
        self._check(self.L.pmom_active_set(self.h, ctypes.c_void_p(maps.data_ptr()), B, ctypes.c_void_p(idx.data_ptr()),
                                           ctypes.c_void_p(n.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return idx, n

    def gather(self, idx, f: int, stream=None):
        import torch
        N = idx.numel()
        dt = torch.complex128 if self.dtype == PMOM_C128 else torch.complex64
        out = torch.empty((N, N), dtype=dt, device="cuda")
        self._check(self.L.pmom_gather(self.h, ctypes.c_void_p(idx.data_ptr()), N, f, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def gather_batch(self, idx, n, f: int, ncap: int, out=None, stream=None):
        """idx: device int32 [B][M], n: device int32 [B] (as from active_set) -> [B][ncap][ncap]
        complex tensor with Z_sub of each candidate in its leading N_b x N_b block."""
        import torch
        B = n.numel()
        dt = torch.complex128 if self.dtype == PMOM_C128 else torch.complex64
        if out is None:
            out = torch.zeros((B, ncap, ncap), dtype=dt, device="cuda")
        self._check(self.L.pmom_gather_batch(self.h, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(n.data_ptr()), B, f,
                                             ncap, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def eval(self, maps, precision: str = "mixed", want_S: bool = True, out=None, stream=None):
        """maps: torch CUDA uint8 [B][layers][ny][nx].  Returns (S [B,F,P,P] complex128 or None, fom, status)."""
        import torch
        B = maps.shape[0]
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        if out is None:
            S = torch.empty((B, self.F, self.P, self.P), dtype=torch.complex128, device="cuda") if want_S else None
            fom = torch.empty((B,), dtype=torch.float64, device="cuda")
            status = torch.empty((B,), dtype=torch.int32, device="cuda")
        else:
            S, fom, status = out
        self._last_kind = "eval"
        self._check(self.L.pmom_eval_candidates(
            self.h, ctypes.c_void_p(maps.data_ptr()), B, prec, ctypes.c_void_p(S.data_ptr() if S is not None else 0),
            ctypes.c_void_p(fom.data_ptr()), ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return S, fom, status

    def eval_bordered(self, reference_map, maps, precision: str = "mixed", want_S: bool = True, out=None,
                      stream=None):
        """Bordered low-rank evaluation of `maps` (torch CUDA uint8 [B][layers][ny][nx]) against the
        torch CUDA uint8 `reference_map` [layers][ny][nx]; same outputs as eval().  Candidates that
        remove or add more than BORDER_K basis functions report CAND_FAR."""
        import torch
        B = maps.shape[0]
        if out is None:
            S = torch.empty((B, self.F, self.P, self.P), dtype=torch.complex128, device="cuda") if want_S else None
            fom = torch.empty((B,), dtype=torch.float64, device="cuda")
            status = torch.empty((B,), dtype=torch.int32, device="cuda")
        else:
            S, fom, status = out
        self._last_kind = "bordered"
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        self._check(self.L.pmom_eval_bordered(
            self.h, ctypes.c_void_p(reference_map.data_ptr()), ctypes.c_void_p(maps.data_ptr()), B, prec,
            ctypes.c_void_p(S.data_ptr() if S is not None else 0), ctypes.c_void_p(fom.data_ptr()),
            ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return S, fom, status

    def eval_host(self, maps: np.ndarray, precision: str = "mixed", S: Optional[np.ndarray] = None,
                  fom: Optional[np.ndarray] = None, status: Optional[np.ndarray] = None, stream=None):
        """Host buffers in and out (pinned numpy views recommended); copies happen inside the call."""
        B = maps.shape[0]
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        fom = np.empty(B, np.float64) if fom is None else fom
        status = np.empty(B, np.int32) if status is None else status
        sp = S.ctypes.data if S is not None else 0
        self._check(self.L.pmom_eval_candidates_host(
            self.h, ctypes.c_void_p(maps.ctypes.data), B, prec, ctypes.c_void_p(sp), ctypes.c_void_p(fom.ctypes.data),
            ctypes.c_void_p(status.ctypes.data), ctypes.c_void_p(_stream_ptr(stream))))
        return S, fom, status

    def graph_capture(self, maps, precision: str = "mixed", out=None, ncap: int = 0, stream=None):
        """Record the evaluation of this batch into a CUDA graph; returns the output tensors that
        each graph_launch() refills."""
        import torch
        B = maps.shape[0]
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        if out is None:
            out = (torch.empty((B, self.F, self.P, self.P), dtype=torch.complex128, device="cuda"),
                   torch.empty((B,), dtype=torch.float64, device="cuda"),
                   torch.empty((B,), dtype=torch.int32, device="cuda"))
        S, fom, status = out
        self._check(self.L.pmom_graph_capture(
            self.h, ctypes.c_void_p(maps.data_ptr()), B, prec, ctypes.c_void_p(S.data_ptr() if S is not None else 0),
            ctypes.c_void_p(fom.data_ptr()), ctypes.c_void_p(status.data_ptr()), int(ncap),
            ctypes.c_void_p(_stream_ptr(stream))))
        self._graph_out = out
        return out

    def graph_launch(self, stream=None):
        self._check(self.L.pmom_graph_launch(self.h, ctypes.c_void_p(_stream_ptr(stream))))
        return self._graph_out

    def autotune_table(self) -> list:
        """The autotuner's choices per support-set bucket that it measured: [{"n_range": (lo, hi),
        "tensor_cores", "groups_per_cta", "slot_cap" (fraction), "us_per_candidate"}]."""
        out = np.zeros((8, 5), dtype=np.int32)
        self._check(self.L.pmom_autotune_table(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        rows = []
        for b in range(8):
            if out[b, 0]:
                lo = 0 if b == 0 else 64 << b
                hi = None if b == 7 else 128 << b
                rows.append({"n_range": [lo, hi], "tensor_cores": bool(out[b, 1]), "groups_per_cta": int(out[b, 2]),
                             "slot_cap": out[b, 3] / 4.0, "us_per_candidate": int(out[b, 4])})
        return rows

    def autotune(self, maps, precision: str = "mixed", stream=None) -> int:
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        ch = ctypes.c_int32(0)
        self._check(self.L.pmom_autotune(self.h, ctypes.c_void_p(maps.data_ptr()), maps.shape[0], prec, ctypes.byref(ch),
                                         ctypes.c_void_p(_stream_ptr(stream))))
        return ch.value

    def eval_noalloc(self, maps, precision: str = "mixed", out=None, stream=None):
        """Like eval(), through the entry point that allocates no device memory during the call
        (temporaries live in the library's fixed 32 MiB device array; see include/pmom.h)."""
        import torch
        B = maps.shape[0]
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        if out is None:
            S = torch.empty((B, self.F, self.P, self.P), dtype=torch.complex128, device="cuda")
            fom = torch.empty((B,), dtype=torch.float64, device="cuda")
            status = torch.empty((B,), dtype=torch.int32, device="cuda")
        else:
            S, fom, status = out
        self._check(self.L.pmom_eval_candidates_noalloc(
            self.h, ctypes.c_void_p(maps.data_ptr()), B, prec, ctypes.c_void_p(S.data_ptr() if S is not None else 0),
            ctypes.c_void_p(fom.data_ptr()), ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return S, fom, status

    def search(self, init_map: np.ndarray, seed: int, d_max: int = 2, m_of_d=(10, 3), max_evals: int = 1000,
               precision: str = "mixed", trace_cap: int = 100000, stream=None):
        """Algorithm 1 on the GPU evaluator.  Returns (best_map, best_fom, evals, trace)."""
        m = list(m_of_d) + [m_of_d[-1]] * (8 - len(m_of_d))
        prm = _SearchParams(seed, d_max, (ctypes.c_int32 * 8)(*m[:8]), max_evals,
                            PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED)
        init = np.ascontiguousarray(init_map, dtype=np.uint8)
        best = np.zeros_like(init)
        bf = ctypes.c_double(0.0)
        ev = ctypes.c_int64(0)
        tr = np.zeros(trace_cap, np.float64)
        tl = ctypes.c_int32(0)
        self._check(self.L.pmom_search(self.h, ctypes.byref(prm), ctypes.c_void_p(init.ctypes.data),
                                       ctypes.c_void_p(best.ctypes.data), ctypes.byref(bf), ctypes.byref(ev),
                                       ctypes.c_void_p(tr.ctypes.data), trace_cap, ctypes.byref(tl),
                                       ctypes.c_void_p(_stream_ptr(stream))))
        return best, bf.value, ev.value, tr[: tl.value].copy()

    def search_resume(self, init_map: np.ndarray, seed: int, d_max: int = 2, m_of_d=(10, 3), max_evals: int = 1000,
                      precision: str = "mixed", state: dict = None, trace_cap: int = 100000, stream=None):
        """Algorithm 1 from or to a checkpoint (pmom_search_resume).  Returns (best_map, best_fom,
        evals, trace of this call, state); pass the state back to continue the same search."""
        m = list(m_of_d) + [m_of_d[-1]] * (8 - len(m_of_d))
        prm = _SearchParams(seed, d_max, (ctypes.c_int32 * 8)(*m[:8]), max_evals,
                            PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED)
        init = np.ascontiguousarray(init_map, dtype=np.uint8)
        cur = init.copy() if state is None else np.ascontiguousarray(state["map"], dtype=np.uint8).copy()
        best = init.copy() if state is None else np.ascontiguousarray(state["best_map"], dtype=np.uint8).copy()
        st = _SearchState(0, 1, 0, 0, 0, 0, 0.0, 0.0, cur.ctypes.data, best.ctypes.data)
        if state is not None:
            st.valid, st.depth, st.counter, st.evals = 1, state["depth"], state["counter"], state["evals"]
            st.restart, st.iteration, st.fom, st.best_fom = state["restart"], state["iteration"], state["fom"], state["best_fom"]
        tr = np.zeros(trace_cap, np.float64)
        tl = ctypes.c_int32(0)
        self._check(self.L.pmom_search_resume(self.h, ctypes.byref(prm), ctypes.c_void_p(init.ctypes.data),
                                              ctypes.byref(st), ctypes.c_void_p(tr.ctypes.data), trace_cap,
                                              ctypes.byref(tl), ctypes.c_void_p(_stream_ptr(stream))))
        out = {"map": cur, "fom": st.fom, "best_map": best, "best_fom": st.best_fom, "evals": st.evals,
               "depth": st.depth, "counter": st.counter, "restart": st.restart, "iteration": st.iteration}
        return best.copy(), st.best_fom, st.evals, tr[: tl.value].copy(), out

    def stats(self) -> dict:
        out = np.zeros(8, dtype=np.int64)
        self._check(self.L.pmom_stats(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return {"tasks": int(out[0]), "refine_iters": int(out[1]), "refine_max": int(out[2]),
                "repaired_tasks": int(out[3]), "tc_wait_timeouts": int(out[4]), "launches": int(out[6])}

    def set_tensor_cores(self, on: bool = True):
        self._check(self.L.pmom_set_tensor_cores(self.h, 1 if on else 0))

    def capacity(self, precision: str = "mixed"):
        """(n_default, n_max): the largest support set of the default shared-memory layout and of
        any layout (larger candidates come back with status CAPACITY)."""
        nd, nm = ctypes.c_int32(), ctypes.c_int32()
        prec = PMOM_FP64 if precision == "fp64" else PMOM_MIXED_REFINED
        self._check(self.L.pmom_capacity(self.h, prec, ctypes.byref(nd), ctypes.byref(nm)))
        return nd.value, nm.value

    def set_timing(self, on: bool = True):
        self._check(self.L.pmom_set_timing(self.h, 1 if on else 0))

    def kernel_times(self) -> dict:
        """Milliseconds of the last eval call's kernels (CUDA events on its stream)."""
        out = np.zeros(4, dtype=np.float64)
        self._check(self.L.pmom_kernel_times(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        if self._last_kind == "bordered":
            return {"ref_lu": out[0], "ref_inverse": out[1], "border": out[2], "fom": out[3]}
        return {"activate": out[0], "eval": out[1], "repair": out[2], "fom": out[3]}

    def sync(self, stream=None):
        self._check(self.L.pmom_sync(self.h, ctypes.c_void_p(_stream_ptr(stream))))
