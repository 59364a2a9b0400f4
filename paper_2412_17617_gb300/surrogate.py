"""Learned pre-ranker binding: a multilayer perceptron on the library's BF16 tensor-core kernels
(pmom_mlp_* in include/pmom.h), trained on (pixel map, |S| dB) pairs that the evaluator produces,
and the pre-ranked search step that exact-evaluates only the network's top-k children.

Marshalling only: forward, backward, Adam, the dB targets and the predicted FoM run in the
library's kernels; the host picks the top-k indices of the predicted FoM and the best of the
exactly evaluated ones.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from .pmom import PmomError, _stream_ptr, load_library

OUT_SCALE = 1.0 / 40.0   # targets are dB / 40 (order-one values for the loss)


class MLP:
    """dims: layer sizes, input first (input = the map's pixel states, one per pixel and layer);
    the output must be 4 F (dB of S11, S21, S31, S32 at each of F frequencies) for predict_fom."""

    def __init__(self, dims: Sequence[int], seed: int = 0):
        self.L = load_library()
        self.dims = [int(d) for d in dims]
        arr = (ctypes.c_int32 * len(self.dims))(*self.dims)
        h = ctypes.c_void_p()
        st = self.L.pmom_mlp_create(len(self.dims) - 1, arr, ctypes.c_uint64(seed), ctypes.byref(h))
        if st != 0:
            raise PmomError(st, "pmom_mlp_create failed")
        self.h = h
        n = ctypes.c_int64()
        self._check(self.L.pmom_mlp_num_params(self.h, ctypes.byref(n)))
        self.n_params = int(n.value)

    def _check(self, st: int):
        if st != 0:
            raise PmomError(st, self.L.pmom_mlp_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.L.pmom_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- parameters (flat FP32 [W_0, b_0, W_1, b_1, ...], W_l row-major dims[l+1] x dims[l])
    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._check(self.L.pmom_mlp_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p), None))
        return out

    def grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._check(self.L.pmom_mlp_get_params(self.h, None, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        self._check(self.L.pmom_mlp_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p)))

    # ---- compute
    def forward(self, x, stream=None):
        """x: torch CUDA uint8 [B][dims[0]] -> torch CUDA float32 [B][dims[-1]]."""
        import torch
        B = x.shape[0]
        y = torch.empty((B, self.dims[-1]), dtype=torch.float32, device="cuda")
        self._check(self.L.pmom_mlp_forward(self.h, ctypes.c_void_p(x.data_ptr()), B, ctypes.c_void_p(y.data_ptr()),
                                            ctypes.c_void_p(_stream_ptr(stream))))
        return y

    def backward(self, x, target, stream=None) -> float:
        """Gradients of the mean squared error (kept in the network); returns the loss."""
        loss = ctypes.c_double()
        self._check(self.L.pmom_mlp_backward(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                             x.shape[0], ctypes.byref(loss), ctypes.c_void_p(_stream_ptr(stream))))
        return float(loss.value)

    def adam(self, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        self._check(self.L.pmom_mlp_adam(self.h, ctypes.c_float(lr), ctypes.c_float(beta1), ctypes.c_float(beta2),
                                         ctypes.c_float(eps), ctypes.c_void_p(_stream_ptr(stream))))

    def predict_fom(self, x, bands_dev, F: int, stream=None):
        """Predicted FoM (Eq. 8-9) of each map from the predicted dB values -> torch float64 [B]."""
        import torch
        B = x.shape[0]
        fom = torch.empty((B,), dtype=torch.float64, device="cuda")
        self._check(self.L.pmom_mlp_predict_fom(self.h, ctypes.c_void_p(x.data_ptr()), B,
                                                ctypes.c_void_p(bands_dev.data_ptr()), F, ctypes.c_float(OUT_SCALE),
                                                ctypes.c_void_p(fom.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return fom

    def timeouts(self) -> int:
        t = ctypes.c_int32()
        self._check(self.L.pmom_mlp_errors(self.h, ctypes.byref(t)))
        return int(t.value)


def targets(S, stream=None):
    """Training targets from evaluated S (torch CUDA complex128 [B][F][P][P]) -> float32 [B][4F]."""
    import torch
    L = load_library()
    B, F, P = S.shape[0], S.shape[1], S.shape[2]
    t = torch.empty((B, 4 * F), dtype=torch.float32, device="cuda")
    st = L.pmom_mlp_targets(ctypes.c_void_p(S.data_ptr()), B, F, P, ctypes.c_float(OUT_SCALE),
                            ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(_stream_ptr(stream)))
    if st != 0:
        raise PmomError(st, "pmom_mlp_targets failed")
    return t


def train(net: MLP, x, t, epochs: int = 20, batch: int = 256, lr: float = 1e-3, seed: int = 0) -> list:
    """Minibatch Adam on (x [N][D] uint8, t [N][4F] float32), both torch CUDA; returns the
    per-epoch mean loss."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = x.shape[0]
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(N, generator=g).cuda()
        tot, cnt = 0.0, 0
        for i in range(0, N - batch + 1, batch):
            idx = perm[i:i + batch]
            xb, tb = x[idx].contiguous(), t[idx].contiguous()
            tot += net.backward(xb, tb)
            net.adam(lr)
            cnt += 1
        hist.append(tot / max(cnt, 1))
    return hist


def preranked_step(ev, net: MLP, bands_dev, parent, children, k: int, precision: str = "mixed"):
    """One search step with pre-ranking: predicted FoM for every child, exact (bordered)
    evaluation of the k best-ranked children against the parent's factors.  Returns (index of the
    best exactly evaluated child, its exact FoM, the indices that were evaluated)."""
    pred = net.predict_fom(children, bands_dev, ev.F).cpu().numpy()
    top = np.argsort(pred, kind="stable")[:k]
    import torch
    sel = children[torch.from_numpy(top).cuda()].contiguous()
    _, fom, status = ev.eval_bordered(parent, sel, precision, want_S=False)
    f = fom.cpu().numpy()
    f = np.where(status.cpu().numpy() == 0, f, np.inf)
    j = int(np.argmin(f))
    return int(top[j]), float(f[j]), top


def walk(ev, start: np.ndarray, budget: int, pick, tabu_len: int = 16, precision: str = "mixed"):
    """Best-neighbour walk over single-pixel flips with a budget of exact evaluations.  Each step
    `pick(parent_dev, children_dev, tabu)` returns the indices of the children to evaluate exactly
    (all of them for the exhaustive walk, the top-k for the pre-ranked one); the walk moves to
    the best evaluated child (bordered update against the parent's factors) and keeps the flipped
    pixels of the last `tabu_len` moves out of reach, so that it does not undo them.  Returns the
    best exact FoM seen and the number of exact evaluations used."""
    import torch
    cur = np.ascontiguousarray(start)
    best, used, tabu = np.inf, 0, []
    while used < budget:
        kids = np.ascontiguousarray(_flips(cur))
        dk = torch.from_numpy(kids).cuda()
        parent = torch.from_numpy(cur).cuda()
        sel = np.asarray(pick(parent, dk, tabu))
        sub = dk[torch.from_numpy(sel).cuda()].contiguous()
        _, fom, status = ev.eval_bordered(parent, sub, precision, want_S=False)
        f = fom.cpu().numpy()
        f = np.where(status.cpu().numpy() == 0, f, np.inf)
        jj = int(np.argmin(f))
        used += len(sel)
        best = min(best, float(f[jj]))
        cur = kids[int(sel[jj])]
        tabu = (tabu + [int(sel[jj])])[-tabu_len:]
    return best, used


def _flips(m: np.ndarray) -> np.ndarray:
    """Every single-pixel change of a two-state map, pixel-major (child i flips pixel i)."""
    L, ny, nx = m.shape
    flat = np.repeat(m.reshape(1, -1), L * ny * nx, axis=0)
    idx = np.arange(L * ny * nx)
    flat[idx, idx] ^= 1
    return flat.reshape(-1, L, ny, nx)


def pick_top(net: MLP, bands_dev, F: int, k: int):
    """Selection rule of the pre-ranked walk: the k children with the lowest predicted FoM."""
    def pick(parent, children, tabu):
        pred = net.predict_fom(children.reshape(children.shape[0], -1), bands_dev, F).cpu().numpy()
        pred[tabu] = np.inf
        return np.argsort(pred, kind="stable")[:k]
    return pick
