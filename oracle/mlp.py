"""Plain float64 reference of the pre-ranker network (TEST INFRASTRUCTURE ONLY: the library's
BF16 tensor-core training and inference kernels are checked against it).

Definition (the library's, stated in include/pmom.h): layer l maps h_l (B x d_l) to
z_l = h_l W_l^T + b_l with W_l of shape d_{l+1} x d_l; h_{l+1} = max(z_l, 0) for every layer but
the last, whose z is the output; loss = mean over the batch and outputs of (out - target)^2.
Parameters are one flat vector [W_0, b_0, W_1, b_1, ...], W row-major.  Gradients by the chain
rule, layer by layer, written out with numpy matrix products.
"""
from __future__ import annotations

import numpy as np


def unpack(params: np.ndarray, dims):
    out, off = [], 0
    for l in range(len(dims) - 1):
        n = dims[l + 1] * dims[l]
        W = params[off:off + n].reshape(dims[l + 1], dims[l])
        off += n
        b = params[off:off + dims[l + 1]]
        off += dims[l + 1]
        out.append((W.astype(np.float64), b.astype(np.float64)))
    assert off == params.size
    return out


def forward(params, dims, X):
    """Returns (output, list of layer inputs h_l, list of pre-activations z_l)."""
    layers = unpack(params, dims)
    h = np.asarray(X, dtype=np.float64)
    hs, zs = [], []
    for l, (W, b) in enumerate(layers):
        hs.append(h)
        z = h @ W.T + b
        zs.append(z)
        h = np.maximum(z, 0.0) if l + 1 < len(layers) else z
    return h, hs, zs


def loss_and_grads(params, dims, X, T):
    out, hs, zs = forward(params, dims, X)
    T = np.asarray(T, dtype=np.float64)
    n = out.size
    d = out - T
    loss = float(np.sum(d * d) / n)
    layers = unpack(params, dims)
    g = []
    dz = 2.0 * d / n
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        dW = dz.T @ hs[l]
        db = dz.sum(axis=0)
        g.append((dW, db))
        if l > 0:
            dz = (dz @ W) * (zs[l - 1] > 0.0)
    g.reverse()
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in g])
    return loss, flat


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
