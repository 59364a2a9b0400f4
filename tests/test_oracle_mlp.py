"""Pins of the pre-ranker network's float64 reference (CPU): its gradients against central finite
differences of its loss, the least-squares optimum of a one-layer (linear) network as a
stationary point, and the BF16 rounding helper against exact cases."""
import numpy as np

from oracle import mlp as R


def _params(dims, rng):
    parts = []
    for l in range(len(dims) - 1):
        parts.append(rng.normal(size=dims[l + 1] * dims[l]) / np.sqrt(dims[l]))
        parts.append(rng.normal(size=dims[l + 1]) * 0.1)
    return np.concatenate(parts)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    dims = [6, 5, 4, 3]
    p = _params(dims, rng)
    X = (rng.random((7, 6)) < 0.5).astype(np.float64)
    T = rng.normal(size=(7, 3))
    loss, g = R.loss_and_grads(p, dims, X, T)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (R.loss_and_grads(p + e, dims, X, T)[0] - R.loss_and_grads(p - e, dims, X, T)[0]) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-7 * max(1.0, np.abs(g).max())
    assert loss > 0


def test_linear_least_squares_optimum_is_stationary():
    rng = np.random.default_rng(6)
    dims = [8, 3]
    X = rng.normal(size=(40, 8))
    T = rng.normal(size=(40, 3))
    A = np.hstack([X, np.ones((40, 1))])
    sol, *_ = np.linalg.lstsq(A, T, rcond=None)   # [9 x 3]: rows of W^T then b
    p = np.concatenate([sol[:8].T.ravel(), sol[8]])
    loss, g = R.loss_and_grads(p, dims, X, T)
    assert np.abs(g).max() <= 1e-12
    # and the loss there is the least-squares residual
    assert abs(loss - np.sum((A @ sol - T) ** 2) / T.size) <= 1e-14


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3], dtype=np.float32)
    r = R.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # halfway between 1 and 1 + 2^-7: ties to even
    assert r[2] == np.float32(1.0 + 2 ** -6)  # halfway between 1 + 2^-7 and 1 + 2^-6: ties to even
    assert r[3] == -2.5
    assert abs(r[4] - 3.0e-3) <= 3.0e-3 * 2 ** -8
