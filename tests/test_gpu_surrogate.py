"""GPU checks of the learned pre-ranker: its BF16 tensor-core forward and backward kernels against
the float64 reference network (same BF16-rounded weights), training on a teacher network, the
dB targets, and the pre-ranked search step against exhaustive exact evaluation.

Tolerances: activations and output gradients are stored in BF16 (8 significant bits) between
layers, so the GPU agrees with the float64 reference to a few BF16 roundings: relative Frobenius
error 2e-2 for outputs and 5e-2 for each layer's gradient.
"""
import numpy as np
import pytest

import pmom_inputs as PI
from oracle import mlp as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import surrogate
    return surrogate


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("dims,B", [([512, 256, 256, 164], 256), ([200, 96, 20], 70), ([37, 130, 9], 300)])
def test_forward_and_gradients_match_reference(S, dims, B):
    """Ragged sizes (not multiples of the 128 x 128 tile or of the 64-wide K chunk) included."""
    net = S.MLP(dims, seed=3)
    rng = np.random.default_rng(1)
    p = net.params()
    pb = R.bf16_round(p)            # the kernels use BF16 copies of the weights; biases stay FP32
    for l, (wo, bo) in enumerate(zip(*_offsets(dims))):
        pb[bo:bo + dims[l + 1]] = p[bo:bo + dims[l + 1]]
    X = (rng.random((B, dims[0])) < 0.5).astype(np.uint8)
    T = rng.normal(size=(B, dims[-1])).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    t = torch.from_numpy(T).cuda()
    y = net.forward(x).cpu().numpy()
    y_ref, _, _ = R.forward(pb, dims, X)
    assert _rel(y, y_ref) <= 2e-2, _rel(y, y_ref)
    loss = net.backward(x, t)
    loss_ref, g_ref = R.loss_and_grads(pb, dims, X, T)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    g = net.grads()
    for l, (wo, bo) in enumerate(zip(*_offsets(dims))):
        nw = dims[l + 1] * dims[l]
        assert _rel(g[wo:wo + nw], g_ref[wo:wo + nw]) <= 5e-2, (l, "W", _rel(g[wo:wo + nw], g_ref[wo:wo + nw]))
        assert _rel(g[bo:bo + dims[l + 1]], g_ref[bo:bo + dims[l + 1]]) <= 5e-2, (l, "b")
    assert net.timeouts() == 0
    net.close()


def _offsets(dims):
    wo, bo, off = [], [], 0
    for l in range(len(dims) - 1):
        wo.append(off)
        off += dims[l + 1] * dims[l]
        bo.append(off)
        off += dims[l + 1]
    return wo, bo


def test_training_learns_a_teacher(S):
    """A student of the same shape fitted to a random teacher's outputs: the loss falls by 10x."""
    dims = [128, 128, 32]
    teacher = S.MLP(dims, seed=11)
    rng = np.random.default_rng(2)
    X = torch.from_numpy((rng.random((4096, 128)) < 0.5).astype(np.uint8)).cuda()
    T = teacher.forward(X).contiguous()
    student = S.MLP(dims, seed=12)
    hist = S.train(student, X, T, epochs=30, batch=256, lr=2e-3)
    assert hist[-1] < 0.1 * hist[0], hist
    teacher.close()
    student.close()


@pytest.fixture(scope="module")
def search_case(S):
    """16x16x2 stripline (41 frequencies, complex64 database from the library's GPU fill): a greedy
    trajectory of exact single-flip steps from a seeded map; every step's 512 evaluated children
    are the pre-ranker's training data (the data a search produces anyway)."""
    from paper_2412_17617_gb300 import Evaluator, band_codes
    w = PI.workload_precision()
    ev = Evaluator(w.grid)
    ev.fill_Z(w.freqs(), "c64")
    codes = band_codes(w.freqs(), w.bands)
    ev.set_fom(codes)
    bands = torch.from_numpy(np.ascontiguousarray(codes)).cuda()
    cur = PI.seed_map(w.grid, w.fill, 0)
    xs, ts, steps = [], [], []
    for it in range(14):
        kids = PI.single_flip_batch(cur, 2)
        dk = torch.from_numpy(kids).cuda()
        Sx, fom, status = ev.eval_bordered(torch.from_numpy(cur).cuda(), dk, "mixed")
        assert int((status != 0).sum()) == 0
        f = fom.cpu().numpy()
        steps.append((cur.copy(), kids, f))
        xs.append(dk.reshape(dk.shape[0], -1))
        ts.append(S.targets(Sx))
        cur = kids[int(np.argmin(f))]
    yield w, ev, bands, xs, ts, steps
    ev.close()


def test_targets_are_db_of_the_fom_entries(S, search_case):
    w, ev, bands, xs, ts, steps = search_case
    cur, kids, f = steps[0]
    Sx, fom, _ = ev.eval(torch.from_numpy(kids[:4]).cuda(), "mixed")
    t = S.targets(Sx).cpu().numpy()
    s = Sx.cpu().numpy()
    F = w.n_freq
    for q, (i, j) in enumerate(((0, 0), (1, 0), (2, 0), (2, 1))):
        ref = 20 * np.log10(np.maximum(np.abs(s[:, :, i, j]), 1e-15)) * S.OUT_SCALE
        assert np.abs(t[:, q * F:(q + 1) * F] - ref).max() <= 1e-5


def test_preranking_beats_random_selection(S, search_case):
    """Train on the first 11 steps' children, then for the next three steps rank the 512 children
    and exact-evaluate only the top 32: the best FoM found must beat the expected best of 32
    children drawn at random (computed exactly from the exhaustive evaluation), on average over
    the three steps; the exact evaluation of the selected children is the arbiter."""
    w, ev, bands, xs, ts, steps = search_case
    n_train, k = 11, 32
    X = torch.cat(xs[:n_train]).contiguous()
    T = torch.cat(ts[:n_train]).contiguous()
    D = X.shape[1]
    net = S.MLP([D, 512, 512, 4 * w.n_freq], seed=7)
    hist = S.train(net, X, T, epochs=40, batch=256, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    ours, rand = [], []
    for cur, kids, f in steps[n_train:]:
        j, fj, top = S.preranked_step(ev, net, bands, torch.from_numpy(cur).cuda(), torch.from_numpy(kids).cuda(), k)
        assert abs(fj - f[j]) <= 1e-6 * abs(f[j])        # the exact FoM of the chosen child
        # expected minimum of k of the n children drawn without replacement
        fs = np.sort(f)
        n = fs.size
        from math import comb
        pr = np.array([comb(n - 1 - i, k - 1) / comb(n, k) for i in range(n)])
        e_rand = float(np.sum(pr * fs))
        best = float(fs[0])
        ours.append((fj - best) / abs(best))
        rand.append((e_rand - best) / abs(best))
    print("relative regret: pre-ranked", ours, "random", rand)
    assert np.mean(ours) < np.mean(rand), (ours, rand)
    net.close()
