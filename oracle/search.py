"""Plain reference of the paper's depth-increasing all-way tree search (Algorithm 1, Section III-A).

TEST INFRASTRUCTURE ONLY (oracle side): it evaluates candidates with the CPU oracle.  The
library's native search (pmom_search) is checked against it decision by decision.

Readings where Algorithm 1 leaves a choice open:
  * a pixel is one (x, y) column; its state is the pattern of its layers' states, a mixed-radix
    number with layer 0 as the lowest digit (radix 2 per layer; radix 3 for the layers below the
    last one on a grid with the via state), so K = 2**layers states on an on/off grid; a node has
    K - 1 children, one per other state of the chosen column;
  * the column j of node (d, k) is drawn uniformly from the columns not yet on the node's path,
    with the counter-based SplitMix64 generator keyed by (seed, restart, iteration, d, k);
  * every child at every depth is evaluated; the best leaf is the argmin over depth-D leaves
    only (ties: lowest leaf index); it is accepted if strictly better than the current F;
  * after M(D) consecutive non-improving iterations the depth grows; when it would exceed Dmax
    the search restarts from a random map (each layer pixel metal with probability 1/2 from the top
    bit of the same generator; on a grid with vias a metal pixel below the last layer is a via when
    the next bit is set) at depth 1, keeping the global best;
  * the search stops once the evaluation budget is used up (a started tree is finished);
  * a candidate whose evaluation failed (non-finite FoM) counts as +infinity.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(x: int) -> int:
    """One output of SplitMix64 (Steele, Lea and Flood, 2014) from state x (state advanced first)."""
    z = (x + GOLDEN) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def key(*parts: int) -> int:
    h = 0
    for p in parts:
        h = splitmix64(h ^ (p & MASK))
    return h


def radices(L: int, n_states: int = 2):
    """Number of states of each layer's pixel in a column (the last layer holds no via)."""
    return [3 if (n_states >= 3 and l < L - 1) else 2 for l in range(L)]


def random_map(seed: int, restart: int, shape, n_states: int = 2) -> np.ndarray:
    L, ny, nx = shape
    out = np.zeros(shape, np.uint8)
    for i in range(L * ny * nx):
        u = key(seed, 0xA5A5, restart, i)
        s = u >> 63
        if s and n_states >= 3 and i < (L - 1) * ny * nx:
            s = 1 + ((u >> 62) & 1)
        out.flat[i] = s
    return out


def column_state(m: np.ndarray, j: int, n_states: int = 2) -> int:
    L, ny, nx = m.shape
    y, x = divmod(j, nx)
    v, w = 0, 1
    for l, r in enumerate(radices(L, n_states)):
        v += int(m[l, y, x]) * w
        w *= r
    return v


def set_column(m: np.ndarray, j: int, s: int, n_states: int = 2) -> np.ndarray:
    L, ny, nx = m.shape
    y, x = divmod(j, nx)
    c = m.copy()
    for l, r in enumerate(radices(L, n_states)):
        c[l, y, x] = s % r
        s //= r
    return c


def tree_search(evaluate, init_map: np.ndarray, seed: int, d_max: int, m_of_d, max_evals: int, n_states: int = 2,
                state: dict = None, return_state: bool = False):
    """evaluate(maps[B][L][ny][nx]) -> FoM[B].  Returns (best_map, best_F, evals, trace) where
    trace[i] is the current F after iteration i of this call; with return_state also the search
    state (current map and F, best map and F, evaluation count, depth, counter, restart and
    iteration keys), from which a later call with state=... continues exactly as the uninterrupted
    search would (max_evals counts every evaluation since the start)."""
    L, ny, nx = init_map.shape
    ncol, K = ny * nx, int(np.prod(radices(L, n_states)))
    if not 1 <= d_max <= ncol:
        raise ValueError(f"d_max = {d_max}: a depth-D tree changes D distinct columns of the {ncol} on the grid")
    if state is not None and not 1 <= int(state["depth"]) <= d_max:
        raise ValueError("resumed depth outside 1..d_max")

    def F_of(maps):
        f = np.asarray(evaluate(np.ascontiguousarray(maps)), dtype=np.float64)
        return np.where(np.isfinite(f), f, np.inf)

    if state is None:
        P = init_map.copy()
        F = float(F_of(P[None])[0])
        evals = 1
        best_P, best_F = P.copy(), F
        D, counter, restart, it = 1, 0, 0, 0
    else:
        P, F = state["map"].copy(), float(state["fom"])
        best_P, best_F = state["best_map"].copy(), float(state["best_fom"])
        evals, D, counter = int(state["evals"]), int(state["depth"]), int(state["counter"])
        restart, it = int(state["restart"]), int(state["iteration"])
    trace = []
    while evals < max_evals:
        nodes = [(frozenset(), P)]
        Fs = None
        for d in range(D):
            children = []
            for k, (S, Pn) in enumerate(nodes):
                free = [c for c in range(ncol) if c not in S]
                j = free[key(seed, restart, it, d, k) % len(free)]
                cur = column_state(Pn, j, n_states)
                for s in range(K):
                    if s != cur:
                        children.append((S | {j}, set_column(Pn, j, s, n_states)))
            Fs = F_of(np.stack([c[1] for c in children]))
            evals += len(children)
            nodes = children
        b = int(np.argmin(Fs))
        if Fs[b] < F:
            P, F = nodes[b][1], float(Fs[b])
            counter = 0
        else:
            counter += 1
        if F < best_F:
            best_P, best_F = P.copy(), F
        if counter >= m_of_d[D - 1]:
            D += 1
            counter = 0
        if D > d_max:
            restart += 1
            P = random_map(seed, restart, (L, ny, nx), n_states)
            F = float(F_of(P[None])[0])
            evals += 1
            D, counter = 1, 0
            if F < best_F:
                best_P, best_F = P.copy(), F
        trace.append(F)
        it += 1
    if return_state:
        st = {"map": P.copy(), "fom": F, "best_map": best_P.copy(), "best_fom": best_F, "evals": evals, "depth": D,
              "counter": counter, "restart": restart, "iteration": it}
        return best_P, best_F, evals, trace, st
    return best_P, best_F, evals, trace
