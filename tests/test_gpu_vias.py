"""GPU checks of the via state (three pixel states): the support set of every map of a small
two-layer grid bit-exact against the oracle (including the rejected via on the last layer), and
the GPU fill of a grid with via strips (vertical triangles, Neumann kernel for vertical currents)
against the oracle's fill entry by entry."""
import dataclasses
import itertools

import numpy as np
import pytest

import pmom_inputs as PI
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    from paper_2412_17617_gb300 import build as B
    B.build()
    from paper_2412_17617_gb300 import pmom
    return pmom


def via_grid(n, pitch=0.5e-3):
    g = PI.grid_tiny(n, PI.MEDIUM_STRIPLINE, 2, pitch_m=pitch)
    return dataclasses.replace(g, name=f"via_{n}x{n}x2", n_states=3)


def test_via_active_set_bit_exact(pm):
    g = via_grid(2)
    OG = O.Grid(g)
    maps = [np.array([lo, hi], np.uint8).reshape(2, 2, 2)
            for lo in itertools.product(range(3), repeat=4) for hi in itertools.product(range(2), repeat=4)]
    bad = np.zeros((2, 2, 2), np.uint8)
    bad[1, 0, 1] = 2                      # a via on the last layer
    allm = np.ascontiguousarray(np.stack(maps + [bad]))
    ev = pm.Evaluator(g)
    idx, n = ev.active_set(torch.from_numpy(allm).cuda())
    idx, n = idx.cpu().numpy(), n.cpu().numpy()
    for b in range(len(maps)):
        ref = O.active_set(OG, allm[b])
        assert n[b] == len(ref)
        assert np.array_equal(idx[b, : n[b]], ref)
    assert n[-1] == -1
    ev.close()


def test_gpu_fill_with_vias_matches_oracle_fill(pm):
    g = via_grid(4)
    freqs = [1.3e9, 6.1e9]
    OG = O.Grid(g)
    Zr, _ = O.fill(OG, freqs)
    ev = pm.Evaluator(g)
    ev.fill_Z(freqs, "c128")
    Zg = ev.copy_Z().cpu().numpy()
    for f in range(len(freqs)):
        assert np.abs(Zg[f] - Zr[f]).max() <= 1e-9 * np.abs(Zr[f]).max()
    ev.close()
