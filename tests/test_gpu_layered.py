"""GPU fill of the layered microstrip (medium 2: PEC ground, dielectric slab up to the highest metal
layer, air above; the mixed-potential kernels of Section II-D's layered-media MPIE by Sommerfeld
integrals) against the oracle's fill entry by entry, the air-slab limit against the homogeneous
image fill, and both evaluation precisions on a layered database against the oracle's solve."""
import dataclasses

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


def _gpu_fill(pm, g, freqs):
    ev = pm.Evaluator(g)
    ev.fill_Z(freqs, "c128")
    Z = ev.copy_Z().cpu().numpy()
    return ev, Z


@pytest.mark.parametrize("layers", [1, 2])
def test_layered_fill_matches_oracle(pm, layers):
    """One and two metal layers in a Rogers-like slab (eps_r 3.66, tan d 0.004): every entry within
    1e-9 of max |Z| (the two-layer case exercises the tables between different heights)."""
    g = dataclasses.replace(PI.grid_tiny(3, PI.MEDIUM_MICROSTRIP, layers), medium=2, eps_r=3.66, tan_d=0.004)
    freqs = [2.4e9, 5.2e9] if layers == 1 else [3.0e9]
    Zr, _ = O.fill(O.Grid(g), freqs)
    ev, Zg = _gpu_fill(pm, g, freqs)
    ev.close()
    for f in range(len(freqs)):
        assert np.abs(Zg[f] - Zr[f]).max() <= 1e-9 * np.abs(Zr[f]).max()


def test_air_slab_equals_image_fill(pm):
    """With eps_r = 1 the grounded slab is free space over a ground plane: the tabulated Sommerfeld
    kernels reproduce the closed-form image pair of medium 0 to interpolation accuracy."""
    g0 = dataclasses.replace(PI.grid_tiny(3), eps_r=1.0, tan_d=0.0)
    freqs = [2.4e9, 5.2e9]
    ev0, Z0 = _gpu_fill(pm, g0, freqs)
    ev2, Z2 = _gpu_fill(pm, dataclasses.replace(g0, medium=2), freqs)
    ev0.close()
    ev2.close()
    assert np.abs(Z2 - Z0).max() <= 1e-7 * np.abs(Z0).max()


def test_layered_database_evaluation(pm):
    """A 4 x 4 layered microstrip: the oracle's layered database loaded into the library, every
    candidate of a seeded batch in both precisions against the oracle's solve; the library's own
    layered fill of the same grid is checked against that database too."""
    g = dataclasses.replace(PI.grid_tiny(4), medium=2, eps_r=3.5, tan_d=0.0, name="layered_4x4")
    freqs = np.array([2.0e9, 2.4e9, 5.2e9])
    OG = O.Grid(g)
    Zr, _ = O.fill(OG, freqs)
    maps = PI.random_maps(g, 12, 0.5, 7)
    S_ref, st = O.eval_batch(OG, Zr, maps)
    assert (st == 0).all()
    bands = O.bands(freqs, PI.PLAIN_BANDS)
    fom_ref = O.fom_batch(S_ref, bands)
    ev = pm.Evaluator(g)
    ev.load_Z(freqs, torch.from_numpy(Zr).cuda())
    ev.set_fom(pm.band_codes(freqs, PI.PLAIN_BANDS))
    dm = torch.from_numpy(maps).cuda()
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        S, fom, status = ev.eval(dm, prec)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all()
        assert np.abs(S.cpu().numpy() - S_ref).max() <= tol * max(1.0, np.abs(S_ref).max())
        assert (np.abs(fom.cpu().numpy() - fom_ref) <= tol * np.abs(fom_ref)).all()
    ev.fill_Z(freqs, "c128")
    Zg = ev.copy_Z().cpu().numpy()
    ev.close()
    for f in range(len(freqs)):
        assert np.abs(Zg[f] - Zr[f]).max() <= 1e-9 * np.abs(Zr[f]).max()
