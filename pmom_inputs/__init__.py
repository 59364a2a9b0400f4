"""Seeded synthetic workloads for the pre-computed MoM candidate evaluator.

This module holds workload *data* only: stack-up and pixel-grid descriptions, port sites,
frequency sweeps, band edges, seed pixel maps and candidate batches.  It contains none of the
method's arithmetic (no mesh, no Green's function, no fill, no solve, no S-parameters, no FoM),
so that both the CPU oracle and the CUDA library can consume the same inputs without sharing
any of the computation they are compared on.

Geometry sources (paper): pixel pitch / map size / stack-up from Table I; eps_r = 3.66 and
tan(delta) = 0.004 for Rogers 4350B from Section IV; the channel bands 5.15-5.925 GHz and
6.425-7.125 GHz and the 3-9 GHz scoring range from Section III-B (Eq. 8-9).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

# Port sides: the feed stub leaves the pixel grid through this edge of the map.
SIDE_RIGHT, SIDE_TOP, SIDE_LEFT, SIDE_BOTTOM = 0, 1, 2, 3

MEDIUM_MICROSTRIP = 0   # metal layers over one ground plane at z = 0
MEDIUM_STRIPLINE = 1    # metal layers between ground planes at z = 0 and z = h_total


@dataclass(frozen=True)
class Port:
    layer: int
    side: int
    pos: int


@dataclass(frozen=True)
class Grid:
    """Pixel grid + stack-up.  Pixel (l, x, y) covers [x*a, (x+1)*a] x [y*a, (y+1)*a] at z = layer_z[l]."""
    name: str
    layers: int
    nx: int
    ny: int
    pitch_m: float
    medium: int
    layer_z_m: Tuple[float, ...]
    h_total_m: float
    eps_r: float
    tan_d: float
    n_states: int
    ports: Tuple[Port, ...]
    diag_pattern: int = 0     # pixel diagonals: 0 alternating, 1 uniform, 2 random (seeded by diag_seed)
    diag_seed: int = 0
    sub: int = 1              # sub-squares per pixel side: 1, 2, 3 = 2, 8, 18 triangles per pixel

    @property
    def n_pixels(self) -> int:
        return self.layers * self.ny * self.nx

    @property
    def n_ports(self) -> int:
        return len(self.ports)


@dataclass(frozen=True)
class Bands:
    """Band edges in Hz.  p1/p2 inclusive, i exclusive, s = the rest of [s_lo, s_hi]."""
    p1: Tuple[float, float]
    p2: Tuple[float, float]
    i: Tuple[float, float]
    s: Tuple[float, float]


@dataclass(frozen=True)
class Workload:
    name: str
    grid: Grid
    f_lo_hz: float
    f_hi_hz: float
    n_freq: int
    fill: float
    batch: int
    z_dtype: str          # "c128" or "c64": storage precision of the pre-computed Z database
    bands: Bands
    z0_ohm: float = 50.0

    def freqs(self) -> np.ndarray:
        return np.linspace(self.f_lo_hz, self.f_hi_hz, self.n_freq)


# ----------------------------------------------------------------------------------------
# Workloads shaped like the paper's diplexers.
# ----------------------------------------------------------------------------------------
H_RO4350 = 0.4866e-3          # dielectric thickness between consecutive planes (Table I)
UNII_BANDS = Bands(p1=(5.15e9, 5.925e9), p2=(6.425e9, 7.125e9), i=(5.925e9, 6.425e9), s=(3e9, 9e9))
# the 8x8 plain case scores channels around 2.4 and 5.2 GHz on a 1-6 GHz sweep
PLAIN_BANDS = Bands(p1=(1.9e9, 2.9e9), p2=(4.7e9, 5.7e9), i=(2.9e9, 4.7e9), s=(1e9, 6e9))


def _three_side_ports(n: int, layer: int = 0) -> Tuple[Port, ...]:
    # port 1 right, port 2 top, port 3 left (Section IV-A port naming)
    mid = n // 2
    return (Port(layer, SIDE_RIGHT, mid), Port(layer, SIDE_TOP, mid), Port(layer, SIDE_LEFT, mid))


def grid_plain_8x8() -> Grid:
    return Grid("plain_8x8_microstrip", 1, 8, 8, 2.0e-3, MEDIUM_MICROSTRIP, (0.5e-3,), 0.5e-3,
                3.5, 0.0, 2, _three_side_ports(8))


def grid_stripline_16x16x2() -> Grid:
    # port 1 right (lower layer); ports 2 and 3 leave on the left, on the lower and upper layer
    h = H_RO4350
    ports = (Port(0, SIDE_RIGHT, 8), Port(0, SIDE_LEFT, 8), Port(1, SIDE_LEFT, 8))
    return Grid("stripline_16x16x2", 2, 16, 16, 0.5625e-3, MEDIUM_STRIPLINE, (h, 2 * h), 3 * h,
                3.66, 0.004, 2, ports)


def grid_stripline_20x20x3(n_states: int = 3) -> Grid:
    """3-layer 20x20 stripline; n_states = 3 adds the via state (void / metal / via to the next
    layer), n_states = 2 is the same stack-up with on/off pixels only."""
    h = H_RO4350
    ports = (Port(0, SIDE_RIGHT, 10), Port(0, SIDE_LEFT, 10), Port(2, SIDE_LEFT, 10))
    name = "stripline_20x20x3_via" if n_states == 3 else "stripline_20x20x3"
    return Grid(name, 3, 20, 20, 0.45e-3, MEDIUM_STRIPLINE, (h, 2 * h, 3 * h), 4 * h, 3.66, 0.004, n_states, ports)


def grid_stripline_32x32x4() -> Grid:
    h = H_RO4350
    ports = (Port(0, SIDE_RIGHT, 16), Port(0, SIDE_LEFT, 16), Port(1, SIDE_LEFT, 16), Port(3, SIDE_BOTTOM, 16))
    return Grid("stripline_32x32x4", 4, 32, 32, 0.3e-3, MEDIUM_STRIPLINE, tuple(h * (i + 1) for i in range(4)),
                5 * h, 3.66, 0.004, 2, ports)


def grid_microstrip_24x24x3() -> Grid:
    """3-layer 24x24 microstrip of 0.4 mm pixels (the 8-state pixel = three on/off layers, Section
    IV-B), Rogers 4350B layers of 0.4866 mm over one ground plane; ports 1 right, 2 top, 3 left on
    the top layer."""
    h = H_RO4350
    return Grid("microstrip_24x24x3", 3, 24, 24, 0.4e-3, MEDIUM_MICROSTRIP, (h, 2 * h, 3 * h), 3 * h, 3.66, 0.004,
                2, _three_side_ports(24, layer=2))


def grid_tiny(n: int = 3, medium: int = MEDIUM_MICROSTRIP, layers: int = 1, pitch_m: float = 2.0e-3) -> Grid:
    """Small grids for brute force and oracle pins."""
    if medium == MEDIUM_MICROSTRIP:
        zs = tuple(0.5e-3 * (i + 1) for i in range(layers))
        return Grid(f"tiny_{n}x{n}x{layers}_microstrip", layers, n, n, pitch_m, medium, zs, zs[-1], 3.5, 0.0, 2,
                    _three_side_ports(n))
    h = H_RO4350
    zs = tuple(h * (i + 1) for i in range(layers))
    ports = (Port(0, SIDE_RIGHT, n // 2), Port(0, SIDE_LEFT, n // 2), Port(layers - 1, SIDE_TOP, n // 2))
    return Grid(f"tiny_{n}x{n}x{layers}_stripline", layers, n, n, pitch_m, medium, zs, h * (layers + 1),
                3.66, 0.004, 2, ports)


def workload_plain() -> Workload:
    """8x8 single-layer microstrip, 11 frequencies 1-6 GHz, complex128 Z, 64 single-pixel flips."""
    return Workload("plain_8x8_f11_b64", grid_plain_8x8(), 1e9, 6e9, 11, 0.5, 64, "c128", PLAIN_BANDS)


def workload_precision() -> Workload:
    """2-layer 16x16 stripline, 41 frequencies 1-7 GHz, complex64 Z, 512 single-bit flips."""
    return Workload("stripline_16x16x2_f41_b512", grid_stripline_16x16x2(), 1e9, 7e9, 41, 0.65, 512, "c64",
                    UNII_BANDS)


def workload_profile() -> Workload:
    """A smaller stripline case (2-layer 10x10, 41 frequencies, complex64) that runs the same
    kernels as the 16x16x2 case with a device footprint small enough for counter captures."""
    h = H_RO4350
    g = Grid("stripline_10x10x2", 2, 10, 10, 0.9e-3, MEDIUM_STRIPLINE, (h, 2 * h), 3 * h, 3.66, 0.004, 2,
             (Port(0, SIDE_RIGHT, 5), Port(0, SIDE_LEFT, 5), Port(1, SIDE_LEFT, 5)))
    return Workload("stripline_10x10x2_f41_b200", g, 1e9, 7e9, 41, 0.65, 200, "c64", UNII_BANDS)


def workload_batching() -> Workload:
    return Workload("stripline_20x20x3_f101_b4096", grid_stripline_20x20x3(), 0.5e9, 8e9, 101, 0.5, 4096, "c64",
                    UNII_BANDS)


def workload_learned() -> Workload:
    """The pre-ranker's configuration: 3-layer 24x24 microstrip, 64 frequencies 3-9 GHz, complex64,
    candidate pools of 10k changes per search step."""
    return Workload("microstrip_24x24x3_f64_b10000", grid_microstrip_24x24x3(), 3e9, 9e9, 64, 0.5, 10000, "c64",
                    UNII_BANDS)


def workload_scale() -> Workload:
    return Workload("stripline_32x32x4_f101_b64", grid_stripline_32x32x4(), 0.5e9, 8e9, 101, 0.5, 64, "c64",
                    UNII_BANDS)


WORKLOADS = {w.name: w for w in (workload_plain(), workload_precision())}


# ----------------------------------------------------------------------------------------
# Seeded maps and candidate batches (numpy PCG64).
# ----------------------------------------------------------------------------------------
def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def seed_map(grid: Grid, fill: float, seed: int) -> np.ndarray:
    """uint8 [layers][ny][nx]; each pixel metal (state 1) with probability `fill`, else void (0)."""
    g = rng(seed)
    return (g.random((grid.layers, grid.ny, grid.nx)) < fill).astype(np.uint8)


def single_flip_batch(seed: np.ndarray, n_states: int = 2) -> np.ndarray:
    """Every single-pixel change of `seed`: for each pixel (row-major over layer, y, x) and each
    other state of that pixel, one candidate.  Shape [B][layers][ny][nx], uint8."""
    L, ny, nx = seed.shape
    out = []
    for l in range(L):
        for y in range(ny):
            for x in range(nx):
                for s in range(n_states):
                    if s == seed[l, y, x]:
                        continue
                    c = seed.copy()
                    c[l, y, x] = s
                    out.append(c)
    return np.ascontiguousarray(np.stack(out).astype(np.uint8))


def depth_flips(seed: np.ndarray, depth: int, count: int, n_states: int, rng_seed: int) -> np.ndarray:
    """`count` candidates that each change `depth` distinct pixels of `seed` to another state
    (pixels and new states drawn uniformly).  Shape [count][layers][ny][nx], uint8."""
    g = rng(rng_seed)
    out = np.repeat(seed[None], count, axis=0).astype(np.uint8)
    flat = out.reshape(count, -1)
    for c in range(count):
        pix = g.choice(flat.shape[1], size=depth, replace=False)
        for j in pix:
            s = int(g.integers(n_states - 1))
            flat[c, j] = s if s < flat[c, j] else s + 1
    return np.ascontiguousarray(out)


def random_maps(grid: Grid, count: int, fill: float, seed: int) -> np.ndarray:
    g = rng(seed)
    return (g.random((count, grid.layers, grid.ny, grid.nx)) < fill).astype(np.uint8)


def workload_maps(w: Workload, seed: int = 0) -> np.ndarray:
    """The candidate batch of a workload: all single flips of a seeded map, trimmed/tiled to w.batch
    (three-state grids: `batching_maps`)."""
    if w.grid.n_states == 3:
        return batching_maps(w, seed)
    base = seed_map(w.grid, w.fill, seed)
    flips = single_flip_batch(base, 2)
    if flips.shape[0] >= w.batch:
        return np.ascontiguousarray(flips[: w.batch])
    reps = -(-w.batch // flips.shape[0])
    return np.ascontiguousarray(np.concatenate([flips] * reps)[: w.batch])


def all_maps(grid: Grid) -> np.ndarray:
    """Every on/off map of a (tiny) grid, in binary counting order over row-major pixels."""
    n = grid.n_pixels
    codes = np.arange(1 << n, dtype=np.int64)
    bits = ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    return np.ascontiguousarray(bits.reshape(-1, grid.layers, grid.ny, grid.nx))


def seed_map_vias(grid: Grid, fill: float, via_frac: float, seed: int) -> np.ndarray:
    """uint8 [layers][ny][nx] with three states: each pixel metal with probability `fill`; a
    metal pixel below the last layer is a via (state 2) with probability `via_frac`."""
    g = rng(seed)
    shape = (grid.layers, grid.ny, grid.nx)
    m = (g.random(shape) < fill).astype(np.uint8)
    v = (g.random(shape) < via_frac) & (m == 1)
    v[-1] = False
    m[v] = 2
    return m


def state_changes(seed: np.ndarray, depth: int, count: int, rng_seed: int) -> np.ndarray:
    """`count` candidates that each change `depth` distinct pixels of a three-state map to another
    state, drawn uniformly among the pixel's valid states (the last layer has no via state).
    Shape [count][layers][ny][nx], uint8."""
    g = rng(rng_seed)
    L, ny, nx = seed.shape
    out = np.repeat(seed[None], count, axis=0).astype(np.uint8)
    flat = out.reshape(count, -1)
    for c in range(count):
        for j in g.choice(flat.shape[1], size=depth, replace=False):
            k = 2 if j >= (L - 1) * ny * nx else 3
            s = int(g.integers(k - 1))
            flat[c, j] = s if s < flat[c, j] else s + 1
    return np.ascontiguousarray(out)


BATCHING_FILLS = tuple(float(f) for f in np.linspace(0.35, 0.75, 8))


def batching_maps(w: Workload, seed: int = 0, count: int = 0) -> np.ndarray:
    """Candidates of the three-state batching workload: eight seed maps of per-layer fill 0.35 ..
    0.75 (20 % of the metal pixels below the top layer are vias), candidate i changing 1 + (i // 8) % 3
    random pixels of seed i % 8, so every prefix of the batch spans the support-set sizes of all
    seeds (about 950 to 2500 on the 20 x 20 x 3 grid).  Shape [count][layers][ny][nx], uint8."""
    count = count or w.batch
    seeds = [seed_map_vias(w.grid, f, 0.2, 1000 * seed + k) for k, f in enumerate(BATCHING_FILLS)]
    out = np.empty((count, w.grid.layers, w.grid.ny, w.grid.nx), np.uint8)
    for i in range(count):
        out[i] = state_changes(seeds[i % len(seeds)], 1 + (i // len(seeds)) % 3, 1, 7919 * seed + i)[0]
    return np.ascontiguousarray(out)
