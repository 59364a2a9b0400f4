"""ctypes front end of the plain C oracle (complex128).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``.  The library under test never imports it and shares no code
with it; both read the same seeded inputs from ``pmom_inputs``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SOURCES = ["or_mesh.c", "or_fill.c", "or_solve.c", "or_layered.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU needed)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    hdr = os.path.join(HERE, "pmom_oracle.h")
    newest = max(os.path.getmtime(p) for p in srcs + [hdr])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fcx-fortran-rules", "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _C128(ctypes.Structure):
    """C99 double complex (same register/memory layout as a struct of two doubles)."""
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class _Grid(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("pitch", ctypes.c_double), ("medium", ctypes.c_int),
                ("layer_z", ctypes.POINTER(ctypes.c_double)), ("h_total", ctypes.c_double),
                ("eps_r", ctypes.c_double), ("tan_d", ctypes.c_double), ("n_states", ctypes.c_int),
                ("n_ports", ctypes.c_int), ("ports", ctypes.POINTER(ctypes.c_int32)),
                ("diag_pattern", ctypes.c_int), ("diag_seed", ctypes.c_uint64), ("sub", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.or_count_bfs.argtypes = [P]
            L.or_bf_table.argtypes = [P, P]
            L.or_active_set.argtypes = [P, P, ctypes.c_int, P, P]
            L.or_fill.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.or_fill.restype = ctypes.c_double
            L.or_fill_subset.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P]
            L.or_fill_subset.restype = ctypes.c_double
            for fn in ("or_green", "or_green_modal"):
                getattr(L, fn).argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double]
                getattr(L, fn).restype = _C128
            L.or_green_images.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
            L.or_green_images.restype = _C128
            for fn in ("or_bessel_k0", "or_bessel_k0_any"):
                getattr(L, fn).argtypes = [_C128]
                getattr(L, fn).restype = _C128
            L.or_green_heights.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int]
            L.or_green_heights.restype = _C128
            L.or_slab_green.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
            L.or_slab_green.restype = _C128
            L.or_tri_potentials.argtypes = [P, P, P, P]
            L.or_tri_rule.argtypes = [ctypes.c_int, P, P]
            L.or_eps_eff.argtypes = [P]
            L.or_eps_eff.restype = ctypes.c_double
            L.or_lu.argtypes = [P, ctypes.c_int, P]
            L.or_lu_solve.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int]
            L.or_eval_map.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_double,
                                      ctypes.c_int, P]
            L.or_eval_batch.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, P, P]
            L.or_fom.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
            L.or_fom.restype = ctypes.c_double
            L.or_bands.argtypes = [P, ctypes.c_int, P, P]
            L.or_triangle.argtypes = [P, ctypes.c_int32, P]
            L.or_orient.argtypes = [P, ctypes.c_int, ctypes.c_int]
            L.or_stub_bfs.argtypes = [P]
            L.or_port_gap.argtypes = [P, ctypes.c_int, P]
            L.or_pair_integrals.argtypes = [P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Grid:
    """Holds the C descriptor (and keeps its arrays alive)."""

    def __init__(self, g):
        self.src = g
        self._z = np.ascontiguousarray(np.array(g.layer_z_m, dtype=np.float64))
        self._ports = np.ascontiguousarray(np.array([[p.layer, p.side, p.pos] for p in g.ports], dtype=np.int32))
        self.c = _Grid(g.layers, g.nx, g.ny, g.pitch_m, g.medium,
                       self._z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), g.h_total_m, g.eps_r, g.tan_d,
                       g.n_states, len(g.ports), self._ports.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       getattr(g, "diag_pattern", 0), getattr(g, "diag_seed", 0), getattr(g, "sub", 1))
        if getattr(g, "sub", 1) not in (1, 2, 3) or (getattr(g, "sub", 1) > 1 and g.n_states > 2):
            raise ValueError("sub-squares per pixel side: 1, 2 or 3; the via state needs 1")
        if g.medium == 2 and g.n_states > 2:
            raise ValueError("the layered microstrip kernels are for horizontal currents: no via state")
        self.ref = ctypes.byref(self.c)
        self.M = lib().or_count_bfs(self.ref)
        self.P = len(g.ports)
        self.table = np.zeros((self.M, 8), dtype=np.int32)
        n = lib().or_bf_table(self.ref, _ptr(self.table))
        assert n == self.M


def _c(z):
    return complex(z.re, z.im)


def bf_table(grid: Grid) -> np.ndarray:
    return grid.table.copy()


def active_set(grid: Grid, pixel_map: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(pixel_map, dtype=np.uint8)
    idx = np.zeros(grid.M, dtype=np.int32)
    n = lib().or_active_set(grid.ref, _ptr(grid.table), grid.M, _ptr(m), _ptr(idx))
    if n < 0:
        raise ValueError("pixel state out of range")
    return idx[:n].copy()


def fill(grid: Grid, freqs, mode: int = 1, threads: int = 0):
    """Parent Z(f), complex128 [F][M][M], symmetrised; also the pre-symmetrisation asymmetry."""
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
    Z = np.zeros((len(f), grid.M, grid.M), dtype=np.complex128)
    if threads <= 0:
        threads = min(len(f), os.cpu_count() or 1)
    asym = lib().or_fill(grid.ref, _ptr(f), len(f), mode, threads, _ptr(Z))
    return Z, asym


def fill_subset(grid: Grid, freqs, bf, mode: int = 0, threads: int = 0):
    """Z of the sub-structure made of BFs `bf` only, filled directly ([F][N][N], symmetrised)."""
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(bf, dtype=np.int32))
    Z = np.zeros((len(f), len(b), len(b)), dtype=np.complex128)
    if threads <= 0:
        threads = min(len(f), os.cpu_count() or 1)
    lib().or_fill_subset(grid.ref, _ptr(f), len(f), mode, threads, _ptr(b), len(b), _ptr(Z))
    return Z


def green(grid: Grid, freq: float, lp: int, lq: int, rho: float, route: str = "default", K: int = 64) -> complex:
    L = lib()
    if route == "images":
        return _c(L.or_green_images(grid.ref, freq, lp, lq, rho, K))
    if route == "modal":
        return _c(L.or_green_modal(grid.ref, freq, lp, lq, rho))
    return _c(L.or_green(grid.ref, freq, lp, lq, rho))


def slab_green(grid: Grid, freq: float, kind: int, z: float, zp: float, rho: float, er_top: float = 1.0,
               reg: bool = False):
    """Grounded-slab kernel (0: G_phi, 1: G_A) by Sommerfeld integrals; returns (G, C)."""
    c = ctypes.c_double(0.0)
    v = lib().or_slab_green(grid.ref, freq, kind, z, zp, rho, er_top, 1 if reg else 0, ctypes.byref(c))
    return _c(v), c.value


def bessel_k0(w: complex, any_arg: bool = False) -> complex:
    f = lib().or_bessel_k0_any if any_arg else lib().or_bessel_k0
    return _c(f(_C128(w.real, w.imag)))


def green_heights(grid: Grid, freq: float, kind: int, zp: float, zq: float, rho: float, route: str = "default",
                  K: int = 64) -> complex:
    """Kernel `kind` (0 Dirichlet: horizontal currents and charges; 1 Neumann: vertical currents)
    between arbitrary heights."""
    r = {"default": 0, "images": 1, "modal": 2}[route]
    return _c(lib().or_green_heights(grid.ref, freq, kind, zp, zq, rho, r, K))


def tri_potentials(tri: np.ndarray, r: np.ndarray):
    t = np.ascontiguousarray(tri, dtype=np.float64)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    i1 = np.zeros(1)
    iv = np.zeros(3)
    lib().or_tri_potentials(_ptr(t), _ptr(rr), _ptr(i1), _ptr(iv))
    return float(i1[0]), iv


def tri_rule(n: int):
    b = ctypes.POINTER(ctypes.c_double)()
    w = ctypes.POINTER(ctypes.c_double)()
    k = lib().or_tri_rule(n, ctypes.byref(b), ctypes.byref(w))
    return (np.ctypeslib.as_array(b, shape=(k, 3)).copy(), np.ctypeslib.as_array(w, shape=(k,)).copy())


def orient(grid: Grid, x: int, y: int) -> int:
    return lib().or_orient(grid.ref, x, y)


def triangle(grid: Grid, key: int) -> np.ndarray:
    v = np.zeros((3, 3))
    lib().or_triangle(grid.ref, int(key), _ptr(v))
    return v


def pair_integrals(grid: Grid, freq: float, kp: int, kq: int) -> np.ndarray:
    out = np.zeros(10, dtype=np.complex128)
    lib().or_pair_integrals(grid.ref, freq, int(kp), int(kq), _ptr(out))
    return out


def eps_eff(grid: Grid) -> float:
    return lib().or_eps_eff(grid.ref)


def lu(A: np.ndarray):
    a = np.ascontiguousarray(A, dtype=np.complex128).copy()
    piv = np.zeros(a.shape[0], dtype=np.int32)
    sing = lib().or_lu(_ptr(a), a.shape[0], _ptr(piv))
    return a, piv, sing


def lu_solve(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(B, dtype=np.complex128).copy()
    if b.ndim == 1:
        b = b[:, None]
    lib().or_lu_solve(_ptr(LU), _ptr(piv), LU.shape[0], _ptr(b), b.shape[1])
    return b


def _z_args(Z: np.ndarray):
    if Z.dtype == np.complex64:
        return np.ascontiguousarray(Z), 1
    return np.ascontiguousarray(Z, dtype=np.complex128), 0


def eval_map(grid: Grid, Z: np.ndarray, pixel_map: np.ndarray, Z0: float = 50.0, form: int = 0):
    """S[F][P][P] (complex128) for one map; status 0 ok, 1 singular."""
    z, zc64 = _z_args(Z)
    m = np.ascontiguousarray(pixel_map, dtype=np.uint8)
    S = np.zeros((z.shape[0], grid.P, grid.P), dtype=np.complex128)
    st = lib().or_eval_map(grid.ref, _ptr(grid.table), grid.M, _ptr(z), zc64, z.shape[0], _ptr(m), Z0, form, _ptr(S))
    if st < 0:
        raise ValueError("pixel state out of range")
    return S, st


def port_gaps(grid: Grid):
    """Per port: the canonical indices of its delta-gap BFs (3p + 1 alone with the two-triangle
    mesh) and their edge lengths (the edge opposite the free vertex of the positive triangle,
    Section II-C)."""
    out = []
    for p in range(grid.P):
        bf = np.zeros(3, np.int32)
        n = lib().or_port_gap(grid.ref, p, _ptr(bf))
        lens = []
        for m in bf[:n]:
            r = grid.table[int(m)]
            v = triangle(grid, int(r[4]))
            f = int(r[6])
            lens.append(float(np.linalg.norm(v[(f + 1) % 3] - v[(f + 2) % 3])))
        out.append((bf[:n].copy(), np.array(lens)))
    return out


def port_lengths(grid: Grid) -> np.ndarray:
    """Length of each port's delta-gap edge (two-triangle mesh: one gap BF per port)."""
    return np.array([lens[0] for _, lens in port_gaps(grid)])


def eval_map_lapack(grid: Grid, Z: np.ndarray, pixel_map: np.ndarray, Z0: float = 50.0) -> np.ndarray:
    """S[F][P][P] of one map by the same definition as eval_map -- gather Z_sub = Z(f)[I, I]
    (Eq. 5, complex64 storage promoted exactly to complex128), unit delta-gap excitation of each
    port's gap BFs, Y_ij = sum over port i's gap of l_k x_k^(j) and S = (1 + Z0 Y)^-1 (1 - Z0 Y)
    (Eq. 6-7) -- with LAPACK's
    dense solve (numpy.linalg.solve) as the solve step, for support sets of thousands of BFs
    where the plain C LU takes minutes."""
    idx = active_set(grid, pixel_map)
    P = grid.P
    gaps = port_gaps(grid)
    V = np.zeros((len(idx), P), np.complex128)
    for p, (bf, lens) in enumerate(gaps):
        pos = np.array([int(np.nonzero(idx == m)[0][0]) for m in bf])
        V[pos, p] = lens
    S = np.zeros((Z.shape[0], P, P), np.complex128)
    eye = np.eye(P)
    for f in range(Z.shape[0]):
        A = Z[f][np.ix_(idx, idx)].astype(np.complex128)
        X = np.linalg.solve(A, V)
        Y = np.stack([V[:, p] @ X for p in range(P)])       # sum over port p's gap of l_k x_k
        S[f] = np.linalg.solve(eye + Z0 * Y, eye - Z0 * Y)
    return S


def eval_batch(grid: Grid, Z: np.ndarray, maps: np.ndarray, Z0: float = 50.0, threads: int = 0):
    z, zc64 = _z_args(Z)
    m = np.ascontiguousarray(maps, dtype=np.uint8)
    B = m.shape[0]
    S = np.zeros((B, z.shape[0], grid.P, grid.P), dtype=np.complex128)
    status = np.zeros(B, dtype=np.int32)
    if threads <= 0:
        threads = os.cpu_count() or 1
    lib().or_eval_batch(grid.ref, _ptr(grid.table), grid.M, _ptr(z), zc64, z.shape[0], _ptr(m), B, Z0, threads,
                        _ptr(S), _ptr(status))
    return S, status


def bands(freqs, b) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
    e = np.ascontiguousarray(np.array([*b.p1, *b.p2, *b.i, *b.s], dtype=np.float64))
    out = np.zeros(len(f), dtype=np.uint8)
    lib().or_bands(_ptr(f), len(f), _ptr(e), _ptr(out))
    return out


def fom(S: np.ndarray, band: np.ndarray) -> float:
    s = np.ascontiguousarray(S, dtype=np.complex128)
    bd = np.ascontiguousarray(band, dtype=np.uint8)
    return lib().or_fom(_ptr(s), s.shape[0], s.shape[1], _ptr(bd))


def fom_batch(S: np.ndarray, band: np.ndarray) -> np.ndarray:
    return np.array([fom(S[b], band) for b in range(S.shape[0])])
