"""Oracle pins for the via state (three pixel states: void / metal / metal with a vertical strip up
to the next layer; the paper names additional states with vias as future work, Section VIII).

Mesh: closed-form BF count, the geometry of the strip triangles and of the three via BFs, and the
support set of every map of a small two-layer grid against a hand count.  Fill: K0 of complex
argument against SciPy, the Dirichlet and Neumann kernels at arbitrary heights by image series
against mode series, the pair integrals of vertical triangles against an independent brute-force
quadrature with direct image sums (which also shows that the vertical current components need
the Neumann kernel), translation invariance, reciprocity and passivity with vias, and a via that
joins two layers carrying the signal like a line on one layer."""
import dataclasses
import itertools

import numpy as np
import pytest
from scipy.special import kv

import pmom_inputs as PI
from oracle import oracle as O

H = PI.H_RO4350
EPS0 = 8.8541878128e-12
MU0 = 4e-7 * np.pi


def via_grid(n, pitch=0.5e-3, tan_d=0.004, ports=None):
    g = PI.grid_tiny(n, PI.MEDIUM_STRIPLINE, 2, pitch_m=pitch)
    kw = {"ports": ports} if ports is not None else {}
    return dataclasses.replace(g, name=f"via_{n}x{n}x2", n_states=3, tan_d=tan_d, **kw)


# ---------------------------------------------------------------------------------- mesh
def test_bf_count_with_vias():
    g = PI.grid_stripline_20x20x3(n_states=3)
    G = O.Grid(g)
    per_layer = 2 * g.nx * (g.nx - 1) + g.nx * g.ny
    assert G.M == 4 * g.n_ports + g.layers * per_layer + 3 * (g.layers - 1) * g.nx * g.ny == 5892
    assert O.Grid(via_grid(3)).M == 4 * 3 + 2 * 21 + 3 * 9


def test_via_geometry():
    """Per via site: Ta and Tb are vertical, lie in the vertical plane of the pixel diagonal and
    tile the rectangle between the two layers; the strip BF joins them along the rectangle's
    diagonal; the lower junction is the pixel's own diagonal edge at z_l shared with its half 0;
    the upper junction is the diagonal edge at z_l+1 shared with half 0 of the pixel above; each
    BF's free vertices lie off its edge."""
    g = via_grid(3)
    G = O.Grid(g)
    T = G.table
    a, zl, zu = g.pitch_m, g.layer_z_m[0], g.layer_z_m[1]
    inner = {int(r[1]): r for r in T if r[0] == 1}
    vias = T[T[:, 0] >= 4].reshape(-1, 3, 8)
    assert len(vias) == g.nx * g.ny
    for strip, join, land in vias:
        assert (strip[0], join[0], land[0]) == (4, 5, 6)
        pix = int(strip[1])
        assert join[1] == pix and land[1] == pix and land[2] == pix + g.nx * g.ny
        ta, tb = O.triangle(G, strip[4]), O.triangle(G, strip[5])
        for t in (ta, tb):
            nrm = np.cross(t[1] - t[0], t[2] - t[0])
            assert abs(nrm[2]) < 1e-12 * np.linalg.norm(nrm)
        area = sum(0.5 * np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0])) for t in (ta, tb))
        assert np.isclose(area, a * np.sqrt(2) * (zu - zl))
        # the pixel diagonal: the edge shared by the pixel's two halves
        ir = inner[pix]
        h0, h1 = O.triangle(G, ir[4]), O.triangle(G, ir[5])
        diag = {tuple(np.round(p, 12)) for p in h0} & {tuple(np.round(p, 12)) for p in h1}
        assert len(diag) == 2
        for row, lay_len in ((strip, np.sqrt(2 * a * a + (zu - zl) ** 2)), (join, a * np.sqrt(2)), (land, a * np.sqrt(2))):
            vp, vm = O.triangle(G, row[4]), O.triangle(G, row[5])
            ep = {tuple(np.round(vp[(row[6] + k) % 3], 12)) for k in (1, 2)}
            em = {tuple(np.round(vm[(row[7] + k) % 3], 12)) for k in (1, 2)}
            assert ep == em
            e = np.array(sorted(ep))
            assert np.isclose(np.linalg.norm(e[0] - e[1]), lay_len)
            assert tuple(np.round(vp[row[6]], 12)) not in ep and tuple(np.round(vm[row[7]], 12)) not in em
        je = {tuple(np.round(O.triangle(G, join[4])[(join[6] + k) % 3], 12)) for k in (1, 2)}
        assert je == diag and join[4] == ir[4]          # the lower junction pairs Ta with half 0
        up = inner[pix + g.nx * g.ny]
        le = {tuple(np.round(O.triangle(G, land[5])[(land[7] + k) % 3], 12)) for k in (1, 2)}
        h0u, h1u = O.triangle(G, up[4]), O.triangle(G, up[5])
        assert le == {tuple(np.round(p, 12)) for p in h0u} & {tuple(np.round(p, 12)) for p in h1u}
        assert land[5] == up[4]
        assert all(np.isclose(p[2], zl) for p in je) and all(np.isclose(p[2], zu) for p in le)


def _all_via_maps(g):
    """Every map of a two-layer grid: states 0-2 on the lower layer, 0-1 on the top layer."""
    n = g.nx * g.ny
    out = []
    for lo in itertools.product(range(3), repeat=n):
        for hi in itertools.product(range(2), repeat=n):
            out.append(np.array([lo, hi], np.uint8).reshape(2, g.ny, g.nx))
    return out


def test_activation_brute_force_with_vias():
    """All 1296 maps of a 2 x 2 two-layer grid: N = 3P + metal pixels + edge-adjacent metal pairs
    (per layer) + ports whose grid pixel is metal + 2 per via + 1 per via with metal above."""
    g = via_grid(2)
    G = O.Grid(g)
    gp = {0: (g.nx - 1, None), 1: (None, g.ny - 1), 2: (0, None), 3: (None, 0)}
    maps = _all_via_maps(g)
    assert len(maps) == 81 * 16
    for m in maps:
        metal = (m >= 1).astype(int)
        n = 3 * g.n_ports + int(metal.sum())
        n += int(np.sum(metal[:, :, :-1] & metal[:, :, 1:]) + np.sum(metal[:, :-1, :] & metal[:, 1:, :]))
        for p in g.ports:
            x, y = gp[p.side]
            n += int(metal[p.layer, p.pos if y is None else y, p.pos if x is None else x])
        via = (m[0] == 2).astype(int)
        n += 2 * int(via.sum()) + int(np.sum(via & metal[1]))
        idx = O.active_set(G, m)
        assert len(idx) == n
        assert np.all(np.diff(idx) > 0)


def test_via_state_rules():
    g = via_grid(3)
    G = O.Grid(g)
    m = np.zeros((2, 3, 3), np.uint8)
    m[0, 1, 1] = 2
    assert len(O.active_set(G, m)) == 3 * 3 + 1 + 2        # inner + strip + lower junction
    m[1, 1, 1] = 1
    assert len(O.active_set(G, m)) == 3 * 3 + 2 + 3
    top = np.zeros((2, 3, 3), np.uint8)
    top[1, 0, 0] = 2                                        # no layer above the last one
    with pytest.raises(ValueError):
        O.active_set(G, top)
    bad = np.zeros((2, 3, 3), np.uint8)
    bad[0, 0, 0] = 3
    with pytest.raises(ValueError):
        O.active_set(G, bad)


def test_single_changes_with_vias():
    """A one-pixel change of a three-layer grid touches at most 9 BFs: a void middle-layer pixel
    with four metal neighbours above a via becomes a via under metal (inner + 4 inter-pixel + the
    landing junction from below + strip + own junction + landing junction)."""
    g = dataclasses.replace(PI.grid_stripline_20x20x3(n_states=3), nx=6, ny=6,
                            ports=(PI.Port(0, 0, 3), PI.Port(0, 2, 3), PI.Port(2, 2, 3)))
    G = O.Grid(g)
    rng = PI.rng(4)
    seed = rng.integers(0, 3, size=(3, 6, 6)).astype(np.uint8)
    seed[2][seed[2] == 2] = 1
    base = set(O.active_set(G, seed).tolist())
    worst = 0
    for c in PI.single_flip_batch(seed, 3):
        if (c[2] == 2).any():
            continue
        d = base.symmetric_difference(O.active_set(G, c).tolist())
        worst = max(worst, len(d))
        assert 1 <= len(d) <= 9
    assert worst >= 5


# ---------------------------------------------------------------------------------- fill
def test_bessel_k0_any_argument_vs_scipy():
    for r in (1e-3, 0.1, 0.7, 2.0, 5.0, 9.0, 14.0, 16.9, 17.1, 25.0, 45.0):
        for ang in (0.0, 0.6, 1.2, 1.45, 1.54, 1.5705):
            w = r * np.exp(1j * ang)
            ref = kv(0, w)
            assert abs(O.bessel_k0(w, any_arg=True) - ref) <= 2e-9 * abs(ref), (r, ang)


@pytest.mark.parametrize("kind", [0, 1])
def test_kernels_at_arbitrary_heights(kind):
    """Image series (600 images; a lossy medium makes it converge) against the mode series at
    rho >= H/2, and against the fill's images-plus-fitted-tail route at rho < H/2."""
    g = via_grid(3, tan_d=0.5)
    G = O.Grid(g)
    Ht = g.h_total_m
    for zp, zq in ((0.3 * Ht, 0.71 * Ht), (0.5 * Ht, 0.5 * Ht), (0.12 * Ht, 0.9 * Ht)):
        for rho in (0.55 * Ht, 1.5 * Ht, 3.0 * Ht):
            a = O.green_heights(G, 5e9, kind, zp, zq, rho, "images", K=600)
            b = O.green_heights(G, 5e9, kind, zp, zq, rho, "modal")
            assert abs(a - b) <= 1e-9 * abs(b)
        for rho in (0.01 * Ht, 0.2 * Ht, 0.45 * Ht):
            a = O.green_heights(G, 5e9, kind, zp, zq, rho, "images", K=600)
            b = O.green_heights(G, 5e9, kind, zp, zq, rho)
            assert abs(a - b) <= 1e-9 * abs(a)


def _gauss_triangle(v, n=14):
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = (x + 1) / 2, w / 2
    U, V = (a.ravel() for a in np.meshgrid(x, x, indexing="ij"))
    W = np.outer(w, w).ravel()
    pts = v[0] + (U * (1 - V))[:, None] * (v[1] - v[0]) + (U * V)[:, None] * (v[2] - v[0])
    area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    return pts, W * U * 2 * area


def _images(k, Ht, r, rq, sign, K=160):
    d = r[:, None, :] - rq[None, :, :]
    rho2 = d[..., 0] ** 2 + d[..., 1] ** 2
    zp, zq = r[:, None, 2], rq[None, :, 2]
    G = 0
    for n in range(-K, K + 1):
        Ra = np.sqrt(rho2 + (zp - zq + 2 * n * Ht) ** 2)
        Rb = np.sqrt(rho2 + (zp + zq + 2 * n * Ht) ** 2)
        G = G + np.exp(-1j * k * Ra) / (4 * np.pi * Ra) + sign * np.exp(-1j * k * Rb) / (4 * np.pi * Rb)
    return G


def _brute_pair(G, g, f, kp, kq, vertical_kernel):
    vp, vq = O.triangle(G, kp), O.triangle(G, kq)
    rp, wp = _gauss_triangle(vp)
    rq, wq = _gauss_triangle(vq)
    k = 2 * np.pi * f * np.sqrt(MU0 * EPS0 * g.eps_r * (1 - 1j * g.tan_d))
    GD = _images(k, g.h_total_m, rp, rq, -1.0)
    GZ = _images(k, g.h_total_m, rp, rq, +1.0 if vertical_kernel == "neumann" else -1.0)
    W = wp[:, None] * wq[None, :]
    out = np.zeros(10, complex)
    out[0] = np.sum(W * GD)
    for a in range(3):
        ra = rp - vp[a]
        for b in range(3):
            rb = rq - vq[b]
            dh = ra[:, None, 0] * rb[None, :, 0] + ra[:, None, 1] * rb[None, :, 1]
            dz = ra[:, None, 2] * rb[None, :, 2]
            out[1 + 3 * a + b] = np.sum(W * (dh * GD + dz * GZ))
    return out


def test_vertical_pair_integrals_vs_brute_force():
    """Well-separated pairs (vertical-vertical, vertical-horizontal): the fill's 7 x 7-point
    integrals against 196 x 196-point Gauss products with direct image sums.  Charges and
    horizontal currents image with a sign change, vertical currents without: using the
    Dirichlet kernel for the vertical components changes the vector integrals by ~100 %."""
    g = via_grid(4, tan_d=0.5)
    G = O.Grid(g)
    T = G.table
    strip, inner = T[T[:, 0] == 4], T[T[:, 0] == 1]
    pairs = [(strip[0][4], strip[-1][5], True), (strip[1][5], strip[-2][4], True),
             (strip[0][4], inner[-1][4], False), (inner[-3][5], strip[2][5], False)]
    for kp, kq, both_vertical in pairs:
        ours = O.pair_integrals(G, 5e9, kp, kq)
        ref = _brute_pair(G, g, 5e9, kp, kq, "neumann")
        assert abs(ours[0] - ref[0]) <= 5e-5 * abs(ref[0])
        assert np.abs(ours[1:] - ref[1:]).max() <= 5e-5 * np.abs(ref[1:]).max()
        if both_vertical:
            wrong = _brute_pair(G, g, 5e9, kp, kq, "dirichlet")
            assert np.abs(wrong[1:] - ref[1:]).max() >= 0.3 * np.abs(ref[1:]).max()


@pytest.fixture(scope="module")
def via_fill():
    g = via_grid(4)
    G = O.Grid(g)
    f = [1.3e9, 6.1e9]
    Zt, asym = O.fill(G, f, mode=1)
    return g, G, f, Zt, asym


def test_lattice_table_fill_equals_direct_fill_with_vias(via_fill):
    g, G, f, Zt, _ = via_fill
    Zd, _ = O.fill(G, f, mode=0)
    assert np.abs(Zd - Zt).max() <= 1e-12 * np.abs(Zd).max()


def test_reciprocity_and_passivity_with_vias(via_fill):
    g, G, f, Z, asym = via_fill
    assert asym < 2e-4
    for Zf in Z:
        herm = 0.5 * (Zf + Zf.conj().T)
        assert np.linalg.eigvalsh(herm).min() >= -1e-10 * np.abs(Zf).max()


def test_via_joins_two_layers():
    """Two strips on different layers overlapping at one pixel, ports on different layers: with a
    via at the overlap the pair transmits like the same strip on one layer (the via is electrically
    tiny at 1 GHz), without it only through the overlap capacitance.  S stays reciprocal and
    passive, and the two S forms (Eq. 6 loaded ports / unloaded Y -> S) agree."""
    ports2 = (PI.Port(0, PI.SIDE_RIGHT, 4), PI.Port(1, PI.SIDE_LEFT, 4))
    ports1 = (PI.Port(0, PI.SIDE_RIGHT, 4), PI.Port(0, PI.SIDE_LEFT, 4))
    mk = lambda ports: PI.Grid("via_8x8x2", 2, 8, 8, 0.5625e-3, PI.MEDIUM_STRIPLINE, (H, 2 * H), 3 * H, 3.66,
                               0.004, 3, ports)
    s21 = {}
    for name, ports in (("two", ports2), ("one", ports1)):
        G = O.Grid(mk(ports))
        Z, _ = O.fill(G, [1e9])
        if name == "one":
            m = np.zeros((2, 8, 8), np.uint8)
            m[0, 4, :] = 1
            cases = {"line": m}
        else:
            m = np.zeros((2, 8, 8), np.uint8)
            m[0, 4, 4:] = 1
            m[1, 4, :5] = 1
            mv = m.copy()
            mv[0, 4, 4] = 2
            cases = {"no_via": m, "via": mv}
        for key, mm in cases.items():
            S, st = O.eval_map(G, Z, mm)
            assert st == 0
            S1, _ = O.eval_map(G, Z, mm, form=1)
            assert np.abs(S1 - S).max() <= 1e-12
            assert np.abs(S - np.swapaxes(S, 1, 2)).max() <= 1e-12
            assert np.linalg.svd(S[0], compute_uv=False).max() <= 1 + 1e-9
            s21[key] = abs(S[0, 1, 0])
    assert abs(s21["via"] / s21["line"] - 1) <= 0.15
    assert s21["no_via"] <= 0.25 * s21["via"]
