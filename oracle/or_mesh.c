/*
 * or_mesh.c -- oracle mesher, basis-function classes and support set.  TEST INFRASTRUCTURE ONLY.
 *
 * Mesh (Section V-A): every pixel is a square of side a cut into s x s sub-squares (s = 1, 2, 3:
 * 2, 8 or 18 triangles per pixel, Fig. mesh_orientation), each split by one diagonal into two right
 * triangles.  With the "alternating" orientation (the default) the diagonal of sub-square (X, Y)
 * of the fine lattice runs from (X, Y+1) to (X+1, Y) when X+Y is even and from (X, Y) to (X+1, Y+1)
 * when X+Y is odd; the "uniform" one always takes the first, the "random" one draws it per fine
 * lattice position from a seeded generator; the pattern is the same on every layer.  One RWG
 * basis function (Section II-B) sits on every edge shared by two triangles:
 *   inner-pixel BF  : an edge inside a pixel               -> active when the pixel is metal
 *   inter-pixel BF  : one of the s edges on a shared side  -> active when both pixels are metal
 *   (pixels touching only at a corner share no edge, so they are not connected: Section VI-A)
 * Ports (Section II-E says only that each port is one BF; the stub geometry is our reading):
 * a feed stub of two pixels leaves the grid through one side, on the lattice continuation.  It
 * carries always-present BFs (the inner edges of both stub pixels and the s edges between the two
 * stub pixels, which form the delta gap of the port, positive triangles outside) and s pixel-port
 * BFs on the side between the stub and the grid pixel it touches (active when that pixel is
 * metal).  With s = 1 the gap is one edge, the port BF.
 * Canonical BF order: port stubs (port-major: inner BFs of the stub pixel next to the grid, gap
 * edges, inner BFs of the outer stub pixel) -> per layer, per pixel row-major (y outer, x inner):
 * inner BFs (per sub-square row-major: diagonal, +x edge, +y edge), the s edges of the +x side,
 * the s edges of the +y side -> pixel-port BFs (port-major) -> via BFs.
 *
 * Via state (n_states = 3, two-triangle mesh; additional states with vias are future work in
 * Section VIII): state 2 on layer l is metal on layer l plus a vertical strip standing on the pixel
 * diagonal, from layer l up to layer l+1.  The strip is a rectangle A = D0@z_l, B = D1@z_l,
 * C = D1@z_{l+1}, D = D0@z_{l+1} (D0, D1 = the diagonal's end corners) cut along A-C into
 * Ta = (A, B, C) and Tb = (A, C, D).  Three BFs per via site (layers 0 .. L-2, per pixel
 * row-major): the strip's own diagonal A-C (Ta -> Tb); the junction A-B with the lower-indexed
 * triangle (half 0) of pixel (l, x, y) (half 0 -> Ta), active with the via; the junction D-C with
 * half 0 of pixel (l+1, x, y) (Tb -> that half), active only when that pixel has metal.  The last
 * layer has no via state.
 */
#include <string.h>

#include "pmom_oracle.h"

static int sub_of(const or_grid* g) { return g->sub > 1 ? g->sub : 1; }

/* half 0, 1: the sub-square's horizontal triangles; 2, 3: Ta, Tb of the via strip above a pixel.
 * Fine-lattice coordinates, offset so that both stub pixels of every port stay non-negative. */
static int32_t tri_key(const or_grid* g, int layer, int X, int Y, int half) {
  int s = sub_of(g), W = 128 * s, off = 4 * s;
  return ((layer * W + (Y + off)) * W + (X + off)) * 4 + half;
}

static void key_decode(const or_grid* g, int32_t key, int* layer, int* X, int* Y, int* half) {
  int s = sub_of(g), W = 128 * s, off = 4 * s;
  *half = key & 3;
  key >>= 2;
  *X = key % W - off;
  key /= W;
  *Y = key % W - off;
  *layer = key / W;
}

void or_key_parts(const or_grid* g, int32_t key, int* layer, int* X, int* Y, int* half) {
  key_decode(g, key, layer, X, Y, half);
}

/* SplitMix64 (Steele, Lea and Flood 2014): state advanced by the golden gamma, then mixed. */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int or_orient(const or_grid* g, int X, int Y) {
  if (g->diag_pattern == 1) return 0;
  if (g->diag_pattern == 2) {
    int s = sub_of(g);
    uint64_t h = splitmix64(0 ^ g->diag_seed);
    h = splitmix64(h ^ (uint64_t)((Y + 4 * s) * (128 * s) + (X + 4 * s)));
    return (int)(h >> 63);
  }
  return (X + Y) & 1;
}

/* Lattice corners of triangle `half` of sub-square (X, Y), in canonical vertex order. */
static void tri_corners(const or_grid* g, int x, int y, int half, int c[3][2]) {
  const int c00[2] = {x, y}, c10[2] = {x + 1, y}, c01[2] = {x, y + 1}, c11[2] = {x + 1, y + 1};
  const int* v[3];
  if (or_orient(g, x, y) == 0) {     /* diagonal c01 - c10 */
    if (half == 0) { v[0] = c00; v[1] = c10; v[2] = c01; }
    else           { v[0] = c10; v[1] = c11; v[2] = c01; }
  } else {                           /* diagonal c00 - c11 */
    if (half == 0) { v[0] = c00; v[1] = c10; v[2] = c11; }
    else           { v[0] = c00; v[1] = c11; v[2] = c01; }
  }
  for (int i = 0; i < 3; ++i) { c[i][0] = v[i][0]; c[i][1] = v[i][1]; }
}

/* End corners D0, D1 of the diagonal of a (one-cell) pixel, in the order they appear in half 0. */
static void diag_ends(const or_grid* g, int x, int y, int d0[2], int d1[2]) {
  if (or_orient(g, x, y) == 0) { d0[0] = x; d0[1] = y + 1; d1[0] = x + 1; d1[1] = y; }
  else                         { d0[0] = x; d0[1] = y;     d1[0] = x + 1; d1[1] = y + 1; }
}

void or_triangle(const or_grid* g, int32_t key, double v[3][3]) {
  int layer, x, y, half, c[3][2];
  key_decode(g, key, &layer, &x, &y, &half);
  double h = g->pitch / sub_of(g);
  if (half >= 2) {
    int d0[2], d1[2];
    diag_ends(g, x, y, d0, d1);
    double zl = g->layer_z[layer], zu = g->layer_z[layer + 1];
    /* Ta = (A, B, C), Tb = (A, C, D) */
    const int* xy[3] = {d0, d1, half == 2 ? d1 : d0};
    double z[3] = {zl, half == 2 ? zl : zu, zu};
    for (int i = 0; i < 3; ++i) {
      v[i][0] = xy[i][0] * h;
      v[i][1] = xy[i][1] * h;
      v[i][2] = z[i];
    }
    return;
  }
  tri_corners(g, x, y, half, c);
  for (int i = 0; i < 3; ++i) {
    v[i][0] = c[i][0] * h;
    v[i][1] = c[i][1] * h;
    v[i][2] = g->layer_z[layer];
  }
}

/* Which half of sub-square (x, y) holds the lattice edge p-q, and the index of its free vertex. */
static int find_half(const or_grid* g, int x, int y, const int p[2], const int q[2], int* free_idx) {
  for (int half = 0; half < 2; ++half) {
    int c[3][2], hit[3] = {0, 0, 0}, nhit = 0;
    tri_corners(g, x, y, half, c);
    for (int i = 0; i < 3; ++i) {
      if ((c[i][0] == p[0] && c[i][1] == p[1]) || (c[i][0] == q[0] && c[i][1] == q[1])) { hit[i] = 1; ++nhit; }
    }
    if (nhit == 2) {
      for (int i = 0; i < 3; ++i) if (!hit[i]) *free_idx = i;
      return half;
    }
  }
  return -1;
}

/* Emit the BF on the edge shared by sub-square P (positive side) and sub-square Q (negative
 * side); the two are fine-lattice neighbours on `layer`. */
static void emit_side(const or_grid* g, int32_t* row, int layer, int px, int py, int qx, int qy) {
  int e0[2], e1[2];
  if (qx == px + 1)      { e0[0] = px + 1; e0[1] = py;     e1[0] = px + 1; e1[1] = py + 1; }
  else if (qx == px - 1) { e0[0] = px;     e0[1] = py;     e1[0] = px;     e1[1] = py + 1; }
  else if (qy == py + 1) { e0[0] = px;     e0[1] = py + 1; e1[0] = px + 1; e1[1] = py + 1; }
  else                   { e0[0] = px;     e0[1] = py;     e1[0] = px + 1; e1[1] = py; }
  int fp = -1, fq = -1;
  int hp = find_half(g, px, py, e0, e1, &fp);
  int hq = find_half(g, qx, qy, e0, e1, &fq);
  row[4] = tri_key(g, layer, px, py, hp);
  row[5] = tri_key(g, layer, qx, qy, hq);
  row[6] = fp;
  row[7] = fq;
}

/* The BF on the diagonal of sub-square (x, y). */
static void emit_diag(const or_grid* g, int32_t* row, int layer, int x, int y) {
  int c0[3][2], c1[3][2];
  tri_corners(g, x, y, 0, c0);
  tri_corners(g, x, y, 1, c1);
  /* free vertex of each half = the corner not on the other half */
  int f0 = -1, f1 = -1;
  for (int i = 0; i < 3; ++i) {
    int shared = 0;
    for (int j = 0; j < 3; ++j) if (c0[i][0] == c1[j][0] && c0[i][1] == c1[j][1]) shared = 1;
    if (!shared) f0 = i;
  }
  for (int i = 0; i < 3; ++i) {
    int shared = 0;
    for (int j = 0; j < 3; ++j) if (c1[i][0] == c0[j][0] && c1[i][1] == c0[j][1]) shared = 1;
    if (!shared) f1 = i;
  }
  row[4] = tri_key(g, layer, x, y, 0);
  row[5] = tri_key(g, layer, x, y, 1);
  row[6] = f0;
  row[7] = f1;
}

/* Stub pixels of a port: s1 touches the grid, s2 is outside it; g is the grid pixel touched. */
static void port_pixels(const or_grid* g, const int32_t* port, int s1[2], int s2[2], int gp[2]) {
  int side = port[1], pos = port[2];
  switch (side) {
    case 0: s1[0] = g->nx;  s1[1] = pos; s2[0] = g->nx + 1; s2[1] = pos; gp[0] = g->nx - 1; gp[1] = pos; break;
    case 1: s1[0] = pos; s1[1] = g->ny;  s2[0] = pos; s2[1] = g->ny + 1; gp[0] = pos; gp[1] = g->ny - 1; break;
    case 2: s1[0] = -1; s1[1] = pos; s2[0] = -2; s2[1] = pos; gp[0] = 0; gp[1] = pos; break;
    default: s1[0] = pos; s1[1] = -1; s2[0] = pos; s2[1] = -2; gp[0] = pos; gp[1] = 0; break;
  }
}

static int pix_index(const or_grid* g, int layer, int x, int y) { return (layer * g->ny + y) * g->nx + x; }

static int has_vias(const or_grid* g) { return g->n_states >= 3 && g->layers >= 2 && sub_of(g) == 1; }

/* inner BFs of one pixel: s^2 diagonals + 2 s (s - 1) edges between its sub-squares */
static int inner_count(int s) { return s * s + 2 * s * (s - 1); }

int or_stub_bfs(const or_grid* g) { return 2 * inner_count(sub_of(g)) + sub_of(g); }

int or_port_gap(const or_grid* g, int p, int32_t* bf) {
  int s = sub_of(g), K = or_stub_bfs(g), ni = inner_count(s);
  for (int k = 0; k < s; ++k) bf[k] = p * K + ni + k;
  return s;
}

int or_count_bfs(const or_grid* g) {
  int s = sub_of(g);
  int per_layer = g->nx * g->ny * inner_count(s) + s * ((g->nx - 1) * g->ny + g->nx * (g->ny - 1));
  int vias = has_vias(g) ? 3 * (g->layers - 1) * g->nx * g->ny : 0;
  return g->n_ports * (or_stub_bfs(g) + s) + g->layers * per_layer + vias;
}

static int32_t* next_row(int32_t* t, int* m, int cls, int pa, int pb, int port) {
  int32_t* r = t + OR_BF_COLS * (*m)++;
  r[0] = cls; r[1] = pa; r[2] = pb; r[3] = port;
  return r;
}

/* Inner BFs of pixel (x, y): per sub-square row-major, its diagonal, then the edge to the +x and
 * to the +y neighbour inside the pixel. */
static void emit_pixel_inner(const or_grid* g, int32_t* t, int* m, int cls, int pa, int port, int layer, int x, int y) {
  int s = sub_of(g);
  for (int j = 0; j < s; ++j)
    for (int i = 0; i < s; ++i) {
      int X = s * x + i, Y = s * y + j;
      emit_diag(g, next_row(t, m, cls, pa, -1, port), layer, X, Y);
      if (i + 1 < s) emit_side(g, next_row(t, m, cls, pa, -1, port), layer, X, Y, X + 1, Y);
      if (j + 1 < s) emit_side(g, next_row(t, m, cls, pa, -1, port), layer, X, Y, X, Y + 1);
    }
}

/* The s edges of the side shared by lattice-neighbour pixels P (positive) and Q (negative). */
static void emit_pixel_side(const or_grid* g, int32_t* t, int* m, int cls, int pa, int pb, int port, int layer,
                            int px, int py, int qx, int qy) {
  int s = sub_of(g);
  for (int k = 0; k < s; ++k) {
    int PX, PY, QX, QY;
    if (qx != px) {   /* vertical side: the sub-squares of row k on either side of it */
      PX = qx > px ? s * px + s - 1 : s * px;
      QX = qx > px ? s * qx : s * qx + s - 1;
      PY = QY = s * py + k;
    } else {          /* horizontal side: the sub-squares of column k */
      PY = qy > py ? s * py + s - 1 : s * py;
      QY = qy > py ? s * qy : s * qy + s - 1;
      PX = QX = s * px + k;
    }
    emit_side(g, next_row(t, m, cls, pa, pb, port), layer, PX, PY, QX, QY);
  }
}

int or_bf_table(const or_grid* g, int32_t* t) {
  int m = 0;
  for (int p = 0; p < g->n_ports; ++p) {
    const int32_t* port = g->ports + 3 * p;
    int s1[2], s2[2], gp[2], layer = port[0];
    port_pixels(g, port, s1, s2, gp);
    emit_pixel_inner(g, t, &m, OR_BF_ALWAYS, -1, p, layer, s1[0], s1[1]);
    emit_pixel_side(g, t, &m, OR_BF_ALWAYS, -1, -1, p, layer, s2[0], s2[1], s1[0], s1[1]);   /* gap, + outside */
    emit_pixel_inner(g, t, &m, OR_BF_ALWAYS, -1, p, layer, s2[0], s2[1]);
  }
  for (int l = 0; l < g->layers; ++l) {
    for (int y = 0; y < g->ny; ++y) {
      for (int x = 0; x < g->nx; ++x) {
        emit_pixel_inner(g, t, &m, OR_BF_INNER, pix_index(g, l, x, y), -1, l, x, y);
        if (x + 1 < g->nx)
          emit_pixel_side(g, t, &m, OR_BF_INTER, pix_index(g, l, x, y), pix_index(g, l, x + 1, y), -1, l, x, y, x + 1, y);
        if (y + 1 < g->ny)
          emit_pixel_side(g, t, &m, OR_BF_INTER, pix_index(g, l, x, y), pix_index(g, l, x, y + 1), -1, l, x, y, x, y + 1);
      }
    }
  }
  for (int p = 0; p < g->n_ports; ++p) {
    const int32_t* port = g->ports + 3 * p;
    int s1[2], s2[2], gp[2], layer = port[0];
    port_pixels(g, port, s1, s2, gp);
    emit_pixel_side(g, t, &m, OR_BF_PIXPORT, pix_index(g, layer, gp[0], gp[1]), -1, p, layer, s1[0], s1[1], gp[0],
                    gp[1]);
  }
  if (has_vias(g)) {
    for (int l = 0; l + 1 < g->layers; ++l) {
      for (int y = 0; y < g->ny; ++y) {
        for (int x = 0; x < g->nx; ++x) {
          int f0 = -1, c[3][2];
          int32_t* r = t + OR_BF_COLS * m++;
          /* strip diagonal A-C: free vertices B (index 1 of Ta) and D (index 2 of Tb) */
          r[0] = OR_BF_VIA_STRIP; r[1] = pix_index(g, l, x, y); r[2] = -1; r[3] = -1;
          r[4] = tri_key(g, l, x, y, 2); r[5] = tri_key(g, l, x, y, 3); r[6] = 1; r[7] = 2;
          /* free vertex of half 0 with respect to the pixel diagonal */
          int d0[2], d1[2];
          diag_ends(g, x, y, d0, d1);
          tri_corners(g, x, y, 0, c);
          for (int i = 0; i < 3; ++i) {
            int on0 = c[i][0] == d0[0] && c[i][1] == d0[1], on1 = c[i][0] == d1[0] && c[i][1] == d1[1];
            if (!on0 && !on1) f0 = i;
          }
          /* junction A-B: half 0 of (l, x, y) -> Ta; free vertex of Ta is C (index 2) */
          r = t + OR_BF_COLS * m++;
          r[0] = OR_BF_VIA_JOIN; r[1] = pix_index(g, l, x, y); r[2] = -1; r[3] = -1;
          r[4] = tri_key(g, l, x, y, 0); r[5] = tri_key(g, l, x, y, 2); r[6] = f0; r[7] = 2;
          /* junction D-C: Tb -> half 0 of (l+1, x, y); free vertex of Tb is A (index 0) */
          r = t + OR_BF_COLS * m++;
          r[0] = OR_BF_VIA_LAND; r[1] = pix_index(g, l, x, y); r[2] = pix_index(g, l + 1, x, y); r[3] = -1;
          r[4] = tri_key(g, l, x, y, 3); r[5] = tri_key(g, l + 1, x, y, 0); r[6] = 0; r[7] = f0;
        }
      }
    }
  }
  return m;
}

int or_active_set(const or_grid* g, const int32_t* t, int M, const uint8_t* map, int32_t* idx) {
  int np = g->layers * g->ny * g->nx, last = (g->layers - 1) * g->ny * g->nx;
  for (int i = 0; i < np; ++i) if (map[i] >= g->n_states) return -1;
  for (int i = last; i < np; ++i) if (map[i] == 2) return -1;   /* no via above the last layer */
  if (!has_vias(g))
    for (int i = 0; i < np; ++i) if (map[i] == 2) return -1;   /* no via state on this mesh */
  int n = 0;
  for (int m = 0; m < M; ++m) {
    const int32_t* r = t + OR_BF_COLS * m;
    int on;
    switch (r[0]) {
      case OR_BF_ALWAYS: on = 1; break;
      case OR_BF_INNER: on = map[r[1]] >= 1; break;
      case OR_BF_INTER: on = map[r[1]] >= 1 && map[r[2]] >= 1; break;
      case OR_BF_PIXPORT: on = map[r[1]] >= 1; break;
      case OR_BF_VIA_STRIP: on = map[r[1]] == 2; break;
      case OR_BF_VIA_JOIN: on = map[r[1]] == 2; break;
      case OR_BF_VIA_LAND: on = map[r[1]] == 2 && map[r[2]] >= 1; break;
      default: on = 0;
    }
    if (on) idx[n++] = m;
  }
  return n;
}
