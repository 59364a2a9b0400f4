/*
 * or_mesh.c -- oracle mesher, basis-function classes and support set.  TEST INFRASTRUCTURE ONLY.
 *
 * Mesh (Section V-A, "alternating" orientation): every pixel is a square of side a split by one
 * diagonal into two right triangles.  The diagonal runs from (x, y+1) to (x+1, y) when x+y is
 * even and from (x, y) to (x+1, y+1) when x+y is odd, on every layer.  One RWG basis function
 * (Section II-B) sits on every edge shared by two triangles:
 *   inner-pixel BF  : the diagonal of a pixel        -> active when the pixel is metal
 *   inter-pixel BF  : the side shared by two pixels  -> active when both pixels are metal
 *   (pixels touching only at a corner share no edge, so they are not connected: Section VI-A)
 * Ports (Section II-E says only that each port is one BF; the stub geometry is our reading):
 * a feed stub of two pixels leaves the grid through one side, on the lattice continuation.  It
 * carries three always-present BFs (the diagonal of each stub pixel and the edge between the
 * two stub pixels, which is the delta-gap port BF, positive triangle outside) and one
 * pixel-port BF on the edge between the stub and the grid pixel it touches (active when that
 * pixel is metal).
 * Canonical BF order: port stubs (port-major: inner stub diagonal, port edge, outer stub
 * diagonal) -> per layer, per pixel row-major (y outer, x inner): diagonal, +x side, +y side
 * -> pixel-port BFs (port-major).
 */
#include <string.h>

#include "pmom_oracle.h"

static int32_t tri_key(int layer, int x, int y, int half) {
  return ((layer * 128 + (y + 4)) * 128 + (x + 4)) * 2 + half;
}

static void key_decode(int32_t key, int* layer, int* x, int* y, int* half) {
  *half = key & 1;
  key >>= 1;
  *x = key % 128 - 4;
  key /= 128;
  *y = key % 128 - 4;
  *layer = key / 128;
}

/* Lattice corners of triangle `half` of pixel (x, y), in canonical vertex order. */
static void tri_corners(int x, int y, int half, int c[3][2]) {
  const int c00[2] = {x, y}, c10[2] = {x + 1, y}, c01[2] = {x, y + 1}, c11[2] = {x + 1, y + 1};
  const int* v[3];
  if (((x + y) & 1) == 0) {          /* diagonal c01 - c10 */
    if (half == 0) { v[0] = c00; v[1] = c10; v[2] = c01; }
    else           { v[0] = c10; v[1] = c11; v[2] = c01; }
  } else {                           /* diagonal c00 - c11 */
    if (half == 0) { v[0] = c00; v[1] = c10; v[2] = c11; }
    else           { v[0] = c00; v[1] = c11; v[2] = c01; }
  }
  for (int i = 0; i < 3; ++i) { c[i][0] = v[i][0]; c[i][1] = v[i][1]; }
}

void or_triangle(const or_grid* g, int32_t key, double v[3][3]) {
  int layer, x, y, half, c[3][2];
  key_decode(key, &layer, &x, &y, &half);
  tri_corners(x, y, half, c);
  for (int i = 0; i < 3; ++i) {
    v[i][0] = c[i][0] * g->pitch;
    v[i][1] = c[i][1] * g->pitch;
    v[i][2] = g->layer_z[layer];
  }
}

/* Which half of pixel (x, y) holds the lattice edge p-q, and the index of its free vertex. */
static int find_half(int x, int y, const int p[2], const int q[2], int* free_idx) {
  for (int half = 0; half < 2; ++half) {
    int c[3][2], hit[3] = {0, 0, 0}, nhit = 0;
    tri_corners(x, y, half, c);
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

/* Emit the BF on the edge shared by pixel P (positive side) and pixel Q (negative side);
 * the two pixels are lattice neighbours on `layer`. */
static void emit_side(int32_t* row, int layer, int px, int py, int qx, int qy) {
  int e0[2], e1[2];
  if (qx == px + 1)      { e0[0] = px + 1; e0[1] = py;     e1[0] = px + 1; e1[1] = py + 1; }
  else if (qx == px - 1) { e0[0] = px;     e0[1] = py;     e1[0] = px;     e1[1] = py + 1; }
  else if (qy == py + 1) { e0[0] = px;     e0[1] = py + 1; e1[0] = px + 1; e1[1] = py + 1; }
  else                   { e0[0] = px;     e0[1] = py;     e1[0] = px + 1; e1[1] = py; }
  int fp = -1, fq = -1;
  int hp = find_half(px, py, e0, e1, &fp);
  int hq = find_half(qx, qy, e0, e1, &fq);
  row[4] = tri_key(layer, px, py, hp);
  row[5] = tri_key(layer, qx, qy, hq);
  row[6] = fp;
  row[7] = fq;
}

static void emit_diag(int32_t* row, int layer, int x, int y) {
  int c0[3][2], c1[3][2];
  tri_corners(x, y, 0, c0);
  tri_corners(x, y, 1, c1);
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
  row[4] = tri_key(layer, x, y, 0);
  row[5] = tri_key(layer, x, y, 1);
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

int or_count_bfs(const or_grid* g) {
  int per_layer = g->nx * g->ny + (g->nx - 1) * g->ny + g->nx * (g->ny - 1);
  return 4 * g->n_ports + g->layers * per_layer;
}

int or_bf_table(const or_grid* g, int32_t* t) {
  int m = 0;
  for (int p = 0; p < g->n_ports; ++p) {
    const int32_t* port = g->ports + 3 * p;
    int s1[2], s2[2], gp[2], layer = port[0];
    port_pixels(g, port, s1, s2, gp);
    int32_t* r;
    r = t + OR_BF_COLS * m++; r[0] = OR_BF_ALWAYS; r[1] = -1; r[2] = -1; r[3] = p; emit_diag(r, layer, s1[0], s1[1]);
    r = t + OR_BF_COLS * m++; r[0] = OR_BF_ALWAYS; r[1] = -1; r[2] = -1; r[3] = p;
    emit_side(r, layer, s2[0], s2[1], s1[0], s1[1]);          /* positive triangle outside */
    r = t + OR_BF_COLS * m++; r[0] = OR_BF_ALWAYS; r[1] = -1; r[2] = -1; r[3] = p; emit_diag(r, layer, s2[0], s2[1]);
  }
  for (int l = 0; l < g->layers; ++l) {
    for (int y = 0; y < g->ny; ++y) {
      for (int x = 0; x < g->nx; ++x) {
        int32_t* r = t + OR_BF_COLS * m++;
        r[0] = OR_BF_INNER; r[1] = pix_index(g, l, x, y); r[2] = -1; r[3] = -1;
        emit_diag(r, l, x, y);
        if (x + 1 < g->nx) {
          r = t + OR_BF_COLS * m++;
          r[0] = OR_BF_INTER; r[1] = pix_index(g, l, x, y); r[2] = pix_index(g, l, x + 1, y); r[3] = -1;
          emit_side(r, l, x, y, x + 1, y);
        }
        if (y + 1 < g->ny) {
          r = t + OR_BF_COLS * m++;
          r[0] = OR_BF_INTER; r[1] = pix_index(g, l, x, y); r[2] = pix_index(g, l, x, y + 1); r[3] = -1;
          emit_side(r, l, x, y, x, y + 1);
        }
      }
    }
  }
  for (int p = 0; p < g->n_ports; ++p) {
    const int32_t* port = g->ports + 3 * p;
    int s1[2], s2[2], gp[2], layer = port[0];
    port_pixels(g, port, s1, s2, gp);
    int32_t* r = t + OR_BF_COLS * m++;
    r[0] = OR_BF_PIXPORT; r[1] = pix_index(g, layer, gp[0], gp[1]); r[2] = -1; r[3] = p;
    emit_side(r, layer, s1[0], s1[1], gp[0], gp[1]);
  }
  return m;
}

int or_active_set(const or_grid* g, const int32_t* t, int M, const uint8_t* map, int32_t* idx) {
  int np = g->layers * g->ny * g->nx;
  for (int i = 0; i < np; ++i) if (map[i] >= g->n_states) return -1;
  int n = 0;
  for (int m = 0; m < M; ++m) {
    const int32_t* r = t + OR_BF_COLS * m;
    int on;
    switch (r[0]) {
      case OR_BF_ALWAYS: on = 1; break;
      case OR_BF_INNER: on = map[r[1]] >= 1; break;
      case OR_BF_INTER: on = map[r[1]] >= 1 && map[r[2]] >= 1; break;
      case OR_BF_PIXPORT: on = map[r[1]] >= 1; break;
      default: on = 0;
    }
    if (on) idx[n++] = m;
  }
  return n;
}
