// Basis-function table of the pixel grid (paper Section II-C; pixels of 2, 8 or 18 triangles with
// alternating, uniform or random diagonals, Section V-A; corner-only contact is no connection,
// Section VI-A).  A pixel is s x s sub-squares of the fine lattice (s = 1, 2, 3), each cut by one
// diagonal.  Table-driven: the two halves of a sub-square, which half owns each side, and which
// triangle corner is the free RWG vertex are fixed per diagonal orientation and looked up instead
// of searched.  A port's delta gap is the s edges between its two stub pixels (one edge, the
// port BF, when s = 1).
//
// Via state (grids with three pixel states, two-triangle pixels; the paper names additional
// states with vias as future work, Section VIII): a vertical strip stands on the pixel diagonal
// D0-D1 from layer l to layer l+1, cut along D0@l - D1@l+1 into the triangles
// Ta = (D0@l, D1@l, D1@l+1) and Tb = (D0@l, D1@l+1, D0@l+1) (triangle keys with half 2 and 3).
// Its three BFs follow the pixel-port BFs, per via layer and pixel row-major: strip diagonal
// (Ta -> Tb), junction with half 0 of the via pixel (half 0 -> Ta) and junction with half 0 of
// the pixel above (Tb -> that half).
#include "pmom_internal.h"

namespace pmom {
namespace {

// Sub-square sides.
enum Side { kBottom = 0, kRight = 1, kTop = 2, kLeft = 3 };

// Orientation o = orient(g, X, Y): o = 0 -> diagonal (X, Y+1)-(X+1, Y); o = 1 -> (X, Y)-(X+1, Y+1).
// Triangle corners in canonical order, as corner codes 0:(X,Y) 1:(X+1,Y) 2:(X,Y+1) 3:(X+1,Y+1):
//   o = 0: half 0 = {0, 1, 2}, half 1 = {1, 3, 2};  o = 1: half 0 = {0, 1, 3}, half 1 = {0, 3, 2}.
// For each orientation and side: the half holding that side and the index of the corner opposite it.
struct HalfFree {
  int8_t half, free_vertex;
};
constexpr HalfFree kSideOwner[2][4] = {
    /* o = 0 */ {{0, 2}, {1, 2}, {1, 0}, {0, 1}},
    /* o = 1 */ {{0, 2}, {0, 0}, {1, 0}, {1, 1}},
};
// Free vertex of each half for the sub-square's own diagonal.
constexpr int8_t kDiagFree[2][2] = {{0, 1}, {1, 2}};

// Fine-lattice triangle key; half 0, 1: the sub-square's own triangles; 2, 3: Ta, Tb of a via strip
int32_t tri_key(const Grid& g, int layer, int X, int Y, int half) {
  const int W = 128 * g.subs(), off = 4 * g.subs();
  return ((layer * W + (Y + off)) * W + (X + off)) * 4 + half;
}

void put_diag(const Grid& g, int32_t* r, int layer, int X, int Y) {
  const int o = orient(g, X, Y);
  r[4] = tri_key(g, layer, X, Y, 0);
  r[5] = tri_key(g, layer, X, Y, 1);
  r[6] = kDiagFree[o][0];
  r[7] = kDiagFree[o][1];
}

// BF on the edge shared by fine-lattice neighbours P (positive triangle) and Q (negative triangle).
void put_side(const Grid& g, int32_t* r, int layer, int px, int py, int qx, int qy) {
  Side sp, sq;
  if (qx == px + 1) { sp = kRight; sq = kLeft; }
  else if (qx == px - 1) { sp = kLeft; sq = kRight; }
  else if (qy == py + 1) { sp = kTop; sq = kBottom; }
  else { sp = kBottom; sq = kTop; }
  const HalfFree a = kSideOwner[orient(g, px, py)][sp];
  const HalfFree b = kSideOwner[orient(g, qx, qy)][sq];
  r[4] = tri_key(g, layer, px, py, a.half);
  r[5] = tri_key(g, layer, qx, qy, b.half);
  r[6] = a.free_vertex;
  r[7] = b.free_vertex;
}

// Feed stub of a port: s1 touches the grid, s2 lies outside it, g is the grid pixel touched.
void stub(const Grid& g, const pmom_port& p, int s1[2], int s2[2], int gp[2]) {
  static const int dir[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
  const int dx = dir[p.side][0], dy = dir[p.side][1];
  if (dx != 0) {
    gp[0] = dx > 0 ? g.nx - 1 : 0;
    gp[1] = p.pos;
  } else {
    gp[0] = p.pos;
    gp[1] = dy > 0 ? g.ny - 1 : 0;
  }
  s1[0] = gp[0] + dx; s1[1] = gp[1] + dy;
  s2[0] = s1[0] + dx; s2[1] = s1[1] + dy;
}

}  // namespace

// SplitMix64 (Steele, Lea and Flood 2014) chained over (diag_seed, fine position) for the random pattern.
int orient(const Grid& g, int X, int Y) {
  if (g.diag_pattern == 1) return 0;
  if (g.diag_pattern == 2) {
    auto mix = [](uint64_t v) {
      uint64_t z = v + 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    const int s = g.subs();
    const uint64_t h = mix(mix(g.diag_seed) ^ static_cast<uint64_t>((Y + 4 * s) * (128 * s) + (X + 4 * s)));
    return static_cast<int>(h >> 63);
  }
  return (X + Y) & 1;
}

int build_bf_table(const Grid& g, std::vector<int32_t>& t) {
  const int s = g.subs(), ni = g.inner_bfs();
  const int M = g.n_ports * (g.stub_bfs() + s) +
                g.layers * (g.nx * g.ny * ni + s * ((g.nx - 1) * g.ny + g.nx * (g.ny - 1))) +
                (g.vias() ? 3 * (g.layers - 1) * g.nx * g.ny : 0);
  t.assign(static_cast<size_t>(M) * kTableCols, -1);
  int m = 0;
  auto row = [&](int kind, int pa, int pb, int port) {
    int32_t* r = &t[static_cast<size_t>(m++) * kTableCols];
    r[0] = kind; r[1] = pa; r[2] = pb; r[3] = port;
    return r;
  };
  auto pix = [&](int l, int x, int y) { return (l * g.ny + y) * g.nx + x; };
  // inner BFs of pixel (x, y): per sub-square row-major, its diagonal, its +x and +y neighbours
  auto inner = [&](int kind, int pa, int port, int l, int x, int y) {
    for (int j = 0; j < s; ++j)
      for (int i = 0; i < s; ++i) {
        const int X = s * x + i, Y = s * y + j;
        put_diag(g, row(kind, pa, -1, port), l, X, Y);
        if (i + 1 < s) put_side(g, row(kind, pa, -1, port), l, X, Y, X + 1, Y);
        if (j + 1 < s) put_side(g, row(kind, pa, -1, port), l, X, Y, X, Y + 1);
      }
  };
  // the s edges of the side shared by neighbour pixels P (positive) and Q (negative)
  auto side = [&](int kind, int pa, int pb, int port, int l, int px, int py, int qx, int qy) {
    for (int k = 0; k < s; ++k) {
      int PX, PY, QX, QY;
      if (qx != px) {
        PX = qx > px ? s * px + s - 1 : s * px;
        QX = qx > px ? s * qx : s * qx + s - 1;
        PY = QY = s * py + k;
      } else {
        PY = qy > py ? s * py + s - 1 : s * py;
        QY = qy > py ? s * qy : s * qy + s - 1;
        PX = QX = s * px + k;
      }
      put_side(g, row(kind, pa, pb, port), l, PX, PY, QX, QY);
    }
  };
  for (int p = 0; p < g.n_ports; ++p) {
    int s1[2], s2[2], gp[2];
    const int l = g.ports[p].layer;
    stub(g, g.ports[p], s1, s2, gp);
    inner(kAlways, -1, p, l, s1[0], s1[1]);
    side(kAlways, -1, -1, p, l, s2[0], s2[1], s1[0], s1[1]);   // delta-gap edges, + outside
    inner(kAlways, -1, p, l, s2[0], s2[1]);
  }
  for (int l = 0; l < g.layers; ++l)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        inner(kInner, pix(l, x, y), -1, l, x, y);
        if (x + 1 < g.nx) side(kInter, pix(l, x, y), pix(l, x + 1, y), -1, l, x, y, x + 1, y);
        if (y + 1 < g.ny) side(kInter, pix(l, x, y), pix(l, x, y + 1), -1, l, x, y, x, y + 1);
      }
  for (int p = 0; p < g.n_ports; ++p) {
    int s1[2], s2[2], gp[2];
    const int l = g.ports[p].layer;
    stub(g, g.ports[p], s1, s2, gp);
    side(kPixPort, pix(l, gp[0], gp[1]), -1, p, l, s1[0], s1[1], gp[0], gp[1]);
  }
  if (g.vias())
    for (int l = 0; l + 1 < g.layers; ++l)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          const int8_t f0 = kDiagFree[orient(g, x, y)][0];   // corner of half 0 off the diagonal
          int32_t* r = row(kViaStrip, pix(l, x, y), -1, -1);
          r[4] = tri_key(g, l, x, y, 2); r[5] = tri_key(g, l, x, y, 3); r[6] = 1; r[7] = 2;
          r = row(kViaJoin, pix(l, x, y), -1, -1);
          r[4] = tri_key(g, l, x, y, 0); r[5] = tri_key(g, l, x, y, 2); r[6] = f0; r[7] = 2;
          r = row(kViaLand, pix(l, x, y), pix(l + 1, x, y), -1);
          r[4] = tri_key(g, l, x, y, 3); r[5] = tri_key(g, l + 1, x, y, 0); r[6] = 0; r[7] = f0;
        }
  return M;
}

}  // namespace pmom
