// Basis-function table of the pixel grid (paper Section II-C; alternating 2-triangle pixels of
// Section V-A; corner-only contact is no connection, Section VI-A).  Table-driven: the two
// halves of a pixel, which half owns each pixel side, and which triangle corner is the free RWG
// vertex are fixed per diagonal orientation and looked up instead of searched.
//
// Via state (grids with three pixel states; the paper names additional states with vias as future
// work, Section VIII): a vertical strip stands on the pixel diagonal D0-D1 from layer l to layer
// l+1, cut along D0@l - D1@l+1 into the triangles Ta = (D0@l, D1@l, D1@l+1) and
// Tb = (D0@l, D1@l+1, D0@l+1) (triangle keys with half 2 and 3).  Its three BFs follow the pixel-port BFs, per via layer and
// pixel row-major: strip diagonal (Ta -> Tb), junction with half 0 of the via pixel (half 0 -> Ta)
// and junction with half 0 of the pixel above (Tb -> that half).
#include "pmom_internal.h"

namespace pmom {
namespace {

// Pixel sides.
enum Side { kBottom = 0, kRight = 1, kTop = 2, kLeft = 3 };

// Orientation o = orient(g, x, y): o = 0 -> diagonal (x, y+1)-(x+1, y); o = 1 -> (x, y)-(x+1, y+1).
// Triangle corners in canonical order, as corner codes 0:(x,y) 1:(x+1,y) 2:(x,y+1) 3:(x+1,y+1):
//   o = 0: half 0 = {0, 1, 2}, half 1 = {1, 3, 2};  o = 1: half 0 = {0, 1, 3}, half 1 = {0, 3, 2}.
// For each orientation and side: the half holding that side and the index of the corner opposite it.
struct HalfFree {
  int8_t half, free_vertex;
};
constexpr HalfFree kSideOwner[2][4] = {
    /* o = 0 */ {{0, 2}, {1, 2}, {1, 0}, {0, 1}},
    /* o = 1 */ {{0, 2}, {0, 0}, {1, 0}, {1, 1}},
};
// Free vertex of each half for the pixel's own diagonal.
constexpr int8_t kDiagFree[2][2] = {{0, 1}, {1, 2}};

// half 0, 1: the pixel's own triangles; 2, 3: Ta, Tb of the via strip standing on it
int32_t tri_key(int layer, int x, int y, int half) { return ((layer * 128 + (y + 4)) * 128 + (x + 4)) * 4 + half; }

void put_diag(const Grid& g, int32_t* r, int layer, int x, int y) {
  const int o = orient(g, x, y);
  r[4] = tri_key(layer, x, y, 0);
  r[5] = tri_key(layer, x, y, 1);
  r[6] = kDiagFree[o][0];
  r[7] = kDiagFree[o][1];
}

// BF on the side shared by lattice neighbours P (positive triangle) and Q (negative triangle).
void put_side(const Grid& g, int32_t* r, int layer, int px, int py, int qx, int qy) {
  Side sp, sq;
  if (qx == px + 1) { sp = kRight; sq = kLeft; }
  else if (qx == px - 1) { sp = kLeft; sq = kRight; }
  else if (qy == py + 1) { sp = kTop; sq = kBottom; }
  else { sp = kBottom; sq = kTop; }
  const HalfFree a = kSideOwner[orient(g, px, py)][sp];
  const HalfFree b = kSideOwner[orient(g, qx, qy)][sq];
  r[4] = tri_key(layer, px, py, a.half);
  r[5] = tri_key(layer, qx, qy, b.half);
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

// SplitMix64 (Steele, Lea and Flood 2014) chained over (diag_seed, position) for the random pattern.
int orient(const Grid& g, int x, int y) {
  if (g.diag_pattern == 1) return 0;
  if (g.diag_pattern == 2) {
    auto mix = [](uint64_t v) {
      uint64_t z = v + 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    const uint64_t h = mix(mix(g.diag_seed) ^ static_cast<uint64_t>((y + 4) * 128 + (x + 4)));
    return static_cast<int>(h >> 63);
  }
  return (x + y) & 1;
}

int build_bf_table(const Grid& g, std::vector<int32_t>& t) {
  const int M = 4 * g.n_ports + g.layers * (g.nx * g.ny + (g.nx - 1) * g.ny + g.nx * (g.ny - 1)) +
                (g.vias() ? 3 * (g.layers - 1) * g.nx * g.ny : 0);
  t.assign(static_cast<size_t>(M) * kTableCols, -1);
  int m = 0;
  auto row = [&](int kind, int pa, int pb, int port) {
    int32_t* r = &t[static_cast<size_t>(m++) * kTableCols];
    r[0] = kind; r[1] = pa; r[2] = pb; r[3] = port;
    return r;
  };
  auto pix = [&](int l, int x, int y) { return (l * g.ny + y) * g.nx + x; };
  for (int p = 0; p < g.n_ports; ++p) {
    int s1[2], s2[2], gp[2];
    const int l = g.ports[p].layer;
    stub(g, g.ports[p], s1, s2, gp);
    put_diag(g, row(kAlways, -1, -1, p), l, s1[0], s1[1]);
    put_side(g, row(kAlways, -1, -1, p), l, s2[0], s2[1], s1[0], s1[1]);   // delta-gap edge, + outside
    put_diag(g, row(kAlways, -1, -1, p), l, s2[0], s2[1]);
  }
  for (int l = 0; l < g.layers; ++l)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        put_diag(g, row(kInner, pix(l, x, y), -1, -1), l, x, y);
        if (x + 1 < g.nx) put_side(g, row(kInter, pix(l, x, y), pix(l, x + 1, y), -1), l, x, y, x + 1, y);
        if (y + 1 < g.ny) put_side(g, row(kInter, pix(l, x, y), pix(l, x, y + 1), -1), l, x, y, x, y + 1);
      }
  for (int p = 0; p < g.n_ports; ++p) {
    int s1[2], s2[2], gp[2];
    const int l = g.ports[p].layer;
    stub(g, g.ports[p], s1, s2, gp);
    put_side(g, row(kPixPort, pix(l, gp[0], gp[1]), -1, p), l, s1[0], s1[1], gp[0], gp[1]);
  }
  if (g.vias())
    for (int l = 0; l + 1 < g.layers; ++l)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          const int8_t f0 = kDiagFree[orient(g, x, y)][0];   // corner of half 0 off the diagonal
          int32_t* r = row(kViaStrip, pix(l, x, y), -1, -1);
          r[4] = tri_key(l, x, y, 2); r[5] = tri_key(l, x, y, 3); r[6] = 1; r[7] = 2;
          r = row(kViaJoin, pix(l, x, y), -1, -1);
          r[4] = tri_key(l, x, y, 0); r[5] = tri_key(l, x, y, 2); r[6] = f0; r[7] = 2;
          r = row(kViaLand, pix(l, x, y), pix(l + 1, x, y), -1);
          r[4] = tri_key(l, x, y, 3); r[5] = tri_key(l + 1, x, y, 0); r[6] = 0; r[7] = f0;
        }
  return M;
}

}  // namespace pmom
