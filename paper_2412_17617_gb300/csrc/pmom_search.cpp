// Depth-increasing all-way tree search (paper Algorithm 1, Section III-A) over the GPU evaluator.
//
// Each level of a tree is evaluated as one batch through the evaluator.  Readings where the
// algorithm leaves a choice open: a pixel is an (x, y) column whose state is the pattern of its
// layers' states, a mixed-radix number with layer 0 as the lowest digit (radix 2, or 3 for the
// layers below the last one on a grid with the via state; K = 2^layers on an on/off grid), so
// every node branches into the K - 1 other states of its chosen column; the column is drawn
// uniformly among those not yet on the node's path with a counter-based SplitMix64 generator
// keyed by (seed, restart, iteration, depth, node); the best depth-D leaf (lowest index on ties)
// is accepted only if strictly better; after M(D) failures the depth grows, and past Dmax the
// search restarts from a random half-filled map at depth 1 (a metal pixel below the last layer
// of a via grid is a via when the generator's next bit is set), keeping the global best; it
// stops once the evaluation budget is spent (a started tree is finished).  A candidate whose
// evaluation failed counts as +infinity.
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "pmom_internal.h"

namespace {

uint64_t mix64(uint64_t x) {   // SplitMix64 output function, state advanced by the golden gamma
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t chain(std::initializer_list<uint64_t> parts) {
  uint64_t h = 0;
  for (uint64_t p : parts) h = mix64(h ^ p);
  return h;
}

struct Shape {
  int L, ny, nx;
  bool vias;
  int cols() const { return ny * nx; }
  size_t pix() const { return static_cast<size_t>(L) * ny * nx; }
  int radix(int l) const { return (vias && l < L - 1) ? 3 : 2; }
  int states() const {
    int k = 1;
    for (int l = 0; l < L; ++l) k *= radix(l);
    return k;
  }
};

int col_state(const uint8_t* m, const Shape& s, int j) {
  int v = 0, w = 1;
  for (int l = 0; l < s.L; ++l) {
    v += m[static_cast<size_t>(l) * s.cols() + j] * w;
    w *= s.radix(l);
  }
  return v;
}

void set_col(uint8_t* m, const Shape& s, int j, int v) {
  for (int l = 0; l < s.L; ++l) {
    m[static_cast<size_t>(l) * s.cols() + j] = static_cast<uint8_t>(v % s.radix(l));
    v /= s.radix(l);
  }
}

}  // namespace

extern "C" pmom_status pmom_search_resume(pmom_ctx* c, const pmom_search_params* prm, const uint8_t* init_map,
                                          pmom_search_state* state, double* trace, int32_t trace_cap,
                                          int32_t* trace_len, void* stream) {
  if (!c || !prm || !state || !state->map || !state->best_map || (!state->valid && !init_map) || prm->d_max < 1 ||
      prm->d_max > 8 || prm->max_evals < 1)
    return PMOM_ERR_INVALID_ARG;
  if (state->valid && (state->depth < 1 || state->depth > prm->d_max || state->counter < 0 || state->evals < 1))
    return PMOM_ERR_INVALID_ARG;
  int32_t M = 0, P = 0;
  pmom_num_bfs(c, &M, &P);
  const pmom::Grid& g = pmom::grid_of(c);
  const Shape sh{g.layers, g.ny, g.nx, g.vias()};
  // a tree of depth D changes D distinct columns: deeper than the column count has no node to draw
  if (prm->d_max > sh.cols()) return PMOM_ERR_INVALID_ARG;
  const size_t npix = sh.pix();
  const int K = sh.states();
  std::vector<uint8_t> batch;
  std::vector<double> fom;
  std::vector<int32_t> status;
  auto evaluate = [&](const std::vector<uint8_t>& maps, int B, std::vector<double>& out) -> pmom_status {
    fom.resize(B);
    status.resize(B);
    const pmom_status st =
        pmom_eval_candidates_host(c, maps.data(), B, prm->precision, nullptr, fom.data(), status.data(), stream);
    if (st) return st;
    out.resize(B);
    for (int b = 0; b < B; ++b) out[b] = std::isfinite(fom[b]) ? fom[b] : std::numeric_limits<double>::infinity();
    return PMOM_OK;
  };
  std::vector<uint8_t> cur, best;
  double F = 0.0, bestF = 0.0;
  int64_t evals = 0;
  int D = 1, counter = 0, tlen = 0;
  uint64_t restart = 0, it = 0;
  std::vector<double> f1;
  pmom_status st = PMOM_OK;
  if (state->valid) {
    cur.assign(state->map, state->map + npix);
    best.assign(state->best_map, state->best_map + npix);
    F = state->fom;
    bestF = state->best_fom;
    evals = state->evals;
    D = state->depth;
    counter = state->counter;
    restart = state->restart;
    it = state->iteration;
  } else {
    cur.assign(init_map, init_map + npix);
    best = cur;
    st = evaluate(cur, 1, f1);
    if (st) return st;
    F = bestF = f1[0];
    evals = 1;
  }
  struct Node {
    std::vector<int> path;   // columns chosen on the way down
    std::vector<uint8_t> map;
  };
  while (evals < prm->max_evals) {
    std::vector<Node> nodes(1, Node{{}, cur});
    std::vector<double> fs;
    for (int d = 0; d < D; ++d) {
      std::vector<Node> children;
      for (size_t k = 0; k < nodes.size(); ++k) {
        std::vector<int> free;
        for (int col = 0; col < sh.cols(); ++col) {
          bool used = false;
          for (int q : nodes[k].path) used |= (q == col);
          if (!used) free.push_back(col);
        }
        const uint64_t u = chain({prm->seed, restart, it, static_cast<uint64_t>(d), static_cast<uint64_t>(k)});
        const int j = free[u % free.size()];
        const int s0 = col_state(nodes[k].map.data(), sh, j);
        for (int v = 0; v < K; ++v) {
          if (v == s0) continue;
          Node ch{nodes[k].path, nodes[k].map};
          ch.path.push_back(j);
          set_col(ch.map.data(), sh, j, v);
          children.push_back(std::move(ch));
        }
      }
      batch.resize(children.size() * npix);
      for (size_t b = 0; b < children.size(); ++b) std::memcpy(&batch[b * npix], children[b].map.data(), npix);
      st = evaluate(batch, static_cast<int>(children.size()), fs);
      if (st) return st;
      evals += static_cast<int64_t>(children.size());
      nodes.swap(children);
    }
    size_t bi = 0;
    for (size_t b = 1; b < fs.size(); ++b)
      if (fs[b] < fs[bi]) bi = b;
    if (fs[bi] < F) {
      cur = nodes[bi].map;
      F = fs[bi];
      counter = 0;
    } else {
      ++counter;
    }
    if (F < bestF) { best = cur; bestF = F; }
    if (counter >= prm->m_of_d[D - 1]) { ++D; counter = 0; }
    if (D > prm->d_max) {
      ++restart;
      const size_t below_top = static_cast<size_t>(sh.L - 1) * sh.cols();
      for (size_t i = 0; i < npix; ++i) {
        const uint64_t u = chain({prm->seed, 0xA5A5ull, restart, i});
        int v = static_cast<int>(u >> 63);
        if (v && sh.vias && i < below_top) v = 1 + static_cast<int>((u >> 62) & 1);
        cur[i] = static_cast<uint8_t>(v);
      }
      st = evaluate(cur, 1, f1);
      if (st) return st;
      F = f1[0];
      ++evals;
      D = 1;
      counter = 0;
      if (F < bestF) { best = cur; bestF = F; }
    }
    if (trace && tlen < trace_cap) trace[tlen] = F;
    ++tlen;
    ++it;
  }
  std::memcpy(state->map, cur.data(), npix);
  std::memcpy(state->best_map, best.data(), npix);
  state->fom = F;
  state->best_fom = bestF;
  state->evals = evals;
  state->depth = D;
  state->counter = counter;
  state->restart = restart;
  state->iteration = it;
  state->valid = 1;
  if (trace_len) *trace_len = tlen < trace_cap ? tlen : trace_cap;
  return PMOM_OK;
}

extern "C" pmom_status pmom_search(pmom_ctx* c, const pmom_search_params* prm, const uint8_t* init_map,
                                   uint8_t* best_map, double* best_fom, int64_t* evals_used, double* trace,
                                   int32_t trace_cap, int32_t* trace_len, void* stream) {
  if (!c || !prm || !init_map || !best_map || !best_fom) return PMOM_ERR_INVALID_ARG;
  const pmom::Grid& g = pmom::grid_of(c);
  std::vector<uint8_t> cur(static_cast<size_t>(g.layers) * g.ny * g.nx);
  pmom_search_state state{};
  state.valid = 0;
  state.map = cur.data();
  state.best_map = best_map;
  const pmom_status st = pmom_search_resume(c, prm, init_map, &state, trace, trace_cap, trace_len, stream);
  if (st) return st;
  *best_fom = state.best_fom;
  if (evals_used) *evals_used = state.evals;
  return PMOM_OK;
}
