// C ABI of the evaluator: context, parent-database residency, FoM bands, and the evaluation
// pipeline (activation -> persistent evaluation -> FP64 repair of unconverged tasks -> FoM).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pmom_internal.h"

struct pmom_ctx {
  int device = 0;
  int num_sms = 0;
  pmom::Grid grid;
  int M = 0;
  std::vector<int32_t> table;
  int4* d_rules = nullptr;
  // parent database
  int F = 0;
  int dtype = PMOM_C64;
  void* d_Z = nullptr;
  size_t z_bytes = 0;
  std::vector<double> freqs;
  // figure of merit
  bool fom_ready = false;
  uint8_t* d_bands = nullptr;
  double Z0 = 50.0;
  // per-batch buffers (grown on demand)
  int b_cap = 0;
  int32_t* d_idx = nullptr;
  int32_t* d_nact = nullptr;
  uint32_t* d_flags = nullptr;
  double2* d_S = nullptr;
  int* d_repair = nullptr;
  int* d_order = nullptr;
  uint8_t* d_maps_stage = nullptr;
  double* d_fom_stage = nullptr;
  int32_t* d_status_stage = nullptr;
  // scalars: [0] task counter, [1] repair count, then 4 x u64 counters
  void* d_small = nullptr;
  // slot workspaces
  void* d_work = nullptr;
  size_t work_bytes = 0;
  int max_slots = 0;   // > 0: task slots limited by free device memory (large support sets)
  cudaStream_t last_stream = nullptr;
  int64_t launches = 0;
  bool timing = false;
  bool timed = false;
  int use_tc = 1;    // tensor-core trailing updates in the single-precision LU
  // autotuner table per support-set bucket (pmom::n_bucket): tensor-core LU, task groups per CTA,
  // resident-task cap in quarters of the full slot count; valid = measured on a batch
  uint8_t tune_valid[pmom::kNBuckets] = {};
  uint8_t tune_tc[pmom::kNBuckets] = {};
  uint8_t tune_groups[pmom::kNBuckets] = {};
  uint8_t tune_cap[pmom::kNBuckets] = {};
  float tune_ms[pmom::kNBuckets] = {};
  // captured evaluation pipeline (pmom_graph_capture / pmom_graph_launch)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_stream = nullptr;   // capture stream (the legacy default stream cannot be captured)
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // bordered evaluation: reference support set, FP64 factors and inverses, per-slot scratch
  int32_t* d_ref_idx = nullptr;    // [M] then n (one int) and the reference's bad-state flag
  uint32_t* d_ref_flags = nullptr;  // [F]
  double2* d_ref_lu = nullptr;
  double2* d_ref_g = nullptr;
  int* d_ref_piv = nullptr;
  size_t ref_cap = 0;               // elements of d_ref_lu / d_ref_g
  double2* d_bwork = nullptr;
  size_t bwork_elems = 0;
  void* d_ref_work = nullptr;       // single-precision reference factors, one evaluation slot per frequency
  size_t ref_work_bytes = 0;
  std::string err;
};

namespace pmom {
const Grid& grid_of(const pmom_ctx* c) { return c->grid; }
}  // namespace pmom

namespace {

pmom_status fail(pmom_ctx* c, pmom_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

pmom_status cuda_fail(pmom_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? PMOM_ERR_OOM : PMOM_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define PMOM_CUDA(ctx, call)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

template <typename T>
void free_dev(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

size_t z_elem(int dtype) { return dtype == PMOM_C128 ? 16 : 8; }

pmom_status ensure_batch(pmom_ctx* c, int B) {
  if (B <= c->b_cap && c->d_idx) return PMOM_OK;
  free_dev(c->d_idx);
  free_dev(c->d_nact);
  free_dev(c->d_flags);
  free_dev(c->d_S);
  free_dev(c->d_repair);
  free_dev(c->d_order);
  free_dev(c->d_maps_stage);
  free_dev(c->d_fom_stage);
  free_dev(c->d_status_stage);
  const int P = c->grid.n_ports;
  PMOM_CUDA(c, cudaMalloc(&c->d_idx, sizeof(int32_t) * static_cast<size_t>(B) * c->M));
  PMOM_CUDA(c, cudaMalloc(&c->d_nact, sizeof(int32_t) * B));
  PMOM_CUDA(c, cudaMalloc(&c->d_flags, sizeof(uint32_t) * B));
  PMOM_CUDA(c, cudaMalloc(&c->d_S, sizeof(double2) * static_cast<size_t>(B) * c->F * P * P));
  PMOM_CUDA(c, cudaMalloc(&c->d_repair, sizeof(int) * static_cast<size_t>(B) * c->F));
  PMOM_CUDA(c, cudaMalloc(&c->d_order, sizeof(int) * static_cast<size_t>(B)));
  PMOM_CUDA(c, cudaMalloc(&c->d_maps_stage, static_cast<size_t>(B) * c->grid.pixels()));
  PMOM_CUDA(c, cudaMalloc(&c->d_fom_stage, sizeof(double) * B));
  PMOM_CUDA(c, cudaMalloc(&c->d_status_stage, sizeof(int32_t) * B));
  c->b_cap = B;
  return PMOM_OK;
}

// Support-set capacity of a launch: the batch's largest set, clipped to what one task group's
// shared memory holds for this precision (larger candidates are flagged, not solved).
int ncap_for(pmom_ctx* c, int precision, int ncap) {
  const int mx = pmom::eval_max_ncap(precision, c->M);
  if (ncap > mx) ncap = mx;
  return ncap < 1 ? 1 : ncap;
}

// The launch configuration the autotuner chose for the batch's largest support set (the
// dominant bucket: the largest tasks carry most of the work): the single-precision kernel
// variant, task groups per CTA and the resident-task cap; per-task LU choice by bucket.
struct LaunchTune {
  int use_tc, max_groups, cap4;
  uint8_t tc_bucket[pmom::kNBuckets];
};
LaunchTune tune_for(const pmom_ctx* c, int ncap) {
  LaunchTune t{};
  const int bd = pmom::n_bucket(ncap);
  for (int b = 0; b < pmom::kNBuckets; ++b) t.tc_bucket[b] = static_cast<uint8_t>(c->tune_valid[b] ? c->tune_tc[b] : c->use_tc);
  t.use_tc = t.tc_bucket[bd];
  t.max_groups = c->tune_valid[bd] ? c->tune_groups[bd] : 0;
  t.cap4 = c->tune_valid[bd] ? c->tune_cap[bd] : 4;
  return t;
}
void apply_tune(const LaunchTune& t, pmom::EvalArgs& a) {
  a.use_tc = t.use_tc;
  a.max_groups = t.max_groups;
  for (int b = 0; b < pmom::kNBuckets; ++b) a.tc_bucket[b] = t.tc_bucket[b];
}

int slots_for(pmom_ctx* c, int precision, int tasks, int ncap, const LaunchTune* t = nullptr) {
  const int use_tc = t ? t->use_tc : c->use_tc;
  const int per_sm = pmom::eval_blocks_per_sm(precision, ncap, c->dtype == PMOM_C128, use_tc, t ? t->max_groups : 0);
  int n = (per_sm > 0 ? per_sm : 1) * c->num_sms;
  if (t && t->cap4 > 0 && t->cap4 < 4) n = (n * t->cap4 + 3) / 4;
  if (c->max_slots > 0 && n > c->max_slots) n = c->max_slots;
  if (n > tasks) n = tasks;
  return n < 1 ? 1 : n;
}

// Slot workspaces for this call: the launch of `precision` and, for the mixed path, the FP64
// repair launch that follows it (they reuse the same memory one after the other).
pmom_status ensure_work(pmom_ctx* c, int precision, int tasks, int ncap) {
  auto need_of = [&](size_t* sb_max) {
    size_t need = 0;
    *sb_max = 0;
    for (int prec = 0; prec < 2; ++prec) {
      if (prec != precision && prec != PMOM_FP64) continue;
      int lda = 0;
      const size_t sb = pmom::eval_slot_bytes(prec, ncap_for(c, prec, ncap), c->grid.n_ports, &lda);
      size_t n = static_cast<size_t>(slots_for(c, prec, tasks, ncap_for(c, prec, ncap)));
      if (prec != PMOM_FP64) {   // the tuned variant may be either LU kernel: room for the larger
        LaunchTune t{};
        t.use_tc = 1 - c->use_tc;
        t.cap4 = 4;
        const size_t n2 = static_cast<size_t>(slots_for(c, prec, tasks, ncap_for(c, prec, ncap), &t));
        if (n2 > n) n = n2;
      }
      if (sb * n > need) need = sb * n;
      if (sb > *sb_max) *sb_max = sb;
    }
    return need;
  };
  c->max_slots = 0;
  size_t sb_max = 0;
  size_t need = need_of(&sb_max);
  if (need <= c->work_bytes && c->d_work) return PMOM_OK;
  free_dev(c->d_work);
  c->work_bytes = 0;
  // large support sets: as many slots as free memory allows (1 GiB kept for the runtime)
  size_t free_b = 0, total_b = 0;
  PMOM_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
  const size_t reserve = size_t(1) << 30;
  if (need + reserve > free_b) {
    const size_t fit = free_b > reserve + sb_max ? (free_b - reserve) / sb_max : 1;
    c->max_slots = static_cast<int>(fit < 1 ? 1 : fit);
    need = need_of(&sb_max);
  }
  PMOM_CUDA(c, cudaMalloc(&c->d_work, need));
  c->work_bytes = need;
  return PMOM_OK;
}

// Device-side state is created on first use, so that a context (and its BF table) can be built
// on a machine without a GPU.
pmom_status ensure_device(pmom_ctx* c) {
  if (c->d_rules) return PMOM_OK;
  PMOM_CUDA(c, cudaGetDevice(&c->device));
  PMOM_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  (void)pmom::tensor_map_encoder_ptr();   // looked up here, outside any stream capture (null: CUDA-core path only)
  std::vector<int4> rules(c->M);
  for (int m = 0; m < c->M; ++m) {
    const int32_t* r = &c->table[static_cast<size_t>(m) * pmom::kTableCols];
    rules[m] = make_int4(r[0], r[1], r[2], 0);
  }
  PMOM_CUDA(c, cudaMalloc(&c->d_small, 256));
  PMOM_CUDA(c, cudaMalloc(&c->d_rules, sizeof(int4) * c->M));
  PMOM_CUDA(c, cudaMemcpy(c->d_rules, rules.data(), sizeof(int4) * c->M, cudaMemcpyHostToDevice));
  return PMOM_OK;
}

}  // namespace

extern "C" {

pmom_status pmom_selftest_wait(int64_t polls, int32_t arrive, int32_t* timed_out, double* elapsed_ms, void* stream) {
  if (polls < 1 || polls > (1ll << 30) || !timed_out || !elapsed_ms) return PMOM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = pmom::launch_wait_selftest(polls, arrive != 0, d_out, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_out, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) return PMOM_ERR_CUDA;
  *timed_out = h;
  *elapsed_ms = ms;
  return PMOM_OK;
}

pmom_status pmom_create(const pmom_grid_desc* g, pmom_ctx** out) {
  if (!g || !out) return PMOM_ERR_INVALID_ARG;
  *out = nullptr;
  if (g->layers < 1 || g->layers > 8 || g->nx < 1 || g->ny < 1 || g->nx > 100 || g->ny > 100 || g->pitch_m <= 0 ||
      g->n_ports < 1 || g->n_ports > pmom::kMaxPorts || !g->ports || !g->layer_z_m || g->medium < 0 || g->medium > 2)
    return PMOM_ERR_INVALID_ARG;
  // layered (grounded-slab) kernels are those of horizontal currents: no via state there
  if (g->medium == 2 && g->n_states >= 3) return PMOM_ERR_UNSUPPORTED;
  if (g->n_states != 2 && g->n_states != 3) return PMOM_ERR_UNSUPPORTED;
  if (g->n_states == 3 && g->layers < 2) return PMOM_ERR_INVALID_ARG;   // a via needs a layer above
  if (g->diag_pattern < 0 || g->diag_pattern > 2) return PMOM_ERR_INVALID_ARG;
  if (g->sub < 0 || g->sub > 3) return PMOM_ERR_INVALID_ARG;
  if (g->sub > 1 && g->n_states == 3) return PMOM_ERR_INVALID_ARG;   // the via stands on a pixel diagonal
  for (int p = 0; p < g->n_ports; ++p) {
    const pmom_port& q = g->ports[p];
    const int lim = (q.side == 0 || q.side == 2) ? g->ny : g->nx;
    if (q.layer < 0 || q.layer >= g->layers || q.side < 0 || q.side > 3 || q.pos < 0 || q.pos >= lim)
      return PMOM_ERR_INVALID_ARG;
  }
  pmom_ctx* c = new pmom_ctx();
  pmom::Grid& gr = c->grid;
  gr.layers = g->layers; gr.nx = g->nx; gr.ny = g->ny; gr.medium = g->medium; gr.n_states = g->n_states;
  gr.diag_pattern = g->diag_pattern; gr.diag_seed = g->diag_seed; gr.sub = g->sub > 1 ? g->sub : 1;
  gr.n_ports = g->n_ports; gr.pitch = g->pitch_m; gr.h_total = g->h_total_m; gr.eps_r = g->eps_r; gr.tan_d = g->tan_d;
  gr.layer_z.assign(g->layer_z_m, g->layer_z_m + g->layers);
  gr.ports.assign(g->ports, g->ports + g->n_ports);
  c->M = pmom::build_bf_table(gr, c->table);
  *out = c;
  return PMOM_OK;
}

pmom_status pmom_destroy(pmom_ctx* c) {
  if (!c) return PMOM_OK;
  free_dev(c->d_rules);
  free_dev(c->d_Z);
  free_dev(c->d_bands);
  free_dev(c->d_idx);
  free_dev(c->d_nact);
  free_dev(c->d_flags);
  free_dev(c->d_S);
  free_dev(c->d_repair);
  free_dev(c->d_maps_stage);
  free_dev(c->d_fom_stage);
  free_dev(c->d_status_stage);
  free_dev(c->d_small);
  free_dev(c->d_work);
  free_dev(c->d_order);
  free_dev(c->d_ref_idx);
  free_dev(c->d_ref_flags);
  free_dev(c->d_ref_lu);
  free_dev(c->d_ref_g);
  free_dev(c->d_ref_piv);
  free_dev(c->d_bwork);
  free_dev(c->d_ref_work);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return PMOM_OK;
}

const char* pmom_last_error(const pmom_ctx* c) { return c ? c->err.c_str() : "null context"; }

pmom_status pmom_num_bfs(const pmom_ctx* c, int32_t* M, int32_t* P) {
  if (!c || !M) return PMOM_ERR_INVALID_ARG;
  *M = c->M;
  if (P) *P = c->grid.n_ports;
  return PMOM_OK;
}

pmom_status pmom_bf_table(const pmom_ctx* c, int32_t* out) {
  if (!c || !out) return PMOM_ERR_INVALID_ARG;
  std::memcpy(out, c->table.data(), sizeof(int32_t) * c->table.size());
  return PMOM_OK;
}

pmom_status pmom_load_Z(pmom_ctx* c, const double* freqs, int32_t F, const void* Z, int32_t dtype, int32_t mem,
                        void* stream) {
  if (!c) return PMOM_ERR_INVALID_ARG;
  if (c) {
    const pmom_status dv = ensure_device(c);
    if (dv) return dv;
  }
  if (!freqs || !Z || (dtype != PMOM_C64 && dtype != PMOM_C128) || (mem != PMOM_MEM_HOST && mem != PMOM_MEM_DEVICE))
    return fail(c, PMOM_ERR_INVALID_ARG, "load_Z: bad argument");
  if (F < 1) return fail(c, PMOM_ERR_Z_SHAPE_MISMATCH, "load_Z: F < 1");
  const size_t bytes = static_cast<size_t>(F) * c->M * c->M * z_elem(dtype);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (bytes != c->z_bytes) {
    free_dev(c->d_Z);
    c->z_bytes = 0;   // no database until the new allocation succeeds
    PMOM_CUDA(c, cudaMalloc(&c->d_Z, bytes));
    c->z_bytes = bytes;
  }
  PMOM_CUDA(c, cudaMemcpyAsync(c->d_Z, Z, bytes, mem == PMOM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  if (mem == PMOM_MEM_HOST) PMOM_CUDA(c, cudaStreamSynchronize(s));
  if (F != c->F) {
    c->fom_ready = false;
    free_dev(c->d_S);
    free_dev(c->d_repair);
    c->b_cap = 0;
    free_dev(c->d_idx);
  }
  c->F = F;
  c->dtype = dtype;
  c->freqs.assign(freqs, freqs + F);
  return PMOM_OK;
}

namespace {

// ------------------------------------------------------------------ database files
constexpr char kZMagic[8] = {'P', 'M', 'O', 'M', 'Z', 'D', 'B', '1'};
constexpr uint32_t kZVersion = 1;
constexpr size_t kZChunk = size_t(64) << 20;   // bytes per host <-> device transfer

uint64_t fnv1a_bytes(const void* p, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
  return h;
}
// FNV-1a over 64-bit words (n a multiple of 8)
uint64_t fnv1a_words(const void* p, size_t n, uint64_t h) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; i += 8) {
    uint64_t w;
    std::memcpy(&w, b + i, 8);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

struct ZHeader {
  char magic[8];
  uint32_t version, dtype;
  int32_t M, F;
  uint64_t table_hash;
};
static_assert(sizeof(ZHeader) == 32, "database header layout");

uint64_t table_hash(const pmom_ctx* c) {
  return fnv1a_bytes(c->table.data(), c->table.size() * sizeof(int32_t));
}

}  // namespace

pmom_status pmom_save_Z(pmom_ctx* c, const char* path, void* stream) {
  if (!c || !path) return PMOM_ERR_INVALID_ARG;
  if (!c->d_Z) return fail(c, PMOM_ERR_NOT_READY, "save_Z: no database");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* fp = std::fopen(tmp.c_str(), "wb");
  if (!fp) return fail(c, PMOM_ERR_IO, "save_Z: cannot open " + tmp);
  ZHeader h;
  std::memcpy(h.magic, kZMagic, 8);
  h.version = kZVersion;
  h.dtype = static_cast<uint32_t>(c->dtype);
  h.M = c->M;
  h.F = c->F;
  h.table_hash = table_hash(c);
  bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 &&
            std::fwrite(c->freqs.data(), sizeof(double), c->freqs.size(), fp) == c->freqs.size();
  void* host = nullptr;
  if (ok && cudaMallocHost(&host, kZChunk) != cudaSuccess) {
    std::fclose(fp);
    std::remove(tmp.c_str());
    return fail(c, PMOM_ERR_OOM, "save_Z: pinned staging buffer");
  }
  uint64_t sum = 0xcbf29ce484222325ull;
  cudaError_t e = cudaSuccess;
  for (size_t off = 0; ok && off < c->z_bytes; off += kZChunk) {
    const size_t n = std::min(kZChunk, c->z_bytes - off);
    e = cudaMemcpyAsync(host, static_cast<const char*>(c->d_Z) + off, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    sum = fnv1a_words(host, n, sum);
    ok = std::fwrite(host, 1, n, fp) == n;
  }
  if (host) cudaFreeHost(host);
  if (ok && e == cudaSuccess) ok = std::fwrite(&sum, sizeof(sum), 1, fp) == 1;
  ok = (std::fclose(fp) == 0) && ok;
  if (e != cudaSuccess) {
    std::remove(tmp.c_str());
    return fail(c, PMOM_ERR_CUDA, std::string("save_Z: ") + cudaGetErrorString(e));
  }
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(c, PMOM_ERR_IO, std::string("save_Z: write failed for ") + path);
  }
  return PMOM_OK;
}

pmom_status pmom_load_Z_file(pmom_ctx* c, const char* path, void* stream) {
  if (!c || !path) return PMOM_ERR_INVALID_ARG;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(c, PMOM_ERR_IO, std::string("load_Z_file: cannot open ") + path);
  auto bail = [&](pmom_status st, const std::string& msg) {
    std::fclose(fp);
    return fail(c, st, "load_Z_file: " + msg);
  };
  ZHeader h;
  if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, kZMagic, 8) != 0 || h.version != kZVersion)
    return bail(PMOM_ERR_IO, "not a database file (magic or version)");
  if (h.dtype != PMOM_C64 && h.dtype != PMOM_C128) return bail(PMOM_ERR_IO, "unknown storage type");
  if (h.M != c->M || h.table_hash != table_hash(c)) return bail(PMOM_ERR_Z_SHAPE_MISMATCH, "written for another grid");
  if (h.F < 1) return bail(PMOM_ERR_Z_SHAPE_MISMATCH, "F < 1");
  const size_t bytes = static_cast<size_t>(h.F) * h.M * h.M * z_elem(static_cast<int>(h.dtype));
  const uint64_t expect = sizeof(h) + sizeof(double) * static_cast<uint64_t>(h.F) + bytes + sizeof(uint64_t);
  if (std::fseek(fp, 0, SEEK_END) != 0) return bail(PMOM_ERR_IO, "seek");
  const long long size = std::ftell(fp);
  if (size < 0 || static_cast<uint64_t>(size) != expect) return bail(PMOM_ERR_IO, "truncated or oversized file");
  std::vector<double> freqs(h.F);
  if (std::fseek(fp, sizeof(h), SEEK_SET) != 0 ||
      std::fread(freqs.data(), sizeof(double), freqs.size(), fp) != freqs.size())
    return bail(PMOM_ERR_IO, "read frequencies");
  // validated: now the device
  const pmom_status dv = ensure_device(c);
  if (dv) {
    std::fclose(fp);
    return dv;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (bytes != c->z_bytes) {
    free_dev(c->d_Z);
    c->z_bytes = 0;
    if (cudaMalloc(&c->d_Z, bytes) != cudaSuccess) {
      c->d_Z = nullptr;
      return bail(PMOM_ERR_OOM, "database allocation");
    }
    c->z_bytes = bytes;
  }
  void* host = nullptr;
  if (cudaMallocHost(&host, kZChunk) != cudaSuccess) return bail(PMOM_ERR_OOM, "pinned staging buffer");
  uint64_t sum = 0xcbf29ce484222325ull, stored = 0;
  bool ok = true;
  cudaError_t e = cudaSuccess;
  for (size_t off = 0; ok && off < bytes; off += kZChunk) {
    const size_t n = std::min(kZChunk, bytes - off);
    ok = std::fread(host, 1, n, fp) == n;
    if (!ok) break;
    sum = fnv1a_words(host, n, sum);
    e = cudaMemcpyAsync(static_cast<char*>(c->d_Z) + off, host, n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
  }
  cudaFreeHost(host);
  if (ok && e == cudaSuccess) ok = std::fread(&stored, sizeof(stored), 1, fp) == 1;
  std::fclose(fp);
  if (e != cudaSuccess || !ok || stored != sum) {
    free_dev(c->d_Z);
    c->z_bytes = 0;
    c->F = 0;
    c->fom_ready = false;
    if (e != cudaSuccess) return fail(c, PMOM_ERR_CUDA, std::string("load_Z_file: ") + cudaGetErrorString(e));
    return fail(c, PMOM_ERR_IO, !ok ? "load_Z_file: read failed" : "load_Z_file: checksum mismatch");
  }
  if (h.F != c->F) {
    c->fom_ready = false;
    free_dev(c->d_S);
    free_dev(c->d_repair);
    c->b_cap = 0;
    free_dev(c->d_idx);
  }
  c->F = h.F;
  c->dtype = static_cast<int>(h.dtype);
  c->freqs = freqs;
  return PMOM_OK;
}

pmom_status pmom_copy_Z(const pmom_ctx* c, void* out, int32_t mem, void* stream) {
  if (!c || !out) return PMOM_ERR_INVALID_ARG;
  if (!c->d_Z) return PMOM_ERR_NOT_READY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out, c->d_Z, c->z_bytes, mem == PMOM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && mem == PMOM_MEM_HOST) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? PMOM_OK : PMOM_ERR_CUDA;
}

pmom_status pmom_set_fom(pmom_ctx* c, const uint8_t* bands, int32_t F, double Z0) {
  if (!c || !bands || !(Z0 > 0)) return fail(c, PMOM_ERR_INVALID_ARG, "set_fom: bad argument");
  if (!c->d_Z) return fail(c, PMOM_ERR_NOT_READY, "set_fom: load or fill Z first");
  if (F != c->F) return fail(c, PMOM_ERR_Z_SHAPE_MISMATCH, "set_fom: band count differs from the database");
  for (int f = 0; f < F; ++f)
    if (bands[f] > 3 && bands[f] != 255) return fail(c, PMOM_ERR_INVALID_ARG, "set_fom: band code");
  free_dev(c->d_bands);
  PMOM_CUDA(c, cudaMalloc(&c->d_bands, F));
  PMOM_CUDA(c, cudaMemcpy(c->d_bands, bands, F, cudaMemcpyHostToDevice));
  c->Z0 = Z0;
  c->fom_ready = true;
  return PMOM_OK;
}

pmom_status pmom_active_set(pmom_ctx* c, const uint8_t* maps, int32_t B, int32_t* idx_out, int32_t* n_out, void* stream) {
  if (!c || !maps || !idx_out || !n_out || B < 1) return fail(c, PMOM_ERR_INVALID_ARG, "active_set: bad argument");
  pmom_status st = ensure_device(c);
  if (st) return st;
  st = ensure_batch(c, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pmom::EvalArgs a{};
  a.rules = c->d_rules; a.M = c->M; a.B = B; a.npix = c->grid.pixels(); a.n_states = c->grid.n_states; a.via_top = c->grid.via_top();
  a.maps = maps; a.idx = idx_out; a.n_act = n_out; a.flags = c->d_flags;
  PMOM_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t) * B, s));
  PMOM_CUDA(c, pmom::launch_activate(a, s));
  return PMOM_OK;
}

pmom_status pmom_gather(pmom_ctx* c, const int32_t* idx, int32_t N, int32_t f, void* out, void* stream) {
  if (!c || !idx || !out || N < 1 || N > c->M) return fail(c, PMOM_ERR_INVALID_ARG, "gather: bad argument");
  if (!c->d_Z) return fail(c, PMOM_ERR_NOT_READY, "gather: no database");
  if (f < 0 || f >= c->F) return fail(c, PMOM_ERR_INVALID_ARG, "gather: frequency index");
  PMOM_CUDA(c, pmom::launch_gather(c->d_Z, c->dtype == PMOM_C128, c->M, f, idx, N, out, static_cast<cudaStream_t>(stream)));
  return PMOM_OK;
}

pmom_status pmom_gather_batch(pmom_ctx* c, const int32_t* idx, const int32_t* n, int32_t B, int32_t f, int32_t ncap,
                              void* out, void* stream) {
  if (!c || !idx || !n || !out || B < 1 || ncap < 1 || ncap > c->M) return fail(c, PMOM_ERR_INVALID_ARG, "gather_batch: bad argument");
  if (!c->d_Z) return fail(c, PMOM_ERR_NOT_READY, "gather_batch: no database");
  if (f < 0 || f >= c->F) return fail(c, PMOM_ERR_INVALID_ARG, "gather_batch: frequency index");
  PMOM_CUDA(c, pmom::launch_gather_batch(c->d_Z, c->dtype == PMOM_C128, c->M, f, idx, n, B, ncap, out,
                                         static_cast<cudaStream_t>(stream)));
  return PMOM_OK;
}

namespace {

// Enqueue the whole evaluation on stream s.  ncap > 0: the caller fixes the shared-memory capacity
// (graph capture: no host round trip); ncap == 0: read the batch's largest support set back first.
pmom_status enqueue_eval(pmom_ctx* c, const uint8_t* maps, int B, int precision, double* S_out, double* fom_out,
                         int32_t* status, cudaStream_t s, int ncap_fixed) {
  const int P = c->grid.n_ports;
  pmom::EvalArgs a{};
  a.rules = c->d_rules; a.M = c->M; a.P = P; a.F = c->F; a.B = B; a.npix = c->grid.pixels();
  a.n_states = c->grid.n_states; a.via_top = c->grid.via_top(); a.maps = maps; a.idx = c->d_idx; a.n_act = c->d_nact; a.Z = c->d_Z;
  a.z_c128 = c->dtype == PMOM_C128;
  for (int p = 0; p < pmom::kMaxPorts; ++p) a.port_len[p] = c->grid.pitch / c->grid.subs();   // gap edges: sub-square sides
  a.gap_stride = c->grid.stub_bfs(); a.gap_off = c->grid.inner_bfs(); a.gap_n = c->grid.subs();
  a.Z0 = c->Z0;
  a.S = S_out ? reinterpret_cast<double2*>(S_out) : c->d_S;
  a.flags = c->d_flags;
  int* small = static_cast<int*>(c->d_small);
  a.task_counter = small;
  a.repair_count = small + 1;
  a.counters = reinterpret_cast<unsigned long long*>(static_cast<char*>(c->d_small) + 64);
  a.repair_list = c->d_repair;
  a.order = c->d_order;
  PMOM_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t) * B, s));
  PMOM_CUDA(c, cudaMemsetAsync(c->d_small, 0, 256, s));
  const bool tm = c->timing && ncap_fixed == 0;
  c->timed = tm;
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[0], s));
  a.n_max = small + 2;
  a.use_tc = c->use_tc;
  PMOM_CUDA(c, pmom::launch_activate(a, s));
  PMOM_CUDA(c, pmom::launch_order(c->d_nact, B, c->M, c->d_order, s));
  c->launches = 2;
  int ncap = ncap_fixed;
  if (ncap <= 0) {
    // the largest support set of the batch sizes the kernels' shared memory and their occupancy
    PMOM_CUDA(c, cudaMemcpyAsync(&ncap, small + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    PMOM_CUDA(c, cudaStreamSynchronize(s));
  }
  ncap = ncap < 1 ? 1 : (ncap > c->M ? c->M : ncap);
  const LaunchTune tune = tune_for(c, ncap);
  apply_tune(tune, a);
  a.ncap = ncap_for(c, precision, ncap);
  const int tasks = B * c->F;
  pmom_status st = ensure_work(c, precision, tasks, ncap);
  if (st) return st;
  a.work = c->d_work;
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[1], s));
  a.slot_bytes = pmom::eval_slot_bytes(precision, a.ncap, P, &a.lda);
  a.ntasks_list = 0;
  PMOM_CUDA(c, pmom::launch_eval(a, precision, slots_for(c, precision, tasks, a.ncap, &tune), s));
  ++c->launches;
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[2], s));
  if (precision == PMOM_MIXED_REFINED) {
    // tasks whose refinement did not converge are solved again on the FP64 path
    PMOM_CUDA(c, cudaMemsetAsync(small, 0, sizeof(int), s));
    a.ncap = ncap_for(c, PMOM_FP64, ncap);
    a.slot_bytes = pmom::eval_slot_bytes(PMOM_FP64, a.ncap, P, &a.lda);
    a.ntasks_list = 1;
    PMOM_CUDA(c, pmom::launch_eval(a, PMOM_FP64, slots_for(c, PMOM_FP64, tasks, a.ncap), s));
    ++c->launches;
  }
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[3], s));
  PMOM_CUDA(c, pmom::launch_ys(a.S, B, c->F, P, c->Z0, c->d_flags, s));
  PMOM_CUDA(c, pmom::launch_fom(a.S, c->d_bands, c->F, P, B, c->d_flags, c->d_nact, fom_out, status, s));
  c->launches += 2;
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[4], s));
  return PMOM_OK;
}

}  // namespace

pmom_status pmom_eval_candidates(pmom_ctx* c, const uint8_t* maps, int32_t B, int32_t precision, double* S_out,
                                 double* fom_out, int32_t* status, void* stream) {
  if (!c || !maps || !fom_out || !status || B < 1 || (precision != PMOM_FP64 && precision != PMOM_MIXED_REFINED))
    return fail(c, PMOM_ERR_INVALID_ARG, "eval: bad argument");
  if (!c->d_Z || !c->fom_ready) return fail(c, PMOM_ERR_NOT_READY, "eval: load Z and set the FoM bands first");
  pmom_status st = ensure_batch(c, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  return enqueue_eval(c, maps, B, precision, S_out, fom_out, status, s, 0);
}

pmom_status pmom_eval_bordered(pmom_ctx* c, const uint8_t* ref_map, const uint8_t* maps, int32_t B, int32_t precision,
                               double* S_out, double* fom_out, int32_t* status, void* stream) {
  if (!c || !ref_map || !maps || !fom_out || !status || B < 1 ||
      (precision != PMOM_FP64 && precision != PMOM_MIXED_REFINED))
    return fail(c, PMOM_ERR_INVALID_ARG, "eval_bordered: bad argument");
  if (!c->d_Z || !c->fom_ready) return fail(c, PMOM_ERR_NOT_READY, "eval_bordered: load Z and set the FoM bands first");
  if (c->grid.subs() > 1)   // its port rows assume one gap BF per port (position 3p+1)
    return fail(c, PMOM_ERR_UNSUPPORTED, "eval_bordered: pixels of more than two triangles");
  pmom_status st = ensure_batch(c, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  const int M = c->M, F = c->F, P = c->grid.n_ports;
  if (!c->d_ref_idx) PMOM_CUDA(c, cudaMalloc(&c->d_ref_idx, sizeof(int32_t) * (M + 2)));
  if (!c->d_ref_flags) PMOM_CUDA(c, cudaMalloc(&c->d_ref_flags, sizeof(uint32_t) * F));
  int32_t* d_ref_n = c->d_ref_idx + M;
  uint32_t* d_ref_bad = reinterpret_cast<uint32_t*>(c->d_ref_idx + M + 1);
  int* small = static_cast<int*>(c->d_small);
  // reference support set (a1), its size read back to size the factors
  pmom::EvalArgs r{};
  r.rules = c->d_rules; r.M = M; r.P = P; r.F = F; r.B = 1; r.npix = c->grid.pixels();
  r.n_states = c->grid.n_states; r.via_top = c->grid.via_top(); r.maps = ref_map; r.idx = c->d_ref_idx; r.n_act = d_ref_n; r.flags = d_ref_bad;
  r.n_max = small + 2;
  PMOM_CUDA(c, cudaMemsetAsync(c->d_small, 0, 256, s));
  PMOM_CUDA(c, cudaMemsetAsync(d_ref_bad, 0, sizeof(uint32_t), s));
  PMOM_CUDA(c, pmom::launch_activate(r, s));
  int n = 0;
  PMOM_CUDA(c, cudaMemcpyAsync(&n, d_ref_n, sizeof(int), cudaMemcpyDeviceToHost, s));
  PMOM_CUDA(c, cudaStreamSynchronize(s));
  if (n <= 0) return fail(c, PMOM_ERR_BAD_STATE_VALUE, "eval_bordered: reference map has a pixel state out of range");
  const int ldn = (n + 3) & ~3;
  const size_t ref_elems = static_cast<size_t>(F) * n * ldn;
  if (ref_elems > c->ref_cap) {
    free_dev(c->d_ref_lu);
    free_dev(c->d_ref_g);
    free_dev(c->d_ref_piv);
    c->ref_cap = 0;
    PMOM_CUDA(c, cudaMalloc(&c->d_ref_lu, sizeof(double2) * ref_elems));
    PMOM_CUDA(c, cudaMalloc(&c->d_ref_g, sizeof(double2) * ref_elems));
    PMOM_CUDA(c, cudaMalloc(&c->d_ref_piv, sizeof(int) * static_cast<size_t>(F) * M));
    c->ref_cap = ref_elems;
  }
  const bool mixed = precision == PMOM_MIXED_REFINED && c->dtype == PMOM_C64 && pmom::ref_inverse_mixed_fits(n);
  const bool tm = c->timing;
  c->timed = tm;
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[0], s));
  PMOM_CUDA(c, cudaMemsetAsync(c->d_ref_flags, 0, sizeof(uint32_t) * F, s));
  if (mixed) {
    // per frequency: single-precision LU of the reference (tensor cores), kept in slot f ...
    int lda = 0;
    const size_t sb = pmom::eval_slot_bytes(PMOM_MIXED_REFINED, n, P, &lda);
    if (sb * F > c->ref_work_bytes) {
      free_dev(c->d_ref_work);
      c->ref_work_bytes = 0;
      PMOM_CUDA(c, cudaMalloc(&c->d_ref_work, sb * F));
      c->ref_work_bytes = sb * F;
    }
    pmom::EvalArgs fa{};
    fa.rules = c->d_rules; fa.M = M; fa.P = P; fa.F = F; fa.B = 1; fa.npix = c->grid.pixels();
    fa.n_states = c->grid.n_states; fa.via_top = c->grid.via_top(); fa.maps = ref_map; fa.idx = c->d_ref_idx; fa.n_act = d_ref_n;
    fa.Z = c->d_Z; fa.z_c128 = 0;
    for (int p = 0; p < pmom::kMaxPorts; ++p) fa.port_len[p] = c->grid.pitch / c->grid.subs();   // gap edges: sub-square sides
    fa.gap_stride = c->grid.stub_bfs(); fa.gap_off = c->grid.inner_bfs(); fa.gap_n = c->grid.subs();
    fa.Z0 = c->Z0; fa.flags = c->d_ref_flags; fa.task_counter = small;
    fa.counters = reinterpret_cast<unsigned long long*>(static_cast<char*>(c->d_small) + 64);
    fa.work = c->d_ref_work; fa.slot_bytes = sb; fa.lda = lda; fa.ncap = n;
    fa.factor_only = 1;
    const LaunchTune ft = tune_for(c, n);
    apply_tune(ft, fa);
    PMOM_CUDA(c, pmom::launch_eval(fa, PMOM_MIXED_REFINED, slots_for(c, PMOM_MIXED_REFINED, F, n, &ft), s));
    if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[1], s));
    // ... its inverse, refined to FP64 accuracy column block by column block ...
    PMOM_CUDA(c, cudaMemsetAsync(small, 0, sizeof(int), s));
    pmom::RefInvArgs ri{};
    ri.F = F; ri.P = P; ri.ncap = n; ri.lda = lda; ri.ldn = ldn; ri.ref_n = d_ref_n; ri.work = c->d_ref_work;
    ri.slot_bytes = sb; ri.G = c->d_ref_g; ri.ref_flags = c->d_ref_flags; ri.task_counter = small;
    const int nblk = (n + 3) / 4;
    int rs = pmom::ref_inverse_mixed_slots(c->num_sms, n);
    if (rs > F * nblk) rs = F * nblk;
    PMOM_CUDA(c, pmom::launch_ref_inverse_mixed(ri, rs, n, s));
    // ... and the FP64 path for any frequency whose factorization or refinement failed
    PMOM_CUDA(c, pmom::launch_ref_factor(c->d_Z, 0, M, c->d_ref_idx, d_ref_n, n, F, c->d_ref_lu, ldn, c->d_ref_piv,
                                         c->d_ref_flags, 1, s));
    PMOM_CUDA(c, pmom::launch_ref_inverse(c->d_ref_lu, ldn, c->d_ref_piv, d_ref_n, n, F, c->d_ref_g, c->d_ref_flags,
                                          1, s));
    PMOM_CUDA(c, pmom::launch_ref_g_to_df(c->d_ref_g, d_ref_n, ldn, c->d_ref_flags, F, s));
  } else {
    // per frequency: FP64 LU of the reference (a4) and its inverse (a5, n right-hand sides)
    PMOM_CUDA(c, pmom::launch_ref_factor(c->d_Z, c->dtype == PMOM_C128, M, c->d_ref_idx, d_ref_n, n, F, c->d_ref_lu,
                                         ldn, c->d_ref_piv, c->d_ref_flags, 0, s));
    if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[1], s));
    PMOM_CUDA(c, pmom::launch_ref_inverse(c->d_ref_lu, ldn, c->d_ref_piv, d_ref_n, n, F, c->d_ref_g, c->d_ref_flags,
                                          0, s));
  }
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[2], s));
  // candidates: support sets, then the bordered update per (candidate, frequency) task
  pmom::EvalArgs a{};
  a.rules = c->d_rules; a.M = M; a.P = P; a.F = F; a.B = B; a.npix = c->grid.pixels();
  a.n_states = c->grid.n_states; a.via_top = c->grid.via_top(); a.maps = maps; a.idx = c->d_idx; a.n_act = c->d_nact; a.flags = c->d_flags;
  a.n_max = small + 2;
  PMOM_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t) * B, s));
  PMOM_CUDA(c, pmom::launch_activate(a, s));
  int nslots = pmom::border_slots(c->num_sms, n, c->dtype == PMOM_C128, mixed);
  if (nslots > B * F) nslots = B * F;
  const size_t se = pmom::border_slot_elems(n);
  if (se * nslots > c->bwork_elems) {
    free_dev(c->d_bwork);
    c->bwork_elems = 0;
    PMOM_CUDA(c, cudaMalloc(&c->d_bwork, sizeof(double2) * se * nslots));
    c->bwork_elems = se * nslots;
  }
  pmom::BorderArgs ba{};
  ba.Z = c->d_Z; ba.z_c128 = c->dtype == PMOM_C128; ba.M = M; ba.P = P; ba.F = F; ba.B = B;
  ba.ref_idx = c->d_ref_idx; ba.ref_n = d_ref_n; ba.ref_flags = c->d_ref_flags; ba.G = c->d_ref_g; ba.ldn = ldn;
  ba.idx = c->d_idx; ba.n_act = c->d_nact;
  double2* Sd = S_out ? reinterpret_cast<double2*>(S_out) : c->d_S;
  ba.S = Sd; ba.flags = c->d_flags;
  for (int p = 0; p < pmom::kMaxPorts; ++p) ba.port_len[p] = c->grid.pitch;   // one gap edge (s = 1)
  ba.task_counter = small;
  ba.work = c->d_bwork; ba.slot_elems = se;
  PMOM_CUDA(c, cudaMemsetAsync(small, 0, sizeof(int), s));
  PMOM_CUDA(c, pmom::launch_border(ba, nslots, n, mixed, s));
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[3], s));
  PMOM_CUDA(c, pmom::launch_ys(Sd, B, F, P, c->Z0, c->d_flags, s));
  PMOM_CUDA(c, pmom::launch_fom(Sd, c->d_bands, F, P, B, c->d_flags, c->d_nact, fom_out, status, s));
  if (tm) PMOM_CUDA(c, cudaEventRecord(c->ev[4], s));
  c->launches = mixed ? 11 : 7;
  return PMOM_OK;
}

pmom_status pmom_graph_capture(pmom_ctx* c, const uint8_t* maps, int32_t B, int32_t precision, double* S_out,
                               double* fom_out, int32_t* status, int32_t ncap, void* stream) {
  if (!c || !maps || !fom_out || !status || B < 1 || ncap < 0 ||
      (precision != PMOM_FP64 && precision != PMOM_MIXED_REFINED))
    return fail(c, PMOM_ERR_INVALID_ARG, "graph_capture: bad argument");
  if (!c->d_Z || !c->fom_ready) return fail(c, PMOM_ERR_NOT_READY, "graph_capture: load Z and set the FoM bands first");
  const int cap = (ncap == 0 || ncap > c->M) ? c->M : ncap;
  // every allocation and launch attribute is settled before the capture starts
  pmom_status st = ensure_batch(c, B);
  if (st) return st;
  st = ensure_work(c, precision, B * c->F, cap);
  if (st) return st;
  slots_for(c, PMOM_FP64, B * c->F, ncap_for(c, PMOM_FP64, cap));
  slots_for(c, precision, B * c->F, ncap_for(c, precision, cap));
  // recording executes nothing, so the graph is captured on the context's own stream; launches may
  // use any stream
  (void)stream;
  if (!c->cap_stream) PMOM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t s = c->cap_stream;
  if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  PMOM_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  st = enqueue_eval(c, maps, B, precision, S_out, fom_out, status, s, cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  c->graph = g;
  PMOM_CUDA(c, cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
  return PMOM_OK;
}

pmom_status pmom_graph_launch(pmom_ctx* c, void* stream) {
  if (!c) return PMOM_ERR_INVALID_ARG;
  if (!c->graph_exec) return fail(c, PMOM_ERR_NOT_READY, "graph_launch: no captured graph");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  PMOM_CUDA(c, cudaGraphLaunch(c->graph_exec, s));
  return PMOM_OK;
}

pmom_status pmom_autotune(pmom_ctx* c, const uint8_t* maps, int32_t B, int32_t precision, int32_t* choice,
                          void* stream) {
  if (!c || !maps || B < 1) return fail(c, PMOM_ERR_INVALID_ARG, "autotune: bad argument");
  if (!c->d_Z || !c->fom_ready) return fail(c, PMOM_ERR_NOT_READY, "autotune: load Z and set the FoM bands first");
  pmom_status st = ensure_batch(c, B);
  if (st) return st;
  if (precision != PMOM_MIXED_REFINED) {   // one variant only
    if (choice) *choice = c->use_tc;
    return PMOM_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the batch's support-set sizes
  pmom::EvalArgs a{};
  a.rules = c->d_rules; a.M = c->M; a.B = B; a.npix = c->grid.pixels(); a.n_states = c->grid.n_states;
  a.via_top = c->grid.via_top(); a.maps = maps; a.idx = c->d_idx; a.n_act = c->d_nact; a.flags = c->d_flags;
  PMOM_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t) * B, s));
  PMOM_CUDA(c, pmom::launch_activate(a, s));
  std::vector<int32_t> n(B);
  PMOM_CUDA(c, cudaMemcpyAsync(n.data(), c->d_nact, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
  PMOM_CUDA(c, cudaStreamSynchronize(s));
  std::vector<int> members[pmom::kNBuckets];
  int nmax = 0, bmax = 0;
  for (int b = 0; b < B; ++b) {
    if (n[b] <= 0) continue;
    members[pmom::n_bucket(n[b])].push_back(b);
    if (n[b] > nmax) { nmax = n[b]; bmax = pmom::n_bucket(n[b]); }
  }
  cudaEvent_t e0, e1;
  PMOM_CUDA(c, cudaEventCreate(&e0));
  PMOM_CUDA(c, cudaEventCreate(&e1));
  const size_t npix = static_cast<size_t>(c->grid.pixels());
  for (int bk = 0; bk < pmom::kNBuckets && !st; ++bk) {
    if (members[bk].empty()) continue;
    // sample: enough tasks for about four rounds of the resident task groups, bounded in work so
    // that each timed run stays near a second
    int k = static_cast<int>(members[bk].size());
    const int want = (8 * c->num_sms + c->F - 1) / c->F;
    if (k > want) k = want;
    int nk = 0;
    for (int i = 0; i < k; ++i) nk = std::max(nk, n[members[bk][i]]);
    while (k > 1 && static_cast<double>(k) * c->F * nk * nk * nk > 3e13) --k;
    for (int i = 0; i < k; ++i)
      PMOM_CUDA(c, cudaMemcpyAsync(c->d_maps_stage + i * npix, maps + members[bk][i] * npix, npix,
                                   cudaMemcpyDeviceToDevice, s));
    float best = 3.4e38f;
    uint8_t bt = 1, bg = 2, bc = 4;
    // variants that differ in what runs: the CUDA-core LU only where its layout holds the bucket's
    // largest support set without the large layout (which always takes the tensor cores), two
    // task groups per CTA only where they fit
    const bool simt_ok = !pmom::eval_is_large(PMOM_MIXED_REFINED, nk, 0);
    for (int tc = 1; tc >= (simt_ok ? 0 : 1) && !st; --tc)
      for (int groups = pmom::eval_groups_max(PMOM_MIXED_REFINED, nk, tc) >= 2 ? 2 : 1; groups >= 1 && !st; --groups)
        for (int cap = 4; cap >= 2 && !st; cap -= 2) {
          c->tune_valid[bk] = 1;
          c->tune_tc[bk] = static_cast<uint8_t>(tc);
          c->tune_groups[bk] = static_cast<uint8_t>(groups);
          c->tune_cap[bk] = static_cast<uint8_t>(cap);
          float ms = 0.f;
          for (int rep = 0; rep < 2 && !st; ++rep) {   // the first run warms caches and sizes workspaces
            PMOM_CUDA(c, cudaEventRecord(e0, s));
            st = enqueue_eval(c, c->d_maps_stage, k, precision, nullptr, c->d_fom_stage, c->d_status_stage, s, 0);
            if (st) break;
            PMOM_CUDA(c, cudaEventRecord(e1, s));
            PMOM_CUDA(c, cudaEventSynchronize(e1));
            PMOM_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
          }
          if (!st && ms < best) { best = ms; bt = static_cast<uint8_t>(tc); bg = static_cast<uint8_t>(groups); bc = static_cast<uint8_t>(cap); }
        }
    c->tune_tc[bk] = bt;
    c->tune_groups[bk] = bg;
    c->tune_cap[bk] = bc;
    c->tune_ms[bk] = best / static_cast<float>(k);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!members[bmax].empty() && c->tune_valid[bmax]) c->use_tc = c->tune_tc[bmax];
  if (choice) *choice = c->use_tc;
  return st;
}

pmom_status pmom_autotune_table(const pmom_ctx* c, int32_t* out) {
  if (!c || !out) return PMOM_ERR_INVALID_ARG;
  for (int b = 0; b < pmom::kNBuckets; ++b) {
    int32_t* o = out + 5 * b;
    o[0] = c->tune_valid[b];
    o[1] = c->tune_valid[b] ? c->tune_tc[b] : c->use_tc;
    o[2] = c->tune_groups[b];
    o[3] = c->tune_cap[b];
    o[4] = static_cast<int32_t>(c->tune_ms[b] * 1000.0f);
  }
  return PMOM_OK;
}

pmom_status pmom_eval_candidates_host(pmom_ctx* c, const uint8_t* maps, int32_t B, int32_t precision, double* S_out,
                                      double* fom_out, int32_t* status, void* stream) {
  if (!c || !maps || !fom_out || !status || B < 1) return fail(c, PMOM_ERR_INVALID_ARG, "eval_host: bad argument");
  if (!c->d_Z || !c->fom_ready) return fail(c, PMOM_ERR_NOT_READY, "eval_host: load Z and set the FoM bands first");
  pmom_status st = ensure_batch(c, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = c->grid.n_ports;
  PMOM_CUDA(c, cudaMemcpyAsync(c->d_maps_stage, maps, static_cast<size_t>(B) * c->grid.pixels(), cudaMemcpyHostToDevice, s));
  st = pmom_eval_candidates(c, c->d_maps_stage, B, precision, nullptr, c->d_fom_stage, c->d_status_stage, stream);
  if (st) return st;
  if (S_out)
    PMOM_CUDA(c, cudaMemcpyAsync(S_out, c->d_S, sizeof(double2) * static_cast<size_t>(B) * c->F * P * P, cudaMemcpyDeviceToHost, s));
  PMOM_CUDA(c, cudaMemcpyAsync(fom_out, c->d_fom_stage, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  PMOM_CUDA(c, cudaMemcpyAsync(status, c->d_status_stage, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
  PMOM_CUDA(c, cudaStreamSynchronize(s));
  return PMOM_OK;
}

pmom_status pmom_stats(pmom_ctx* c, int64_t* out8) {
  if (!c || !out8) return PMOM_ERR_INVALID_ARG;
  PMOM_CUDA(c, cudaStreamSynchronize(c->last_stream));
  unsigned long long cnt[5] = {0, 0, 0, 0, 0};
  PMOM_CUDA(c, cudaMemcpy(cnt, static_cast<char*>(c->d_small) + 64, sizeof(cnt), cudaMemcpyDeviceToHost));
  out8[0] = static_cast<int64_t>(cnt[3]);
  out8[1] = static_cast<int64_t>(cnt[0]);
  out8[2] = static_cast<int64_t>(cnt[1]);
  out8[3] = static_cast<int64_t>(cnt[2]);
  out8[4] = static_cast<int64_t>(cnt[4]);
  out8[5] = 0;
  out8[6] = c->launches;
  out8[7] = 0;
  return PMOM_OK;
}

pmom_status pmom_set_tensor_cores(pmom_ctx* c, int32_t on) {
  if (!c) return PMOM_ERR_INVALID_ARG;
  c->use_tc = on != 0;
  for (int b = 0; b < pmom::kNBuckets; ++b) c->tune_valid[b] = 0;   // an explicit choice replaces the table
  return PMOM_OK;
}

pmom_status pmom_capacity(pmom_ctx* c, int32_t precision, int32_t* n_default, int32_t* n_max) {
  if (!c || !n_default || !n_max || (precision != PMOM_FP64 && precision != PMOM_MIXED_REFINED))
    return fail(c, PMOM_ERR_INVALID_ARG, "capacity: bad argument");
  pmom_status st = ensure_device(c);
  if (st) return st;
  *n_max = pmom::eval_max_ncap(precision, c->M);
  // largest N that stays on the default layout (the layout size grows with N: binary search)
  int lo = 0, hi = c->M + 1;   // default(lo) (lo = 0 trivially), !default(hi)
  while (hi - lo > 1) {
    const int mid = lo + (hi - lo) / 2;
    if (!pmom::eval_is_large(precision, mid, c->use_tc)) lo = mid; else hi = mid;
  }
  *n_default = lo;
  return PMOM_OK;
}

pmom_status pmom_set_timing(pmom_ctx* c, int32_t on) {
  if (!c) return PMOM_ERR_INVALID_ARG;
  if (on && !c->ev[0])
    for (auto& e : c->ev) PMOM_CUDA(c, cudaEventCreate(&e));
  c->timing = on != 0;
  return PMOM_OK;
}

pmom_status pmom_kernel_times(pmom_ctx* c, double* ms4) {
  if (!c || !ms4) return PMOM_ERR_INVALID_ARG;
  if (!c->timed) return fail(c, PMOM_ERR_NOT_READY, "kernel_times: no timed eval call yet");
  PMOM_CUDA(c, cudaEventSynchronize(c->ev[4]));
  for (int i = 0; i < 4; ++i) {
    float ms = 0.f;
    PMOM_CUDA(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    ms4[i] = ms;
  }
  return PMOM_OK;
}

pmom_status pmom_sync(pmom_ctx* c, void* stream) {
  if (!c) return PMOM_ERR_INVALID_ARG;
  PMOM_CUDA(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  PMOM_CUDA(c, cudaGetLastError());
  return PMOM_OK;
}

pmom_status pmom_fill_Z(pmom_ctx* c, const double* freqs, int32_t F, int32_t dtype, void* stream) {
  if (c) {
    const pmom_status dv = ensure_device(c);
    if (dv) return dv;
  }
  if (!c || !freqs || F < 1 || (dtype != PMOM_C64 && dtype != PMOM_C128))
    return fail(c, PMOM_ERR_INVALID_ARG, "fill_Z: bad argument");
  for (int f = 0; f < F; ++f)
    if (!(freqs[f] > 0)) return fail(c, PMOM_ERR_INVALID_ARG, "fill_Z: frequencies must be positive");
  if (c->grid.medium == 1)
    for (double z : c->grid.layer_z)
      if (!(z > 0 && z < c->grid.h_total)) return fail(c, PMOM_ERR_INVALID_ARG, "fill_Z: layer outside the plates");
  void* dz = nullptr;
  std::string msg;
  pmom_status st = pmom::fill_Z(c->grid, c->table, c->M, freqs, F, dtype, static_cast<cudaStream_t>(stream), &dz, &msg);
  if (st) return fail(c, st, msg);
  free_dev(c->d_Z);
  c->d_Z = dz;
  c->z_bytes = static_cast<size_t>(F) * c->M * c->M * z_elem(dtype);
  if (F != c->F) {
    c->fom_ready = false;
    free_dev(c->d_S);
    free_dev(c->d_repair);
    free_dev(c->d_idx);
    c->b_cap = 0;
  }
  c->F = F;
  c->dtype = dtype;
  c->freqs.assign(freqs, freqs + F);
  return PMOM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free evaluation
// Some callers cannot let the library allocate device memory inside a call: device memory
// handed to another framework's pool at start-up, or loops that cannot take the allocator's
// latency and the synchronization of cudaFree.  For them every temporary of the evaluation comes
// out of one fixed device array declared here; the kernels are the same ones
// pmom_eval_candidates launches, given pointers into this array instead of context workspaces.
namespace {

constexpr size_t kNoAllocBytes = PMOM_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_base[kNoAllocMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" pmom_status pmom_eval_candidates_noalloc(pmom_ctx* c, const uint8_t* maps, int32_t B, int32_t precision,
                                                    double* S_out, double* fom_out, int32_t* status, void* stream) {
  if (!c || !maps || !fom_out || !status || B < 1 || (precision != PMOM_FP64 && precision != PMOM_MIXED_REFINED))
    return fail(c, PMOM_ERR_INVALID_ARG, "eval_noalloc: bad argument");
  if (!c->d_Z || !c->fom_ready || !c->d_rules)
    return fail(c, PMOM_ERR_NOT_READY, "eval_noalloc: load Z and set the FoM bands first");
  int dev = 0;
  PMOM_CUDA(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(c, PMOM_ERR_INVALID_ARG, "eval_noalloc: device index");
  unsigned char* base = nullptr;
  {
    // once per device, with that device current: the host-side symbol is not a device address
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      g_noalloc_base[dev] = static_cast<unsigned char*>(p);
    }
    base = g_noalloc_base[dev];
  }
  const int P = c->grid.n_ports, F = c->F, M = c->M;
  // carve the scratch: counters | idx | N | flags | repair list | S (if the caller passed none) | slots
  size_t off = 0;
  const size_t o_small = off; off = align256(off + 256);
  const size_t o_idx = off; off = align256(off + sizeof(int32_t) * static_cast<size_t>(B) * M);
  const size_t o_nact = off; off = align256(off + sizeof(int32_t) * B);
  const size_t o_flags = off; off = align256(off + sizeof(uint32_t) * B);
  const size_t o_rep = off; off = align256(off + sizeof(int) * static_cast<size_t>(B) * F);
  const size_t o_S = off;
  if (!S_out) off = align256(off + sizeof(double2) * static_cast<size_t>(B) * F * P * P);
  const size_t o_work = off;
  int lda = 0;   // the same leading dimension for both precisions
  const size_t slot_main = pmom::eval_slot_bytes(precision, M, P, &lda);
  const size_t slot_fp64 = pmom::eval_slot_bytes(PMOM_FP64, M, P, &lda);
  const size_t slot_max = slot_main > slot_fp64 ? slot_main : slot_fp64;
  if (o_work + slot_max > kNoAllocBytes) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "eval_noalloc: batch needs %zu bytes of scratch (one task workspace %zu) but the fixed array holds %zu",
                  o_work + slot_max, slot_max, kNoAllocBytes);
    return fail(c, PMOM_ERR_INVALID_ARG, msg);
  }
  const int fit = static_cast<int>((kNoAllocBytes - o_work) / slot_max);
  const int tasks = B * F;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* small = reinterpret_cast<int*>(base + o_small);
  pmom::EvalArgs a{};
  a.rules = c->d_rules; a.M = M; a.P = P; a.F = F; a.B = B; a.npix = c->grid.pixels();
  a.n_states = c->grid.n_states; a.via_top = c->grid.via_top(); a.maps = maps;
  a.idx = reinterpret_cast<int32_t*>(base + o_idx);
  a.n_act = reinterpret_cast<int32_t*>(base + o_nact);
  a.flags = reinterpret_cast<uint32_t*>(base + o_flags);
  a.Z = c->d_Z;
  a.z_c128 = c->dtype == PMOM_C128;
  for (int p = 0; p < pmom::kMaxPorts; ++p) a.port_len[p] = c->grid.pitch / c->grid.subs();   // gap edges: sub-square sides
  a.gap_stride = c->grid.stub_bfs(); a.gap_off = c->grid.inner_bfs(); a.gap_n = c->grid.subs();
  a.Z0 = c->Z0;
  a.S = S_out ? reinterpret_cast<double2*>(S_out) : reinterpret_cast<double2*>(base + o_S);
  a.task_counter = small;
  a.repair_count = small + 1;
  a.counters = reinterpret_cast<unsigned long long*>(base + o_small + 64);
  a.repair_list = reinterpret_cast<int*>(base + o_rep);
  a.work = base + o_work;
  a.lda = lda;
  a.ncap = M;   // no host round trip here: shared memory sized for the whole parent
  const LaunchTune nt = tune_for(c, M);   // the autotuner's table, as pmom_eval_candidates
  apply_tune(nt, a);
  // the array keeps the previous call's contents: zero what the kernels accumulate into
  PMOM_CUDA(c, cudaMemsetAsync(base + o_small, 0, 256, s));
  PMOM_CUDA(c, cudaMemsetAsync(a.flags, 0, sizeof(uint32_t) * B, s));
  PMOM_CUDA(c, pmom::launch_activate(a, s));
  a.slot_bytes = slot_main;
  a.ntasks_list = 0;
  int n = slots_for(c, precision, tasks, M, &nt);
  PMOM_CUDA(c, pmom::launch_eval(a, precision, n < fit ? n : fit, s));
  if (precision == PMOM_MIXED_REFINED) {
    PMOM_CUDA(c, cudaMemsetAsync(small, 0, sizeof(int), s));
    a.slot_bytes = slot_fp64;
    a.ntasks_list = 1;
    n = slots_for(c, PMOM_FP64, tasks, M);
    PMOM_CUDA(c, pmom::launch_eval(a, PMOM_FP64, n < fit ? n : fit, s));
  }
  PMOM_CUDA(c, pmom::launch_ys(a.S, B, F, P, c->Z0, a.flags, s));
  PMOM_CUDA(c, pmom::launch_fom(a.S, c->d_bands, F, P, B, a.flags, a.n_act, fom_out, status, s));
  return PMOM_OK;
}
