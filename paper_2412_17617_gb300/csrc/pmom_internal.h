// Internal declarations of the GB300 candidate evaluator (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pmom.h"

namespace pmom {

constexpr int kMaxPorts = 4;
constexpr int kTableCols = 8;

// Activation rule of one basis function, as the kernels read it.  kVia*: the three BFs of a via
// site (state 2: metal plus a vertical strip up to the next layer): the strip's own diagonal, its
// junction with the via pixel, and its junction with the pixel above (active when that one is metal).
enum RuleKind : int32_t { kAlways = 0, kInner = 1, kInter = 2, kPixPort = 3, kViaStrip = 4, kViaJoin = 5, kViaLand = 6 };

struct Grid {
  int layers = 0, nx = 0, ny = 0, medium = 0, n_states = 2, n_ports = 0;
  int diag_pattern = 0;    // 0 alternating, 1 uniform, 2 random (pmom_grid_desc)
  uint64_t diag_seed = 0;
  int sub = 1;             // sub-squares per pixel side (pmom_grid_desc)
  double pitch = 0, h_total = 0, eps_r = 1, tan_d = 0;
  std::vector<double> layer_z;
  std::vector<pmom_port> ports;
  int pixels() const { return layers * nx * ny; }
  int subs() const { return sub > 1 ? sub : 1; }
  // inner BFs of one pixel (s^2 diagonals + 2 s (s - 1) inner edges) and always-present BFs of a
  // port stub (both stub pixels' inner BFs + the s gap edges); port p's gap BFs are
  // p * stub_bfs() + inner_bfs() + k, k < s, in the table and in every support set
  int inner_bfs() const { return subs() * subs() + 2 * subs() * (subs() - 1); }
  int stub_bfs() const { return 2 * inner_bfs() + subs(); }
  bool vias() const { return n_states >= 3 && layers >= 2 && subs() == 1; }
  // first pixel index that cannot hold the via state (the last layer has no layer above it)
  int via_top() const { return vias() ? (layers - 1) * nx * ny : pixels(); }
};

// Diagonal orientation of lattice pixel (x, y): 0 -> (x, y+1)-(x+1, y), 1 -> (x, y)-(x+1, y+1)
// (pmom_mesh.cpp).
int orient(const Grid& g, int x, int y);

// Grid of a context (pmom_api.cu).
const Grid& grid_of(const pmom_ctx* c);

// Builds the canonical BF table (see pmom_bf_table in pmom.h).  Returns M.
int build_bf_table(const Grid& g, std::vector<int32_t>& table);

// Support-set size buckets of the autotuner: [0, 128), [128, 256), ..., [4096, 8192), >= 8192.
constexpr int kNBuckets = 8;
__host__ __device__ inline int n_bucket(int N) {
  int b = 0;
  for (int t = 128; b < kNBuckets - 1 && N >= t; t <<= 1) ++b;
  return b;
}

// Device-side launch parameters of the evaluation kernels.
struct EvalArgs {
  const int4* rules;       // [M] {kind, pixA, pixB, 0}
  int M, P, F, B, npix, n_states;
  int via_top;             // pixels at index >= via_top reject state 2 (Grid::via_top)
  const uint8_t* maps;     // [B][npix]
  int32_t* idx;            // [B][M]
  int32_t* n_act;          // [B]
  const void* Z;           // [F][M][M] resident database
  int z_c128;              // 1: double2 storage, 0: float2
  double port_len[kMaxPorts];
  int gap_stride, gap_off, gap_n;   // port p's gap BFs: p * gap_stride + gap_off + k, k < gap_n
  double Z0;
  double2* S;              // [B][F][P][P]
  uint32_t* flags;         // [B] bit flags per candidate
  int* task_counter;       // persistent queue head
  int* repair_list;        // [B*F] tasks the mixed path hands to FP64
  int* repair_count;
  unsigned long long* counters;  // [5]: refinement iterations, max iterations, repaired, tasks, tensor-core wait timeouts
  void* work;              // slot workspaces
  size_t slot_bytes;
  int lda;                 // leading dimension of the per-slot matrix
  int ntasks_list;         // 0: all B*F tasks; 1: tasks from repair_list
  int ncap;                // largest N of the batch (sizes the shared-memory panel); <= M
  int* n_max;              // activation writes max N here (atomicMax)
  int use_tc;              // single-precision LU: trailing updates on the tensor cores (tcgen05)
  int factor_only;         // 1: task t factors into workspace slot t (kept) and ends after the LU
  const int* order;        // [B] candidates in task order (largest support set first), or null
  int nslots;              // workspace slots of this launch (set by the launcher)
  uint8_t tc_bucket[kNBuckets];   // per support-set bucket (n_bucket): tensor-core LU (1) or CUDA-core (0)
  int max_groups;          // task groups per CTA at most (0: as many as fit)
};

enum CandFlag : uint32_t {
  kFlagSingular = 1u, kFlagNonfinite = 2u, kFlagRepaired = 4u, kFlagBadState = 8u, kFlagCapacity = 16u,
  kFlagFar = 32u
};

// Bordered evaluation against a reference map (pmom_border.cu).
constexpr int kBorderK = 8;   // BFs a candidate may remove from / add to the reference support set
struct BorderArgs {
  const void* Z;              // [F][M][M] resident database
  int z_c128;
  int M, P, F, B;
  const int32_t* ref_idx;     // [n] reference support set (ascending)
  const int32_t* ref_n;       // n (device)
  const uint32_t* ref_flags;  // [F] 1: the reference matrix is singular at f
  const void* G;              // [F][n][ldn] reference inverses: double2, or float-float float4 (df route)
  int ldn;
  const int32_t* idx;         // [B][M] candidates' support sets
  const int32_t* n_act;       // [B]
  double2* S;                 // [B][F][P][P]: Y written here, converted by launch_ys
  uint32_t* flags;            // [B]
  double port_len[kMaxPorts];
  int* task_counter;
  double2* work;              // per-slot scratch
  size_t slot_elems;
};
// FP64 reference factorization and inverse; gated = 1: only the frequencies whose single-precision
// reference failed (the fallback after launch_ref_inverse_mixed).
cudaError_t launch_ref_factor(const void* Z, int z_c128, int M, const int32_t* ref_idx, const int32_t* ref_n, int n,
                              int F, double2* LU, int ldn, int* piv, uint32_t* ref_flags, int gated, cudaStream_t s);
cudaError_t launch_ref_inverse(const double2* LU, int ldn, const int* piv, const int32_t* ref_n, int n, int F,
                               double2* G, const uint32_t* ref_flags, int gated, cudaStream_t s);
// Refined reference inverse from single-precision factors kept in evaluation workspace slot f.
struct RefInvArgs {
  int F, P, ncap, lda, ldn;
  const int32_t* ref_n;
  const void* work;
  size_t slot_bytes;
  double2* G;
  uint32_t* ref_flags;
  int* task_counter;
};
bool ref_inverse_mixed_fits(int n);
int ref_inverse_mixed_slots(int num_sms, int n);
cudaError_t launch_ref_inverse_mixed(const RefInvArgs& r, int nslots, int n, cudaStream_t s);
// In place double2 -> float-float (float4) for the frequencies the FP64 fallback redid.
cudaError_t launch_ref_g_to_df(double2* G, const int32_t* ref_n, int ldn, const uint32_t* ref_flags, int F,
                               cudaStream_t s);
size_t border_slot_elems(int n);
// df = 1: W = G B in float-float arithmetic (complex64 databases; ignored for complex128)
int border_slots(int num_sms, int n, int z_c128, int df);
cudaError_t launch_border(const BorderArgs& a, int nslots, int n, int df, cudaStream_t s);

// Launchers (pmom_eval.cu).
cudaError_t launch_activate(const EvalArgs& a, cudaStream_t s);
// Self-test of the bounded mbarrier wait (pmom_eval.cu): d_out[0] = 1 when the wait gave up.
cudaError_t launch_wait_selftest(long long polls, int arrive, int* d_out, cudaStream_t s);
cudaError_t launch_eval(const EvalArgs& a, int precision, int nslots, cudaStream_t s);
// Candidates sorted by support-set size, largest first (longest-processing-time order for the
// persistent queue); one block, B <= 65536.
cudaError_t launch_order(const int32_t* n_act, int B, int M, int* order, cudaStream_t s);
// Y -> S in place for every (candidate, frequency) task of the batch (Eq. 6-7).
cudaError_t launch_ys(double2* S, int B, int F, int P, double Z0, uint32_t* flags, cudaStream_t s);
cudaError_t launch_fom(const double2* S, const uint8_t* bands, int F, int P, int B, const uint32_t* flags,
                       const int32_t* n_act, double* fom, int32_t* status, cudaStream_t s);
cudaError_t launch_gather(const void* Z, int z_c128, int M, int f, const int32_t* idx, int N, void* out,
                          cudaStream_t s);
// Batched gather of B support sets (idx [B][M], n [B] on the device) into out [B][ncap][ncap].
cudaError_t launch_gather_batch(const void* Z, int z_c128, int M, int f, const int32_t* idx, const int32_t* n, int B,
                                int ncap, void* out, cudaStream_t s);
// Workspace of one task slot for support sets up to ncap (leading dimension returned in *lda).
size_t eval_slot_bytes(int precision, int ncap, int P, int* lda);
size_t eval_smem_bytes(int precision, int ncap, int use_tc);
int eval_blocks_per_sm(int precision, int ncap, int z_c128, int use_tc, int max_groups = 0);
// Large-support-set layout (narrow panels, solve vectors in global memory): chosen when the default
// layout does not fit one CTA; pmom_eval_large.cu holds its kernels.
bool eval_is_large(int precision, int ncap, int use_tc);
int eval_max_ncap(int precision, int M);
// Task groups per CTA that the layout of this launch allows (1 or 2).
int eval_groups_max(int precision, int ncap, int use_tc);
cudaError_t launch_eval_large(const EvalArgs& a, int precision, int nslots, cudaStream_t s);
// cuTensorMapEncodeTiled looked up through the runtime's driver entry point (null if unavailable),
// kept after the first successful lookup.  The tensor-core launches encode their operand maps with
// it; the first device use of a context looks it up, so a later graph capture makes no lookup.
void* tensor_map_encoder_ptr();
int eval_blocks_per_sm_large(int precision, int ncap, int z_c128, int max_groups = 0);

// GPU fill of Z(f) (pmom_fill.cu): allocates *d_Z_out (F*M*M elements of dtype) on success.
pmom_status fill_Z(const Grid& g, const std::vector<int32_t>& table, int M, const double* freqs, int F, int dtype,
                   cudaStream_t s, void** d_Z_out, std::string* err);

}  // namespace pmom
