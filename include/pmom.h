/*
 * pmom.h -- C ABI of the GB300 pre-computed MoM candidate evaluator.
 *
 * The library implements the evaluation step of the paper's inverse-design loop: for a batch of
 * candidate pixel maps it selects each candidate's active RWG basis functions, gathers the
 * corresponding rows and columns of the pre-computed parent interaction matrix Z(f), solves for
 * every port excitation at every frequency, converts the port currents to S-parameters and
 * scores the two-passband diplexer figure of merit.
 *
 * Conventions shared by every call:
 *   - All entry points return a pmom_status (0 = PMOM_OK).  On failure pmom_last_error(ctx)
 *     returns a message owned by the context (valid until the next call on that context).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Device work is
 *     asynchronous on that stream; CUDA faults surface at the next call or at pmom_sync().
 *   - "device" pointers are CUDA device (or managed) memory of the current device; "host"
 *     pointers are ordinary or pinned host memory.  The caller owns every buffer it passes; the
 *     library owns its copy of Z, its basis-function tables and its workspaces until
 *     pmom_destroy().
 *   - A context is bound to the device that is current when pmom_create() runs and must only be
 *     used from one host thread at a time.
 *   - Pixel maps are uint8 [layers][ny][nx] per candidate (row-major, x fastest).  State 0 is
 *     void, 1 is metal.
 */
#ifndef PMOM_H
#define PMOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pmom_status;
enum {
  PMOM_OK = 0,
  PMOM_ERR_INVALID_ARG = 1,      /* null pointer, size out of range, inconsistent grid */
  PMOM_ERR_OOM = 2,              /* a device allocation failed */
  PMOM_ERR_BAD_STATE_VALUE = 3,  /* a pixel state >= n_states, or a via on the last layer (reported per
                                    candidate as well) */
  PMOM_ERR_Z_SHAPE_MISMATCH = 4, /* Z / frequency / band shapes disagree with the grid */
  PMOM_ERR_CUDA = 5,             /* a CUDA runtime call failed; see pmom_last_error */
  PMOM_ERR_NOT_READY = 6,        /* call order: Z or the FoM bands not loaded yet */
  PMOM_ERR_UNSUPPORTED = 7,      /* a feature the library does not implement (e.g. more than three pixel
                                    states, the bordered update on pixels of more than two triangles) */
  PMOM_ERR_IO = 8                /* database file: open / read / write failed, not a database file,
                                    truncated, or its checksum disagrees */
};

/* Storage of the parent matrix database. */
enum { PMOM_C64 = 0, PMOM_C128 = 1 };
/* Where a buffer lives. */
enum { PMOM_MEM_HOST = 0, PMOM_MEM_DEVICE = 1 };
/* Arithmetic of the evaluation.
 *   PMOM_FP64          : complex128 LU with partial pivoting on the CUDA cores (plain path).
 *   PMOM_MIXED_REFINED : complex64 LU (single precision) + iterative refinement whose residual
 *                        V - Z_sub x is formed in double-class precision from the exact stored
 *                        Z entries, until the correction stops shrinking (see pmom_stats). */
enum { PMOM_FP64 = 0, PMOM_MIXED_REFINED = 1 };
/* Per-candidate status codes (status_out). */
enum {
  PMOM_CAND_OK = 0,
  PMOM_CAND_SINGULAR = 1,        /* an exactly zero pivot at some frequency */
  PMOM_CAND_NONFINITE = 2,       /* NaN/Inf in S or FoM */
  PMOM_CAND_REPAIRED = 3,        /* mixed path did not converge at some frequency; that frequency
                                    was re-solved on the FP64 path (results are valid) */
  PMOM_CAND_BAD_STATE = 5,       /* a pixel state >= n_states or a via on the last layer; S/FoM not computed */
  PMOM_CAND_CAPACITY = 6,        /* support set larger than a captured graph's capacity; not computed */
  PMOM_CAND_FAR = 7              /* bordered evaluation: more than PMOM_BORDER_K basis functions removed
                                    or added relative to the reference map; not computed */
};

typedef struct {
  int32_t layer; /* metal layer of the feed stub */
  int32_t side;  /* 0: +x (right), 1: +y (top), 2: -x (left), 3: -y (bottom) */
  int32_t pos;   /* pixel row (sides 0/2) or column (sides 1/3) the stub leaves through */
} pmom_port;

/* Pixel grid and stack-up (paper Section II-A/II-D, Table I). */
typedef struct {
  int32_t layers, nx, ny;
  double pitch_m;              /* pixel side a */
  int32_t medium;              /* 0: microstrip (ground at z = 0, homogeneous effective medium),
                                  1: stripline (grounds at 0, h_total), 2: layered microstrip (PEC
                                  ground, a dielectric slab up to the highest layer, air above;
                                  Sommerfeld kernels of horizontal currents: with n_states 3 it is
                                  refused with UNSUPPORTED) */
  const double* layer_z_m;     /* [layers], host; heights of the metal layers */
  double h_total_m;            /* stripline plate spacing */
  double eps_r, tan_d;         /* homogenised substrate */
  int32_t n_states;            /* 2: void / metal; 3: void / metal / metal with a via up to the next
                                  layer (layers >= 2; the last layer rejects state 2) */
  int32_t n_ports;             /* 1..4 */
  const pmom_port* ports;      /* [n_ports], host */
  int32_t diag_pattern;        /* pixel diagonals (Section V-A, Fig. mesh_orientation a-c), the same on
                                  every layer and on the port stubs: 0 alternating (diagonal
                                  (x, y+1)-(x+1, y) when x+y is even, else (x, y)-(x+1, y+1)),
                                  1 uniform (always the first), 2 random (the first when the top bit
                                  of SplitMix64 chained over diag_seed and (y+4)*128 + x+4 is 0) */
  uint64_t diag_seed;          /* pattern 2 only */
  int32_t sub;                 /* sub-squares per pixel side, on the same fine lattice pattern: 1, 2 or 3
                                  (2, 8 or 18 triangles per pixel, Section V-A; 0 reads as 1).  With
                                  s > 1 a port's delta gap is the s edges between its stub pixels,
                                  driven together (V_k = l_k) with the port current summed over them;
                                  the via state and the bordered update need s = 1 */
} pmom_grid_desc;

typedef struct pmom_ctx pmom_ctx;

/* Build the basis-function tables of the grid (two alternating triangles per pixel, RWG on every
 * shared edge, four BF classes: Section II-C; corner-only contact is no connection: Section VI-A).
 * Copies the descriptor; `out` receives a new context.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
pmom_status pmom_create(const pmom_grid_desc* grid, pmom_ctx** out);
pmom_status pmom_destroy(pmom_ctx* ctx);
const char* pmom_last_error(const pmom_ctx* ctx);

/* Number M of basis functions of the all-metal parent (rows of Z), and ports P. */
pmom_status pmom_num_bfs(const pmom_ctx* ctx, int32_t* M, int32_t* P);

/* BF table, host int32 [M][8]: class (0 always-present, 1 inner-pixel, 2 inter-pixel,
 * 3 pixel-port, 4 via strip, 5 via junction with its own pixel, 6 via junction with the pixel
 * above), pixel A, pixel B, port, key(T+), key(T-), free vertex in T+, free vertex in T-.
 * pixel = (layer*ny + y)*nx + x; key = (((layer*128 + y+4)*128 + x+4)*4 + half), half 0 being the
 * triangle that holds the pixel's lower (-y) side and halves 2, 3 the two triangles of the via
 * strip standing on the pixel diagonal (D0, D1 its ends): (D0@l, D1@l, D1@l+1), (D0@l, D1@l+1,
 * D0@l+1).  Canonical BF order: port stubs (per port: inner stub diagonal, delta-gap edge, outer
 * stub diagonal), then per layer and pixel (row-major): diagonal, +x side, +y side, then one
 * pixel-port BF per port, then (three-state grids) per via layer 0..L-2 and pixel: strip, own
 * junction, upper junction.  A via BF is active when its pixel has state 2 (the upper junction also
 * needs metal on the pixel above). */
pmom_status pmom_bf_table(const pmom_ctx* ctx, int32_t* table_host);

/* Load the parent database Z[F][M][M] (row-major; complex interleaved re,im) for F frequencies
 * (Phase 2 of the paper's flow, Section II-A).  dtype: PMOM_C64 or PMOM_C128; mem: where Z lives.
 * The library copies Z into memory it owns (device-to-device for PMOM_MEM_DEVICE); the caller may
 * free its buffer when the call returns (after pmom_sync for device sources).
 * Errors: INVALID_ARG, Z_SHAPE_MISMATCH (F < 1), OOM, CUDA. */
pmom_status pmom_load_Z(pmom_ctx* ctx, const double* freqs_hz_host, int32_t F, const void* Z, int32_t dtype,
                        int32_t mem, void* stream);

/* Copy the resident database (as loaded or filled) out to a caller buffer of F*M*M complex
 * elements of the resident dtype.  mem says where `out` lives. */
pmom_status pmom_copy_Z(const pmom_ctx* ctx, void* out, int32_t mem, void* stream);

/* Fill the parent database on the GPU (MPIE with RWG basis, Eq. 1-2) at F frequencies and keep
 * it resident as dtype; replaces a loaded Z.  Green's functions of the stack-up: one ground image
 * in a homogeneous effective medium (medium 0), the parallel-plate functions (medium 1), or the
 * grounded slab's mixed-potential kernels (medium 2, the layered-media MPIE of Section II-D):
 * G_A and G_phi as Sommerfeld integrals of the transmission-line voltages of the stack-up, each
 * a quasi-static term plus a remainder tabulated per frequency and pair of layer heights on
 * rho = i d/16 (d the slab thickness) and interpolated cubically. */
pmom_status pmom_fill_Z(pmom_ctx* ctx, const double* freqs_hz_host, int32_t F, int32_t dtype, void* stream);

/* Figure-of-merit bands (Eq. 8-9): band_of_freq host uint8 [F] with 0 = f_p1, 1 = f_p2,
 * 2 = f_i, 3 = f_s, 255 = not scored; Z0 = port reference impedance (Eq. 6).
 * Errors: Z_SHAPE_MISMATCH if F differs from the loaded database. */
pmom_status pmom_set_fom(pmom_ctx* ctx, const uint8_t* band_of_freq_host, int32_t F, double Z0);

/* Support sets (Eq. 3): for each of B device maps, idx_out[b][0..N_b) = ascending indices of the
 * active BFs and n_out[b] = N_b (-1 if a state is out of range).  idx_out: device int32 [B][M]. */
pmom_status pmom_active_set(pmom_ctx* ctx, const uint8_t* maps_dev, int32_t B, int32_t* idx_out_dev,
                            int32_t* n_out_dev, void* stream);

/* Z_sub = S^T Z(f) S (Eq. 4-5) for one device index list of length N at frequency f, written to
 * out_dev as N*N complex elements of the resident dtype (row-major).  Bit-exact copy of entries. */
pmom_status pmom_gather(pmom_ctx* ctx, const int32_t* idx_dev, int32_t N, int32_t f, void* out_dev, void* stream);

/* Batched gather (Eq. 4-5) at frequency f: for each b < B with 0 < N_b = n_dev[b] <= ncap,
 * out_dev[b][i][j] = Z(f)[I_b[i]][I_b[j]] for i, j < N_b (out_dev: B x ncap x ncap elements of the
 * resident dtype, row-major; other entries untouched), idx_dev as written by pmom_active_set.
 * Each CTA stages whole parent rows in shared memory by bulk asynchronous copies and compacts them
 * with coalesced stores -- the gather step of the evaluation kernel as a launch of its own, for
 * callers that factor elsewhere and for measuring it.  Bit-exact copy of entries.  Errors:
 * INVALID_ARG, NOT_READY (no database). */
pmom_status pmom_gather_batch(pmom_ctx* ctx, const int32_t* idx_dev, const int32_t* n_dev, int32_t B, int32_t f,
                              int32_t ncap, void* out_dev, void* stream);

/* Evaluate B candidates at every loaded frequency (Eq. 2-9).
 *   maps_dev   : device uint8 [B][layers][ny][nx]
 *   precision  : PMOM_FP64 or PMOM_MIXED_REFINED
 *   S_out_dev  : device double [B][F][P][P][2] (re, im; S[i][j] = response at port i+1 to port j+1),
 *                or NULL to skip writing S
 *   fom_out_dev: device double [B] (lower is better)
 *   status_dev : device int32 [B] (PMOM_CAND_*)
 * Errors: INVALID_ARG, NOT_READY (no Z or no bands), OOM, CUDA. */
pmom_status pmom_eval_candidates(pmom_ctx* ctx, const uint8_t* maps_dev, int32_t B, int32_t precision,
                                 double* S_out_dev, double* fom_out_dev, int32_t* status_dev, void* stream);

/* CUDA-graph form of pmom_eval_candidates for repeated evaluation of same-shaped batches (the
 * inner loop of the tree search): records the whole pipeline (activation, ordering, persistent
 * evaluation, FP64 repair, Y->S, FoM) for these device buffers into one graph; pmom_graph_launch
 * replays it on `stream` with no host synchronisation.  The maps' contents may change between
 * launches; the pointers and B may not.  ncap: the largest support set the graph must handle
 * (0 = M); a candidate with more active BFs reports PMOM_CAND_CAPACITY instead of being solved.
 * All allocations happen before the capture starts.  Capturing replaces a previous graph. */
pmom_status pmom_graph_capture(pmom_ctx* ctx, const uint8_t* maps_dev, int32_t B, int32_t precision,
                               double* S_out_dev, double* fom_out_dev, int32_t* status_dev, int32_t ncap,
                               void* stream);
pmom_status pmom_graph_launch(pmom_ctx* ctx, void* stream);

/* Autotuner (batching of Phase 3, Fig. 1, over the uneven support sets of Eq. 3): groups the
 * batch's candidates by support-set size in buckets [0, 128), [128, 256), ..., [4096, 8192),
 * >= 8192, and for each bucket present times, on a sample of its candidates (enough tasks for
 * about four rounds of the resident task groups), every combination of the single-precision LU
 * variant (tensor-core or CUDA-core updates), the task groups per CTA (2 or 1) and the
 * resident-task cap (all slots or half); the fastest is kept per bucket for later calls.  Each
 * task then takes its bucket's LU variant inside one launch, whose groups per CTA and slot cap
 * are those of the batch's largest-support-set bucket.  *choice_out = the LU variant of that
 * bucket (1: tensor cores).  Synchronous; FP64 has a single variant.  pmom_set_tensor_cores
 * clears the table. */
pmom_status pmom_autotune(pmom_ctx* ctx, const uint8_t* maps_dev, int32_t B, int32_t precision, int32_t* choice_out,
                          void* stream);

/* The autotuner's table: out_host int32 [8][5] per bucket = {measured (0/1), tensor-core LU (0/1),
 * task groups per CTA, slot cap in quarters of the full count, best time per candidate of the
 * sample in microseconds}. */
pmom_status pmom_autotune_table(const pmom_ctx* ctx, int32_t* out_host);

/* Same computation with host buffers: the call copies the maps to the device, evaluates, copies
 * S (if S_out_host != NULL), FoM and status back and synchronizes `stream` before returning.
 * Pinned host buffers make the copies asynchronous DMA. */
pmom_status pmom_eval_candidates_host(pmom_ctx* ctx, const uint8_t* maps_host, int32_t B, int32_t precision,
                                      double* S_out_host, double* fom_out_host, int32_t* status_host,
                                      void* stream);

/* Allocation-free evaluation.  Some callers cannot let a library call cudaMalloc or cudaFree
 * while they run: a host that hands all device memory to another framework's caching pool at
 * start-up (a late cudaMalloc then fails or fragments that pool), and real-time loops for which
 * the allocator's latency, and the device synchronization that cudaFree implies, are not
 * acceptable.  The paper has no counterpart to this entry point; it is a deployment convenience.
 * Same arguments and results as pmom_eval_candidates (S_out_dev may be NULL only if the batch's
 * S still fits the scratch), but every temporary (support sets, per-task workspaces, counters)
 * lives in one fixed array of PMOM_NOALLOC_SCRATCH_BYTES (32 MiB) that the library declares in
 * device memory and that stays reserved on every GPU that loads the library until the process
 * exits.  The call issues no cudaMalloc/cudaFree.  Preconditions: Z loaded or filled and the
 * FoM bands set on `ctx` (those earlier calls may allocate).  A batch whose scratch does not fit
 * is rejected with PMOM_ERR_INVALID_ARG and a message stating the bytes needed (in practice the
 * FP64 workspace of one task must fit: M up to about 1400 for the mixed path).  Workspaces are
 * sized for the whole parent (M BFs), so the tasks share min(resident task slots,
 * (32 MiB - batch bookkeeping) / workspace(M)) workspaces: near the limit only one or two, and the
 * batch then runs on one or two SMs (results unchanged, throughput far below
 * pmom_eval_candidates).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the one array and it keeps the
 * previous call's contents: the entry point clears the parts that must start at zero itself,
 * but two calls that overlap on the GPU (different streams, contexts or host threads without
 * ordering) race on the array and corrupt each other.  pmom_stats / pmom_kernel_times do not
 * report these calls. */
#define PMOM_NOALLOC_SCRATCH_BYTES (32u << 20)
pmom_status pmom_eval_candidates_noalloc(pmom_ctx* ctx, const uint8_t* maps_dev, int32_t B, int32_t precision,
                                         double* S_out_dev, double* fom_out_dev, int32_t* status_dev, void* stream);

/* Single-precision LU variant: on != 0 (default) runs the trailing-matrix updates on the
 * tensor cores (tcgen05, TF32 operands split hi + lo, fp32 accumulation in TMEM); 0 runs them on
 * the CUDA cores.  Both meet the same accuracy after refinement; the switch exists for tuning.
 * The tensor-core variant stages its operand tiles with tensor-map (TMA) copies: each launch
 * encodes its maps on the host through the CUDA runtime's driver entry point
 * (cuTensorMapEncodeTiled); if that lookup or encoding fails, the evaluation call returns
 * PMOM_ERR_CUDA (invalid value) without launching the evaluation kernel. */
pmom_status pmom_set_tensor_cores(pmom_ctx* ctx, int32_t on);

/* Bordered low-rank evaluation of candidates close to a reference map (the single-pixel changes
 * of a search step).  A change removes a set R and adds a set A of basis functions relative to the
 * reference support set S (Eq. 3; a flip touches the pixel's inner BF, its inter-pixel BFs and a
 * pixel-port BF, Section II-C).  Per frequency the call factors the reference Z_sub = Z(f)[S, S]
 * in FP64 and forms its inverse G; each candidate's port solutions then follow exactly (up to
 * rounding) from the block-inverse identities
 *     (Z_TT)^-1 = G_TT - G_TR G_RR^-1 G_RT   (T = S \ R)
 * and the Schur complement C = Z_AA - Z_AT (Z_TT)^-1 Z_TA of the bordered system, in
 * O(|S|^2 |A| + |S| k (k + P)) work instead of a new O(N^3) factorization; Y and S follow Eq. 6-7
 * and the FoM Eq. 8-9 as in pmom_eval_candidates.
 *   precision : PMOM_FP64 -- the reference LU, its inverse and the products G * Z(f)[S, A] in FP64;
 *               PMOM_MIXED_REFINED (complex64 databases) -- the reference LU in single precision on
 *               the tensor cores, the inverse refined column block by column block with
 *               float-float residuals to a normwise backward error of 1e-12 (frequencies that
 *               do not get there are redone in FP64), the products in float-float arithmetic;
 *               complex128 databases always take the FP64 route
 *   reference_map_dev : device uint8 [layers][ny][nx]
 *   maps_dev, S_out_dev, fom_out_dev, status_dev : as pmom_eval_candidates
 * Candidates with |R| or |A| above PMOM_BORDER_K report PMOM_CAND_FAR (evaluate them with
 * pmom_eval_candidates).  The call reads the reference's support-set size back (one stream
 * synchronization) and allocates F * |S|^2 * 32 bytes of reference factors on first use.
 * Errors: INVALID_ARG, NOT_READY, BAD_STATE_VALUE (reference map), OOM, CUDA. */
#define PMOM_BORDER_K 8
pmom_status pmom_eval_bordered(pmom_ctx* ctx, const uint8_t* reference_map_dev, const uint8_t* maps_dev, int32_t B,
                               int32_t precision, double* S_out_dev, double* fom_out_dev, int32_t* status_dev,
                               void* stream);

/* ---- Learned pre-ranker (a multilayer perceptron trained on the evaluator's own outputs) ----
 * The search step of Algorithm 1 evaluates every child of a node; the pre-ranker predicts each
 * child's |S| in dB from its pixel map so that only the best-ranked children get an exact
 * evaluation (the exact solver stays the arbiter of every accepted change).  The paper has no
 * learned component; this follows the search's candidate structure (Section III-A).
 * Network: layer l maps h_l (B x dims[l]) to h_l W_l^T + b_l (W_l: dims[l+1] x dims[l]),
 * ReLU on all but the last layer; input = the map's pixel states as 0/1; BF16 weights and
 * activations, FP32 accumulation (tensor cores, tcgen05 kind::f16), FP32 master weights, Adam.
 * Parameters are one flat FP32 vector [W_0, b_0, W_1, b_1, ...] (W row-major). */
typedef struct pmom_mlp pmom_mlp;
/* dims: n_layers + 1 sizes (input first); initial weights He-uniform from SplitMix64(seed),
 * biases 0.  Needs the GPU.  Errors: INVALID_ARG, OOM, CUDA. */
pmom_status pmom_mlp_create(int32_t n_layers, const int32_t* dims, uint64_t seed, pmom_mlp** out);
pmom_status pmom_mlp_destroy(pmom_mlp* net);
const char* pmom_mlp_last_error(const pmom_mlp* net);
pmom_status pmom_mlp_num_params(const pmom_mlp* net, int64_t* count);
/* Copy the FP32 parameters and/or the last gradients to host float [count] (either may be NULL;
 * synchronizes the device). */
pmom_status pmom_mlp_get_params(pmom_mlp* net, float* params_host, float* grads_host);
/* Replace the parameters (host float [count]); resets the Adam state. */
pmom_status pmom_mlp_set_params(pmom_mlp* net, const float* params_host);
/* y_dev (device float [B][dims[L]]) = network(x_dev), x_dev device uint8 [B][dims[0]]. */
pmom_status pmom_mlp_forward(pmom_mlp* net, const uint8_t* x_dev, int32_t B, float* y_dev, void* stream);
/* Gradients of the mean squared error against target_dev (device float [B][dims[L]]) into the
 * network's gradient buffer; loss_host (optional) receives the loss (synchronizes). */
pmom_status pmom_mlp_backward(pmom_mlp* net, const uint8_t* x_dev, const float* target_dev, int32_t B,
                              double* loss_host, void* stream);
/* One Adam step with the last gradients. */
pmom_status pmom_mlp_adam(pmom_mlp* net, float lr, float beta1, float beta2, float eps, void* stream);
/* Predicted FoM (Eq. 8-9) of each map: the network's outputs are read as dB of S11, S21, S31, S32
 * (output q * F + f, times out_scale) and scored with band codes (device uint8 [F], as for
 * pmom_set_fom); fom_dev device double [B].  Needs dims[L] == 4 F. */
pmom_status pmom_mlp_predict_fom(pmom_mlp* net, const uint8_t* x_dev, int32_t B, const uint8_t* bands_dev,
                                 int32_t F, float out_scale, double* fom_dev, void* stream);
/* Training targets from evaluated S (device double [B][F][P][P][2], P = 3 or 4, as written by
 * pmom_eval_candidates): target_dev[b][q * F + f] = out_scale * dB(S_q(f)) for q = S11, S21,
 * S31, S32 (the entries the FoM of Eq. 8-9 reads), dB = 20 log10(max(|S|, 1e-15)). */
pmom_status pmom_mlp_targets(const double* S_dev, int32_t B, int32_t F, int32_t P, float out_scale,
                             float* target_dev, void* stream);
/* Tensor-core completion waits that ran out since creation (their GEMM tiles were skipped). */
pmom_status pmom_mlp_errors(pmom_mlp* net, int32_t* timeouts);

/* Support-set capacity of one task on this GPU for `precision` (PMOM_FP64 or
 * PMOM_MIXED_REFINED): *n_default = the largest N the default shared-memory layout holds (wide
 * panels, solve vectors in shared memory, up to two tasks per SM); *n_max = the largest N any
 * layout holds (narrow panels, solve vectors in the task's global workspace, one task per SM).
 * Candidates with N > *n_max are returned with status PMOM_CAND_CAPACITY.  Both are capped at M.
 * Needs the GPU.  Errors: INVALID_ARG, CUDA. */
pmom_status pmom_capacity(pmom_ctx* ctx, int32_t precision, int32_t* n_default, int32_t* n_max);

/* Depth-increasing all-way tree search (paper Algorithm 1, Section III-A; hyper-parameters of
 * Section III-C: Dmax = 2 with M(1) = 10, M(2) = 3 for the 8-state case).  A pixel is an (x, y)
 * column whose state is the bit pattern of its layers; every tree node branches into all other
 * states of one column drawn uniformly (counter-based SplitMix64 keyed by seed, restart,
 * iteration, depth and node) among the columns not yet on its path; each tree level is one
 * evaluator batch.  The best depth-D leaf is accepted only if its FoM is strictly lower; after
 * m_of_d[D-1] failures the depth grows; past d_max the search restarts from a random half-filled
 * map.  Stops when max_evals evaluations are used (a started tree is finished).
 *   init_map_host / best_map_host: uint8 [layers][ny][nx]; trace_host (optional): the current
 *   FoM after each iteration, up to trace_cap entries. */
typedef struct {
  uint64_t seed;
  int32_t d_max;          /* 1..8, and at most nx * ny (INVALID_ARG otherwise) */
  int32_t m_of_d[8];      /* non-improving iterations tolerated at each depth */
  int64_t max_evals;      /* FoM evaluation budget */
  int32_t precision;      /* PMOM_FP64 or PMOM_MIXED_REFINED */
} pmom_search_params;
pmom_status pmom_search(pmom_ctx* ctx, const pmom_search_params* params, const uint8_t* init_map_host,
                        uint8_t* best_map_host, double* best_fom, int64_t* evals_used, double* trace_host,
                        int32_t trace_cap, int32_t* trace_len, void* stream);

/* Database files (the paper's Phase 2 result, pre-computed once and reused).  Layout, little
 * endian: "PMOMZDB1", uint32 version 1, uint32 dtype (PMOM_C64 / PMOM_C128), int32 M, int32 F,
 * uint64 hash of the BF table (FNV-1a 64 over its M x 8 int32 in memory order), double freqs[F],
 * the database [F][M][M] (interleaved re, im), uint64 checksum of the database (FNV-1a 64 over its
 * 64-bit words).  pmom_save_Z writes the context's database (to path + ".tmp", then renamed);
 * pmom_load_Z_file checks the header, the BF-table hash and the file size before any device work,
 * then streams the data to the device (replacing the current database, as pmom_load_Z) and
 * checks the checksum, dropping the database on a mismatch.  Both synchronize `stream`.
 * Errors: INVALID_ARG, NOT_READY (save without a database), Z_SHAPE_MISMATCH (another grid: M or
 * BF table differ), IO, OOM, CUDA. */
pmom_status pmom_save_Z(pmom_ctx* ctx, const char* path, void* stream);
pmom_status pmom_load_Z_file(pmom_ctx* ctx, const char* path, void* stream);

/* Checkpoint of a search (pmom_search_resume): the caller owns the struct and both maps
 * ([layers][ny][nx] host bytes).  valid = 0 starts from init_map; a state returned by an earlier
 * call continues exactly where that call stopped (the same decisions as one uninterrupted run),
 * restart and iteration being the generator keys of R17. */
typedef struct {
  int32_t valid;
  int32_t depth, counter;
  int64_t evals;          /* evaluations since the search started */
  uint64_t restart, iteration;
  double fom, best_fom;   /* FoM of the current map and of the best map */
  uint8_t* map;           /* current map, host, caller-owned */
  uint8_t* best_map;      /* best map, host, caller-owned */
} pmom_search_state;
/* Algorithm 1 as pmom_search, from or to a checkpoint: runs until state->evals reaches
 * params->max_evals (a started tree is finished), then leaves the state valid.  trace_host
 * receives the current FoM after each iteration of this call.  Errors as pmom_search, and
 * INVALID_ARG for a state without maps. */
pmom_status pmom_search_resume(pmom_ctx* ctx, const pmom_search_params* params, const uint8_t* init_map_host,
                               pmom_search_state* state, double* trace_host, int32_t trace_cap, int32_t* trace_len,
                               void* stream);

/* Counters of the last eval call (host int64 [8]): tasks, refinement iterations summed over tasks,
 * max iterations of one task, tasks re-solved in FP64, tensor-core waits that ran out (the
 * task's candidate then reports PMOM_CAND_NONFINITE), reserved, kernel launches issued,
 * reserved.  Synchronizes the context's last stream. */
pmom_status pmom_stats(pmom_ctx* ctx, int64_t* out8);

/* Kernel timing of later eval calls: on != 0 makes each eval record CUDA events on its stream
 * around its kernels; pmom_kernel_times then returns the last call's milliseconds for
 * [0] activation, [1] evaluation, [2] FP64 repair, [3] Y -> S and FoM (host double [4];
 * synchronizes).  After pmom_eval_bordered the four are [0] reference gather + FP64 LU,
 * [1] reference inverse, [2] candidate activation + bordered update, [3] Y -> S and FoM. */
pmom_status pmom_set_timing(pmom_ctx* ctx, int32_t on);
pmom_status pmom_kernel_times(pmom_ctx* ctx, double* ms4_host);

/* Wait for all work the context issued on `stream`. */
pmom_status pmom_sync(pmom_ctx* ctx, void* stream);

/* Failure-detection self-test of the bounded completion wait that every tensor-core path uses
 * (a stalled wait flags the task, PMOM_CAND_NONFINITE, instead of hanging the GPU): one warp waits
 * on an mbarrier expecting one arrival, polling at most `polls` times (1 .. 2^30); with
 * arrive != 0 it arrives first, otherwise nothing ever arrives.  *timed_out_host = 1 when the wait
 * gave up, 0 when it saw the phase complete; *elapsed_ms_host = the kernel's CUDA-event time.  No
 * context; synchronizes `stream`; the device stays usable.  Errors: INVALID_ARG, CUDA. */
pmom_status pmom_selftest_wait(int64_t polls, int32_t arrive, int32_t* timed_out_host, double* elapsed_ms_host,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PMOM_H */
