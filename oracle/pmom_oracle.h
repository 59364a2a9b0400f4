/*
 * pmom_oracle.h -- plain CPU reference of the pre-computed MoM candidate evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the oracle the CUDA library is checked against; it is
 * used by tests/, by the smoke check and by the CPU-baseline leg of bench.py, never by the
 * library itself.  It shares no code with the library.  Everything is complex128 and follows the
 * paper's definitions step by step, with no blocking, fusion or reordering:
 *
 *   mesh + basis-function classes ....... Section II-C (four BF categories), Section VI-A
 *                                          (diagonal-only contact is not a connection),
 *                                          Section V-A (two alternating triangles per pixel)
 *   support set and selection ........... Eq. (3)-(5)
 *   EFIE / MPIE fill of Z(f) ............ Eq. (1)-(2), RWG basis (Section II-B)
 *   port excitation, S-parameters ....... Eq. (6)-(7)
 *   figure of merit ..................... Eq. (8)-(9)
 *
 * Where the paper is silent (Green's function of the stack-up, quadrature, port stub geometry,
 * dB convention, band edges) the readings are stated next to the code that takes them.
 */
#ifndef PMOM_ORACLE_H
#define PMOM_ORACLE_H

#include <complex.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int layers, nx, ny;
  double pitch;            /* pixel side a [m] */
  int medium;              /* 0: microstrip (one ground plane at z = 0) in the homogeneous effective-medium
                              reading, 1: stripline (planes at 0 and h_total), 2: microstrip as a
                              grounded dielectric slab under air (Sommerfeld kernels) */
  const double* layer_z;   /* [layers] metal heights [m] */
  double h_total;          /* stripline plate spacing [m] (microstrip: unused) */
  double eps_r, tan_d;
  int n_states;            /* 2: void/metal; 3: void/metal/metal with a via to the next layer */
  int n_ports;
  const int32_t* ports;    /* [n_ports][3] = layer, side (0 right, 1 top, 2 left, 3 bottom), pos */
  int diag_pattern;        /* pixel diagonals (Section V-A, Fig. mesh_orientation a-c): 0 alternating, 1 uniform, 2 random */
  uint64_t diag_seed;      /* pattern 2: seed of the per-position orientation draw */
  int sub;                 /* sub-squares per pixel side: 1, 2 or 3 (2, 8 or 18 triangles per pixel,
                              Section V-A); 0 reads as 1; vias need 1 */
} or_grid;

/* Basis-function classes (Section II-C), plus the three BFs of a via site (state 2). */
enum { OR_BF_ALWAYS = 0, OR_BF_INNER = 1, OR_BF_INTER = 2, OR_BF_PIXPORT = 3,
       OR_BF_VIA_STRIP = 4, OR_BF_VIA_JOIN = 5, OR_BF_VIA_LAND = 6 };

/* One BF-table row = 8 int32:
 *   [0] class  [1] pixel A  [2] pixel B  [3] port (or -1)
 *   [4] key of T+  [5] key of T-  [6] free-vertex index in T+  [7] free-vertex index in T-
 * pixel index = (layer*ny + y)*nx + x; triangle key = (((layer*W + Y+4s)*W + X+4s)*4 + half) with
 * W = 128 s and (X, Y) the sub-square on the fine lattice (the pixel itself when s = 1); half 0/1 =
 * the sub-square's triangles, 2/3 = the triangles Ta/Tb of the via strip from the pixel up to
 * layer+1.  Via rows: [1] = the via pixel (l, x, y); [2] = (l+1, x, y) for the landing junction. */
#define OR_BF_COLS 8

int or_count_bfs(const or_grid* g);
/* Always-present BFs per port stub (3 when s = 1), and the delta-gap BFs of port p: their
 * canonical indices (s of them; 3p+1 when s = 1), which are also their positions in every
 * support set (the stub BFs come first).  Returns s. */
int or_stub_bfs(const or_grid* g);
int or_port_gap(const or_grid* g, int p, int32_t* bf);
/* Fine-lattice parts of a triangle key. */
void or_key_parts(const or_grid* g, int32_t key, int* layer, int* X, int* Y, int* half);
int or_bf_table(const or_grid* g, int32_t* table);
/* Eq. (3): ascending indices of the BFs active under `map` ([layers][ny][nx] states).
 * Returns N >= 0, or -1 if a state is out of range. */
int or_active_set(const or_grid* g, const int32_t* table, int M, const uint8_t* map, int32_t* idx);

/* Diagonal orientation of lattice pixel (x, y) (stub pixels included; the same on every layer):
 * 0 -> diagonal (x, y+1)-(x+1, y), 1 -> (x, y)-(x+1, y+1).  Alternating: (x + y) mod 2; uniform: 0;
 * random: the top bit of SplitMix64 chained over (diag_seed, (y+4)*128 + x+4). */
int or_orient(const or_grid* g, int x, int y);

/* Triangle geometry of a key (3 vertices, metres). */
void or_triangle(const or_grid* g, int32_t key, double v[3][3]);

/* Z(f) of the all-metal parent, complex128, row-major [F][M][M].
 * mode 0: every triangle pair integrated; mode 1: pairs related by a lattice translation share
 * one integration.  Returns max |Z - Z^T| / max |Z| before symmetrisation (Z <- (Z + Z^T)/2). */
double or_fill(const or_grid* g, const double* freqs, int F, int mode, int threads, double complex* Z);
/* Z(f) of the sub-structure made of the listed BFs only ([F][N][N]), filled directly by the same
 * per-pair code (the premise of Eq. 4-5: it equals the parent's rows and columns bf). */
double or_fill_subset(const or_grid* g, const double* freqs, int F, int mode, int threads, const int32_t* bf, int N,
                      double complex* Z);

/* Green's function of the stack-up between metal layers lp and lq at lateral distance rho. */
double complex or_green(const or_grid* g, double freq, int lp, int lq, double rho);
/* Same, by the slow reference route only (stripline: plain image series with K images). */
double complex or_green_images(const or_grid* g, double freq, int lp, int lq, double rho, int K);
double complex or_green_modal(const or_grid* g, double freq, int lp, int lq, double rho);
double complex or_bessel_k0(double complex w);
/* K0 for any Re w >= 0 (series / asymptotic; used for the TEM term of the Neumann mode series). */
double complex or_bessel_k0_any(double complex w);
/* Kernel `kind` (0: Dirichlet G_D, 1: Neumann G_N) between arbitrary heights zp, zq [m];
 * route 0: the fill's evaluation, 1: image series with K images, 2: mode series. */
double complex or_green_heights(const or_grid* g, double freq, int kind, double zp, double zq, double rho,
                                int route, int K);
/* Grounded-slab (microstrip) kernels by Sommerfeld integrals: kind 0 = G_phi (eps0-normalised scalar
 * potential), 1 = G_A (horizontal vector potential), between heights z, zp inside or on the slab
 * (thickness = the highest metal layer) at lateral distance rho; er_top = relative permittivity of
 * the half-space above.  reg != 0 subtracts C / (4 pi R); C (the quasi-static constant) -> c_out. */
double complex or_slab_green(const or_grid* g, double freq, int kind, double z, double zp, double rho,
                             double er_top, int reg, double* c_out);
/* The fill's table of the Sommerfeld remainder at rho_i = i h (i < n); C and k1 returned. */
void or_slab_table(const or_grid* g, double freq, int kind, double z, double zp, double er_top, double h, int n,
                   double complex* out, double* c_out, double complex* k1_out);
/* Analytic potential integrals over a planar triangle (used by the singular part of the fill). */
void or_tri_potentials(const double tri[3][3], const double r[3], double* I1, double Iv[3]);
/* Quadrature rules on the reference triangle: n = 7 or 13; returns barycentric rows and weights. */
int or_tri_rule(int n, const double** bary, const double** w);
double or_eps_eff(const or_grid* g);
void or_pair_integrals(const or_grid* g, double freq, int32_t kp, int32_t kq, double complex out[10]);

/* Dense LU with partial pivoting (|a| modulus, ties to the lowest row), row-major, in place. */
int or_lu(double complex* A, int n, int32_t* piv);
void or_lu_solve(const double complex* LU, const int32_t* piv, int n, double complex* B, int nrhs);

/* Per-candidate evaluation (Eq. 5-7): S[F][P][P] for one map.  zc64 != 0: Z is complex64
 * storage (promoted exactly to complex128).  form 0: unloaded delta-gap solve + Y->S,
 * form 1: ports loaded with Z0 and Eq. (6).  Returns 0, 1 (singular), -1 (bad state). */
int or_eval_map(const or_grid* g, const int32_t* table, int M, const void* Z, int zc64, int F,
                const uint8_t* map, double Z0, int form, double complex* S);
/* Batch version, threads over (candidate, frequency); status[B]. */
void or_eval_batch(const or_grid* g, const int32_t* table, int M, const void* Z, int zc64, int F,
                   const uint8_t* maps, int B, double Z0, int threads, double complex* S, int32_t* status);

/* Eq. (8)-(9).  band[f]: 0 p1, 1 p2, 2 i, 3 s, 255 none. */
double or_fom(const double complex* S, int F, int P, const uint8_t* band);
void or_bands(const double* freqs, int F, const double* edges /* p1lo,p1hi,p2lo,p2hi,ilo,ihi,slo,shi */,
              uint8_t* band);

#ifdef __cplusplus
}
#endif
#endif
