/*
 * or_solve.c -- oracle candidate evaluation.  TEST INFRASTRUCTURE ONLY.
 *
 * For one pixel map and one frequency (Section II-C and II-E):
 *   support set I (Eq. 3, ascending) -> Z_sub = S^T Z_parent S (Eq. 4-5, i.e. rows and columns I)
 *   -> solve Z_sub X = V for every port excitation (Eq. 2) -> port currents I_i = l_i x_i (Eq. 7)
 *   -> S-parameters.  A port's delta gap is its gap BFs (one with the two-triangle mesh, s with
 *   s x s sub-squares per pixel); a unit gap voltage drives each of them with V_k = l_k, and the
 *   port current is the sum over them.  Two equivalent forms are provided:
 *      form 0: unloaded delta-gap solve, V = l_k at the gap BFs of port j;
 *              Y_ij = sum over the gap of port i of l_k x_k^(j);  S = (1 + Z0 Y)^-1 (1 - Z0 Y)
 *      form 1: every port carries its Z0 load across its gap (Z_kk' += Z0 l_k l_k' for gap BFs
 *              k, k' of one port; Z_pp += Z0 l_p^2 with one gap BF) and an EMF of 1 V drives
 *              port j; S_ij = delta_ij - 2 Z0 I_i / V_j (Eq. 6)
 * FoM of Eq. (8)-(9) with S in dB = 20 log10(max(|S|, 1e-15)); lower is better.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "pmom_oracle.h"

int or_lu(double complex* A, int n, int32_t* piv) {
  int singular = 0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = cabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = cabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double complex t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
    }
    if (best == 0.0) { singular = 1; continue; }
    double complex akk = A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double complex l = A[(size_t)i * n + k] / akk;
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return singular;
}

void or_lu_solve(const double complex* LU, const int32_t* piv, int n, double complex* B, int nrhs) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k)
      for (int c = 0; c < nrhs; ++c) {
        double complex t = B[(size_t)k * nrhs + c];
        B[(size_t)k * nrhs + c] = B[(size_t)p * nrhs + c];
        B[(size_t)p * nrhs + c] = t;
      }
  }
  for (int i = 0; i < n; ++i)              /* L y = P b, unit diagonal */
    for (int k = 0; k < i; ++k)
      for (int c = 0; c < nrhs; ++c) B[(size_t)i * nrhs + c] -= LU[(size_t)i * n + k] * B[(size_t)k * nrhs + c];
  for (int i = n - 1; i >= 0; --i) {       /* U x = y */
    for (int k = i + 1; k < n; ++k)
      for (int c = 0; c < nrhs; ++c) B[(size_t)i * nrhs + c] -= LU[(size_t)i * n + k] * B[(size_t)k * nrhs + c];
    for (int c = 0; c < nrhs; ++c) B[(size_t)i * nrhs + c] /= LU[(size_t)i * n + i];
  }
}

static double port_edge_length(const or_grid* g, const int32_t* table, int m) {
  const int32_t* r = table + OR_BF_COLS * m;
  double v[3][3];
  or_triangle(g, r[4], v);
  int f = r[6];
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = v[(f + 1) % 3][k] - v[(f + 2) % 3][k];
  return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* S for one map at one frequency; Zf is that frequency's M x M parent matrix. */
static int eval_one(const or_grid* g, const int32_t* table, int M, const void* Zf, int zc64, const int32_t* idx,
                    int N, double Z0, int form, double complex* S) {
  int P = g->n_ports;
  double complex* A = (double complex*)malloc(sizeof(double complex) * (size_t)N * N);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      size_t off = (size_t)idx[a] * M + idx[b];
      if (zc64) {
        const float* z = (const float*)Zf;
        A[(size_t)a * N + b] = (double)z[2 * off] + I * (double)z[2 * off + 1];
      } else {
        A[(size_t)a * N + b] = ((const double complex*)Zf)[off];
      }
    }
  /* the gap BFs of each port: canonical indices, which are also their positions in the support
   * set (the always-present stub BFs come first), and their edge lengths */
  int32_t gap[4][3];
  double lg[4][3];
  int ng = 0;
  for (int p = 0; p < P; ++p) {
    ng = or_port_gap(g, p, gap[p]);
    for (int k = 0; k < ng; ++k) {
      if (gap[p][k] >= N || idx[gap[p][k]] != gap[p][k]) { free(A); return 1; }
      lg[p][k] = port_edge_length(g, table, gap[p][k]);
    }
  }
  if (form == 1)
    for (int p = 0; p < P; ++p)
      for (int k = 0; k < ng; ++k)
        for (int q = 0; q < ng; ++q) A[(size_t)gap[p][k] * N + gap[p][q]] += Z0 * lg[p][k] * lg[p][q];
  double complex* X = (double complex*)calloc((size_t)N * P, sizeof(double complex));
  for (int j = 0; j < P; ++j)
    for (int k = 0; k < ng; ++k) X[(size_t)gap[j][k] * P + j] = lg[j][k] * 1.0;
  int32_t* piv = (int32_t*)malloc(sizeof(int32_t) * N);
  int sing = or_lu(A, N, piv);
  or_lu_solve(A, piv, N, X, P);
  /* port currents: I_ij = sum over the gap of port i of l_k x_k^(j) */
  double complex Ip[16];
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double complex c = 0.0;
      for (int k = 0; k < ng; ++k) c += lg[i][k] * X[(size_t)gap[i][k] * P + j];
      Ip[i * P + j] = c;
    }
  if (form == 0) {
    /* Y = I (unit gap voltages); S = (1 + Z0 Y)^-1 (1 - Z0 Y) */
    double complex Ap[16], Bp[16];
    int32_t pv[4];
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) {
        Ap[i * P + j] = (i == j ? 1.0 : 0.0) + Z0 * Ip[i * P + j];
        Bp[i * P + j] = (i == j ? 1.0 : 0.0) - Z0 * Ip[i * P + j];
      }
    or_lu(Ap, P, pv);
    or_lu_solve(Ap, pv, P, Bp, P);
    memcpy(S, Bp, sizeof(double complex) * P * P);
  } else {
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) S[i * P + j] = (i == j ? 1.0 : 0.0) - 2.0 * Z0 * Ip[i * P + j] / 1.0;
  }
  free(A); free(X); free(piv);
  return sing;
}

int or_eval_map(const or_grid* g, const int32_t* table, int M, const void* Z, int zc64, int F,
                const uint8_t* map, double Z0, int form, double complex* S) {
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * M);
  int N = or_active_set(g, table, M, map, idx);
  if (N < 0) { free(idx); return -1; }
  int P = g->n_ports, status = 0;
  size_t esz = zc64 ? 8 : 16;
  for (int f = 0; f < F; ++f) {
    const char* Zf = (const char*)Z + (size_t)f * M * M * esz;
    if (eval_one(g, table, M, Zf, zc64, idx, N, Z0, form, S + (size_t)f * P * P)) status = 1;
  }
  free(idx);
  return status;
}

typedef struct {
  const or_grid* g;
  const int32_t* table;
  int M, F, B, zc64, nthreads, tid;
  const void* Z;
  const uint8_t* maps;
  double Z0;
  double complex* S;
  int32_t* status;
  const int32_t* idx;   /* [B][M] */
  const int32_t* N;     /* [B] */
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* J = (batch_job*)arg;
  int P = J->g->n_ports;
  size_t esz = J->zc64 ? 8 : 16;
  for (long t = J->tid; t < (long)J->B * J->F; t += J->nthreads) {
    int b = (int)(t / J->F), f = (int)(t % J->F);
    if (J->N[b] < 0) continue;
    const char* Zf = (const char*)J->Z + (size_t)f * J->M * J->M * esz;
    if (eval_one(J->g, J->table, J->M, Zf, J->zc64, J->idx + (size_t)b * J->M, J->N[b], J->Z0, 0,
                 J->S + ((size_t)b * J->F + f) * P * P))
      J->status[b] = 1;   /* benign race: every writer stores the same value */
  }
  return NULL;
}

void or_eval_batch(const or_grid* g, const int32_t* table, int M, const void* Z, int zc64, int F,
                   const uint8_t* maps, int B, double Z0, int threads, double complex* S, int32_t* status) {
  int np = g->layers * g->ny * g->nx;
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)B * M);
  int32_t* N = (int32_t*)malloc(sizeof(int32_t) * B);
  for (int b = 0; b < B; ++b) {
    N[b] = or_active_set(g, table, M, maps + (size_t)b * np, idx + (size_t)b * M);
    status[b] = N[b] < 0 ? -1 : 0;
  }
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
  batch_job* jobs = (batch_job*)malloc(sizeof(batch_job) * threads);
  for (int i = 0; i < threads; ++i) {
    batch_job j = {g, table, M, F, B, zc64, threads, i, Z, maps, Z0, S, status, idx, N};
    jobs[i] = j;
    pthread_create(&th[i], NULL, batch_worker, &jobs[i]);
  }
  for (int i = 0; i < threads; ++i) pthread_join(th[i], NULL);
  free(th); free(jobs); free(idx); free(N);
}

static double sdb(double complex s) {
  double a = cabs(s);
  if (a < 1e-15) a = 1e-15;
  return 20.0 * log10(a);
}

double or_fom(const double complex* S, int F, int P, const uint8_t* band) {
  double fom = 0.0;
  for (int f = 0; f < F; ++f) {
    const double complex* s = S + (size_t)f * P * P;
    double s11 = sdb(s[0 * P + 0]), s21 = sdb(s[1 * P + 0]), s31 = sdb(s[2 * P + 0]), s32 = sdb(s[2 * P + 1]);
    double rw_p1 = pow(10.0, (s21 + 1.0) / 10.0), rw_p2 = pow(10.0, (s31 + 1.0) / 10.0);
    double rw_s1 = pow(10.0, (-s21 - 35.0) / 15.0), rw_s2 = pow(10.0, (-s31 - 35.0) / 15.0);
    double rw_s3 = pow(10.0, (-s21 - 20.0) / 18.0), rw_s4 = pow(10.0, (-s31 - 20.0) / 18.0);
    double rw_oi = pow(10.0, (-s32 - 20.0) / 15.0);
    double rw_m1 = pow(10.0, (-15.0 - s11) / 10.0), rw_m2 = pow(10.0, (-15.0 - s11) / 10.0);
    switch (band[f]) {
      case 0: fom += 1.0 / rw_p1 + 1.0 / rw_m1 + 1.0 / rw_s2; break;
      case 1: fom += 1.0 / rw_p2 + 1.0 / rw_m2 + 1.0 / rw_s1; break;
      case 2: fom += 1.0 / rw_oi; break;
      case 3: fom += 1.0 / rw_s3 + 1.0 / rw_s4; break;
      default: break;
    }
  }
  return fom;
}

void or_bands(const double* freqs, int F, const double* e, uint8_t* band) {
  for (int f = 0; f < F; ++f) {
    double x = freqs[f];
    if (x >= e[0] && x <= e[1]) band[f] = 0;
    else if (x >= e[2] && x <= e[3]) band[f] = 1;
    else if (x > e[4] && x < e[5]) band[f] = 2;
    else if (x >= e[6] && x <= e[7]) band[f] = 3;
    else band[f] = 255;
  }
}
