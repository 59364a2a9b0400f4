/*
 * or_fill.c -- oracle EFIE (MPIE) fill of the parent interaction matrix Z(f).  TEST INFRASTRUCTURE ONLY.
 *
 * Eq. (1)-(2) with RWG functions (Section II-B), Galerkin testing, e^{+jwt} convention:
 *   Z_mn = jw mu  <f_m, G f_n>  +  1/(jw eps) <div f_m, G div' f_n>
 * with f = s (l / 2A) (r - v_free) and div f = s l / A on T+ (s = +1) and T- (s = -1).
 *
 * Green's function (the paper uses FEKO's layered-media MPIE, Section II-D; that code is not
 * available, so the stack-up is read as a homogeneous dielectric eps_r (1 - j tan d)):
 *   microstrip: one PEC ground at z = 0, homogeneous medium of Hammerstad-Jensen eps_eff at
 *               w = pitch, one negative image:  G = g(R) - g(R_image)
 *   stripline : PEC planes at z = 0 and z = H, dielectric between them.  Horizontal currents and
 *               charges both see the Dirichlet Green's function of the slab, which we evaluate in
 *               two exact representations:
 *                 image series  G = sum_n g(rho, z - z' + 2nH) - g(rho, z + z' + 2nH)
 *                 mode series   G = 1/(pi H) sum_{m>=1} sin(m pi z/H) sin(m pi z'/H) K0(gamma_m rho),
 *                               gamma_m = sqrt((m pi/H)^2 - k^2)
 *               For rho >= H/2 the mode series is summed to round-off.  For rho < H/2 the image
 *               terms |n| <= K are summed explicitly and the remaining images, which are smooth
 *               and even in rho, are represented by c0 + c1 rho^2 + c2 rho^4 matched to the mode
 *               series at rho = H/2, 3H/4, H.
 *   g(R) = exp(-jkR) / (4 pi R),  k = w sqrt(mu0 eps0 eps_r (1 - j tan d)).
 *
 * Quadrature: Radon's 7-point degree-5 rule on both triangles of a well-separated pair;
 * Dunavant's 13-point degree-7 rule for near pairs (centroid distance < 2 x longest edge),
 * where 1/(4 pi R) of the direct term is integrated analytically over the source triangle
 * (Wilton et al. 1984) and the smooth remainder G - 1/(4 pi R) numerically.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "pmom_oracle.h"

#define OR_PI 3.14159265358979323846
#define C0 299792458.0
#define MU0 (4.0e-7 * OR_PI)
#define EPS0 (1.0 / (MU0 * C0 * C0))
#define MAXL 8
#define IMG_K 16

/* ---------------------------------------------------------------- quadrature rules */
static double rule7_b[7][3], rule7_w[7], rule13_b[13][3], rule13_w[13];
static int rules_ready = 0;
static pthread_once_t rules_once = PTHREAD_ONCE_INIT;

static void set_sym(double b[][3], double* w, int* n, double a, double c, double wt) {
  /* point (a, c, c) and its distinct permutations */
  double pts[3][3] = {{a, c, c}, {c, a, c}, {c, c, a}};
  for (int i = 0; i < 3; ++i) { b[*n][0] = pts[i][0]; b[*n][1] = pts[i][1]; b[*n][2] = pts[i][2]; w[(*n)++] = wt; }
}

static void init_rules(void) {
  int n = 0;
  double s15 = sqrt(15.0);
  rule7_b[0][0] = rule7_b[0][1] = rule7_b[0][2] = 1.0 / 3.0; rule7_w[0] = 9.0 / 40.0; n = 1;
  set_sym(rule7_b, rule7_w, &n, (9.0 - 2.0 * s15) / 21.0, (6.0 + s15) / 21.0, (155.0 + s15) / 1200.0);
  set_sym(rule7_b, rule7_w, &n, (9.0 + 2.0 * s15) / 21.0, (6.0 - s15) / 21.0, (155.0 - s15) / 1200.0);
  n = 0;
  rule13_b[0][0] = rule13_b[0][1] = rule13_b[0][2] = 1.0 / 3.0; rule13_w[0] = -0.149570044467682; n = 1;
  set_sym(rule13_b, rule13_w, &n, 0.479308067841920, 0.260345966079040, 0.175615257433208);
  set_sym(rule13_b, rule13_w, &n, 0.869739794195568, 0.065130102902216, 0.053347235608838);
  const double a = 0.048690315425316, b = 0.312865496004874, c = 0.638444188569810, wt = 0.077113760890257;
  const double perm[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
  for (int i = 0; i < 6; ++i) {
    rule13_b[n][0] = perm[i][0]; rule13_b[n][1] = perm[i][1]; rule13_b[n][2] = perm[i][2]; rule13_w[n++] = wt;
  }
  rules_ready = 1;
}

int or_tri_rule(int n, const double** bary, const double** w) {
  pthread_once(&rules_once, init_rules);
  if (n == 7) { *bary = &rule7_b[0][0]; *w = rule7_w; return 7; }
  if (n == 13) { *bary = &rule13_b[0][0]; *w = rule13_w; return 13; }
  return 0;
}

/* ---------------------------------------------------------------- small vector helpers */
static void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* ---------------------------------------------------------------- analytic potentials */
/* R + l written without cancellation when l < 0 (R^2 = R0^2 + l^2). */
static double r_plus_l(double R, double l, double R02) { return l >= 0.0 ? R + l : R02 / (R - l); }

void or_tri_potentials(const double tri[3][3], const double r[3], double* I1, double Iv[3]) {
  double e1[3], e2[3], n[3];
  sub3(tri[1], tri[0], e1);
  sub3(tri[2], tri[0], e2);
  cross3(e1, e2, n);
  double nn = norm3(n);
  for (int i = 0; i < 3; ++i) n[i] /= nn;
  double rv[3];
  sub3(r, tri[0], rv);
  double d = dot3(n, rv), ad = fabs(d);
  double rho[3] = {r[0] - d * n[0], r[1] - d * n[1], r[2] - d * n[2]};
  double s1 = 0.0, sv[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i) {
    const double* a = tri[i];
    const double* b = tri[(i + 1) % 3];
    double lv[3], lhat[3], u[3], am[3], bm[3];
    sub3(b, a, lv);
    double len = norm3(lv);
    for (int k = 0; k < 3; ++k) lhat[k] = lv[k] / len;
    cross3(lhat, n, u);                   /* outward edge normal in the plane */
    sub3(a, rho, am);
    sub3(b, rho, bm);
    double lm = dot3(am, lhat), lp = dot3(bm, lhat), t = dot3(am, u);
    double R02 = t * t + d * d;
    double Rm = sqrt(R02 + lm * lm), Rp = sqrt(R02 + lp * lp);
    double Lg = 0.0;
    if (R02 > 1e-30 * len * len) Lg = log(r_plus_l(Rp, lp, R02) / r_plus_l(Rm, lm, R02));
    if (R02 > 1e-30 * len * len) {
      s1 += t * Lg;
      if (ad > 0.0) s1 -= ad * (atan(t * lp / (R02 + ad * Rp)) - atan(t * lm / (R02 + ad * Rm)));
    }
    double vv = R02 * Lg + lp * Rp - lm * Rm;
    for (int k = 0; k < 3; ++k) sv[k] += 0.5 * u[k] * vv;
  }
  *I1 = s1;
  Iv[0] = sv[0]; Iv[1] = sv[1]; Iv[2] = sv[2];
}

/* ---------------------------------------------------------------- Green's functions */
double complex or_bessel_k0(double complex w) {
  /* K0(w) = int_0^inf exp(-w cosh t) dt (Re w > 0); the trapezoidal rule converges
   * geometrically for this analytic, double-exponentially decaying integrand.  Near t = 0 the
   * integrand is a Gaussian of width 1/sqrt|w|, so the step shrinks for large |w|. */
  double h = 0.6 / sqrt(cabs(w));
  if (h > 0.2) h = 0.2;
  double complex s = 0.5 * cexp(-w);
  for (int j = 1; j < 20000; ++j) {
    double c = cosh(j * h);
    if (creal(w) * (c - 1.0) > 40.0) break;   /* terms below e^-40 of the first */
    s += cexp(-w * c);
  }
  return h * s;
}

double or_eps_eff(const or_grid* g) {
  if (g->medium != 0) return g->eps_r;
  /* Hammerstad & Jensen (1980) effective permittivity of a strip of width w = pitch at height h */
  double h = g->layer_z[0];
  for (int l = 1; l < g->layers; ++l) if (g->layer_z[l] > h) h = g->layer_z[l];
  double u = g->pitch / h, er = g->eps_r;
  double a = 1.0 + log((pow(u, 4) + pow(u / 52.0, 2)) / (pow(u, 4) + 0.432)) / 49.0 + log(1.0 + pow(u / 18.1, 3)) / 18.7;
  double b = 0.564 * pow((er - 0.9) / (er + 3.0), 0.053);
  return 0.5 * (er + 1.0) + 0.5 * (er - 1.0) * pow(1.0 + 10.0 / u, -a * b);
}

typedef struct {
  const or_grid* g;
  double omega, H, rho_s;
  double complex k, eps;
  double complex fit[MAXL][MAXL][3];
} medium_t;

static double complex gfree(double complex k, double R) { return cexp(-I * k * R) / (4.0 * OR_PI * R); }

/* (exp(-jkR) - 1) / (4 pi R), finite at R = 0 */
static double complex gfree_reg(double complex k, double R) {
  double complex x = -I * k * R;
  if (cabs(x) < 1e-3) return (-I * k) * (1.0 + x / 2.0 + x * x / 6.0 + x * x * x / 24.0) / (4.0 * OR_PI);
  return (cexp(x) - 1.0) / (4.0 * OR_PI * R);
}

static double complex strip_images(const medium_t* md, double zp, double zq, double rho, int K, int reg) {
  double H = md->H, r2 = rho * rho;
  double complex s = 0.0;
  for (int a = 0; a <= K; ++a) {
    for (int sg = (a == 0 ? 1 : -1); sg <= 1; sg += 2) {
      int n = a * sg;
      double zp_ = (zp - zq) + 2.0 * n * H, zm_ = (zp + zq) + 2.0 * n * H;
      double Rp = sqrt(r2 + zp_ * zp_), Rm = sqrt(r2 + zm_ * zm_);
      if (n == 0 && reg) s += gfree_reg(md->k, Rp);
      else s += gfree(md->k, Rp);
      s -= gfree(md->k, Rm);
    }
  }
  return s;
}

static double complex strip_modal(const medium_t* md, double zp, double zq, double rho) {
  double H = md->H;
  double complex s = 0.0;
  for (int m = 1; m < 4000; ++m) {
    double km = m * OR_PI / H;
    double complex gam = csqrt(km * km - md->k * md->k);
    if (creal(gam) * rho > 40.0) break;
    s += sin(km * zp) * sin(km * zq) * or_bessel_k0(gam * rho);
  }
  return s / (OR_PI * H);
}

static void medium_init(medium_t* md, const or_grid* g, double freq) {
  md->g = g;
  md->omega = 2.0 * OR_PI * freq;
  double er = or_eps_eff(g);
  md->eps = EPS0 * er * (1.0 - I * g->tan_d);
  md->k = md->omega * csqrt(MU0 * md->eps);
  md->H = g->h_total;
  md->rho_s = 0.5 * g->h_total;
  if (g->medium == 1) {
    for (int p = 0; p < g->layers; ++p) {
      for (int q = 0; q < g->layers; ++q) {
        double zp = g->layer_z[p], zq = g->layer_z[q];
        double x[3];
        double complex y[3];
        for (int i = 0; i < 3; ++i) {
          double rho = md->rho_s * (1.0 + 0.5 * i);
          x[i] = rho * rho;
          y[i] = strip_modal(md, zp, zq, rho) - strip_images(md, zp, zq, rho, IMG_K, 0);
        }
        /* quadratic in x = rho^2 through the three points (Newton divided differences) */
        double complex d01 = (y[1] - y[0]) / (x[1] - x[0]);
        double complex d12 = (y[2] - y[1]) / (x[2] - x[1]);
        double complex d012 = (d12 - d01) / (x[2] - x[0]);
        double complex c2 = d012;
        double complex c1 = d01 - d012 * (x[0] + x[1]);
        double complex c0 = y[0] - d01 * x[0] + d012 * x[0] * x[1];
        md->fit[p][q][0] = c0; md->fit[p][q][1] = c1; md->fit[p][q][2] = c2;
      }
    }
  }
}

/* G (reg = 0) or G - 1/(4 pi R_direct) (reg = 1) between layers lp, lq at lateral distance rho. */
static double complex green_eval(const medium_t* md, int lp, int lq, double rho, int reg) {
  const or_grid* g = md->g;
  double zp = g->layer_z[lp], zq = g->layer_z[lq];
  if (g->medium == 0) {
    double Rd = sqrt(rho * rho + (zp - zq) * (zp - zq)), Ri = sqrt(rho * rho + (zp + zq) * (zp + zq));
    return (reg ? gfree_reg(md->k, Rd) : gfree(md->k, Rd)) - gfree(md->k, Ri);
  }
  if (rho >= md->rho_s) {
    double complex G = strip_modal(md, zp, zq, rho);
    if (reg) G -= 1.0 / (4.0 * OR_PI * sqrt(rho * rho + (zp - zq) * (zp - zq)));
    return G;
  }
  const double complex* c = md->fit[lp][lq];
  double x = rho * rho;
  return strip_images(md, zp, zq, rho, IMG_K, reg) + c[0] + x * (c[1] + x * c[2]);
}

double complex or_green(const or_grid* g, double freq, int lp, int lq, double rho) {
  medium_t md;
  medium_init(&md, g, freq);
  return green_eval(&md, lp, lq, rho, 0);
}

double complex or_green_images(const or_grid* g, double freq, int lp, int lq, double rho, int K) {
  medium_t md;
  medium_init(&md, g, freq);
  return strip_images(&md, g->layer_z[lp], g->layer_z[lq], rho, K, 0);
}

double complex or_green_modal(const or_grid* g, double freq, int lp, int lq, double rho) {
  medium_t md;
  medium_init(&md, g, freq);
  return strip_modal(&md, g->layer_z[lp], g->layer_z[lq], rho);
}

/* ---------------------------------------------------------------- triangle-pair integrals */
typedef struct {
  double v[3][3];
  double c[3];
  double area, lmax;
  int layer;
} tri_t;

static void tri_setup(tri_t* t, const double v[3][3], int layer) {
  memcpy(t->v, v, sizeof(t->v));
  double e1[3], e2[3], n[3];
  sub3(v[1], v[0], e1);
  sub3(v[2], v[0], e2);
  cross3(e1, e2, n);
  t->area = 0.5 * norm3(n);
  t->lmax = 0.0;
  for (int i = 0; i < 3; ++i) {
    double e[3];
    sub3(v[(i + 1) % 3], v[i], e);
    double l = norm3(e);
    if (l > t->lmax) t->lmax = l;
    t->c[i] = (v[0][i] + v[1][i] + v[2][i]) / 3.0;
  }
  t->layer = layer;
}

static void tri_point(const tri_t* t, const double* b, double* r) {
  for (int k = 0; k < 3; ++k) r[k] = b[0] * t->v[0][k] + b[1] * t->v[1][k] + b[2] * t->v[2][k];
}

/* out[0] = int int G ; out[1 + 3a + b] = int int (r - v_a).(r' - v_b) G  over T_p x T_q */
static void pair_integrals(const medium_t* md, const tri_t* p, const tri_t* q, double complex out[10]) {
  for (int i = 0; i < 10; ++i) out[i] = 0.0;
  double dc[3];
  sub3(p->c, q->c, dc);
  double lm = p->lmax > q->lmax ? p->lmax : q->lmax;
  /* lattice geometry puts many pairs exactly on the threshold: resolve ties as "near" */
  int near = norm3(dc) < 2.0 * lm * (1.0 + 1e-9);
  const double *bo, *wo, *bi, *wi;
  int no = or_tri_rule(near ? 13 : 7, &bo, &wo);
  int ni = or_tri_rule(near ? 13 : 7, &bi, &wi);
  for (int i = 0; i < no; ++i) {
    double r[3], ra[3][3];
    tri_point(p, bo + 3 * i, r);
    for (int a = 0; a < 3; ++a) sub3(r, p->v[a], ra[a]);
    double wpo = wo[i] * p->area;
    if (near) {
      double I1, Iv[3];
      or_tri_potentials(q->v, r, &I1, Iv);
      double d = r[2] - q->v[0][2];
      double r0[3] = {r[0], r[1], r[2] - d};    /* projection on the (horizontal) plane of T_q */
      out[0] += wpo * I1 / (4.0 * OR_PI);
      for (int b = 0; b < 3; ++b) {
        double vb[3], t[3];
        sub3(r0, q->v[b], vb);
        for (int k = 0; k < 3; ++k) t[k] = Iv[k] + vb[k] * I1;
        for (int a = 0; a < 3; ++a) out[1 + 3 * a + b] += wpo * dot3(ra[a], t) / (4.0 * OR_PI);
      }
    }
    for (int j = 0; j < ni; ++j) {
      double rq[3];
      tri_point(q, bi + 3 * j, rq);
      double rho = hypot(r[0] - rq[0], r[1] - rq[1]);
      double complex G = green_eval(md, p->layer, q->layer, rho, near);
      double complex wG = wpo * wi[j] * q->area * G;
      out[0] += wG;
      double rb[3][3];
      for (int b = 0; b < 3; ++b) sub3(rq, q->v[b], rb[b]);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out[1 + 3 * a + b] += wG * dot3(ra[a], rb[b]);
    }
  }
}

/* ---------------------------------------------------------------- fill */
typedef struct {
  const or_grid* g;
  const int32_t* table;
  int M, F, mode, nthreads, tid;
  const double* freqs;
  double complex* Z;
  int T;
  const int32_t* tri_keys;     /* [T] */
  int32_t* key_to_tri;         /* key -> triangle index */
} fill_job;

static void key_parts(int32_t key, int* layer, int* x, int* y, int* half) {
  *half = key & 1;
  key >>= 1;
  *x = key % 128 - 4;
  key /= 128;
  *y = key % 128 - 4;
  *layer = key / 128;
}

static void* fill_worker(void* arg) {
  fill_job* J = (fill_job*)arg;
  const or_grid* g = J->g;
  int T = J->T, M = J->M;
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * T);
  for (int t = 0; t < T; ++t) {
    double v[3][3];
    int layer, x, y, half;
    or_triangle(g, J->tri_keys[t], v);
    key_parts(J->tri_keys[t], &layer, &x, &y, &half);
    tri_setup(&tris[t], v, layer);
  }
  /* pair-integral storage: direct mode keeps all T x T pairs; table mode keeps one entry per
   * (layer pair, orientation/half pair, lattice offset) */
  int W = (g->nx > g->ny ? g->nx : g->ny) + 5, NW = 2 * W + 1;
  size_t nslots = J->mode == 0 ? (size_t)T * T : (size_t)g->layers * g->layers * 16 * NW * NW;
  double complex* slot = (double complex*)malloc(sizeof(double complex) * 10 * nslots);
  unsigned char* have = (unsigned char*)malloc(nslots);
  int32_t* pair_slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)T * T);
  for (int p = 0; p < T; ++p) {
    int lp, xp, yp, hp;
    key_parts(J->tri_keys[p], &lp, &xp, &yp, &hp);
    for (int q = 0; q < T; ++q) {
      int lq, xq, yq, hq;
      key_parts(J->tri_keys[q], &lq, &xq, &yq, &hq);
      size_t s;
      if (J->mode == 0) s = (size_t)p * T + q;
      else {
        int op = (xp + yp) & 1, oq = (xq + yq) & 1;
        s = ((((((size_t)lp * g->layers + lq) * 2 + op) * 2 + hp) * 2 + oq) * 2 + hq) * NW * NW +
            (size_t)(xq - xp + W) * NW + (yq - yp + W);
      }
      pair_slot[(size_t)p * T + q] = (int32_t)s;
    }
  }
  for (int f = J->tid; f < J->F; f += J->nthreads) {
    medium_t md;
    medium_init(&md, g, J->freqs[f]);
    memset(have, 0, nslots);
    for (int p = 0; p < T; ++p) {
      for (int q = 0; q < T; ++q) {
        size_t s = (size_t)pair_slot[(size_t)p * T + q];
        if (have[s]) continue;
        pair_integrals(&md, &tris[p], &tris[q], slot + 10 * s);
        have[s] = 1;
      }
    }
    double complex jwmu = I * md.omega * MU0;
    double complex inv_jweps = 1.0 / (I * md.omega * md.eps);
    double complex* Zf = J->Z + (size_t)f * M * M;
    for (int m = 0; m < M; ++m) {
      const int32_t* rm = J->table + OR_BF_COLS * m;
      int tm[2] = {J->key_to_tri[rm[4]], J->key_to_tri[rm[5]]};
      int fm[2] = {rm[6], rm[7]};
      double em[3];
      /* edge length = distance between the two non-free vertices of T+ */
      sub3(tris[tm[0]].v[(fm[0] + 1) % 3], tris[tm[0]].v[(fm[0] + 2) % 3], em);
      double lm = norm3(em);
      for (int n = 0; n < M; ++n) {
        const int32_t* rn = J->table + OR_BF_COLS * n;
        int tn[2] = {J->key_to_tri[rn[4]], J->key_to_tri[rn[5]]};
        int fn[2] = {rn[6], rn[7]};
        double en[3];
        sub3(tris[tn[0]].v[(fn[0] + 1) % 3], tris[tn[0]].v[(fn[0] + 2) % 3], en);
        double ln = norm3(en);
        double complex z = 0.0;
        for (int s = 0; s < 2; ++s) {
          for (int t = 0; t < 2; ++t) {
            double sg = (s == t) ? 1.0 : -1.0;
            const tri_t* P = &tris[tm[s]];
            const tri_t* Q = &tris[tn[t]];
            const double complex* v = slot + 10 * (size_t)pair_slot[(size_t)tm[s] * T + tn[t]];
            double aa = P->area * Q->area;
            z += sg * lm * ln * (jwmu / (4.0 * aa) * v[1 + 3 * fm[s] + fn[t]] + inv_jweps / aa * v[0]);
          }
        }
        Zf[(size_t)m * M + n] = z;
      }
    }
  }
  free(tris);
  free(slot);
  free(have);
  free(pair_slot);
  return NULL;
}

double or_fill(const or_grid* g, const double* freqs, int F, int mode, int threads, double complex* Z) {
  int M = or_count_bfs(g);
  int32_t* table = (int32_t*)malloc(sizeof(int32_t) * OR_BF_COLS * M);
  or_bf_table(g, table);
  /* distinct triangles referenced by the BFs */
  int32_t* key_to_tri = (int32_t*)malloc(sizeof(int32_t) * (1 << 21));
  for (int i = 0; i < (1 << 21); ++i) key_to_tri[i] = -1;
  int32_t* keys = (int32_t*)malloc(sizeof(int32_t) * 2 * M);
  int T = 0;
  for (int m = 0; m < M; ++m) {
    for (int s = 0; s < 2; ++s) {
      int32_t k = table[OR_BF_COLS * m + 4 + s];
      if (key_to_tri[k] < 0) { key_to_tri[k] = T; keys[T++] = k; }
    }
  }
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
  fill_job* jobs = (fill_job*)malloc(sizeof(fill_job) * threads);
  for (int i = 0; i < threads; ++i) {
    fill_job j = {g, table, M, F, mode, threads, i, freqs, Z, T, keys, key_to_tri};
    jobs[i] = j;
    pthread_create(&th[i], NULL, fill_worker, &jobs[i]);
  }
  for (int i = 0; i < threads; ++i) pthread_join(th[i], NULL);
  /* reciprocity check, then symmetrise (Z <- (Z + Z^T) / 2) */
  double amax = 0.0, dmax = 0.0;
  for (int f = 0; f < F; ++f) {
    double complex* Zf = Z + (size_t)f * M * M;
    for (int m = 0; m < M; ++m) {
      for (int n = 0; n < M; ++n) {
        double a = cabs(Zf[(size_t)m * M + n]);
        if (a > amax) amax = a;
        if (n > m) {
          double d = cabs(Zf[(size_t)m * M + n] - Zf[(size_t)n * M + m]);
          if (d > dmax) dmax = d;
          double complex s = 0.5 * (Zf[(size_t)m * M + n] + Zf[(size_t)n * M + m]);
          Zf[(size_t)m * M + n] = s;
          Zf[(size_t)n * M + m] = s;
        }
      }
    }
  }
  free(th);
  free(jobs);
  free(keys);
  free(key_to_tri);
  free(table);
  return amax > 0.0 ? dmax / amax : 0.0;
}

/* Test hook: the ten integrals of one triangle pair (keys of the grid's lattice). */
void or_pair_integrals(const or_grid* g, double freq, int32_t kp, int32_t kq, double complex out[10]) {
  medium_t md;
  medium_init(&md, g, freq);
  double v[3][3];
  int layer, x, y, half;
  tri_t P, Q;
  or_triangle(g, kp, v);
  key_parts(kp, &layer, &x, &y, &half);
  tri_setup(&P, v, layer);
  or_triangle(g, kq, v);
  key_parts(kq, &layer, &x, &y, &half);
  tri_setup(&Q, v, layer);
  pair_integrals(&md, &P, &Q, out);
}
