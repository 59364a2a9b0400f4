/*
 * or_fill.c -- oracle EFIE (MPIE) fill of the parent interaction matrix Z(f).  TEST INFRASTRUCTURE ONLY.
 *
 * Eq. (1)-(2) with RWG functions (Section II-B), Galerkin testing, e^{+jwt} convention:
 *   Z_mn = jw mu  <f_m, G_A f_n>  +  1/(jw eps) <div f_m, G_phi div' f_n>
 * with f = s (l / 2A) (r - v_free) and div f = s l / A on T+ (s = +1) and T- (s = -1).
 *
 * Green's function (the paper uses FEKO's layered-media MPIE, Section II-D; that code is not
 * available, so the stack-up is read as a homogeneous dielectric eps_r (1 - j tan d)).  PEC planes
 * image a horizontal current and a charge with the opposite sign and a vertical current with the
 * same sign, so G_phi and the horizontal components of the dyadic G_A are the Dirichlet function
 * G_D of the stack-up and its vertical component is the Neumann function G_N (for a homogeneous
 * medium between PEC planes this mixed-potential form is exact: dG_N/dz = -dG_D/dz'):
 *   microstrip: one PEC ground at z = 0, homogeneous medium of Hammerstad-Jensen eps_eff at
 *               w = pitch, one image:  G_D = g(R) - g(R_image),  G_N = g(R) + g(R_image)
 *   stripline : PEC planes at z = 0 and z = H, dielectric between them, in two exact representations:
 *                 image series  G = sum_n g(rho, z - z' + 2nH) -/+ g(rho, z + z' + 2nH)
 *                 mode series   G_D = 1/(pi H) sum_{m>=1} sin(m pi z/H) sin(m pi z'/H) K0(gamma_m rho)
 *                               G_N = 1/(2 pi H) sum_{m>=0} e_m cos(m pi z/H) cos(m pi z'/H) K0(gamma_m rho)
 *                               gamma_m = sqrt((m pi/H)^2 - k^2), e_0 = 1, e_m = 2
 *               For rho >= H/2 the mode series is summed to round-off.  For rho < H/2 the image
 *               terms |n| <= K are summed explicitly and the remaining images, which are smooth
 *               and even in rho, are represented by c0 + c1 rho^2 + c2 rho^4 matched to the mode
 *               series at rho = H/2, 3H/4, H, separately for every pair of heights (z, z') that
 *               the quadrature visits (metal layers, and the points of vertical via triangles).
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
  if (g->medium == 1) return g->eps_r;
  /* Hammerstad & Jensen (1980) effective permittivity of a strip of width w = pitch at height h */
  double h = g->layer_z[0];
  for (int l = 1; l < g->layers; ++l) if (g->layer_z[l] > h) h = g->layer_z[l];
  double u = g->pitch / h, er = g->eps_r;
  double a = 1.0 + log((pow(u, 4) + pow(u / 52.0, 2)) / (pow(u, 4) + 0.432)) / 49.0 + log(1.0 + pow(u / 18.1, 3)) / 18.7;
  double b = 0.564 * pow((er - 0.9) / (er + 3.0), 0.053);
  return 0.5 * (er + 1.0) + 0.5 * (er - 1.0) * pow(1.0 + 10.0 / u, -a * b);
}

/* K0(w) for any Re w >= 0, in particular near the imaginary axis (the TEM term of the Neumann mode
 * series, where the fixed-step trapezoidal rule above is inaccurate):
 *   |w| > 17                 Hankel's asymptotic expansion (Abramowitz & Stegun 9.7.2);
 *   Re w <= |w| / 10         the ascending series -(ln(w/2) + gamma_E) I0(w) + sum_k (w^2/4)^k / (k!)^2 H_k
 *                            (A&S 9.6.13), whose cancellation stays below e^{1.1 |w|};
 *   otherwise                the trapezoidal rule on int_0^inf exp(-w cosh t) dt with a step
 *                            h = 2 pi d / 40, d = pi/2 - |arg w| the half-width of the strip in
 *                            which the integrand stays bounded (error ~ e^{-2 pi d / h}). */
double complex or_bessel_k0_any(double complex w) {
  double aw = cabs(w);
  if (aw > 17.0) {
    double complex a = 1.0, sum = 1.0;
    for (int k = 1; k < 60; ++k) {
      double complex na = a * (-(2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k * w);
      if (cabs(na) >= cabs(a)) break;
      a = na;
      sum += a;
      if (cabs(a) < 1e-17) break;
    }
    return csqrt(OR_PI / (2.0 * w)) * cexp(-w) * sum;
  }
  if (creal(w) <= 0.1 * aw) {
    double complex q = w * w / 4.0, t = 1.0, I0 = 1.0, S = 0.0;
    double Hk = 0.0;
    for (int k = 1; k < 400; ++k) {
      t *= q / ((double)k * (double)k);
      Hk += 1.0 / k;
      I0 += t;
      S += t * Hk;
      if (k > aw && cabs(t) * (Hk + 1.0) < 1e-18) break;
    }
    return -(clog(w / 2.0) + 0.57721566490153286061) * I0 + S;
  }
  double d = 0.5 * OR_PI - fabs(carg(w));
  double h = 2.0 * OR_PI * d / 40.0;
  if (h > 0.2) h = 0.2;
  if (h > 0.6 / sqrt(aw)) h = 0.6 / sqrt(aw);
  double complex s = 0.5 * cexp(-w);
  for (int j = 1; j < 200000; ++j) {
    double c = cosh(j * h);
    if (creal(w) * (c - 1.0) > 40.0) break;
    s += cexp(-w * c);
  }
  return h * s;
}

/* Kernel kinds: 0 = Dirichlet G_D (horizontal currents, charges), 1 = Neumann G_N (vertical currents). */
typedef struct {
  const or_grid* g;
  double omega, H, rho_s;
  double complex k, eps;
  int nz;                 /* distinct heights: the metal layers first (id = layer), then via points */
  const double* z;
  double complex* fit;    /* stripline: [kind][nz][nz][3] tail coefficients */
  /* layered microstrip (medium 2): Sommerfeld remainders of G_phi (0) and G_A (1) per pair of
   * heights on rho_i = i htab, their quasi-static constants, the slab wavenumber (md->k) */
  int layered, ntab;
  double htab;
  double complex* tab;    /* [2][nz][nz][ntab] */
  double* ctab;           /* [2][nz][nz] */
} medium_t;

static double complex gfree(double complex k, double R) { return cexp(-I * k * R) / (4.0 * OR_PI * R); }

/* (exp(-jkR) - 1) / (4 pi R), finite at R = 0 */
static double complex gfree_reg(double complex k, double R) {
  double complex x = -I * k * R;
  if (cabs(x) < 1e-3) return (-I * k) * (1.0 + x / 2.0 + x * x / 6.0 + x * x * x / 24.0) / (4.0 * OR_PI);
  return (cexp(x) - 1.0) / (4.0 * OR_PI * R);
}

static double complex strip_images(const medium_t* md, int kind, double zp, double zq, double rho, int K, int reg) {
  double H = md->H, r2 = rho * rho, sg2 = kind == 0 ? -1.0 : 1.0;
  double complex s = 0.0;
  for (int a = 0; a <= K; ++a) {
    for (int sg = (a == 0 ? 1 : -1); sg <= 1; sg += 2) {
      int n = a * sg;
      double zp_ = (zp - zq) + 2.0 * n * H, zm_ = (zp + zq) + 2.0 * n * H;
      double Rp = sqrt(r2 + zp_ * zp_), Rm = sqrt(r2 + zm_ * zm_);
      if (n == 0 && reg) s += gfree_reg(md->k, Rp);
      else s += gfree(md->k, Rp);
      s += sg2 * gfree(md->k, Rm);
    }
  }
  return s;
}

static double complex strip_modal(const medium_t* md, int kind, double zp, double zq, double rho) {
  double H = md->H;
  double complex s = 0.0;
  if (kind == 1) s = 0.5 * or_bessel_k0_any(csqrt(-md->k * md->k) * rho);   /* m = 0 (TEM), e_0 / 2 */
  for (int m = 1; m < 4000; ++m) {
    double km = m * OR_PI / H;
    double complex gam = csqrt(km * km - md->k * md->k);
    if (creal(gam) * rho > 40.0) break;
    double w = kind == 0 ? sin(km * zp) * sin(km * zq) : cos(km * zp) * cos(km * zq);
    s += w * or_bessel_k0(gam * rho);
  }
  return s / (OR_PI * H);
}

static void medium_init(medium_t* md, const or_grid* g, double freq, int nz, const double* z) {
  md->g = g;
  md->omega = 2.0 * OR_PI * freq;
  md->layered = g->medium == 2;
  md->tab = NULL;
  md->ctab = NULL;
  if (md->layered) {
    /* the slab's permittivity enters through the kernels; the scalar term is eps0-normalised */
    md->eps = EPS0;
  } else {
    double er = or_eps_eff(g);
    md->eps = EPS0 * er * (1.0 - I * g->tan_d);
  }
  md->k = md->omega * csqrt(MU0 * md->eps);
  md->H = g->h_total;
  md->rho_s = 0.5 * g->h_total;
  md->nz = nz;
  md->z = z;
  md->fit = NULL;
  if (md->layered && nz > 0) {
    double d = z[0];
    for (int i = 1; i < nz; ++i) if (z[i] > d) d = z[i];
    double rho_max = g->pitch * sqrt((g->nx + 6.0) * (g->nx + 6.0) + (g->ny + 6.0) * (g->ny + 6.0));
    md->htab = d / 16.0;
    md->ntab = (int)ceil(rho_max / md->htab) + 4;
    md->tab = (double complex*)malloc(sizeof(double complex) * 2 * nz * nz * md->ntab);
    md->ctab = (double*)malloc(sizeof(double) * 2 * nz * nz);
    for (int kind = 0; kind < 2; ++kind)
      for (int p = 0; p < nz; ++p)
        for (int q = p; q < nz; ++q) {
          double complex* t = md->tab + ((size_t)(kind * nz + p) * nz + q) * md->ntab;
          double c;
          double complex k1;
          or_slab_table(g, freq, kind, z[p], z[q], 1.0, md->htab, md->ntab, t, &c, &k1);
          md->ctab[(kind * nz + p) * nz + q] = md->ctab[(kind * nz + q) * nz + p] = c;
          md->k = k1;
          if (q != p)   /* reciprocity */
            memcpy(md->tab + ((size_t)(kind * nz + q) * nz + p) * md->ntab, t, sizeof(double complex) * md->ntab);
        }
  }
  if (g->medium == 1) {
    md->fit = (double complex*)malloc(sizeof(double complex) * 2 * nz * nz * 3);
    for (int kind = 0; kind < 2; ++kind) {
      for (int p = 0; p < nz; ++p) {
        for (int q = 0; q < nz; ++q) {
          double complex* c = md->fit + ((size_t)(kind * nz + p) * nz + q) * 3;
          if (q < p) {   /* both kernels are symmetric in (z, z') */
            const double complex* t = md->fit + ((size_t)(kind * nz + q) * nz + p) * 3;
            c[0] = t[0]; c[1] = t[1]; c[2] = t[2];
            continue;
          }
          double x[3];
          double complex y[3];
          for (int i = 0; i < 3; ++i) {
            double rho = md->rho_s * (1.0 + 0.5 * i);
            x[i] = rho * rho;
            y[i] = strip_modal(md, kind, z[p], z[q], rho) - strip_images(md, kind, z[p], z[q], rho, IMG_K, 0);
          }
          /* quadratic in x = rho^2 through the three points (Newton divided differences) */
          double complex d01 = (y[1] - y[0]) / (x[1] - x[0]);
          double complex d12 = (y[2] - y[1]) / (x[2] - x[1]);
          double complex d012 = (d12 - d01) / (x[2] - x[0]);
          c[2] = d012;
          c[1] = d01 - d012 * (x[0] + x[1]);
          c[0] = y[0] - d01 * x[0] + d012 * x[0] * x[1];
        }
      }
    }
  }
}

static void medium_free(medium_t* md) {
  free(md->fit);
  free(md->tab);
  free(md->ctab);
  md->fit = NULL;
  md->tab = NULL;
  md->ctab = NULL;
}

/* Cubic Lagrange interpolation of a table on rho_i = i h. */
static double complex table_interp(const double complex* t, int n, double h, double rho) {
  double x = rho / h;
  int i = (int)floor(x);
  int j0 = i - 1;
  if (j0 < 0) j0 = 0;
  if (j0 > n - 4) j0 = n - 4;
  double u = x - j0;
  double l0 = -(u - 1) * (u - 2) * (u - 3) / 6.0, l1 = u * (u - 2) * (u - 3) / 2.0;
  double l2 = -u * (u - 1) * (u - 3) / 2.0, l3 = u * (u - 1) * (u - 2) / 6.0;
  return l0 * t[j0] + l1 * t[j0 + 1] + l2 * t[j0 + 2] + l3 * t[j0 + 3];
}

/* G (reg = 0) or G - 1/(4 pi R_direct) (reg = 1) of kernel `kind` between heights z[ip], z[iq] at
 * lateral distance rho. */
static double complex green_eval(const medium_t* md, int kind, int ip, int iq, double rho, int reg) {
  const or_grid* g = md->g;
  double zp = md->z[ip], zq = md->z[iq];
  if (md->layered) {   /* kind 0: G_phi, 2: G_A (horizontal) */
    int tk = kind == 2 ? 1 : 0;
    double c = md->ctab[(tk * md->nz + ip) * md->nz + iq];
    double R = sqrt(rho * rho + (zp - zq) * (zp - zq));
    double complex direct = reg ? c * gfree_reg(md->k, R) : c * gfree(md->k, R);
    return direct + table_interp(md->tab + ((size_t)(tk * md->nz + ip) * md->nz + iq) * md->ntab, md->ntab, md->htab, rho);
  }
  if (g->medium == 0) {
    double Rd = sqrt(rho * rho + (zp - zq) * (zp - zq)), Ri = sqrt(rho * rho + (zp + zq) * (zp + zq));
    double complex gi = gfree(md->k, Ri);
    return (reg ? gfree_reg(md->k, Rd) : gfree(md->k, Rd)) + (kind == 0 ? -gi : gi);
  }
  if (rho >= md->rho_s) {
    double complex G = strip_modal(md, kind, zp, zq, rho);
    if (reg) G -= 1.0 / (4.0 * OR_PI * sqrt(rho * rho + (zp - zq) * (zp - zq)));
    return G;
  }
  const double complex* c = md->fit + ((size_t)(kind * md->nz + ip) * md->nz + iq) * 3;
  double x = rho * rho;
  return strip_images(md, kind, zp, zq, rho, IMG_K, reg) + c[0] + x * (c[1] + x * c[2]);
}

double complex or_green(const or_grid* g, double freq, int lp, int lq, double rho) {
  medium_t md;
  medium_init(&md, g, freq, g->layers, g->layer_z);
  double complex G = green_eval(&md, 0, lp, lq, rho, 0);
  medium_free(&md);
  return G;
}

double complex or_green_images(const or_grid* g, double freq, int lp, int lq, double rho, int K) {
  medium_t md;
  medium_init(&md, g, freq, 0, NULL);
  double complex G = strip_images(&md, 0, g->layer_z[lp], g->layer_z[lq], rho, K, 0);
  medium_free(&md);
  return G;
}

double complex or_green_modal(const or_grid* g, double freq, int lp, int lq, double rho) {
  medium_t md;
  medium_init(&md, g, freq, 0, NULL);
  double complex G = strip_modal(&md, 0, g->layer_z[lp], g->layer_z[lq], rho);
  medium_free(&md);
  return G;
}

double complex or_green_heights(const or_grid* g, double freq, int kind, double zp, double zq, double rho,
                                int route, int K) {
  double z[2] = {zp, zq};
  medium_t md;
  medium_init(&md, g, freq, route == 0 ? 2 : 0, z);
  double complex G;
  if (route == 1) G = strip_images(&md, kind, zp, zq, rho, K, 0);
  else if (route == 2) G = strip_modal(&md, kind, zp, zq, rho);
  else G = green_eval(&md, kind, 0, 1, rho, 0);
  medium_free(&md);
  return G;
}

/* ---------------------------------------------------------------- triangle-pair integrals */
typedef struct {
  double v[3][3];
  double c[3];
  double n[3];            /* unit normal */
  double area, lmax;
  int layer, vert;        /* vert: a vertical (via) triangle */
  int zid[2][13];         /* height id of every point of the 7-point (0) and 13-point (1) rule */
} tri_t;

static void tri_setup(tri_t* t, const double v[3][3], int layer) {
  memcpy(t->v, v, sizeof(t->v));
  double e1[3], e2[3], n[3];
  sub3(v[1], v[0], e1);
  sub3(v[2], v[0], e2);
  cross3(e1, e2, n);
  double nn = norm3(n);
  t->area = 0.5 * nn;
  for (int i = 0; i < 3; ++i) t->n[i] = n[i] / nn;
  t->lmax = 0.0;
  for (int i = 0; i < 3; ++i) {
    double e[3];
    sub3(v[(i + 1) % 3], v[i], e);
    double l = norm3(e);
    if (l > t->lmax) t->lmax = l;
    t->c[i] = (v[0][i] + v[1][i] + v[2][i]) / 3.0;
  }
  t->layer = layer;
  t->vert = !(v[0][2] == v[1][2] && v[0][2] == v[2][2]);
  for (int r = 0; r < 2; ++r)
    for (int i = 0; i < 13; ++i) t->zid[r][i] = layer;
}

/* Height of a quadrature point: exactly the layer height on a horizontal triangle. */
static double point_z(const tri_t* t, const double* b) {
  if (!t->vert) return t->v[0][2];
  return t->v[0][2] + b[1] * (t->v[1][2] - t->v[0][2]) + b[2] * (t->v[2][2] - t->v[0][2]);
}

static void tri_point(const tri_t* t, const double* b, double* r) {
  for (int k = 0; k < 2; ++k) r[k] = b[0] * t->v[0][k] + b[1] * t->v[1][k] + b[2] * t->v[2][k];
  r[2] = point_z(t, b);
}

/* Height ids of the quadrature points of vertical triangles: the distinct heights are appended to
 * `z` (which starts with the layer heights) in ascending order, so that the id order of any two
 * heights, and with it every fitted tail, does not depend on which triangles are present; returns
 * the new count. */
static int assign_heights(tri_t* tris, int T, double* z, int nz) {
  int n0 = nz;
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = 0; t < T; ++t) {
      if (!tris[t].vert) continue;
      for (int r = 0; r < 2; ++r) {
        const double *b, *w;
        int n = or_tri_rule(r == 0 ? 7 : 13, &b, &w);
        for (int i = 0; i < n; ++i) {
          double zz = point_z(&tris[t], b + 3 * i);
          int id = -1;
          for (int j = 0; j < nz; ++j) if (z[j] == zz) { id = j; break; }
          if (pass == 0) {
            if (id < 0) z[nz++] = zz;
          } else {
            tris[t].zid[r][i] = id;
          }
        }
      }
    }
    if (pass == 0) {   /* sort the appended heights (insertion sort: a few dozen values) */
      for (int i = n0 + 1; i < nz; ++i) {
        double v = z[i];
        int j = i - 1;
        while (j >= n0 && z[j] > v) { z[j + 1] = z[j]; --j; }
        z[j + 1] = v;
      }
    }
  }
  return nz;
}

/* out[0] = int int G_D ; out[1 + 3a + b] = int int (r - v_a) . G_A (r' - v_b), where G_A acts with
 * G_D on the horizontal and G_N on the vertical components, over T_p x T_q */
static void pair_integrals(const medium_t* md, const tri_t* p, const tri_t* q, double complex out[10]) {
  for (int i = 0; i < 10; ++i) out[i] = 0.0;
  double dc[3];
  sub3(p->c, q->c, dc);
  double lm = p->lmax > q->lmax ? p->lmax : q->lmax;
  /* lattice geometry puts many pairs exactly on the threshold: resolve ties as "near" */
  int near = norm3(dc) < 2.0 * lm * (1.0 + 1e-9);
  int both_vert = p->vert && q->vert;
  const double *bo, *wo, *bi, *wi;
  int no = or_tri_rule(near ? 13 : 7, &bo, &wo);
  int ni = or_tri_rule(near ? 13 : 7, &bi, &wi);
  for (int i = 0; i < no; ++i) {
    double r[3], ra[3][3];
    tri_point(p, bo + 3 * i, r);
    for (int a = 0; a < 3; ++a) sub3(r, p->v[a], ra[a]);
    double wpo = wo[i] * p->area;
    int izp = p->zid[near][i];
    if (near) {
      /* the subtracted 1 / (4 pi R) carries each kernel's quasi-static constant (1 but in a
       * layered medium, where G_phi and G_A have their own) */
      double cphi = 1.0, cA = 1.0;
      if (md->layered) {
        int izq0 = q->zid[1][0];
        cphi = md->ctab[(0 * md->nz + izp) * md->nz + izq0];
        cA = md->ctab[(1 * md->nz + izp) * md->nz + izq0];
      }
      double I1, Iv[3], rv[3];
      or_tri_potentials(q->v, r, &I1, Iv);
      sub3(r, q->v[0], rv);
      double d = dot3(q->n, rv);
      double r0[3] = {r[0] - d * q->n[0], r[1] - d * q->n[1], r[2] - d * q->n[2]};   /* projection on T_q's plane */
      out[0] += cphi * wpo * I1 / (4.0 * OR_PI);
      for (int b = 0; b < 3; ++b) {
        double vb[3], t[3];
        sub3(r0, q->v[b], vb);
        for (int k = 0; k < 3; ++k) t[k] = Iv[k] + vb[k] * I1;
        for (int a = 0; a < 3; ++a) out[1 + 3 * a + b] += cA * wpo * dot3(ra[a], t) / (4.0 * OR_PI);
      }
    }
    for (int j = 0; j < ni; ++j) {
      double rq[3];
      tri_point(q, bi + 3 * j, rq);
      int izq = q->zid[near][j];
      double rho = hypot(r[0] - rq[0], r[1] - rq[1]);
      double complex GD = green_eval(md, 0, izp, izq, rho, near);
      /* horizontal vector part: the same kernel in a homogeneous medium, G_A in a layered one */
      double complex GA = md->layered ? green_eval(md, 2, izp, izq, rho, near) : GD;
      double complex GN = both_vert ? green_eval(md, 1, izp, izq, rho, near) : 0.0;
      double complex w = wpo * wi[j] * q->area;
      out[0] += w * GD;
      double rb[3][3];
      for (int b = 0; b < 3; ++b) sub3(rq, q->v[b], rb[b]);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double dh = ra[a][0] * rb[b][0] + ra[a][1] * rb[b][1], dz = ra[a][2] * rb[b][2];
          out[1 + 3 * a + b] += w * (dh * GA + (both_vert ? dz * GN : 0.0));
        }
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
  const tri_t* tris;           /* [T], with height ids */
  int nz;
  const double* z;             /* [nz] heights */
} fill_job;


static void* fill_worker(void* arg) {
  fill_job* J = (fill_job*)arg;
  const or_grid* g = J->g;
  int T = J->T, M = J->M;
  const tri_t* tris = J->tris;
  /* pair-integral storage: direct mode keeps all T x T pairs; table mode keeps one entry per
   * (layer pair, orientation/triangle pair, lattice offset) */
  int sub = g->sub > 1 ? g->sub : 1;
  int W = ((g->nx > g->ny ? g->nx : g->ny) + 5) * sub, NW = 2 * W + 1;
  size_t nslots = J->mode == 0 ? (size_t)T * T : (size_t)g->layers * g->layers * 64 * NW * NW;
  double complex* slot = (double complex*)malloc(sizeof(double complex) * 10 * nslots);
  unsigned char* have = (unsigned char*)malloc(nslots);
  int32_t* pair_slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)T * T);
  for (int p = 0; p < T; ++p) {
    int lp, xp, yp, hp;
    or_key_parts(g, J->tri_keys[p], &lp, &xp, &yp, &hp);
    for (int q = 0; q < T; ++q) {
      int lq, xq, yq, hq;
      or_key_parts(g, J->tri_keys[q], &lq, &xq, &yq, &hq);
      size_t s;
      if (J->mode == 0) s = (size_t)p * T + q;
      else {
        int op = or_orient(g, xp, yp), oq = or_orient(g, xq, yq);
        s = ((((((size_t)lp * g->layers + lq) * 2 + op) * 4 + hp) * 2 + oq) * 4 + hq) * NW * NW +
            (size_t)(xq - xp + W) * NW + (yq - yp + W);
      }
      pair_slot[(size_t)p * T + q] = (int32_t)s;
    }
  }
  for (int f = J->tid; f < J->F; f += J->nthreads) {
    medium_t md;
    medium_init(&md, g, J->freqs[f], J->nz, J->z);
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
    medium_free(&md);
  }
  free(slot);
  free(have);
  free(pair_slot);
  return NULL;
}

/* Distinct triangles of the grid's BFs with their geometry and height ids; returns T. */
static int collect_triangles(const or_grid* g, const int32_t* table, int M, int32_t* key_to_tri, int32_t* keys,
                             tri_t** tris_out, double** z_out, int* nz_out) {
  int T = 0;
  for (int m = 0; m < M; ++m) {
    for (int s = 0; s < 2; ++s) {
      int32_t k = table[OR_BF_COLS * m + 4 + s];
      if (key_to_tri[k] < 0) { key_to_tri[k] = T; keys[T++] = k; }
    }
  }
  tri_t* tris = (tri_t*)malloc(sizeof(tri_t) * T);
  for (int t = 0; t < T; ++t) {
    double v[3][3];
    int layer, x, y, half;
    or_triangle(g, keys[t], v);
    or_key_parts(g, keys[t], &layer, &x, &y, &half);
    tri_setup(&tris[t], v, layer);
  }
  double* z = (double*)malloc(sizeof(double) * (g->layers + 40 * T + 1));
  for (int l = 0; l < g->layers; ++l) z[l] = g->layer_z[l];
  *nz_out = assign_heights(tris, T, z, g->layers);
  *tris_out = tris;
  *z_out = z;
  return T;
}

/* Z of the BFs listed in `table` (M rows): the parent's, or a sub-structure's. */
static double fill_table(const or_grid* g, const int32_t* table, int M, const double* freqs, int F, int mode,
                         int threads, double complex* Z) {
  /* distinct triangles referenced by the BFs */
  int32_t kmax = 0;
  for (int m = 0; m < M; ++m)
    for (int s = 0; s < 2; ++s) if (table[OR_BF_COLS * m + 4 + s] > kmax) kmax = table[OR_BF_COLS * m + 4 + s];
  int32_t* key_to_tri = (int32_t*)malloc(sizeof(int32_t) * ((size_t)kmax + 1));
  for (int32_t i = 0; i <= kmax; ++i) key_to_tri[i] = -1;
  int32_t* keys = (int32_t*)malloc(sizeof(int32_t) * 2 * M);
  tri_t* tris;
  double* z;
  int nz;
  int T = collect_triangles(g, table, M, key_to_tri, keys, &tris, &z, &nz);
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
  fill_job* jobs = (fill_job*)malloc(sizeof(fill_job) * threads);
  for (int i = 0; i < threads; ++i) {
    fill_job j = {g, table, M, F, mode, threads, i, freqs, Z, T, keys, key_to_tri, tris, nz, z};
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
  free(tris);
  free(z);
  return amax > 0.0 ? dmax / amax : 0.0;
}

double or_fill(const or_grid* g, const double* freqs, int F, int mode, int threads, double complex* Z) {
  int M = or_count_bfs(g);
  int32_t* table = (int32_t*)malloc(sizeof(int32_t) * OR_BF_COLS * M);
  or_bf_table(g, table);
  double asym = fill_table(g, table, M, freqs, F, mode, threads, Z);
  free(table);
  return asym;
}

double or_fill_subset(const or_grid* g, const double* freqs, int F, int mode, int threads, const int32_t* bf, int N,
                      double complex* Z) {
  int M = or_count_bfs(g);
  int32_t* table = (int32_t*)malloc(sizeof(int32_t) * OR_BF_COLS * M);
  or_bf_table(g, table);
  int32_t* sub = (int32_t*)malloc(sizeof(int32_t) * OR_BF_COLS * (N > 0 ? N : 1));
  for (int a = 0; a < N; ++a) memcpy(sub + OR_BF_COLS * a, table + OR_BF_COLS * bf[a], sizeof(int32_t) * OR_BF_COLS);
  double asym = fill_table(g, sub, N, freqs, F, mode, threads, Z);
  free(sub);
  free(table);
  return asym;
}

/* Test hook: the ten integrals of one triangle pair (keys of the grid's lattice). */
void or_pair_integrals(const or_grid* g, double freq, int32_t kp, int32_t kq, double complex out[10]) {
  int32_t keys[2] = {kp, kq};
  tri_t tr[2];
  for (int i = 0; i < 2; ++i) {
    double v[3][3];
    int layer, x, y, half;
    or_triangle(g, keys[i], v);
    or_key_parts(g, keys[i], &layer, &x, &y, &half);
    tri_setup(&tr[i], v, layer);
  }
  double* z = (double*)malloc(sizeof(double) * (g->layers + 80));
  for (int l = 0; l < g->layers; ++l) z[l] = g->layer_z[l];
  int nz = assign_heights(tr, 2, z, g->layers);
  medium_t md;
  medium_init(&md, g, freq, nz, z);
  pair_integrals(&md, &tr[0], &tr[1], out);
  medium_free(&md);
  free(z);
}
