/*
 * or_layered.c -- Green's functions of a grounded dielectric slab by Sommerfeld integrals.
 * TEST INFRASTRUCTURE ONLY.
 *
 * The paper's fill is FEKO's layered-media MPIE (Section II-D).  For a microstrip stack-up --
 * PEC ground at z = 0, a dielectric slab eps_1 = eps_r (1 - j tan d) up to z = d, a homogeneous
 * half-space eps_top above (air) -- the kernels of the mixed-potential form for horizontal
 * currents and their charges (formulation C of Michalski and Zheng, 1990) follow from the voltage
 * V(z|z') that a unit shunt current source at z' drives at z on the transmission line of each
 * polarisation (TE: Y = k_z / (w mu0); TM: Y = w eps0 eps_i / k_z; the line is shorted at z = 0
 * and matched by the half-space above d):
 *   vector potential, horizontal part    G_A~  = V_TE / (j w mu0)
 *   scalar potential (eps0 normalised)   G_phi~ = (j w eps0 / k_rho^2) (V_TM - V_TE)
 * and the spatial kernels are their Sommerfeld transforms
 *   G(rho) = (1 / 2 pi) int_0^inf G~(k_rho) J0(k_rho rho) k_rho dk_rho.
 * With these the interaction of Eq. (1) reads Z_mn = j w mu0 <f_m, G_A f_n>
 * + 1 / (j w eps0) <div f_m, G_phi div f_n>.  In a homogeneous medium eps above the ground both
 * reduce to the image form: G_A = g(R) - g(R_image), G_phi = (eps0 / eps) (g(R) - g(R_image)).
 *
 * Evaluation: the quasi-static part C e^{-j k1 R} / (4 pi R) (C = 1 for G_A; for G_phi 1 / eps_r
 * inside the slab and 2 / (eps_r + eps_top) when either point lies on the interface) is
 * subtracted in the spectral domain (its transform is C e^{-j k_z1 |z - z'|} / (2 j k_z1)) and
 * added back in closed form; the remainder is integrated along a half-ellipse in the first
 * quadrant from 0 to beyond every branch point and surface-wave pole (e^{+jwt}: they lie on or
 * below the real axis), then along the real axis: for rho > 0 in partitions between the zeros
 * of J0, summed with Wynn's epsilon algorithm; for rho = 0 through k_rho = k_a / u.
 */
#include <math.h>
#include <stdlib.h>

#include "pmom_oracle.h"

#define SL_PI 3.14159265358979323846
#define SL_C0 299792458.0
#define SL_MU0 (4.0e-7 * SL_PI)
#define SL_EPS0 (1.0 / (SL_MU0 * SL_C0 * SL_C0))

typedef struct {
  double omega, d;
  double complex k0t, k1;      /* wavenumbers of the top half-space and of the slab */
  double complex er1, ert;     /* relative permittivities (slab complex) */
  double ka, kb;               /* half-ellipse: from 0 to 2 ka, height kb */
} slab_t;

/* Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre recurrence). */
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(SL_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double z1 = z;
      z = z1 - p1 / pp;
      if (fabs(z - z1) < 1e-15) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

/* k_z = sqrt(k^2 - k_rho^2) on the branch Im k_z <= 0 (fields e^{-j k_z |z|} that decay) */
static double complex kz_of(double complex k, double complex kr) {
  double complex v = csqrt(k * k - kr * kr);
  if (cimag(v) > 0.0) v = -v;
  return v;
}

/* Transmission-line voltage at z for a unit shunt current at z' (0 < z, z' <= d), written with
 * q = j k_z1 (Re q >= 0) and e(x) = exp(-2 q x) so that no term overflows. */
static double complex tl_voltage(const slab_t* s, int te, double complex kr, double z, double zp) {
  double complex kz1 = kz_of(s->k1, kr), kz0 = kz_of(s->k0t, kr);
  double complex Y1, Y0;
  if (te) {
    Y1 = kz1 / (s->omega * SL_MU0);
    Y0 = kz0 / (s->omega * SL_MU0);
  } else {
    Y1 = s->omega * SL_EPS0 * s->er1 / kz1;
    Y0 = s->omega * SL_EPS0 * s->ert / kz0;
  }
  double complex q = I * kz1;
  double l = s->d - zp;
  double complex ez = cexp(-2.0 * q * zp), el = cexp(-2.0 * q * l);
  double complex coth_zp = (1.0 + ez) / (1.0 - ez);
  double complex t = (1.0 - el) / (1.0 + el);
  double complex Vs = 1.0 / (Y1 * coth_zp + Y1 * (Y0 + Y1 * t) / (Y1 + Y0 * t));
  if (z <= zp) {
    return Vs * cexp(q * (z - zp)) * (1.0 - cexp(-2.0 * q * z)) / (1.0 - ez);
  }
  double a = s->d - z, b = l;
  double complex r = Y0 / Y1, ea = cexp(-2.0 * q * a);
  return Vs * cexp(q * (a - b)) * ((1.0 + ea) + r * (1.0 - ea)) / ((1.0 + el) + r * (1.0 - el));
}

/* kind 0: G_phi~, kind 1: G_A~ (horizontal) */
static double complex spectral(const slab_t* s, int kind, double complex kr, double z, double zp) {
  double complex vte = tl_voltage(s, 1, kr, z, zp);
  if (kind == 1) return vte / (I * s->omega * SL_MU0);
  double complex vtm = tl_voltage(s, 0, kr, z, zp);
  return I * s->omega * SL_EPS0 / (kr * kr) * (vtm - vte);
}

static double quasi_static_c(const slab_t* s, int kind, double z, double zp) {
  if (kind == 1) return 1.0;
  if (z >= s->d || zp >= s->d) return 2.0 / creal(s->er1 + s->ert);
  return 1.0 / creal(s->er1);
}

static double complex asym_spectral(const slab_t* s, double c, double complex kr, double z, double zp) {
  double complex kz1 = kz_of(s->k1, kr);
  return c * cexp(-I * kz1 * fabs(z - zp)) / (2.0 * I * kz1);
}

/* J0 of a complex argument by its ascending series (|w| stays moderate on the half-ellipse) */
static double complex bessel_j0c(double complex w) {
  double complex q = -w * w / 4.0, t = 1.0, s = 1.0;
  for (int m = 1; m < 200; ++m) {
    t *= q / ((double)m * m);
    s += t;
    if (cabs(t) < 1e-18 * (1.0 + cabs(s)) && m > cabs(w)) break;
  }
  return s;
}

static double complex spec_remainder(const slab_t* s, int kind, double c, double complex kr, double z, double zp) {
  return spectral(s, kind, kr, z, zp) - asym_spectral(s, c, kr, z, zp);
}

/* Wynn's epsilon algorithm on the partial sums S[0..n-1] (n <= 64): eps_{-1} = 0, eps_0 = S,
 * eps_{k+1}[i] = eps_{k-1}[i+1] + 1 / (eps_k[i+1] - eps_k[i]); the even columns estimate the
 * limit, and the last entry of the last even column is returned. */
static double complex wynn(const double complex* S, int n) {
  double complex em1[65], e0[65], e1[65];
  if (n > 64) n = 64;
  for (int i = 0; i < n; ++i) { em1[i] = 0.0; e0[i] = S[i]; }
  double complex best = S[n - 1];
  int len = n;
  for (int k = 1; len > 1; ++k) {
    for (int i = 0; i + 1 < len; ++i) {
      double complex dd = e0[i + 1] - e0[i];
      if (cabs(dd) == 0.0) return best;   /* converged exactly */
      e1[i] = em1[i + 1] + 1.0 / dd;
    }
    --len;
    if (k % 2 == 0) best = e1[len - 1];
    for (int i = 0; i <= len; ++i) em1[i] = e0[i];
    for (int i = 0; i < len; ++i) e0[i] = e1[i];
  }
  return best;
}

/* (1 / 2 pi) int_0^inf R(k_rho) J0(k_rho rho) k_rho dk_rho of the remainder */
static double complex sommerfeld_remainder(const slab_t* s, int kind, double z, double zp, double rho) {
  double c = quasi_static_c(s, kind, z, zp);
  enum { NE = 96, NP = 24 };
  double xe[NE], we[NE], xp[NP], wp[NP];
  gauss_legendre(NE, xe, we);
  gauss_legendre(NP, xp, wp);
  double complex sum = 0.0;
  /* half-ellipse k(t) = ka (1 - cos t) + j kb sin t, split in four pieces */
  for (int piece = 0; piece < 4; ++piece) {
    double t0 = SL_PI * piece / 4.0, t1 = SL_PI * (piece + 1) / 4.0;
    for (int i = 0; i < NE; ++i) {
      double t = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * xe[i];
      double complex kr = s->ka * (1.0 - cos(t)) + I * s->kb * sin(t);
      double complex dk = (s->ka * sin(t) + I * s->kb * cos(t)) * 0.5 * (t1 - t0) * we[i];
      sum += spec_remainder(s, kind, c, kr, z, zp) * bessel_j0c(kr * rho) * kr * dk;
    }
  }
  double k_start = 2.0 * s->ka;
  /* graded panels from k_start (the scale of the branch points and poles the path has just
   * passed), widths growing by 1.5 and capped at half a period of J0, up to k_switch, past which
   * the remainder has settled into its smooth decay (scale: the slab thickness, or the height
   * difference when that is smaller) */
  double dz = fabs(z - zp), scale = (dz > 0.0 && dz < s->d) ? dz : s->d;
  double k_switch = 40.0 / scale;
  if (k_switch < 2.0 * k_start) k_switch = 2.0 * k_start;
  double width = rho > 0.0 ? SL_PI / rho : 1e300, w = 0.25 * k_start;
  for (double a = k_start; a < k_switch;) {
    double b = a + (w < width ? w : width);
    if (b > k_switch) b = k_switch;
    for (int i = 0; i < NP; ++i) {
      double kr = 0.5 * (a + b) + 0.5 * (b - a) * xp[i];
      sum += spec_remainder(s, kind, c, kr, z, zp) * j0(kr * rho) * kr * 0.5 * (b - a) * wp[i];
    }
    a = b;
    w *= 1.5;
  }
  if (rho <= 0.0) {
    /* tail k = k_switch / u, u in (0, 1]: the remainder falls off like k^-3 or faster */
    for (int piece = 0; piece < 8; ++piece) {
      double u0 = piece / 8.0, u1 = (piece + 1) / 8.0;
      for (int i = 0; i < NP; ++i) {
        double u = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * xp[i];
        double kr = k_switch / u;
        sum += spec_remainder(s, kind, c, kr, z, zp) * kr * (k_switch / (u * u)) * 0.5 * (u1 - u0) * wp[i];
      }
    }
  } else {
    /* tail: partitions between the large-argument zeros of J0, summed with Wynn's epsilon */
    double complex S[64];
    int nmax = 64;
    double complex acc = 0.0;
    int n0 = (int)ceil((k_switch * rho + SL_PI / 4.0) / SL_PI);
    double a = k_switch;
    for (int n = 0; n < 64; ++n) {
      double b = ((n0 + n) * SL_PI + SL_PI / 4.0) / rho;
      if (b <= a) b = a + SL_PI / rho;
      double complex part = 0.0;
      for (int i = 0; i < NP; ++i) {
        double kr = 0.5 * (a + b) + 0.5 * (b - a) * xp[i];
        part += spec_remainder(s, kind, c, kr, z, zp) * j0(kr * rho) * kr * 0.5 * (b - a) * wp[i];
      }
      acc += part;
      S[n] = acc;
      a = b;
      if (n >= 12 && cabs(part) < 1e-17 * cabs(acc)) { nmax = n + 1; break; }
    }
    sum += wynn(S, nmax < 40 ? nmax : 40);
  }
  return sum / (2.0 * SL_PI);
}

static void slab_init(slab_t* s, const or_grid* g, double freq, double er_top, double rho_max) {
  double d = g->layer_z[0];
  for (int l = 1; l < g->layers; ++l) if (g->layer_z[l] > d) d = g->layer_z[l];
  s->omega = 2.0 * SL_PI * freq;
  s->d = d;
  s->er1 = g->eps_r * (1.0 - I * g->tan_d);
  s->ert = er_top;
  double k0 = s->omega / SL_C0;
  s->k0t = k0 * csqrt(s->ert);
  s->k1 = k0 * csqrt(s->er1);
  double kmax = cabs(s->k1) > cabs(s->k0t) ? cabs(s->k1) : cabs(s->k0t);
  s->ka = 1.5 * kmax + k0;
  s->kb = 0.25 * kmax;
  if (rho_max > 0.0 && s->kb * rho_max > 1.0) s->kb = 1.0 / rho_max;
}

/* Layered kernel kind (0: G_phi, 1: G_A horizontal) between heights z, zp at lateral distance
 * rho; reg != 0 subtracts C / (4 pi R), C the quasi-static constant returned in *c_out. */
double complex or_slab_green(const or_grid* g, double freq, int kind, double z, double zp, double rho,
                             double er_top, int reg, double* c_out) {
  slab_t s;
  slab_init(&s, g, freq, er_top, rho > 0.0 ? 2.0 * rho : 0.0);
  double c = quasi_static_c(&s, kind, z, zp);
  double R = sqrt(rho * rho + (z - zp) * (z - zp));
  double complex direct;
  if (reg) {
    double complex x = -I * s.k1 * R;
    direct = cabs(x) < 1e-3 ? c * (-I * s.k1) * (1.0 + x / 2.0 + x * x / 6.0) / (4.0 * SL_PI)
                            : c * (cexp(x) - 1.0) / (4.0 * SL_PI * R);
  } else {
    direct = c * cexp(-I * s.k1 * R) / (4.0 * SL_PI * R);
  }
  if (c_out) *c_out = c;
  return direct + sommerfeld_remainder(&s, kind, z, zp, rho);
}

/* Table of the Sommerfeld remainder of kernel `kind` between heights z, zp at rho_i = i h,
 * i < n, for the fill: G = C e^{-j k1 R} / (4 pi R) + remainder(rho).  Returns C and k1. */
void or_slab_table(const or_grid* g, double freq, int kind, double z, double zp, double er_top, double h, int n,
                   double complex* out, double* c_out, double complex* k1_out) {
  slab_t s;
  slab_init(&s, g, freq, er_top, h * (n - 1));
  for (int i = 0; i < n; ++i) out[i] = sommerfeld_remainder(&s, kind, z, zp, h * i);
  *c_out = quasi_static_c(&s, kind, z, zp);
  *k1_out = s.k1;
}
