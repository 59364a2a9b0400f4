// GPU fill of the parent interaction matrix Z(f) (paper Phase 2, Eq. 1-2, RWG basis).
//
// Galerkin MPIE, e^{+jwt}:  Z_mn = jw mu0 <f_m, G f_n> + <div f_m, G div f_n> / (jw eps),
// eps = eps0 eps_r (1 - j tan d) (microstrip: Hammerstad-Jensen eps_eff of a strip w = pitch).
// Green's functions of the homogeneous stack-up.  The ground planes mirror horizontal currents and
// charges with a sign change and vertical (via) currents without one, so the scalar potential and
// the horizontal part of the vector potential use the Dirichlet function G_D and the vertical part
// the Neumann function G_N (exact mixed-potential form for a homogeneous medium between PEC planes):
//   microstrip  G_D = g(R) - g(R'), G_N = g(R) + g(R'), R' to the image below the ground z = 0
//   stripline   plates z = 0, H: for lateral distance rho >= H/2 the waveguide-mode sums
//               G_D = (1/(pi H)) sum_{m>=1} sin(m pi z/H) sin(m pi z'/H) K0(gamma_m rho),
//               G_N = (1/(2 pi H)) [K0(gamma_0 rho) + 2 sum_{m>=1} cos(m pi z/H) cos(m pi z'/H) K0(gamma_m rho)];
//               below H/2 the images with |n| <= 16 plus a quadratic in rho^2 matched to the mode
//               sum at rho = H/2, 3H/4, H (the remaining images are smooth and even in rho), one
//               quadratic per kernel and pair of heights: the metal layers and the heights of the
//               quadrature points on vertical via triangles.
//   grounded slab (medium 2: PEC ground at z = 0, dielectric eps_r (1 - j tan d) up to the highest
//               metal layer d, air above): the mixed-potential kernels of the layered medium for
//               horizontal currents, G_A = S0{V_TE / (jw mu0)} and G_phi = S0{(jw eps0 / k_rho^2)
//               (V_TM - V_TE)} (V the voltages of the TE and TM transmission lines of the stack-up,
//               S0 the Sommerfeld transform), each the quasi-static term C e^{-jk1 R}/(4 pi R) plus a
//               remainder tabulated on rho = i h, h = d/16, per frequency and pair of heights (cubic
//               interpolation); the scalar term is eps0-normalised and the analytic singular
//               integrals carry each kernel's C (1 for G_A; 1/eps_r in the slab, 2/(eps_r + 1) on
//               its surface for G_phi).  The remainder integral runs along a half-ellipse in the
//               first quadrant past the branch points and surface-wave poles, then over graded
//               panels of the real axis and, for rho > 0, over partitions between the zeros of J0
//               summed with Wynn's epsilon algorithm; one thread per table entry.
// Triangle pairs related by a lattice translation (same layers, orientations, halves and
// offset) share one integration: one thread integrates one such class at one frequency
// (7-point rule x 7-point rule when the centroids are at least two longest edges apart; else
// 13 x 13 with the 1/(4 pi R) part of the direct term integrated analytically over the source
// triangle).  A second kernel assembles Z_mn from the class table and stores (Z_mn + Z_nm)/2.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "pmom_internal.h"

namespace pmom {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 4.0e-7 * kPi;
constexpr int kImages = 16;
constexpr int kMaxLayers = 8;

struct FillTri {
  double v[3][3];
  double c[3];
  double n[3];          // unit normal
  double area, lmax;
  int layer, vert;      // vert: a vertical via triangle
  int16_t zid[2][13];   // height id of each point of the 7-point (0) and 13-point (1) rule
};

struct Medium {
  double omega, H, rho_s;
  double2 k;       // complex wavenumber (the slab's for the layered medium)
  double2 eps;     // complex permittivity (eps0 for the layered medium: the kernels carry the slab)
  int stripline;
  int layered;     // grounded slab: tabulated Sommerfeld kernels
  int nz;          // distinct heights (metal layers first, id = layer)
  int ntab;        // layered: table points on rho = i htab
  double htab;
};

// Grounded slab of one frequency (layered medium): slab thickness d, wavenumbers and relative
// permittivities of the slab (1) and the half-space above (t), and the half-ellipse of the
// Sommerfeld path (0 to 2 ka, height kb).
struct Slab {
  double omega, d;
  double2 k0t, k1, er1, ert;
  double ka, kb;
};
constexpr int kGlE = 96;   // Gauss-Legendre points per quarter of the half-ellipse
constexpr int kGlP = 24;   // per real-axis panel
__constant__ double kGlE_x[kGlE], kGlE_w[kGlE], kGlP_x[kGlP], kGlP_w[kGlP];

// ------------------------------------------------------------------ complex double helpers
__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 ca(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cexp_(double2 a) {
  double s, c;
  sincos(a.y, &s, &c);
  const double e = exp(a.x);
  return make_double2(e * c, e * s);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// principal square root; the part that would cancel (r - |a.x| when |a.y| << |a.x|) is formed
// from the other one, so nearly real arguments never take sqrt of a rounded-negative number
__device__ __forceinline__ double2 csqrt_(double2 a) {
  const double r = hypot(a.x, a.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  if (a.x >= 0.0) {
    const double re = sqrt(0.5 * (r + a.x));
    return make_double2(re, a.y / (2.0 * re));
  }
  double im = sqrt(0.5 * (r - a.x));
  if (a.y < 0.0) im = -im;
  return make_double2(a.y / (2.0 * im), im);
}

// exp(-j k R) / (4 pi R)
__device__ __forceinline__ double2 g_free(double2 k, double R) {
  // -j k R = (k.y R) + j(-k.x R)
  return cscale(cexp_(make_double2(k.y * R, -k.x * R)), 1.0 / (4.0 * kPi * R));
}
// (exp(-j k R) - 1) / (4 pi R), finite as R -> 0
__device__ __forceinline__ double2 g_free_smooth(double2 k, double R) {
  const double2 x = make_double2(k.y * R, -k.x * R);
  if (x.x * x.x + x.y * x.y < 1e-6) {
    // -jk (1 + x/2 + x^2/6 + x^3/24)
    double2 t = ca(make_double2(1.0, 0.0), cscale(x, 0.5));
    const double2 x2 = cm(x, x);
    t = ca(t, cscale(x2, 1.0 / 6.0));
    t = ca(t, cscale(cm(x2, x), 1.0 / 24.0));
    return cscale(cm(make_double2(k.y, -k.x), t), 1.0 / (4.0 * kPi));
  }
  const double2 e = cexp_(x);
  return cscale(make_double2(e.x - 1.0, e.y), 1.0 / (4.0 * kPi * R));
}

// K0(w), Re w > 0: trapezoidal rule on K0(w) = int_0^inf exp(-w cosh t) dt.
__device__ double2 bessel_k0(double2 w) {
  const double aw = hypot(w.x, w.y);
  double h = 0.6 / sqrt(aw);
  h = h > 0.2 ? 0.2 : h;
  double2 sum = cscale(cexp_(make_double2(-w.x, -w.y)), 0.5);
  for (int j = 1; j < 20000; ++j) {
    const double ch = cosh(j * h);
    if (w.x * (ch - 1.0) > 40.0) break;
    sum = ca(sum, cexp_(make_double2(-w.x * ch, -w.y * ch)));
  }
  return cscale(sum, h);
}

// K0(w) for any Re w >= 0 (the TEM term of G_N lies near the imaginary axis, where the fixed-step
// rule of bessel_k0 fails): Hankel's asymptotic expansion sqrt(pi/2w) e^-w sum_k a_k for |w| > 17
// (Abramowitz & Stegun 9.7.2); the ascending series -(ln(w/2) + gamma_E) I0(w) + sum_k
// (w^2/4)^k H_k / (k!)^2 (A&S 9.6.13) when Re w <= |w|/10; else the trapezoidal rule with its step
// scaled to the width pi/2 - |arg w| of the strip where exp(-w cosh t) stays bounded.
__device__ double2 bessel_k0_tem(double2 w) {
  const double aw = hypot(w.x, w.y);
  if (aw > 17.0) {
    double2 a = make_double2(1.0, 0.0), acc = a;
    const double2 inv8w = cdiv(make_double2(0.125, 0.0), w);
    for (int k = 1; k < 60; ++k) {
      const double2 na = cscale(cm(a, inv8w), -(2.0 * k - 1.0) * (2.0 * k - 1.0) / k);
      if (hypot(na.x, na.y) >= hypot(a.x, a.y)) break;
      a = na;
      acc = ca(acc, a);
      if (hypot(a.x, a.y) < 1e-17) break;
    }
    const double2 pre = csqrt_(cdiv(make_double2(0.5 * kPi, 0.0), w));
    return cm(cm(pre, cexp_(make_double2(-w.x, -w.y))), acc);
  }
  if (w.x <= 0.1 * aw) {
    const double2 q = cscale(cm(w, w), 0.25);
    double2 t = make_double2(1.0, 0.0), i0 = t, sum = make_double2(0.0, 0.0);
    double hk = 0.0;
    for (int k = 1; k < 400; ++k) {
      t = cscale(cm(t, q), 1.0 / (static_cast<double>(k) * k));
      hk += 1.0 / k;
      i0 = ca(i0, t);
      sum = ca(sum, cscale(t, hk));
      if (k > aw && hypot(t.x, t.y) * (hk + 1.0) < 1e-18) break;
    }
    const double2 lg = make_double2(log(0.5 * aw) + 0.57721566490153286061, atan2(w.y, w.x));
    return cs(sum, cm(lg, i0));
  }
  const double d = 0.5 * kPi - fabs(atan2(w.y, w.x));
  const double h = fmin(fmin(2.0 * kPi * d / 40.0, 0.2), 0.6 / sqrt(aw));
  double2 acc = cscale(cexp_(make_double2(-w.x, -w.y)), 0.5);
  for (int j = 1; j < 200000; ++j) {
    const double ch = cosh(j * h);
    if (w.x * (ch - 1.0) > 40.0) break;
    acc = ca(acc, cexp_(make_double2(-w.x * ch, -w.y * ch)));
  }
  return cscale(acc, h);
}

// kind 0: G_D mode sum; kind 1: G_N mode sum (with the TEM term m = 0)
__device__ double2 strip_modes(const Medium& md, int kind, double zp, double zq, double rho) {
  double2 s = make_double2(0.0, 0.0);
  const double2 k2 = cm(md.k, md.k);
  if (kind == 1) s = cscale(bessel_k0_tem(cscale(csqrt_(make_double2(-k2.x, -k2.y)), rho)), 0.5);
  for (int m = 1; m < 4000; ++m) {
    const double km = m * kPi / md.H;
    const double2 gam = csqrt_(make_double2(km * km - k2.x, -k2.y));
    if (gam.x * rho > 40.0) break;
    const double w = kind == 0 ? sin(km * zp) * sin(km * zq) : cos(km * zp) * cos(km * zq);
    s = ca(s, cscale(bessel_k0(cscale(gam, rho)), w));
  }
  return cscale(s, 1.0 / (kPi * md.H));
}

// ------------------------------------------------------------------ grounded slab kernels
__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 jmul(double2 a) { return make_double2(-a.y, a.x); }   // j a

// k_z = sqrt(k^2 - k_rho^2) on the branch with Im k_z <= 0 (fields e^{-j k_z |z|} decay)
__device__ double2 kz_branch(double2 k, double2 kr) {
  const double2 v = csqrt_(cs(cm(k, k), cm(kr, kr)));
  return v.y > 0.0 ? make_double2(-v.x, -v.y) : v;
}

// Voltage at height z of the TE (te) or TM line for a unit shunt current at zp (0 < z, zp <= d):
// the line is shorted at the ground and loaded by the half-space admittance above d; written with
// q = j k_z1 (Re q >= 0) and decaying exponentials only.
__device__ double2 slab_voltage(const Slab& s, bool te, double2 kr, double z, double zp) {
  constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
  const double2 kz1 = kz_branch(s.k1, kr), kz0 = kz_branch(s.k0t, kr);
  double2 Y1, Y0;
  if (te) {
    Y1 = cscale(kz1, 1.0 / (s.omega * kMu0));
    Y0 = cscale(kz0, 1.0 / (s.omega * kMu0));
  } else {
    Y1 = cdiv(cscale(s.er1, s.omega * kEps0), kz1);
    Y0 = cdiv(cscale(s.ert, s.omega * kEps0), kz0);
  }
  const double2 q = jmul(kz1);
  const double l = s.d - zp;
  const double2 one = make_double2(1.0, 0.0);
  const double2 ez = cexp_(cscale(q, -2.0 * zp)), el = cexp_(cscale(q, -2.0 * l));
  const double2 coth_down = cdiv(ca(one, ez), cs(one, ez));          // shorted line below zp
  const double2 th_up = cdiv(cs(one, el), ca(one, el));              // tanh(q l) above zp
  const double2 y_up = cdiv(cm(Y1, ca(Y0, cm(Y1, th_up))), ca(Y1, cm(Y0, th_up)));
  const double2 Vs = cdiv(one, ca(cm(Y1, coth_down), y_up));
  if (z <= zp) {
    // Vs sinh(q z) / sinh(q zp)
    return cdiv(cm(cm(Vs, cexp_(cscale(q, z - zp))), cs(one, cexp_(cscale(q, -2.0 * z)))), cs(one, ez));
  }
  const double a = s.d - z;
  const double2 r = cdiv(Y0, Y1), ea = cexp_(cscale(q, -2.0 * a));
  const double2 num = ca(ca(one, ea), cm(r, cs(one, ea)));
  const double2 den = ca(ca(one, el), cm(r, cs(one, el)));
  return cdiv(cm(cm(Vs, cexp_(cscale(q, a - l))), num), den);
}

// quasi-static constant of kernel `kind` (0: G_phi, 1: G_A)
__device__ __host__ inline double slab_c(double d, double er1_re, double ert_re, int kind, double z, double zp) {
  if (kind == 1) return 1.0;
  if (z >= d || zp >= d) return 2.0 / (er1_re + ert_re);
  return 1.0 / er1_re;
}

// spectral kernel minus its quasi-static part C e^{-j k_z1 |z - zp|} / (2 j k_z1)
__device__ double2 slab_spectral_rem(const Slab& s, int kind, double c, double2 kr, double z, double zp) {
  constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
  const double2 vte = slab_voltage(s, true, kr, z, zp);
  double2 g;
  if (kind == 1) {
    g = cdiv(vte, make_double2(0.0, s.omega * kMu0));
  } else {
    const double2 vtm = slab_voltage(s, false, kr, z, zp);
    g = cdiv(cm(make_double2(0.0, s.omega * kEps0), cs(vtm, vte)), cm(kr, kr));
  }
  const double2 kz1 = kz_branch(s.k1, kr);
  const double2 e = cexp_(cscale(jmul(kz1), -fabs(z - zp)));
  return cs(g, cdiv(cscale(e, c), cscale(jmul(kz1), 2.0)));
}

// J0 of a complex argument, ascending series (the arguments on the half-ellipse stay moderate)
__device__ double2 j0_complex(double2 w) {
  const double2 q = cscale(cm(w, w), -0.25);
  double2 t = make_double2(1.0, 0.0), sum = t;
  const double aw = cabs_(w);
  for (int m = 1; m < 200; ++m) {
    t = cscale(cm(t, q), 1.0 / (static_cast<double>(m) * m));
    sum = ca(sum, t);
    if (cabs_(t) < 1e-18 * (1.0 + cabs_(sum)) && m > aw) break;
  }
  return sum;
}

// Wynn's epsilon table over partial sums S[0..n-1] (n <= 40): the last entry of the last even
// column is the estimate of the limit
__device__ double2 wynn_limit(const double2* S, int n) {
  double2 em1[40], e0[40], e1[40];
  for (int i = 0; i < n; ++i) { em1[i] = make_double2(0.0, 0.0); e0[i] = S[i]; }
  double2 best = S[n - 1];
  int len = n;
  for (int k = 1; len > 1; ++k) {
    for (int i = 0; i + 1 < len; ++i) {
      const double2 dd = cs(e0[i + 1], e0[i]);
      if (dd.x == 0.0 && dd.y == 0.0) return best;
      e1[i] = ca(em1[i + 1], cdiv(make_double2(1.0, 0.0), dd));
    }
    --len;
    if (k % 2 == 0) best = e1[len - 1];
    for (int i = 0; i <= len; ++i) em1[i] = e0[i];
    for (int i = 0; i < len; ++i) e0[i] = e1[i];
  }
  return best;
}

// (1 / 2 pi) int_0^inf R(k_rho) J0(k_rho rho) k_rho dk_rho of the remainder R of kernel `kind`
__device__ double2 slab_remainder(const Slab& s, int kind, double z, double zp, double rho) {
  const double c = slab_c(s.d, s.er1.x, s.ert.x, kind, z, zp);
  double2 sum = make_double2(0.0, 0.0);
  for (int piece = 0; piece < 4; ++piece) {   // half-ellipse k(t) = ka (1 - cos t) + j kb sin t
    const double t0 = kPi * piece / 4.0, t1 = kPi * (piece + 1) / 4.0;
    for (int i = 0; i < kGlE; ++i) {
      const double t = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * kGlE_x[i];
      double st, ct;
      sincos(t, &st, &ct);
      const double2 kr = make_double2(s.ka * (1.0 - ct), s.kb * st);
      const double2 dk = cscale(make_double2(s.ka * st, s.kb * ct), 0.5 * (t1 - t0) * kGlE_w[i]);
      const double2 f = cm(cm(slab_spectral_rem(s, kind, c, kr, z, zp), j0_complex(cscale(kr, rho))), cm(kr, dk));
      sum = ca(sum, f);
    }
  }
  const double k_start = 2.0 * s.ka;
  const double dz = fabs(z - zp), scale = (dz > 0.0 && dz < s.d) ? dz : s.d;
  double k_switch = 40.0 / scale;
  if (k_switch < 2.0 * k_start) k_switch = 2.0 * k_start;
  const double period = rho > 0.0 ? kPi / rho : 1e300;
  double w = 0.25 * k_start;
  for (double a = k_start; a < k_switch;) {   // graded real-axis panels
    double b = a + (w < period ? w : period);
    if (b > k_switch) b = k_switch;
    for (int i = 0; i < kGlP; ++i) {
      const double kr = 0.5 * (a + b) + 0.5 * (b - a) * kGlP_x[i];
      const double wt = j0(kr * rho) * kr * 0.5 * (b - a) * kGlP_w[i];
      sum = ca(sum, cscale(slab_spectral_rem(s, kind, c, make_double2(kr, 0.0), z, zp), wt));
    }
    a = b;
    w *= 1.5;
  }
  if (rho <= 0.0) {   // tail k = k_switch / u, u in (0, 1]
    for (int piece = 0; piece < 8; ++piece) {
      const double u0 = piece / 8.0, u1 = (piece + 1) / 8.0;
      for (int i = 0; i < kGlP; ++i) {
        const double u = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * kGlP_x[i];
        const double kr = k_switch / u;
        const double wt = kr * (k_switch / (u * u)) * 0.5 * (u1 - u0) * kGlP_w[i];
        sum = ca(sum, cscale(slab_spectral_rem(s, kind, c, make_double2(kr, 0.0), z, zp), wt));
      }
    }
  } else {            // tail: partitions between the large-argument zeros of J0, Wynn-accelerated
    double2 S[40];
    int ns = 0;
    double2 acc = make_double2(0.0, 0.0);
    const int n0 = static_cast<int>(ceil((k_switch * rho + 0.25 * kPi) / kPi));
    double a = k_switch;
    for (int n = 0; n < 64; ++n) {
      double b = ((n0 + n) * kPi + 0.25 * kPi) / rho;
      if (b <= a) b = a + kPi / rho;
      double2 part = make_double2(0.0, 0.0);
      for (int i = 0; i < kGlP; ++i) {
        const double kr = 0.5 * (a + b) + 0.5 * (b - a) * kGlP_x[i];
        const double wt = j0(kr * rho) * kr * 0.5 * (b - a) * kGlP_w[i];
        part = ca(part, cscale(slab_spectral_rem(s, kind, c, make_double2(kr, 0.0), z, zp), wt));
      }
      acc = ca(acc, part);
      if (n < 40) S[ns++] = acc;
      a = b;
      if (n >= 12 && cabs_(part) < 1e-17 * cabs_(acc)) break;
    }
    sum = ca(sum, wynn_limit(S, ns));
  }
  return cscale(sum, 1.0 / (2.0 * kPi));
}

// One thread per table entry: remainder of kernel `kind` between heights z[p] <= z[q] (p <= q,
// mirrored to (q, p) by reciprocity) at rho = i htab, for every frequency.
// tab layout: [F][2][nz][nz][ntab].
__global__ void slab_table_kernel(const Slab* __restrict__ slabs, const double* __restrict__ z, int nz, int ntab,
                                  double htab, int F, double2* __restrict__ tab) {
  const int npair = nz * (nz + 1) / 2;
  const long gid = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long total = static_cast<long>(F) * 2 * npair * ntab;
  if (gid >= total) return;
  const int i = static_cast<int>(gid % ntab);
  long r = gid / ntab;
  int pr = static_cast<int>(r % npair);
  r /= npair;
  const int kind = static_cast<int>(r % 2), f = static_cast<int>(r / 2);
  int p = 0;
  while (pr >= nz - p) { pr -= nz - p; ++p; }
  const int q = p + pr;
  const double2 v = slab_remainder(slabs[f], kind, z[p], z[q], htab * i);
  const size_t base = (static_cast<size_t>(f) * 2 + kind) * nz * nz;
  tab[(base + static_cast<size_t>(p) * nz + q) * ntab + i] = v;
  if (q != p) tab[(base + static_cast<size_t>(q) * nz + p) * ntab + i] = v;
}

// cubic Lagrange interpolation of a table on rho = i h
__device__ double2 table_cubic(const double2* t, int n, double h, double rho) {
  const double x = rho / h;
  int j0 = static_cast<int>(floor(x)) - 1;
  if (j0 < 0) j0 = 0;
  if (j0 > n - 4) j0 = n - 4;
  const double u = x - j0;
  const double l0 = -(u - 1) * (u - 2) * (u - 3) / 6.0, l1 = u * (u - 2) * (u - 3) / 2.0;
  const double l2 = -u * (u - 1) * (u - 3) / 2.0, l3 = u * (u - 1) * (u - 2) / 6.0;
  return ca(ca(cscale(t[j0], l0), cscale(t[j0 + 1], l1)), ca(cscale(t[j0 + 2], l2), cscale(t[j0 + 3], l3)));
}

// layered kernel tk (0: G_phi, 1: G_A) between heights z[ip], z[iq]: C e^{-jk1 R}/(4 pi R) (its
// regular part when smooth) plus the tabulated remainder
__device__ double2 green_slab(const Medium& md, const double* z, const double2* tab, const double* ctab, int tk,
                              int ip, int iq, double rho, bool smooth) {
  const double c = ctab[(tk * md.nz + ip) * md.nz + iq];
  const double dz = z[ip] - z[iq], R = sqrt(rho * rho + dz * dz);
  const double2 direct = cscale(smooth ? g_free_smooth(md.k, R) : g_free(md.k, R), c);
  return ca(direct, table_cubic(tab + (static_cast<size_t>(tk * md.nz + ip) * md.nz + iq) * md.ntab, md.ntab, md.htab, rho));
}

// image sum |n| <= kImages (second family subtracted for G_D, added for G_N); `smooth` replaces
// the direct term by its R -> 0 regular part
__device__ double2 strip_images(const Medium& md, int kind, double zp, double zq, double rho, bool smooth) {
  double2 s = make_double2(0.0, 0.0);
  const double r2 = rho * rho;
  for (int n = -kImages; n <= kImages; ++n) {
    const double a = zp - zq + 2.0 * n * md.H, b = zp + zq + 2.0 * n * md.H;
    const double Ra = sqrt(r2 + a * a), Rb = sqrt(r2 + b * b);
    s = ca(s, (n == 0 && smooth) ? g_free_smooth(md.k, Ra) : g_free(md.k, Ra));
    s = kind == 0 ? cs(s, g_free(md.k, Rb)) : ca(s, g_free(md.k, Rb));
  }
  return s;
}

// Kernel `kind` between heights z[ip], z[iq] at lateral distance rho; smooth = true returns
// G - 1/(4 pi R_direct).
__device__ double2 green(const Medium& md, const double* z, const double2* fit, int kind, int ip, int iq, double rho,
                         bool smooth) {
  const double zp = z[ip], zq = z[iq];
  if (!md.stripline) {
    const double Rd = sqrt(rho * rho + (zp - zq) * (zp - zq)), Ri = sqrt(rho * rho + (zp + zq) * (zp + zq));
    const double2 gd = smooth ? g_free_smooth(md.k, Rd) : g_free(md.k, Rd), gi = g_free(md.k, Ri);
    return kind == 0 ? cs(gd, gi) : ca(gd, gi);
  }
  if (rho >= md.rho_s) {
    double2 G = strip_modes(md, kind, zp, zq, rho);
    if (smooth) G.x -= 1.0 / (4.0 * kPi * sqrt(rho * rho + (zp - zq) * (zp - zq)));
    return G;
  }
  const double2* c = fit + 3 * ((static_cast<size_t>(kind) * md.nz + ip) * md.nz + iq);
  const double x = rho * rho;
  return ca(strip_images(md, kind, zp, zq, rho, smooth), ca(c[0], cscale(ca(c[1], cscale(c[2], x)), x)));
}

// ------------------------------------------------------------------ quadrature (barycentric)
// Radon 7-point, degree 5; Dunavant 13-point, degree 7.
__constant__ double kQ7[7][4];
__constant__ double kQ13[13][4];

void host_rules(double q7[7][4], double q13[13][4]) {
  const double s = std::sqrt(15.0);
  const double a1 = (6.0 - s) / 21.0, w1 = (155.0 - s) / 1200.0;
  const double a2 = (6.0 + s) / 21.0, w2 = (155.0 + s) / 1200.0;
  double r7[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 0.225},
                     {1 - 2 * a1, a1, a1, w1}, {a1, 1 - 2 * a1, a1, w1}, {a1, a1, 1 - 2 * a1, w1},
                     {1 - 2 * a2, a2, a2, w2}, {a2, 1 - 2 * a2, a2, w2}, {a2, a2, 1 - 2 * a2, w2}};
  std::memcpy(q7, r7, sizeof(r7));
  const double b1 = 0.260345966079040, v1 = 0.175615257433208;
  const double b2 = 0.065130102902216, v2 = 0.053347235608838;
  const double c1 = 0.048690315425316, c2 = 0.312865496004874, c3 = 0.638444188569810, v3 = 0.077113760890257;
  double r13[13][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, -0.149570044467682},
                       {1 - 2 * b1, b1, b1, v1}, {b1, 1 - 2 * b1, b1, v1}, {b1, b1, 1 - 2 * b1, v1},
                       {1 - 2 * b2, b2, b2, v2}, {b2, 1 - 2 * b2, b2, v2}, {b2, b2, 1 - 2 * b2, v2},
                       {c1, c2, c3, v3}, {c1, c3, c2, v3}, {c2, c1, c3, v3},
                       {c2, c3, c1, v3}, {c3, c1, c2, v3}, {c3, c2, c1, v3}};
  std::memcpy(q13, r13, sizeof(r13));
}

// Analytic integrals over planar triangle T of 1/R and (rho' - rho)/R for observation point r
// (Wilton et al. 1984): I1 and the in-plane vector Iv.
__device__ void potentials(const FillTri& t, const double r[3], double* I1, double Iv[3]) {
  double e1[3], e2[3], n[3];
  for (int i = 0; i < 3; ++i) { e1[i] = t.v[1][i] - t.v[0][i]; e2[i] = t.v[2][i] - t.v[0][i]; }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int i = 0; i < 3; ++i) n[i] /= nn;
  const double d = n[0] * (r[0] - t.v[0][0]) + n[1] * (r[1] - t.v[0][1]) + n[2] * (r[2] - t.v[0][2]);
  const double ad = fabs(d);
  const double p[3] = {r[0] - d * n[0], r[1] - d * n[1], r[2] - d * n[2]};
  double s = 0.0, sv[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    const double* A = t.v[i];
    const double* B = t.v[(i + 1) % 3];
    double l[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double len = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    for (int k = 0; k < 3; ++k) l[k] /= len;
    const double u[3] = {l[1] * n[2] - l[2] * n[1], l[2] * n[0] - l[0] * n[2], l[0] * n[1] - l[1] * n[0]};
    const double am[3] = {A[0] - p[0], A[1] - p[1], A[2] - p[2]};
    const double bm[3] = {B[0] - p[0], B[1] - p[1], B[2] - p[2]};
    const double lm = am[0] * l[0] + am[1] * l[1] + am[2] * l[2];
    const double lp = bm[0] * l[0] + bm[1] * l[1] + bm[2] * l[2];
    const double tt = am[0] * u[0] + am[1] * u[1] + am[2] * u[2];
    const double R02 = tt * tt + d * d;
    const double Rm = sqrt(R02 + lm * lm), Rp = sqrt(R02 + lp * lp);
    double lg = 0.0;
    if (R02 > 1e-30 * len * len) {
      const double num = lp >= 0 ? Rp + lp : R02 / (Rp - lp);
      const double den = lm >= 0 ? Rm + lm : R02 / (Rm - lm);
      lg = log(num / den);
      s += tt * lg;
      if (ad > 0) s -= ad * (atan(tt * lp / (R02 + ad * Rp)) - atan(tt * lm / (R02 + ad * Rm)));
    }
    const double vv = R02 * lg + lp * Rp - lm * Rm;
    for (int k = 0; k < 3; ++k) sv[k] += 0.5 * u[k] * vv;
  }
  *I1 = s;
  Iv[0] = sv[0]; Iv[1] = sv[1]; Iv[2] = sv[2];
}

// Tail quadratics of both kernels for every pair of heights at frequency blockIdx.x:
// fits[f][kind][ip][iq][3].
__global__ void fit_kernel(const Medium* __restrict__ media, const double* __restrict__ z, double2* __restrict__ fits) {
  const int f = blockIdx.x;
  const Medium md = media[f];
  const int nz = md.nz, pairs = 2 * nz * nz;
  for (int t = threadIdx.x; t < pairs; t += blockDim.x) {
    double2* c = fits + (static_cast<size_t>(f) * pairs + t) * 3;
    if (!md.stripline) {
      c[0] = c[1] = c[2] = make_double2(0.0, 0.0);
      continue;
    }
    const int kind = t / (nz * nz), ip = (t / nz) % nz, iq = t % nz;
    double x[3];
    double2 y[3];
    for (int i = 0; i < 3; ++i) {
      const double rho = md.rho_s * (1.0 + 0.5 * i);
      x[i] = rho * rho;
      y[i] = cs(strip_modes(md, kind, z[ip], z[iq], rho), strip_images(md, kind, z[ip], z[iq], rho, false));
    }
    // Lagrange form of the quadratic in x through the three points, expanded to c0 + c1 x + c2 x^2
    double2 c0 = make_double2(0, 0), c1 = c0, c2 = c0;
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      const double den = (x[i] - x[j]) * (x[i] - x[k]);
      c2 = ca(c2, cscale(y[i], 1.0 / den));
      c1 = ca(c1, cscale(y[i], -(x[j] + x[k]) / den));
      c0 = ca(c0, cscale(y[i], x[j] * x[k] / den));
    }
    c[0] = c0; c[1] = c1; c[2] = c2;
  }
}

// One thread: integrals of one translation class at one frequency.
// out[0] = int int G_D, out[1 + 3a + b] = int int (r - v_a) . G_A (r' - v_b) with G_A = G_D on the
// horizontal and G_N on the vertical components.
// Layered medium: G_phi for the scalar part, G_A for the horizontal vector part, and the analytic
// singular integrals weighted by their quasi-static constants (tabs, ctabs: per frequency
// [2][nz][nz][ntab] remainders and [2][nz][nz] constants).
__global__ void __launch_bounds__(128) class_kernel(const FillTri* __restrict__ tris, const int2* __restrict__ rep, int U,
                                                     const Medium* __restrict__ media, const double* __restrict__ z,
                                                     const double2* __restrict__ fits, int F, double2* __restrict__ out,
                                                     const double2* __restrict__ tabs, const double* __restrict__ ctabs) {
  const long gid = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= static_cast<long>(U) * F) return;
  const int f = static_cast<int>(gid / U), u = static_cast<int>(gid % U);
  const Medium md = media[f];
  const double2* fit = fits + static_cast<size_t>(f) * 2 * md.nz * md.nz * 3;
  const double2* tab = md.layered ? tabs + static_cast<size_t>(f) * 2 * md.nz * md.nz * md.ntab : nullptr;
  const double* ctab = md.layered ? ctabs + static_cast<size_t>(f) * 2 * md.nz * md.nz : nullptr;
  const FillTri& p = tris[rep[u].x];
  const FillTri& q = tris[rep[u].y];
  double2 acc[10];
  for (int i = 0; i < 10; ++i) acc[i] = make_double2(0.0, 0.0);
  const double dc = sqrt((p.c[0] - q.c[0]) * (p.c[0] - q.c[0]) + (p.c[1] - q.c[1]) * (p.c[1] - q.c[1]) +
                         (p.c[2] - q.c[2]) * (p.c[2] - q.c[2]));
  const double lmax = fmax(p.lmax, q.lmax);
  const bool near = dc < 2.0 * lmax * (1.0 + 1e-9);
  const bool both_vert = p.vert && q.vert;
  const int nq = near ? 13 : 7, rs = near ? 1 : 0;
  const double(*Q)[4] = near ? kQ13 : kQ7;
  for (int i = 0; i < nq; ++i) {
    const int ip = p.zid[rs][i];
    double r[3];
    for (int k = 0; k < 2; ++k) r[k] = Q[i][0] * p.v[0][k] + Q[i][1] * p.v[1][k] + Q[i][2] * p.v[2][k];
    r[2] = z[ip];
    const double wo = Q[i][3] * p.area;
    double ra[3][3];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) ra[a][k] = r[k] - p.v[a][k];
    if (near) {
      double I1, Iv[3];
      potentials(q, r, &I1, Iv);
      const double s = wo / (4.0 * kPi);
      double cphi = 1.0, cA = 1.0;
      if (md.layered) {
        const int iq0 = q.zid[1][0];
        cphi = ctab[(0 * md.nz + ip) * md.nz + iq0];
        cA = ctab[(1 * md.nz + ip) * md.nz + iq0];
      }
      acc[0].x += cphi * s * I1;
      // projection of r on the plane of q
      const double d = q.n[0] * (r[0] - q.v[0][0]) + q.n[1] * (r[1] - q.v[0][1]) + q.n[2] * (r[2] - q.v[0][2]);
      const double r0[3] = {r[0] - d * q.n[0], r[1] - d * q.n[1], r[2] - d * q.n[2]};
      for (int b = 0; b < 3; ++b) {
        double tv[3];
        for (int k = 0; k < 3; ++k) tv[k] = Iv[k] + (r0[k] - q.v[b][k]) * I1;
        for (int a = 0; a < 3; ++a) acc[1 + 3 * a + b].x += cA * s * (ra[a][0] * tv[0] + ra[a][1] * tv[1] + ra[a][2] * tv[2]);
      }
    }
    for (int j = 0; j < nq; ++j) {
      const int iq = q.zid[rs][j];
      double rq[3];
      for (int k = 0; k < 2; ++k) rq[k] = Q[j][0] * q.v[0][k] + Q[j][1] * q.v[1][k] + Q[j][2] * q.v[2][k];
      rq[2] = z[iq];
      const double rho = hypot(r[0] - rq[0], r[1] - rq[1]);
      const double w = wo * Q[j][3] * q.area;
      // scalar kernel, horizontal vector kernel (the same in a homogeneous medium), vertical one
      double2 GD, GA, GN = make_double2(0.0, 0.0);
      if (md.layered) {
        GD = cscale(green_slab(md, z, tab, ctab, 0, ip, iq, rho, near), w);
        GA = cscale(green_slab(md, z, tab, ctab, 1, ip, iq, rho, near), w);
      } else {
        GD = cscale(green(md, z, fit, 0, ip, iq, rho, near), w);
        GA = GD;
        if (both_vert) GN = cscale(green(md, z, fit, 1, ip, iq, rho, near), w);
      }
      acc[0] = ca(acc[0], GD);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const double dh = ra[a][0] * (rq[0] - q.v[b][0]) + ra[a][1] * (rq[1] - q.v[b][1]);
          const double dz = ra[a][2] * (rq[2] - q.v[b][2]);
          acc[1 + 3 * a + b] = ca(acc[1 + 3 * a + b], ca(cscale(GA, dh), cscale(GN, dz)));
        }
    }
  }
  double2* o = out + gid * 10;
  for (int i = 0; i < 10; ++i) o[i] = acc[i];
}

struct BfGeom {
  int tp, tm;        // triangle indices of T+ and T-
  int fp, fm;        // free vertex indices
  double len;        // edge length
};

__device__ __forceinline__ double2 zmn(const BfGeom& m, const BfGeom& n, const FillTri* tris, const int* pair_class, int T,
                                       const double2* cls, double2 jwmu, double2 inv_jweps) {
  double2 z = make_double2(0.0, 0.0);
  const int tm[2] = {m.tp, m.tm}, fm[2] = {m.fp, m.fm};
  const int tn[2] = {n.tp, n.tm}, fn[2] = {n.fp, n.fm};
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      const double2* v = cls + static_cast<size_t>(pair_class[tm[s] * T + tn[t]]) * 10;
      const double aa = tris[tm[s]].area * tris[tn[t]].area;
      const double sg = (s == t ? 1.0 : -1.0) * m.len * n.len;
      const double2 vec = cm(cscale(jwmu, 0.25 / aa), v[1 + 3 * fm[s] + fn[t]]);
      const double2 sca = cm(cscale(inv_jweps, 1.0 / aa), v[0]);
      z = ca(z, cscale(ca(vec, sca), sg));
    }
  return z;
}

template <typename ZT>
__global__ void assemble_kernel(const BfGeom* __restrict__ bfs, int M, const FillTri* __restrict__ tris,
                                const int* __restrict__ pair_class, int T, const double2* __restrict__ cls_all, int U,
                                const Medium* __restrict__ media, ZT* __restrict__ Z) {
  const int f = blockIdx.y;
  const long e = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= static_cast<long>(M) * M) return;
  const int m = static_cast<int>(e / M), n = static_cast<int>(e % M);
  const Medium md = media[f];
  const double2 jwmu = make_double2(0.0, md.omega * kMu0);
  const double2 inv_jweps = cdiv(make_double2(1.0, 0.0), cm(make_double2(0.0, md.omega), md.eps));
  const double2* cls = cls_all + static_cast<size_t>(f) * U * 10;
  const BfGeom bm = bfs[m], bn = bfs[n];
  const double2 a = zmn(bm, bn, tris, pair_class, T, cls, jwmu, inv_jweps);
  const double2 b = zmn(bn, bm, tris, pair_class, T, cls, jwmu, inv_jweps);
  const double2 z = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
  ZT out;
  out.x = z.x;
  out.y = z.y;
  Z[static_cast<size_t>(f) * M * M + e] = out;
}

double hj_eps_eff(const Grid& g) {
  double h = 0.0;
  for (double z : g.layer_z) h = std::max(h, z);
  const double u = g.pitch / h, er = g.eps_r;
  const double a = 1.0 + std::log((std::pow(u, 4) + std::pow(u / 52.0, 2)) / (std::pow(u, 4) + 0.432)) / 49.0 +
                   std::log(1.0 + std::pow(u / 18.1, 3)) / 18.7;
  const double b = 0.564 * std::pow((er - 0.9) / (er + 3.0), 0.053);
  return 0.5 * (er + 1.0) + 0.5 * (er - 1.0) * std::pow(1.0 + 10.0 / u, -a * b);
}

// Geometry of a triangle key (half 0, 1: the pixel's triangles; 2, 3: the via strip's Ta, Tb).
// Fine-lattice parts of a triangle key (the mesher's encoding: W = 128 s, offset 4 s).
void key_parts(const Grid& g, int32_t key, int* layer, int* x, int* y, int* half) {
  const int W = 128 * g.subs(), off = 4 * g.subs();
  *half = key & 3;
  int k = key >> 2;
  *x = k % W - off;
  k /= W;
  *y = k % W - off;
  *layer = k / W;
}

void key_triangle(const Grid& g, int32_t key, FillTri* t) {
  int half, x, y, layer;
  key_parts(g, key, &layer, &x, &y, &half);
  const double h = g.pitch / g.subs();   // sub-square side
  static const int corner[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};
  static const int tri[2][2][3] = {{{0, 1, 2}, {1, 3, 2}}, {{0, 1, 3}, {0, 3, 2}}};
  static const int dend[2][2] = {{2, 1}, {0, 3}};   // diagonal end corners D0, D1 per orientation
  const int o = orient(g, x, y);
  if (half < 2) {
    for (int i = 0; i < 3; ++i) {
      const int cc = tri[o][half][i];
      t->v[i][0] = (x + corner[cc][0]) * h;
      t->v[i][1] = (y + corner[cc][1]) * h;
      t->v[i][2] = g.layer_z[layer];
    }
  } else {
    // Ta = (D0@l, D1@l, D1@l+1), Tb = (D0@l, D1@l+1, D0@l+1)
    const int cs3[2][3] = {{dend[o][0], dend[o][1], dend[o][1]}, {dend[o][0], dend[o][1], dend[o][0]}};
    const int up[2][3] = {{0, 0, 1}, {0, 1, 1}};
    for (int i = 0; i < 3; ++i) {
      const int cc = cs3[half - 2][i];
      t->v[i][0] = (x + corner[cc][0]) * h;
      t->v[i][1] = (y + corner[cc][1]) * h;
      t->v[i][2] = g.layer_z[layer + up[half - 2][i]];
    }
  }
  double e1[3], e2[3];
  for (int i = 0; i < 3; ++i) { e1[i] = t->v[1][i] - t->v[0][i]; e2[i] = t->v[2][i] - t->v[0][i]; }
  const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double lmax = 0.0;
  for (int i = 0; i < 3; ++i) {
    t->n[i] = n[i] / nn;
    t->c[i] = (t->v[0][i] + t->v[1][i] + t->v[2][i]) / 3.0;
    const int j = (i + 1) % 3;
    const double dx = t->v[j][0] - t->v[i][0], dy = t->v[j][1] - t->v[i][1], dz = t->v[j][2] - t->v[i][2];
    lmax = std::max(lmax, std::sqrt(dx * dx + dy * dy + dz * dz));
  }
  t->area = 0.5 * nn;
  t->lmax = lmax;
  t->layer = layer;
  t->vert = half >= 2;
  for (int r = 0; r < 2; ++r)
    for (int i = 0; i < 13; ++i) t->zid[r][i] = static_cast<int16_t>(layer);
}

// Gauss-Legendre nodes and weights of order n on [-1, 1]: Newton's method on P_n from the
// Chebyshev-like first guess cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by the three-term
// recurrence.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;   // P_0, P_1
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(t), p0 = P_{n-1}(t)
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-15) break;
    }
    x[i] = -t;
    x[n - 1 - i] = t;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

}  // namespace
}  // namespace pmom

namespace pmom {

pmom_status fill_Z(const Grid& g, const std::vector<int32_t>& table, int M, const double* freqs, int F, int dtype,
                   cudaStream_t s, void** d_Z_out, std::string* err) {
  if (g.layers > kMaxLayers) return PMOM_ERR_UNSUPPORTED;
  // the layered kernels are those of horizontal currents: no via strips in a grounded slab
  if (g.medium == 2 && g.vias()) return PMOM_ERR_UNSUPPORTED;
  // distinct triangles
  std::unordered_map<int32_t, int> tri_of;
  std::vector<FillTri> tris;
  std::vector<int32_t> keys;
  for (int m = 0; m < M; ++m)
    for (int sd = 0; sd < 2; ++sd) {
      const int32_t k = table[static_cast<size_t>(m) * kTableCols + 4 + sd];
      if (!tri_of.count(k)) {
        tri_of[k] = static_cast<int>(tris.size());
        FillTri t;
        key_triangle(g, k, &t);
        tris.push_back(t);
        keys.push_back(k);
      }
    }
  const int T = static_cast<int>(tris.size());
  double q7[7][4], q13[13][4];
  host_rules(q7, q13);
  // heights visited by the quadrature: the layers, then the points of vertical triangles
  std::vector<double> heights(g.layer_z.begin(), g.layer_z.end());
  for (FillTri& t : tris) {
    if (!t.vert) continue;
    for (int r = 0; r < 2; ++r) {
      const int n = r ? 13 : 7;
      for (int i = 0; i < n; ++i) {
        const double* b = r ? q13[i] : q7[i];
        const double zz = t.v[0][2] + b[1] * (t.v[1][2] - t.v[0][2]) + b[2] * (t.v[2][2] - t.v[0][2]);
        size_t id = 0;
        while (id < heights.size() && heights[id] != zz) ++id;
        if (id == heights.size()) heights.push_back(zz);
        t.zid[r][i] = static_cast<int16_t>(id);
      }
    }
  }
  const int nz = static_cast<int>(heights.size());
  // translation classes
  std::unordered_map<long long, int> cls_of;
  std::vector<int2> rep;
  std::vector<int> pair_class(static_cast<size_t>(T) * T);
  // diagonal orientation of each triangle's pixel: with the alternating pattern the second
  // triangle's follows from the first's and the offset, with the uniform and random ones it does
  // not, so both enter the class
  std::vector<int> ori(T);
  std::vector<int4> parts(T);   // layer, x, y, half on the fine lattice
  for (int t = 0; t < T; ++t) {
    int l, x, y, h;
    key_parts(g, keys[t], &l, &x, &y, &h);
    parts[t] = make_int4(l, x, y, h);
    ori[t] = orient(g, x, y);
  }
  for (int p = 0; p < T; ++p) {
    const int lp = parts[p].x, xp = parts[p].y, yp = parts[p].z, hp = parts[p].w;
    for (int q = 0; q < T; ++q) {
      const int lq = parts[q].x, xq = parts[q].y, yq = parts[q].z, hq = parts[q].w;
      const long long key =
          ((((((((static_cast<long long>(lp) * 8 + lq) * 2 + ori[p]) * 2 + ori[q]) * 4 + hp) * 4 + hq) * 2048 +
             (xq - xp + 1024)) * 2048) + (yq - yp + 1024));
      auto it = cls_of.find(key);
      int c;
      if (it == cls_of.end()) {
        c = static_cast<int>(rep.size());
        cls_of.emplace(key, c);
        rep.push_back(make_int2(p, q));
      } else {
        c = it->second;
      }
      pair_class[static_cast<size_t>(p) * T + q] = c;
    }
  }
  const int U = static_cast<int>(rep.size());
  std::vector<BfGeom> bfs(M);
  for (int m = 0; m < M; ++m) {
    const int32_t* r = &table[static_cast<size_t>(m) * kTableCols];
    BfGeom b;
    b.tp = tri_of[r[4]];
    b.tm = tri_of[r[5]];
    b.fp = r[6];
    b.fm = r[7];
    const FillTri& t = tris[b.tp];
    const double* v1 = t.v[(b.fp + 1) % 3];
    const double* v2 = t.v[(b.fp + 2) % 3];
    b.len = std::sqrt((v1[0] - v2[0]) * (v1[0] - v2[0]) + (v1[1] - v2[1]) * (v1[1] - v2[1]) + (v1[2] - v2[2]) * (v1[2] - v2[2]));
    bfs[m] = b;
  }
  std::vector<Medium> media(F);
  const bool layered = g.medium == 2;
  const double er = g.medium == 0 ? hj_eps_eff(g) : g.eps_r;
  const double eps0 = 1.0 / (kMu0 * kC0 * kC0);
  // layered medium: the slab up to the highest metal layer, tables on rho = i d/16 out to the
  // diagonal of the grid with a three-pixel margin on every side
  double d_slab = 0.0;
  for (double zz : g.layer_z) d_slab = std::max(d_slab, zz);
  const double htab = d_slab / 16.0;
  const double rho_max = g.pitch * std::sqrt((g.nx + 6.0) * (g.nx + 6.0) + (g.ny + 6.0) * (g.ny + 6.0));
  const int ntab = layered ? static_cast<int>(std::ceil(rho_max / htab)) + 4 : 0;
  std::vector<Slab> slabs(layered ? F : 0);
  std::vector<double> ctabs(layered ? static_cast<size_t>(F) * 2 * nz * nz : 0);
  for (int f = 0; f < F; ++f) {
    Medium& md = media[f];
    md.omega = 2.0 * kPi * freqs[f];
    md.eps = layered ? make_double2(eps0, 0.0) : make_double2(eps0 * er, -eps0 * er * g.tan_d);
    // k = w sqrt(mu0 eps), principal root
    const std::complex<double> kk = md.omega * std::sqrt(std::complex<double>(kMu0 * md.eps.x, kMu0 * md.eps.y));
    md.k = make_double2(kk.real(), kk.imag());
    md.stripline = g.medium == 1;
    md.layered = layered;
    md.H = g.h_total;
    md.rho_s = 0.5 * g.h_total;
    md.nz = nz;
    md.ntab = ntab;
    md.htab = htab;
    if (layered) {
      Slab& sl = slabs[f];
      sl.omega = md.omega;
      sl.d = d_slab;
      const std::complex<double> er1(g.eps_r, -g.eps_r * g.tan_d), ert(1.0, 0.0);
      const double k0 = md.omega / kC0;
      const std::complex<double> k1 = k0 * std::sqrt(er1), k0t = k0 * std::sqrt(ert);
      sl.er1 = make_double2(er1.real(), er1.imag());
      sl.ert = make_double2(ert.real(), ert.imag());
      sl.k1 = make_double2(k1.real(), k1.imag());
      sl.k0t = make_double2(k0t.real(), k0t.imag());
      const double kmax = std::max(std::abs(k1), std::abs(k0t));
      sl.ka = 1.5 * kmax + k0;
      sl.kb = 0.25 * kmax;
      const double rho_tab = htab * (ntab - 1);
      if (sl.kb * rho_tab > 1.0) sl.kb = 1.0 / rho_tab;
      md.k = sl.k1;   // the quasi-static term propagates with the slab's wavenumber
      for (int kind = 0; kind < 2; ++kind)
        for (int p = 0; p < nz; ++p)
          for (int q = 0; q < nz; ++q)
            ctabs[((static_cast<size_t>(f) * 2 + kind) * nz + p) * nz + q] =
                slab_c(d_slab, er1.real(), ert.real(), kind, heights[p], heights[q]);
    }
  }
  FillTri* d_tris = nullptr;
  double* d_z = nullptr;
  int2* d_rep = nullptr;
  int* d_pc = nullptr;
  BfGeom* d_bfs = nullptr;
  Medium* d_media = nullptr;
  double2* d_fit = nullptr;
  double2* d_cls = nullptr;
  Slab* d_slabs = nullptr;
  double2* d_tab = nullptr;
  double* d_ctab = nullptr;
  void* d_Z = nullptr;
  const size_t zel = dtype == PMOM_C128 ? sizeof(double2) : sizeof(float2);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chk(cudaMemcpyToSymbolAsync(kQ7, q7, sizeof(q7), 0, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyToSymbolAsync(kQ13, q13, sizeof(q13), 0, cudaMemcpyHostToDevice, s));
  chk(cudaMalloc(&d_tris, sizeof(FillTri) * T));
  chk(cudaMalloc(&d_rep, sizeof(int2) * U));
  chk(cudaMalloc(&d_pc, sizeof(int) * pair_class.size()));
  chk(cudaMalloc(&d_bfs, sizeof(BfGeom) * M));
  chk(cudaMalloc(&d_media, sizeof(Medium) * F));
  chk(cudaMalloc(&d_z, sizeof(double) * nz));
  chk(cudaMalloc(&d_fit, sizeof(double2) * 3 * 2 * static_cast<size_t>(nz) * nz * F));
  chk(cudaMalloc(&d_cls, sizeof(double2) * 10 * static_cast<size_t>(U) * F));
  if (layered) {
    double gx[kGlE], gw[kGlE], px[kGlP], pw[kGlP];
    gauss_legendre(kGlE, gx, gw);
    gauss_legendre(kGlP, px, pw);
    chk(cudaMemcpyToSymbolAsync(kGlE_x, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyToSymbolAsync(kGlE_w, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyToSymbolAsync(kGlP_x, px, sizeof(px), 0, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyToSymbolAsync(kGlP_w, pw, sizeof(pw), 0, cudaMemcpyHostToDevice, s));
    chk(cudaMalloc(&d_slabs, sizeof(Slab) * F));
    chk(cudaMalloc(&d_tab, sizeof(double2) * static_cast<size_t>(F) * 2 * nz * nz * ntab));
    chk(cudaMalloc(&d_ctab, sizeof(double) * ctabs.size()));
    if (e == cudaSuccess) {
      chk(cudaMemcpyAsync(d_slabs, slabs.data(), sizeof(Slab) * F, cudaMemcpyHostToDevice, s));
      chk(cudaMemcpyAsync(d_ctab, ctabs.data(), sizeof(double) * ctabs.size(), cudaMemcpyHostToDevice, s));
    }
  }
  chk(cudaMalloc(&d_Z, zel * static_cast<size_t>(F) * M * M));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(d_tris, tris.data(), sizeof(FillTri) * T, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(d_rep, rep.data(), sizeof(int2) * U, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(d_pc, pair_class.data(), sizeof(int) * pair_class.size(), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(d_bfs, bfs.data(), sizeof(BfGeom) * M, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(d_media, media.data(), sizeof(Medium) * F, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(d_z, heights.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, s));
  }
  if (e == cudaSuccess) {
    fit_kernel<<<F, 128, 0, s>>>(d_media, d_z, d_fit);
    chk(cudaGetLastError());
    if (layered) {
      const long entries = static_cast<long>(F) * 2 * (nz * (nz + 1) / 2) * ntab;
      slab_table_kernel<<<static_cast<unsigned>((entries + 127) / 128), 128, 0, s>>>(d_slabs, d_z, nz, ntab, htab, F, d_tab);
      chk(cudaGetLastError());
    }
    const long work = static_cast<long>(U) * F;
    class_kernel<<<static_cast<unsigned>((work + 127) / 128), 128, 0, s>>>(d_tris, d_rep, U, d_media, d_z, d_fit, F, d_cls,
                                                                           d_tab, d_ctab);
    chk(cudaGetLastError());
    const dim3 grid(static_cast<unsigned>((static_cast<long>(M) * M + 255) / 256), F);
    if (dtype == PMOM_C128)
      assemble_kernel<double2><<<grid, 256, 0, s>>>(d_bfs, M, d_tris, d_pc, T, d_cls, U, d_media, static_cast<double2*>(d_Z));
    else
      assemble_kernel<float2><<<grid, 256, 0, s>>>(d_bfs, M, d_tris, d_pc, T, d_cls, U, d_media, static_cast<float2*>(d_Z));
    chk(cudaGetLastError());
    chk(cudaStreamSynchronize(s));
  }
  cudaFree(d_tris);
  cudaFree(d_rep);
  cudaFree(d_pc);
  cudaFree(d_bfs);
  cudaFree(d_media);
  cudaFree(d_fit);
  cudaFree(d_z);
  cudaFree(d_cls);
  cudaFree(d_slabs);
  cudaFree(d_tab);
  cudaFree(d_ctab);
  if (e != cudaSuccess) {
    if (d_Z) cudaFree(d_Z);
    *err = std::string("fill_Z: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PMOM_ERR_OOM : PMOM_ERR_CUDA;
  }
  *d_Z_out = d_Z;
  return PMOM_OK;
}

}  // namespace pmom
