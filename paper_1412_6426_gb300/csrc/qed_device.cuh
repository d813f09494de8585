// Device-side building blocks of the QED particle step (sm_103a).
//
// Units: momentum m c, time hbar/(m c^2), length hbar/(m c), fields E_S.
// In these units the bracket [dt e^2 m c/hbar^2] of Eqs. (24), (27), (30)
// is alpha*dt and the Lorentz force is q (E + v x B).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qed {

constexpr double kAlpha = 7.2973525693e-3;          // fine-structure constant
constexpr double kSqrt3Over2Pi = 0.27566444771089602; // sqrt(3)/(2 pi), correctly rounded
constexpr double kTwoPi = 6.283185307179586;
constexpr double kPi = 3.141592653589793;

enum Species { kElectron = 0, kPositron = 1, kPhoton = 2, kIon = 3, kNSpecies = 4 };
enum Purpose : uint32_t { kEmit = 1, kPair = 2, kChild = 3, kKeep = 4, kThin = 5, kSchwinger = 6 };
constexpr unsigned kSchwingerKind = 0x80;   // flag in the product kind of vacuum pairs
enum FieldMode {
  kFieldGrid = 0, kFieldUniform = 1, kFieldGaussianLP = 2, kFieldRotatingE = 3, kFieldEnsemble = 4,
  kFieldStandingWave = 5
};

// Device status bits (folded into a qed_status by the host).
enum StatusBit : int {
  kStCapacity = 1, kStNonfinite = 2, kStTimeout = 4, kStPmGt1 = 8, kStCourant = 16
};

// ---------------------------------------------------------------------------
// Rate tables.  g1(z) = F1(z) z^{-1/3}, g2(z) = F2(z) z^{-1/3} (Sec. IV.E,
// F1(x) = x int_x^inf K_{5/3}, F2(x) = x K_{2/3}(x)) are stored as piecewise
// polynomials: binade e of z (z in [2^e, 2^{e+1})) split into S equal
// sub-intervals, each a degree-D polynomial in t in [-1, 1].  For e >= 0 the
// stored function is g * exp(z).  Below 2^EMIN the two-term series
// g1 = g1(0) - (pi/sqrt 3) z^{2/3}, g2 = g2(0) is used; at and above 2^EMAX
// both are zero (exp(-512) is far below any uniform draw).
template <typename R> struct TabCfg;
template <> struct TabCfg<double> { static constexpr int EMIN = -60, EMAX = 9, S = 4, D = 10; };
template <> struct TabCfg<float> { static constexpr int EMIN = -40, EMAX = 9, S = 2, D = 5; };

template <typename R> struct Tab {
  static constexpr int EMIN = TabCfg<R>::EMIN, EMAX = TabCfg<R>::EMAX;
  static constexpr int S = TabCfg<R>::S, D = TabCfg<R>::D;
  static constexpr int NB = EMAX - EMIN;
  static constexpr int NC = D + 1;
  static constexpr int kCoefs = 2 * NB * S * NC;  // both functions
  // header: g1(0), g2(0), pi/sqrt(3), unused
  static constexpr int kHeader = 4;
  static constexpr int kSize = kHeader + kCoefs;
};

__device__ __forceinline__ void split_binade(double z, int &e, double &m) {
  unsigned long long b = (unsigned long long)__double_as_longlong(z);
  e = (int)((b >> 52) & 0x7ffull) - 1023;
  m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
}
__device__ __forceinline__ void split_binade(float z, int &e, float &m) {
  unsigned b = __float_as_uint(z);
  e = (int)((b >> 23) & 0xffu) - 127;
  m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
}

__device__ __forceinline__ double exp_r(double x) { return exp(x); }
__device__ __forceinline__ float exp_r(float x) { return __expf(x); }
__device__ __forceinline__ double log_r(double x) { return log(x); }
__device__ __forceinline__ float log_r(float x) { return __logf(x); }
__device__ __forceinline__ double cbrt_r(double x) { return cbrt(x); }
__device__ __forceinline__ float cbrt_r(float x) { return cbrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double floor_r(double x) { return floor(x); }
__device__ __forceinline__ float floor_r(float x) { return floorf(x); }
__device__ __forceinline__ double ceil_r(double x) { return ceil(x); }
__device__ __forceinline__ float ceil_r(float x) { return ceilf(x); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fabs_r(double x) { return fabs(x); }
__device__ __forceinline__ float fabs_r(float x) { return fabsf(x); }

// g1(z), g2(z) for z > 0 from the table T (layout of Tab<R>).
template <typename R>
__device__ __forceinline__ void syn_g(const R *__restrict__ T, R z, R &g1, R &g2) {
  using C = Tab<R>;
  int e;
  R m;
  split_binade(z, e, m);
  if (e < C::EMIN) {
    // two-term series (the next terms are O(z^{4/3}) relative)
    R z23 = cbrt_r(z * z);
    g1 = __ldg(T + 0) - __ldg(T + 2) * z23;
    g2 = __ldg(T + 1);
    return;
  }
  if (e >= C::EMAX) { g1 = R(0); g2 = R(0); return; }
  R u = (m - R(1)) * R(C::S);
  int s = (int)u;
  s = s > C::S - 1 ? C::S - 1 : s;
  R t = R(2) * (u - R(s)) - R(1);
  const R *c1 = T + C::kHeader + (((e - C::EMIN) * C::S + s) * C::NC);
  const R *c2 = c1 + C::NB * C::S * C::NC;
  R a1 = __ldg(c1 + C::D), a2 = __ldg(c2 + C::D);
#pragma unroll
  for (int j = C::D - 1; j >= 0; --j) {
    a1 = fma_r(a1, t, __ldg(c1 + j));
    a2 = fma_r(a2, t, __ldg(c2 + j));
  }
  if (e >= 0) {
    R ez = exp_r(-z);
    a1 *= ez;
    a2 *= ez;
  }
  g1 = a1;
  g2 = a2;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products, with the key bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniforms strictly inside (0,1).  FP64: 52 bits (top 26 of two words);
// FP32: the top 23 bits of the first word.  Both add one half of the last
// unit, so every value is exact and neither 0 nor 1 occurs.
__device__ __forceinline__ double uniform_pair(unsigned a, unsigned b, double *) {
  return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 4503599627370496.0);
}
__device__ __forceinline__ float uniform_pair(unsigned a, unsigned, float *) {
  return ((float)(a >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// r1, r2 of the particle with this id at (step, sub-step, purpose).
template <typename R>
__device__ __forceinline__ void draw2(uint64_t id, unsigned step, unsigned sub, unsigned purpose,
                                      unsigned seed, R &r1, R &r2) {
  uint4 o = philox4x32_10(make_uint4(step, sub, purpose, seed),
                          make_uint2((unsigned)id, (unsigned)(id >> 32)));
  r1 = uniform_pair(o.x, o.y, (R *)nullptr);
  r2 = uniform_pair(o.z, o.w, (R *)nullptr);
}

// Id of a product: mixes the parent id, step, sub-step and the product's
// species, so ids (and the products' streams) do not depend on the order in
// which threads create them.
__device__ __forceinline__ uint64_t child_id(uint64_t parent, unsigned step, unsigned sub,
                                             unsigned kind, unsigned seed) {
  uint4 o = philox4x32_10(make_uint4(step, sub, kChild | (kind << 8), seed),
                          make_uint2((unsigned)parent, (unsigned)(parent >> 32)));
  return (uint64_t)o.x | ((uint64_t)o.y << 32);
}

// ---------------------------------------------------------------------------
template <typename R> struct V3 { R x, y, z; };

template <typename R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// chi of a lepton, Eq. (4): sqrt((gamma E + p x B)^2 - (p.E)^2), p in m c.
template <typename R>
__device__ __forceinline__ R chi_lepton(V3<R> p, R gamma, V3<R> E, V3<R> B) {
  V3<R> c = cross(p, B);
  R ax = gamma * E.x + c.x, ay = gamma * E.y + c.y, az = gamma * E.z + c.z;
  R pe = dot(p, E);
  R s = ax * ax + ay * ay + az * az - pe * pe;
  return s > R(0) ? sqrt_r(s) : R(0);
}

// H_eff of Eq. (3): sqrt((E + v x B)^2 - (p_hat . E)^2).
template <typename R>
__device__ __forceinline__ R heff_lepton(V3<R> p, R gamma, V3<R> E, V3<R> B) {
  R ig = R(1) / gamma;
  V3<R> v = {p.x * ig, p.y * ig, p.z * ig};
  V3<R> c = cross(v, B);
  R ax = E.x + c.x, ay = E.y + c.y, az = E.z + c.z;
  R pm = sqrt_r(dot(p, p));
  R pe = pm > R(0) ? dot(p, E) / pm : R(0);
  R s = ax * ax + ay * ay + az * az - pe * pe;
  return s > R(0) ? sqrt_r(s) : R(0);
}

// FP32 forms of chi, H_eff and the sub-interval count, with the hardware
// reciprocal square root, fast division and base-2 logarithm/exponential (a
// few ulp; the FP32 path is held to statistics and to 1e-5 between events):
// they decide sub-interval counts and probabilities, not the push itself.
// FP64 keeps the correctly rounded forms above.
__device__ __forceinline__ float sqrt_fast(float s) { return s > 0.f ? s * rsqrtf(s) : 0.f; }
template <>
__device__ __forceinline__ float chi_lepton<float>(V3<float> p, float gamma, V3<float> E, V3<float> B) {
  V3<float> c = cross(p, B);
  float ax = gamma * E.x + c.x, ay = gamma * E.y + c.y, az = gamma * E.z + c.z;
  float pe = dot(p, E);
  return sqrt_fast(ax * ax + ay * ay + az * az - pe * pe);
}
template <>
__device__ __forceinline__ float heff_lepton<float>(V3<float> p, float gamma, V3<float> E, V3<float> B) {
  const float ig = __fdividef(1.f, gamma);
  V3<float> v = {p.x * ig, p.y * ig, p.z * ig};
  V3<float> c = cross(v, B);
  float ax = E.x + c.x, ay = E.y + c.y, az = E.z + c.z;
  const float pp = dot(p, p);
  float pe = pp > 0.f ? dot(p, E) * rsqrtf(pp) : 0.f;
  return sqrt_fast(ax * ax + ay * ay + az * az - pe * pe);
}

// A photon's energy |p| and 1/|p| (0 for p = 0).  FP32: one reciprocal
// square root; FP64: correctly rounded square root and division.
__device__ __forceinline__ void photon_norm(const V3<float> &p, float &eps, float &ie) {
  const float pp = dot(p, p);
  ie = pp > 0.f ? rsqrtf(pp) : 0.f;
  eps = pp * ie;
}
__device__ __forceinline__ void photon_norm(const V3<double> &p, double &eps, double &ie) {
  eps = sqrt(dot(p, p));
  ie = eps > 0.0 ? 1.0 / eps : 0.0;
}

// H^gamma_eff of Eq. (32) for unit direction n.
template <typename R>
__device__ __forceinline__ R heff_photon(V3<R> n, V3<R> E, V3<R> B) {
  V3<R> c = cross(n, B);
  R ax = E.x + c.x, ay = E.y + c.y, az = E.z + c.z;
  R ne = dot(n, E);
  R s = ax * ax + ay * ay + az * az - ne * ne;
  return s > R(0) ? sqrt_r(s) : R(0);
}

// Sub-interval count (Sec. IV.H): N = ceil(t_span/dt_q) in [1, nmax], with
// dt_q from Eq. (28) for leptons and Eq. (33) for photons, scaled by kappa.
// (137/2pi)(lambda_C/c) = 137 and 130 (lambda_C/c) = 130*2pi in these units.
template <typename R>
__device__ __forceinline__ int nsub_lepton(R t_span, R gamma, R heff, R kappa, int nmax,
                                           int &capped) {
  capped = 0;
  if (!(heff > R(0))) return 1;
  R ih = R(1) / heff;
  R a = R(0.67) * cbrt_r(gamma) * cbrt_r(ih * ih);
  R b = R(2) * ih;
  R dtq = kappa * R(137) * (a < b ? a : b);
  R ratio = t_span / dtq;
  if (!(ratio > R(1))) return 1;
  R n = ceil_r(ratio);
  if (n > R(nmax)) { capped = 1; return nmax; }
  return (int)n;
}

template <>
__device__ __forceinline__ float heff_photon<float>(V3<float> n, V3<float> E, V3<float> B) {
  V3<float> c = cross(n, B);
  float ax = E.x + c.x, ay = E.y + c.y, az = E.z + c.z;
  float ne = dot(n, E);
  return sqrt_fast(ax * ax + ay * ay + az * az - ne * ne);
}

// FP32: (gamma / H^2)^(1/3) from one base-2 logarithm pair and exponential.
template <>
__device__ __forceinline__ int nsub_lepton<float>(float t_span, float gamma, float heff, float kappa, int nmax,
                                                  int &capped) {
  capped = 0;
  if (!(heff > 0.f)) return 1;
  const float ih = __fdividef(1.f, heff);
  const float a = 0.67f * exp2f((__log2f(gamma) - 2.f * __log2f(heff)) * (1.f / 3.f));
  const float b = 2.f * ih;
  const float dtq = kappa * 137.f * (a < b ? a : b);
  const float ratio = __fdividef(t_span, dtq);
  if (!(ratio > 1.f)) return 1;
  const float n = ceilf(ratio);
  if (n > (float)nmax) { capped = 1; return nmax; }
  return (int)n;
}

template <typename R>
__device__ __forceinline__ int nsub_photon(R t_span, R heff_g, R kappa, int nmax, int &capped) {
  capped = 0;
  if (!(heff_g > R(0))) return 1;
  R dtq = kappa * R(130.0 * kTwoPi) / heff_g;
  R ratio = t_span / dtq;
  if (!(ratio > R(1))) return 1;
  R n = ceil_r(ratio);
  if (n > R(nmax)) { capped = 1; return nmax; }
  return (int)n;
}

// Modified event generator, Eq. (25) with f_m = r1^3 (Sec. IV.G), written in
// terms of r1 so that no factor 1/delta appears:
//   3 r1^2 G(r1^3) = sqrt3/(2pi) chi (1-delta) 3 c [g1(z) + 1.5 chi delta z g2(z)],
//   z = (2/3) delta/(chi (1-delta)),  c = z^{1/3}/r1 = ((2/3)/(chi (1-delta)))^{1/3},
// and P_m = alpha h/gamma times that.
template <typename R>
__device__ __forceinline__ R prob_emit(const R *__restrict__ T, R r1, R chi, R gamma, R h) {
  if (!(chi > R(0))) return R(0);
  R delta = r1 * r1 * r1;
  R omd = R(1) - delta;
  if (!(omd > R(0))) return R(0);
  R c3 = R(2.0 / 3.0) / (chi * omd);
  R z = delta * c3;
  R g1, g2;
  syn_g(T, z, g1, g2);
  R br = g1 + R(1.5) * chi * delta * z * g2;
  return R(kAlpha) * h / gamma * R(kSqrt3Over2Pi) * chi * omd * R(3) * cbrt_r(c3) * br;
}

// Alternative event generator (Sec. IV.F): the density P(delta) of Eq. (24)
// itself at delta = r1,
//   P = alpha h/gamma sqrt3/(2pi) chi (1-delta)/delta z^{1/3} [g1 + 1.5 chi delta z g2].
template <typename R>
__device__ __forceinline__ R prob_alternative(const R *__restrict__ T, R delta, R chi, R gamma, R h) {
  if (!(chi > R(0)) || !(delta > R(0))) return R(0);
  R omd = R(1) - delta;
  if (!(omd > R(0))) return R(0);
  R z = R(2.0 / 3.0) * delta / (chi * omd);
  R g1, g2;
  syn_g(T, z, g1, g2);
  R br = g1 + R(1.5) * chi * delta * z * g2;
  return R(kAlpha) * h / gamma * R(kSqrt3Over2Pi) * chi * omd / delta * cbrt_r(z) * br;
}

// Standard event generator (Sec. IV.F) from tables built in FP64 at init:
// rows j = 0 .. kStdRows-1 at ln chi_j = kStdLnChiLo + j kStdDLn, each the
// normalised cumulative W(s^3)/W(1) at s = i/(kStdCols-1) (s = delta^{1/3},
// so delta_min -> 0 needs no cutoff), and ln W(1) per row.  Interpolation
// is linear in ln chi and in s.  Below the table, chi < chi_lo, the
// spectrum depends on delta/chi only and W(1) grows as chi: both are scaled
// from the first row.  Above it the last row is used.
constexpr int kStdRows = 4097, kStdCols = 1025;
constexpr double kStdLnChiLo = -13.815510557964274;   // ln 1e-6
constexpr double kStdDLn = 23.025850929940457 / 4096; // up to chi = 1e4

template <typename R>
__device__ __forceinline__ void std_row(R chi, int &j, R &f, R &scale) {
  R lx = (log_r(chi) - R(kStdLnChiLo)) * R(1.0 / kStdDLn);
  scale = R(1);
  if (!(lx >= R(0))) {
    scale = chi * R(1.0e6);          // chi / chi_lo
    lx = R(0);
  }
  if (lx > R(kStdRows - 1)) lx = R(kStdRows - 1);
  j = (int)lx;
  if (j > kStdRows - 2) j = kStdRows - 2;
  f = lx - R(j);
}

// Total probability W(1) of an interval h: alpha h/gamma times the table's W.
template <typename R>
__device__ __forceinline__ R std_total(const R *__restrict__ lnw, R chi, R gamma, R h) {
  if (!(chi > R(0))) return R(0);
  int j;
  R f, sc;
  std_row(chi, j, f, sc);
  const R l = lnw[j] + f * (lnw[j + 1] - lnw[j]);
  return R(kAlpha) * h / gamma * exp_r(l) * sc;
}

// Photon energy: the root of W(delta)/W(1) = u.  Bisection over the s grid
// finds the cell; inside it two Newton steps on
//   C(s) = C(s_lo) + int_{s_lo}^{s} f(t) dt / W(1),   f(t) = 3 t^2 G(t^3, chi),
// with the integral by Simpson's rule and f from the synchrotron tables,
// replace linear interpolation (which is poor where C flattens, delta -> 1).
template <typename R>
__device__ __noinline__ R std_delta(const R *__restrict__ T, const R *__restrict__ cdf, const R *__restrict__ lnw,
                                    R chi, R u) {
  int j;
  R f, sc;
  std_row(chi, j, f, sc);
  const R *a = cdf + (size_t)j * kStdCols, *b = a + kStdCols;
  int lo = 0, hi = kStdCols - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    const R c = a[mid] + f * (b[mid] - a[mid]);
    if (c <= u) lo = mid; else hi = mid;
  }
  const R clo = a[lo] + f * (b[lo] - a[lo]), chi_ = a[hi] + f * (b[hi] - a[hi]);
  const R ds = R(1.0 / (kStdCols - 1));
  const R slo = R(lo) * ds, shi = R(hi) * ds;
  R s = slo + (chi_ > clo ? (u - clo) / (chi_ - clo) : R(0)) * ds;
  // the shape below the table is the first row's (chi_lo)
  const R chi_e = sc != R(1) ? R(1.0e-6) : chi;
  const R w1 = exp_r(lnw[j] + f * (lnw[j + 1] - lnw[j]));
  const R unit = R(1) / R(kAlpha);       // prob_emit(T, t, chi, 1, 1/alpha) = f(t)
  for (int it = 0; it < 2; ++it) {
    const R fm = prob_emit(T, R(0.5) * (slo + s), chi_e, R(1), unit);
    const R fs = prob_emit(T, s, chi_e, R(1), unit);
    const R f0 = prob_emit(T, slo, chi_e, R(1), unit);
    const R c = clo + (s - slo) * (f0 + R(4) * fm + fs) * R(1.0 / 6.0) / w1;
    if (!(fs > R(0))) break;
    R sn = s - (c - u) * w1 / fs;
    sn = sn < slo ? slo : (sn > shi ? shi : sn);
    s = sn;
  }
  return s * s * s * sc;
}

// The standard generator in FP64 at the particle's own chi, without tables
// in chi: W(x) = int_0^{x^(1/3)} f(s) ds with f(s) = 3 s^2 G(s^3, chi) (the
// modified generator's density; no cutoff is needed in s = delta^(1/3)),
// summed over kStdPanels panels of equal width in s, each by 8-point
// Gauss-Legendre (the roots of P_8 and their weights, to 20 digits).  The root of
// W(delta) = u W(1) lies in the first panel where the running sum reaches
// u W(1); inside it a safeguarded Newton iteration on the partial panel
// integral converges to the last bit of s.
constexpr int kStdPanels = 256;

__device__ __forceinline__ double std_f(const double *__restrict__ T, double s, double chi) {
  return prob_emit(T, s, chi, 1.0, 1.0 / kAlpha);
}

static __device__ __noinline__ double std_gl8(const double *__restrict__ T, double chi, double a, double b) {
  const double x[4] = {0.18343464249564980494, 0.52553240991632898582, 0.79666647741362673959,
                       0.96028985649753623168};
  const double w[4] = {0.36268378337836198297, 0.31370664587788728734, 0.22238103445337447054,
                       0.10122853629037625915};
  const double m = 0.5 * (a + b), r = 0.5 * (b - a);
  double acc = 0.0;
#pragma unroll
  for (int k = 3; k >= 0; --k) acc += w[k] * (std_f(T, m - r * x[k], chi) + std_f(T, m + r * x[k], chi));
  return r * acc;
}

// W(1) / (alpha h / gamma) at chi.
static __device__ __noinline__ double std_total_exact(const double *__restrict__ T, double chi) {
  double acc = 0.0;
  for (int k = 0; k < kStdPanels; ++k)
    acc += std_gl8(T, chi, (double)k / kStdPanels, (double)(k + 1) / kStdPanels);
  return acc;
}

// delta with W(delta) = u W(1) at chi.
static __device__ __noinline__ double std_delta_exact(const double *__restrict__ T, double chi, double u) {
  const double target = u * std_total_exact(T, chi);
  double below = 0.0;
  int k = 0;
  for (; k < kStdPanels - 1; ++k) {
    const double pk = std_gl8(T, chi, (double)k / kStdPanels, (double)(k + 1) / kStdPanels);
    if (!(below + pk < target)) break;
    below += pk;
  }
  const double a = (double)k / kStdPanels;
  double lo = a, hi = (double)(k + 1) / kStdPanels, s = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double g = below + std_gl8(T, chi, a, s) - target;
    if (g < 0.0) lo = s; else hi = s;
    const double fs = std_f(T, s, chi);
    double sn = fs > 0.0 ? s - g / fs : 0.5 * (lo + hi);
    if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
    if (sn == s || hi - lo <= 0x1p-53 * hi) { s = sn; break; }
    s = sn;
  }
  return s * s * s;
}

// Pair generator, Eq. (30), with (3/2) chi_g z_p = 1/(de (1-de)):
//   P_p = alpha h sqrt3/(2pi) (chi_g/eps) z^{1/3} [g2(z) - de(1-de) g1(z)].
template <typename R>
__device__ __forceinline__ R prob_pair(const R *__restrict__ T, R de, R chig, R eps, R h) {
  if (!(chig > R(0)) || !(eps > R(0))) return R(0);
  R d = de * (R(1) - de);
  if (!(d > R(0))) return R(0);
  R z = R(2.0 / 3.0) / (chig * d);
  R g1, g2;
  syn_g(T, z, g1, g2);
  return R(kAlpha) * h * R(kSqrt3Over2Pi) * (chig / eps) * cbrt_r(z) * (g2 - d * g1);
}

// gamma = sqrt(1 + p^2/m^2) and 1/(m gamma) of a momentum p (units m_e c) of
// a particle of mass m (units m_e), from 1/m^2 and 1/m.  FP32: one
// reciprocal square root (a few ulp; the FP32 path is held to 1e-5 between
// events); FP64: correctly rounded square root and division.
__device__ __forceinline__ void lorentz(const V3<float> &p, float inv_m, float inv_m2, float &g, float &ig_m) {
  const float x = 1.0f + (p.x * p.x + p.y * p.y + p.z * p.z) * inv_m2;
  const float r = rsqrtf(x);
  g = x * r;
  ig_m = inv_m * r;
}
__device__ __forceinline__ void lorentz(const V3<double> &p, double inv_m, double inv_m2, double &g, double &ig_m) {
  g = sqrt(1.0 + (p.x * p.x + p.y * p.y + p.z * p.z) * inv_m2);
  ig_m = inv_m / g;
}

// Boris push (Appendix A): half E, rotation by B, half E.  The generic form;
// FP32 and FP64 use the specialisations below.
template <typename R>
__device__ __forceinline__ void boris(V3<R> &p, V3<R> E, V3<R> B, R q, R m, R h) {
  R a = R(0.5) * q * h;
  V3<R> um = {p.x + a * E.x, p.y + a * E.y, p.z + a * E.z};
  R gm = sqrt_r(R(1) + dot(um, um) / (m * m));
  R f = a / (m * gm);
  V3<R> t = {f * B.x, f * B.y, f * B.z};
  R k = R(2) / (R(1) + dot(t, t));
  V3<R> s = {k * t.x, k * t.y, k * t.z};
  V3<R> c1 = cross(um, t);
  V3<R> up = {um.x + c1.x, um.y + c1.y, um.z + c1.z};
  V3<R> c2 = cross(up, s);
  p = {um.x + c2.x + a * E.x, um.y + c2.y + a * E.y, um.z + c2.z + a * E.z};
}

// FP32: 1/gamma from one reciprocal square root and the rotation factor
// 2/(1 + t^2) from a fast division (a few ulp each: the rotation then keeps
// |p| to ~1e-7 per push, with random sign), no other division.
template <>
__device__ __forceinline__ void boris<float>(V3<float> &p, V3<float> E, V3<float> B, float q, float m, float h) {
  const float a = 0.5f * q * h;
  const V3<float> um = {p.x + a * E.x, p.y + a * E.y, p.z + a * E.z};
  const float im = __frcp_rn(m);
  const float f = a * im * rsqrtf(1.0f + dot(um, um) * im * im);
  const V3<float> t = {f * B.x, f * B.y, f * B.z};
  const float k = __fdividef(2.0f, 1.0f + dot(t, t));
  const V3<float> sv = {k * t.x, k * t.y, k * t.z};
  const V3<float> c1 = cross(um, t);
  const V3<float> up = {um.x + c1.x, um.y + c1.y, um.z + c1.z};
  const V3<float> c2 = cross(up, sv);
  p = {um.x + c2.x + a * E.x, um.y + c2.y + a * E.y, um.z + c2.z + a * E.z};
}

// FP64: every product, sum and quotient rounded on its own (the _rn
// intrinsics are never contracted into FMAs), in a fixed order -- sums left
// to right, s = 2t / (1 + t^2) -- so that the push is a function of (p, E,
// B, q, m, h) alone, exact to the last bit of IEEE binary64 arithmetic.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dot_rn(V3<double> a, V3<double> b) {
  return add_rn(add_rn(mul_rn(a.x, b.x), mul_rn(a.y, b.y)), mul_rn(a.z, b.z));
}
__device__ __forceinline__ V3<double> cross_rn(V3<double> a, V3<double> b) {
  return {sub_rn(mul_rn(a.y, b.z), mul_rn(a.z, b.y)), sub_rn(mul_rn(a.z, b.x), mul_rn(a.x, b.z)),
          sub_rn(mul_rn(a.x, b.y), mul_rn(a.y, b.x))};
}

template <>
__device__ __forceinline__ void boris<double>(V3<double> &p, V3<double> E, V3<double> B, double q, double m,
                                              double h) {
  const double a = mul_rn(mul_rn(0.5, q), h);
  const V3<double> um = {add_rn(p.x, mul_rn(a, E.x)), add_rn(p.y, mul_rn(a, E.y)), add_rn(p.z, mul_rn(a, E.z))};
  const double gm = __dsqrt_rn(add_rn(1.0, __ddiv_rn(dot_rn(um, um), mul_rn(m, m))));
  const double f = __ddiv_rn(a, mul_rn(m, gm));
  const V3<double> t = {mul_rn(f, B.x), mul_rn(f, B.y), mul_rn(f, B.z)};
  const double den = add_rn(1.0, dot_rn(t, t));
  const V3<double> sv = {__ddiv_rn(mul_rn(2.0, t.x), den), __ddiv_rn(mul_rn(2.0, t.y), den),
                         __ddiv_rn(mul_rn(2.0, t.z), den)};
  const V3<double> c1 = cross_rn(um, t);
  const V3<double> up = {add_rn(um.x, c1.x), add_rn(um.y, c1.y), add_rn(um.z, c1.z)};
  const V3<double> c2 = cross_rn(up, sv);
  p = {add_rn(add_rn(um.x, c2.x), mul_rn(a, E.x)), add_rn(add_rn(um.y, c2.y), mul_rn(a, E.y)),
       add_rn(add_rn(um.z, c2.z), mul_rn(a, E.z))};
}

}  // namespace qed
