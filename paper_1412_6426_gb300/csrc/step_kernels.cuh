// Kernels of the particle step, shared by two translation units: step.cu
// instantiates them for the plain method, step_ext.cu (EXT = true) for runs
// with independent ensembles or the generator factors of Sec. VI, so that
// the plain kernels keep their register budget.
#pragma once
#include <cmath>

#include "qed_internal.h"

namespace qed {
namespace {

// Working state of one particle during the step: unbounded per-axis cell
// coordinates plus offsets in [0,1).
template <typename R> struct Pt {
  int ci[3];
  R off[3];
  V3<R> p;
  R w;
  uint64_t id;
};

// A product waiting to evolve for the rest of the step.  Its id is formed
// by the pass that takes it (product_id of the parent's id, the sub-interval
// of its birth and its kind), out of the parent's sub-interval loop.
template <typename R> struct Pend {
  R off[3];
  R w;
  V3<R> p;
  R trem;
  V3<R> E, B;
  int ci[3];
  int sp;
  uint64_t parent;
  unsigned sub, kind;
};

// Per-thread counts of the frequent events, summed per warp at the end of a
// kernel.  Rare events (P > 1, capped intervals, absorbed particles,
// overflows, non-finite values) go straight to the global counters, so that
// this struct stays small enough to live in registers.
struct Cnt {
  unsigned sub_l = 0, sub_g = 0;       // sub-intervals of leptons, of photons
  unsigned psteps[4] = {0, 0, 0, 0};   // live particles advanced, per species
  unsigned emis = 0, pairs = 0;
  unsigned made_ph = 0, made_pair = 0;   // products made (all N_g samples, after the 1/f_g keep)
};

template <typename R>
__device__ __forceinline__ void count_rare(const StepArgs<R> &a, int counter, unsigned v) {
  if (v) atomicAdd(a.counters + counter, (unsigned long long)v);
}

// ----- store access --------------------------------------------------------
__device__ __forceinline__ void load(const StepArgs<float> &a, int sp, long long i, Pt<float> &q,
                                     int &cell) {
  float4 P = __ldg((const float4 *)a.pos[sp] + i);
  float4 M = __ldg((const float4 *)a.mom[sp] + i);
  q.off[0] = P.x; q.off[1] = P.y; q.off[2] = P.z; q.w = P.w;
  q.p = {M.x, M.y, M.z};
  cell = __float_as_int(M.w);
}
__device__ __forceinline__ void load(const StepArgs<double> &a, int sp, long long i, Pt<double> &q,
                                     int &cell) {
  const double2 *P = (const double2 *)a.pos[sp] + 2 * i;
  const double2 *M = (const double2 *)a.mom[sp] + 2 * i;
  double2 p0 = __ldg(P), p1 = __ldg(P + 1), m0 = __ldg(M), m1 = __ldg(M + 1);
  q.off[0] = p0.x; q.off[1] = p0.y; q.off[2] = p1.x; q.w = p1.y;
  q.p = {m0.x, m0.y, m1.x};
  cell = (int)m1.y;
}
__device__ __forceinline__ void unpack(const float4 &P, const float4 &M, Pt<float> &q, int &cell) {
  q.off[0] = P.x; q.off[1] = P.y; q.off[2] = P.z; q.w = P.w;
  q.p = {M.x, M.y, M.z};
  cell = __float_as_int(M.w);
}
template <typename H>
__device__ __forceinline__ void unpack(const H &P, const H &M, Pt<double> &q, int &cell) {
  q.off[0] = P.a.x; q.off[1] = P.a.y; q.off[2] = P.b.x; q.w = P.b.y;
  q.p = {M.a.x, M.a.y, M.b.x};
  cell = (int)M.b.y;
}
__device__ __forceinline__ void store(const StepArgs<float> &a, int sp, long long i,
                                      const Pt<float> &q, int cell, bool with_id) {
  ((float4 *)a.pos[sp])[i] = make_float4(q.off[0], q.off[1], q.off[2], q.w);
  ((float4 *)a.mom[sp])[i] = make_float4(q.p.x, q.p.y, q.p.z, __int_as_float(cell));
  if (with_id) a.id[sp][i] = q.id;
}
__device__ __forceinline__ void store_pos(const StepArgs<float> &a, int sp, long long i, const Pt<float> &q) {
  ((float4 *)a.pos[sp])[i] = make_float4(q.off[0], q.off[1], q.off[2], q.w);
}
__device__ __forceinline__ void store_pos(const StepArgs<double> &a, int sp, long long i, const Pt<double> &q) {
  double2 *P = (double2 *)a.pos[sp] + 2 * i;
  P[0] = make_double2(q.off[0], q.off[1]);
  P[1] = make_double2(q.off[2], q.w);
}
__device__ __forceinline__ void store(const StepArgs<double> &a, int sp, long long i,
                                      const Pt<double> &q, int cell, bool with_id) {
  double2 *P = (double2 *)a.pos[sp] + 2 * i;
  double2 *M = (double2 *)a.mom[sp] + 2 * i;
  P[0] = make_double2(q.off[0], q.off[1]);
  P[1] = make_double2(q.off[2], q.w);
  M[0] = make_double2(q.p.x, q.p.y);
  M[1] = make_double2(q.p.z, (double)cell);
  if (with_id) a.id[sp][i] = q.id;
}

// Smallest uniform the generators can draw (r2 > this always).
__device__ __forceinline__ double r2_floor(double) { return 0x1p-53; }
__device__ __forceinline__ float r2_floor(float) { return 0x1p-24f; }

// ----- fields --------------------------------------------------------------
// Per-step constants of the analytic fields, formed once per block in FP64
// by one thread, so that the per-particle FP32 work needs no FP64 at all.
struct alignas(8) StepConst {
  double ud[6];              // uniform / rotating: E and B
  float uf[6];
  // Gaussian pulse: carrier phase in cycles = frac(c0 + i * kfix) + off * kf,
  // with c0 and kfix fractions of a cycle in 64-bit fixed point, so the
  // cell-index term is exact whatever the size of the lattice
  unsigned long long c0, kfix;
  float kf;                  // omega dx / 2 pi (cycles per cell)
  float eta0, zeta0;         // eta = eta0 + x_rel, zeta = zeta0 - x_rel
  float y0, z0;              // offsets of the lattice origin from the focus
  float zr, inv_zr;          // Rayleigh length and its inverse
  float inv_w0sq;            // 1 / w0^2
  float curv;                // -omega / (4 pi): curvature phase in cycles per r^2/R
  float env_k;               // -2 ln 2 / tau^2
  float amp0, phi0_cyc;      // E0 and the phase offset in cycles
  // Bound on a photon's effective field anywhere in this step and whether a
  // photon that cannot pair (eps hmax < chi*) may take the straight flight:
  // analytic fields, when every H <= hmax gives one sub-interval (the
  // flight is then the general path's bit for bit); the Yee mesh, when no
  // H <= hmax caps the sub-intervals (the flight then differs from N
  // sub-interval moves by rounding only, and no field is gathered).
  double hmax;
  float hmax_f;              // hmax rounded up, for the FP32 comparison
  int one_interval;
  // the step's start time and index (they key the random streams)
  double t;
  unsigned step;
  unsigned pad_;
};

// Device clock, advanced by the first kernel of every step.
struct Clock {
  double t;
  long long step;
};

__device__ __forceinline__ unsigned long long cycles_fixed(double cyc) {
  cyc -= floor(cyc);
  if (!(cyc < 1.0)) cyc = 0.0;
  return __double2ull_rn(ldexp(cyc, 64) > 1.8446744073709550e19 ? 0.0 : ldexp(cyc, 64));
}

// Largest chi_g for which no pair draw can succeed when the sub-interval is
// not capped: there h <= dt_q = kappa 130 (2 pi)/H, so P_p is at most
// sqrt3/(2pi) alpha kappa 130 (2 pi) F2(z_min) = 1.6431 kappa F2(z_min),
// z_min = 8/(3 chi_g).  z* solves 3.2862 kappa F2(z*) = r2_floor / 2 on the
// decreasing branch of F2 (beyond its maximum at 0.4169), by bisection on the
// table (a factor 4 of margin); chi* = 8/(3 z*).
template <typename R>
__device__ double photon_chi_star(const R *tab, double kappa) {
  const double target = 0.5 * (double)r2_floor(R(0)) / (3.2862 * kappa);
  if (!(target < 0.6)) return 0.0;
  double lo = 0.4169, hi = 740.0;    // F2(lo) > target >= F2(hi)
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    R g1, g2;
    syn_g(tab, (R)mid, g1, g2);
    const double f2 = cbrt(mid) * (double)g2;
    if (f2 > target) lo = mid; else hi = mid;
  }
  return 8.0 / (3.0 * hi);
}

template <typename R>
__device__ void step_constants(const StepArgs<R> &a, StepConst &k) {
  const Clock *clk = (const Clock *)a.clock;
  k.t = clk->t;
  k.step = (unsigned)clk->step;
  // H^g_eff = |E + n x B|_perp <= |E| + |B| (Eq. (32))
  k.hmax = INFINITY;
  if (a.field_mode == kFieldUniform)
    k.hmax = sqrt(a.fp[0] * a.fp[0] + a.fp[1] * a.fp[1] + a.fp[2] * a.fp[2]) +
             sqrt(a.fp[3] * a.fp[3] + a.fp[4] * a.fp[4] + a.fp[5] * a.fp[5]);
  else if (a.field_mode == kFieldRotatingE)
    k.hmax = fabs(a.fp[0]);
  else if (a.field_mode == kFieldStandingWave)
    // |E| + |B| = |E0| (|sin wx cos wt| + |cos wx sin wt|) <= |E0| (Cauchy-Schwarz)
    k.hmax = fabs(a.fp[0]);
  else if (a.field_mode == kFieldGaussianLP)
    k.hmax = 2.0 * fabs(a.fp[0]);             // |E| = |B| <= E0 everywhere
  else if (a.field_mode == kFieldEnsemble)
    k.hmax = a.ens_hmax;
  else if (a.field_mode == kFieldGrid && a.grid_max) {
    // CIC weights are a convex combination: |E| <= |(max|Ex|, max|Ey|, max|Ez|)|
    double m[6];
    for (int c = 0; c < 6; ++c) m[c] = sizeof(R) == 4 ? (double)__uint_as_float((unsigned)a.grid_max[c])
                                                       : __longlong_as_double((long long)a.grid_max[c]);
    k.hmax = (sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) + sqrt(m[3] * m[3] + m[4] * m[4] + m[5] * m[5])) *
             (1.0 + 1e-6);
    // compaction groups the photons that cannot pair (two-class split)
    if (a.eps_star_out) *a.eps_star_out = k.hmax > 0.0 ? 0.999 * (*a.chi_star) / k.hmax : 0.0;
  }
  // N = ceil(dt H / (kappa 130 2 pi)) is 1 for every H <= hmax (margin 1e-3);
  // on the mesh: N stays below nsub_max for every H <= hmax
  if (a.field_mode == kFieldGrid)
    k.one_interval = (double)a.dt * k.hmax <= 0.999 * (double)a.nsub_max * (double)a.kappa * 130.0 * kTwoPi;
  else
    k.one_interval = (double)a.dt * k.hmax <= 0.999 * (double)a.kappa * 130.0 * kTwoPi;
  k.hmax_f = (float)(k.hmax * 1.00001);
  for (int c = 0; c < 6; ++c) k.ud[c] = 0.0;
  if (a.field_mode == kFieldUniform) {
    for (int c = 0; c < 6; ++c) k.ud[c] = a.fp[c];
  } else if (a.field_mode == kFieldRotatingE) {
    double cyc = a.fp[1] * k.t * (1.0 / kTwoPi);
    double f = cyc - rint(cyc), s, c;
    sincospi(2.0 * f, &s, &c);
    k.ud[0] = a.fp[0] * c;
    k.ud[1] = a.fp[0] * s;
  } else if (a.field_mode == kFieldStandingWave) {
    // amplitudes of E_y (times sin wx) and B_z (times cos wx) at this step
    double cyc = a.fp[1] * k.t * (1.0 / kTwoPi);
    double f = cyc - rint(cyc), s, c;
    sincospi(2.0 * f, &s, &c);
    k.ud[1] = a.fp[0] * c;
    k.ud[5] = -a.fp[0] * s;
    // FP32 phase of wx in cycles, lattice part in 64-bit fixed point
    k.c0 = cycles_fixed(a.fp[1] * a.x0[0] * (1.0 / kTwoPi));
    const double K = a.fp[1] * a.dd[0] * (1.0 / kTwoPi);
    k.kfix = cycles_fixed(K);
    k.kf = (float)K;
  } else if (a.field_mode == kFieldGaussianLP) {
    double T0 = (k.t - a.fp[7]) - a.fp[4] + a.x0[0];
    k.c0 = cycles_fixed(a.fp[1] * T0 * (1.0 / kTwoPi));
    double K = a.fp[1] * a.dd[0] * (1.0 / kTwoPi);
    k.kfix = cycles_fixed(K);
    k.kf = (float)K;
    k.eta0 = (float)T0;
    k.zeta0 = (float)(a.fp[4] - a.x0[0]);
    k.y0 = (float)(a.x0[1] - a.fp[5]);
    k.z0 = (float)(a.x0[2] - a.fp[6]);
    const double zr = 0.5 * a.fp[1] * a.fp[2] * a.fp[2];
    k.zr = (float)zr;
    k.inv_zr = (float)(1.0 / zr);
    k.inv_w0sq = (float)(1.0 / (a.fp[2] * a.fp[2]));
    k.curv = (float)(-0.5 * a.fp[1] / kTwoPi);
    k.env_k = (float)(-2.0 * 0.6931471805599453 / (a.fp[3] * a.fp[3]));
    k.amp0 = (float)a.fp[0];
    k.phi0_cyc = (float)(a.fp[8] / kTwoPi);
  }
  for (int c = 0; c < 6; ++c) k.uf[c] = (float)k.ud[c];
}

// Analytic fields at the particle position and the step's time (modes of qed.h).
// FP32: no FP64 instruction; the carrier phase comes from StepConst.
__device__ void field_analytic(const StepArgs<float> &a, const StepConst &k, const Pt<float> &q,
                               V3<float> &E, V3<float> &B) {
  if (a.field_mode == kFieldStandingWave) {
    const unsigned long long ph = k.c0 + (unsigned long long)(unsigned)q.ci[0] * k.kfix;
    float cyc = (float)(unsigned)(ph >> 32) * 2.3283064365386963e-10f + q.off[0] * k.kf;
    cyc -= rintf(cyc);
    float s, c;
    sincospif(2.f * cyc, &s, &c);
    E = {0.f, k.uf[1] * s, 0.f};
    B = {0.f, 0.f, k.uf[5] * c};
    return;
  }
  if (a.field_mode != kFieldGaussianLP) {
    E = {k.uf[0], k.uf[1], k.uf[2]};
    B = {k.uf[3], k.uf[4], k.uf[5]};
    return;
  }
  E = {0.f, 0.f, 0.f};
  B = {0.f, 0.f, 0.f};
  const float xr = ((float)q.ci[0] + q.off[0]) * a.d[0];
  const float zeta = k.zeta0 - xr, eta = k.eta0 + xr;
  const float y = k.y0 + ((float)q.ci[1] + q.off[1]) * a.d[1];
  const float z = k.z0 + ((float)q.ci[2] + q.off[2]) * a.d[2];
  const float rz = zeta * k.inv_zr;
  const float rs = rsqrtf(1.f + rz * rz);        // w0 / w(zeta)
  const float iq = rs * rs;                      // w0^2 / w(zeta)^2
  const float r2 = y * y + z * z;
  const float invR = rz * k.inv_zr * iq;         // zeta / (zeta^2 + zr^2)
  const unsigned long long ph = k.c0 + (unsigned long long)(unsigned)q.ci[0] * k.kfix;
  float cyc = (float)(unsigned)(ph >> 32) * 2.3283064365386963e-10f + q.off[0] * k.kf +
              k.curv * r2 * invR + atanf(rz) * 0.15915494309189535f + k.phi0_cyc;
  cyc -= rintf(cyc);
  float s, c;
  sincospif(2.f * cyc, &s, &c);
  const float amp = k.amp0 * rs * __expf(-r2 * k.inv_w0sq * iq + k.env_k * eta * eta);
  E.y = amp * c;
  B.z = -E.y;
}

// FP64: the same fields with every quantity in FP64.
__device__ void field_analytic(const StepArgs<double> &a, const StepConst &k, const Pt<double> &q,
                               V3<double> &E, V3<double> &B) {
  if (a.field_mode == kFieldStandingWave) {
    const double xa = a.x0[0] + ((double)q.ci[0] + q.off[0]) * a.dd[0];
    double s, c;
    sincos(a.fp[1] * xa, &s, &c);
    E = {0.0, k.ud[1] * s, 0.0};
    B = {0.0, 0.0, k.ud[5] * c};
    return;
  }
  if (a.field_mode != kFieldGaussianLP) {
    E = {k.ud[0], k.ud[1], k.ud[2]};
    B = {k.ud[3], k.ud[4], k.ud[5]};
    return;
  }
  E = {0.0, 0.0, 0.0};
  B = {0.0, 0.0, 0.0};
  // zeta: distance travelled past the focus along -x; eta: retarded time
  const double xa = a.x0[0] + ((double)q.ci[0] + q.off[0]) * a.dd[0];
  const double zeta = a.fp[4] - xa;
  const double eta = (k.t - a.fp[7]) - zeta;
  const double y = a.x0[1] - a.fp[5] + ((double)q.ci[1] + q.off[1]) * a.dd[1];
  const double z = a.x0[2] - a.fp[6] + ((double)q.ci[2] + q.off[2]) * a.dd[2];
  const double w = a.fp[1], w0 = a.fp[2], tau = a.fp[3];
  const double zr = 0.5 * w * w0 * w0;
  const double rz = zeta / zr;
  const double wz2 = w0 * w0 * (1.0 + rz * rz);
  const double r2 = y * y + z * z;
  const double invR = zeta / (zeta * zeta + zr * zr);
  const double phase = w * eta - 0.5 * w * r2 * invR + atan(rz) + a.fp[8];
  const double env = exp(-2.0 * 0.6931471805599453 * eta * eta / (tau * tau));
  const double amp = a.fp[0] * sqrt(w0 * w0 / wz2) * exp(-r2 / wz2) * env;
  E.y = amp * cos(phase);
  B.z = -E.y;
}

// Ensemble mode: the field of the particle's ensemble at the step's time,
// evaluated once per step by k_step_constants.
template <typename R>
__device__ __forceinline__ void field_ensemble(const StepArgs<R> &a, uint64_t id, V3<R> &E, V3<R> &B) {
  const unsigned long long e = a.ens_shift >= 64 ? 0ull : (unsigned long long)(id >> a.ens_shift);
  if (e >= (unsigned long long)a.n_ens) {
    E = {R(0), R(0), R(0)};
    B = {R(0), R(0), R(0)};
    return;
  }
  const R *f = a.ens_field + e * kEnsFieldStride;
  E = {__ldg(f), __ldg(f + 1), __ldg(f + 2)};
  B = {__ldg(f + 3), __ldg(f + 4), __ldg(f + 5)};
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// CIC gather of one staggered component (stagger sx, sy, sz in {0, 1/2}).
// wrapi for an index that is almost always in range already (one compare).
__device__ __forceinline__ int wrap_fast(int i, int n) { return (unsigned)i < (unsigned)n ? i : wrapi(i, n); }

// CIC weights along one axis for a component at stagger 0 or 1/2: the lower
// node (wrapped), the upper node (wrapped) and the fraction towards it.
template <typename R> struct Axis {
  int i0, i1;
  R fr;
};

template <typename R>
__device__ __forceinline__ Axis<R> cic_axis(int ci, R off, bool half, int n) {
  if (!half) return {ci, ci + 1 == n ? 0 : ci + 1, off};   // off in [0, 1): nodes ci, ci + 1
  R v = off - R(0.5);
  int b = ci;
  if (v < R(0)) { v += R(1); b -= 1; }
  return {wrap_fast(b, n), wrap_fast(b + 1, n), v};
}

// Node indices in 32 bits (the mesh holds fewer than 2^31 cells): one
// multiply-add forms each load's address.  The trilinear weights are
// applied as nested linear interpolations (four along x, two along y, one
// along z: a + f (b - a) each), 14 operations instead of the 8 weight
// products and 8 multiply-adds.
template <typename R>
__device__ __forceinline__ R cic(const R *__restrict__ f, const Axis<R> &x, const Axis<R> &y, const Axis<R> &z,
                                 unsigned nx, unsigned nxy) {
  const unsigned r00 = z.i0 * nxy + y.i0 * nx, r01 = z.i0 * nxy + y.i1 * nx;
  const unsigned r10 = z.i1 * nxy + y.i0 * nx, r11 = z.i1 * nxy + y.i1 * nx;
  const unsigned x0 = (unsigned)x.i0, x1 = (unsigned)x.i1;
  const R f000 = __ldg(f + (r00 + x0)), f100 = __ldg(f + (r00 + x1));
  const R f010 = __ldg(f + (r01 + x0)), f110 = __ldg(f + (r01 + x1));
  const R f001 = __ldg(f + (r10 + x0)), f101 = __ldg(f + (r10 + x1));
  const R f011 = __ldg(f + (r11 + x0)), f111 = __ldg(f + (r11 + x1));
  const R a0 = fma_r(x.fr, f100 - f000, f000), a1 = fma_r(x.fr, f110 - f010, f010);
  const R a2 = fma_r(x.fr, f101 - f001, f001), a3 = fma_r(x.fr, f111 - f011, f011);
  const R b0 = fma_r(y.fr, a1 - a0, a0), b1 = fma_r(y.fr, a3 - a2, a2);
  return fma_r(z.fr, b1 - b0, b0);
}

// CIC gather of the six staggered components (Yee positions in qed.h); the
// per-axis nodes and fractions of both staggers are formed once.
template <typename R>
__device__ void gather_grid(const StepArgs<R> &a, const Pt<R> &q, V3<R> &E, V3<R> &B) {
  const Axis<R> x0 = cic_axis(q.ci[0], q.off[0], false, a.n[0]), xh = cic_axis(q.ci[0], q.off[0], true, a.n[0]);
  const Axis<R> y0 = cic_axis(q.ci[1], q.off[1], false, a.n[1]), yh = cic_axis(q.ci[1], q.off[1], true, a.n[1]);
  const Axis<R> z0 = cic_axis(q.ci[2], q.off[2], false, a.n[2]), zh = cic_axis(q.ci[2], q.off[2], true, a.n[2]);
  const unsigned nx = a.n[0], nxy = (unsigned)a.n[0] * a.n[1];
  E.x = cic(a.E[0], xh, y0, z0, nx, nxy);
  E.y = cic(a.E[1], x0, yh, z0, nx, nxy);
  E.z = cic(a.E[2], x0, y0, zh, nx, nxy);
  B.x = cic(a.B[0], x0, yh, zh, nx, nxy);
  B.y = cic(a.B[1], xh, y0, zh, nx, nxy);
  B.z = cic(a.B[2], xh, yh, z0, nx, nxy);
}

// ----- Esirkepov deposit (linear shape) ------------------------------------
// The particle moves from offset os in cell cs to q (less than one cell per
// axis).  Along each axis the shapes before and after cover three nodes at
// most: nodes cs + lo + t, t = 0, 1, 2, with lo = min(0, end cell - cs).  In
// the frame of node cs - 1 (where the weights are formed) node t is lo + 1 +
// t.  The current along an axis is the running sum of that axis' weights
// over its first two edges (the sum over all three is zero: the charge is
// conserved), so a particle touches 2 x 3 x 3 nodes per component.
//
// With S0, S1 the shape weights before and after the move, dS = S1 - S0 and
// A = (S0 + S1)/2, Esirkepov's transverse factor of the x current,
//   S0y S0z + dSy S0z/2 + S0y dSz/2 + dSy dSz/3,
// is A_y A_z + dSy dSz/12 (and likewise for y and z), so every term is one
// fused multiply-add and one product.
template <typename R> struct EsirTerms {
  int lo[3];
  R A[3][3], dS[3][3], dS12[3][3];
  R P[3][2];   // per component: prefactor times the running sum over edges 0 and 1
};

template <typename R>
__device__ __forceinline__ bool esir_terms(const StepArgs<R> &a, const int *cs, const R *os, const Pt<R> &q, R qw,
                                           EsirTerms<R> &t) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int dc = q.ci[c] - cs[c];
    const R ua = R(1) + os[c];
    const R ub = R(dc + 1) + q.off[c];
    if (!(fabs_r(ub - ua) < R(1))) return false;
    t.lo[c] = dc < 0 ? dc : 0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const R node = R(t.lo[c] + 1 + m);
      R s0 = R(1) - fabs_r(ua - node);
      R s1 = R(1) - fabs_r(ub - node);
      s0 = s0 > R(0) ? s0 : R(0);
      s1 = s1 > R(0) ? s1 : R(0);
      t.A[c][m] = R(0.5) * (s0 + s1);
      t.dS[c][m] = s1 - s0;
      t.dS12[c][m] = t.dS[c][m] * R(1.0 / 12.0);
    }
    const R pref = -qw * a.jscale[c];
    t.P[c][0] = pref * t.dS[c][0];
    t.P[c][1] = pref * (t.dS[c][0] + t.dS[c][1]);
  }
  return true;
}

// add(component, node offsets (di, dj, dk) from cs + lo, value) for every
// current term of the Esirkepov scheme (Appendix C); the terms of nodes
// outside the move's support are zero, and add() skips them.
template <typename R, typename Add>
__device__ __forceinline__ void esir_apply(const EsirTerms<R> &t, Add add) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R w = fma_r(t.A[1][j], t.A[2][k], t.dS12[1][j] * t.dS[2][k]);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const R v = t.P[0][i] * w;
        add(0, i, j, k, v);
      }
    }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R w = fma_r(t.A[0][i], t.A[2][k], t.dS12[0][i] * t.dS[2][k]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R v = t.P[1][j] * w;
        add(1, i, j, k, v);
      }
    }
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R w = fma_r(t.A[0][i], t.A[1][j], t.dS12[0][i] * t.dS[1][j]);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const R v = t.P[2][k] * w;
        add(2, i, j, k, v);
      }
    }
}

// Esirkepov deposit into the global current (atomics).
template <typename R>
__device__ __noinline__ void deposit(const StepArgs<R> &a, const int *cs, const R *os, const Pt<R> &q, R qw) {
  EsirTerms<R> t;
  if (!esir_terms(a, cs, os, q, qw, t)) { atomicOr(a.status, kStCourant); return; }
  const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
  int I[3], Jj[3], K[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    I[m] = wrap_fast(cs[0] + t.lo[0] + m, a.n[0]);
    Jj[m] = wrap_fast(cs[1] + t.lo[1] + m, a.n[1]);
    K[m] = wrap_fast(cs[2] + t.lo[2] + m, a.n[2]);
  }
  esir_apply(t, [&](int c, int i, int j, int k, R v) {
    if (v != R(0)) atomicAdd(a.J[c] + K[k] * nxy + Jj[j] * nx + I[i], v);
  });
}

// ----- movement and boundaries ---------------------------------------------
template <typename R>
__device__ __forceinline__ void move(const StepArgs<R> &a, Pt<R> &q, V3<R> v, R h) {
  const R dv[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R o = q.off[c] + dv[c] * h * a.inv_d[c];
    R fl = floor_r(o);
    if (fl != R(0)) {
      q.ci[c] += (int)fl;
      o -= fl;
      if (o >= R(1)) { o -= R(1); q.ci[c] += 1; }
    }
    q.off[c] = o;
  }
}

// Periodic wrap or removal at the end of a particle's step; returns the
// linear cell or -1 when the particle left an open lattice.
template <typename R>
__device__ __forceinline__ int finish_cell(const StepArgs<R> &a, Pt<R> &q) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (a.periodic[c]) q.ci[c] = wrap_fast(q.ci[c], a.n[c]);
    else if (q.ci[c] < 0 || q.ci[c] >= a.n[c]) return -1;
  }
  return (q.ci[2] * a.n[1] + q.ci[1]) * a.n[0] + q.ci[0];
}

__device__ __forceinline__ double log10_r(double x) { return log10(x); }
__device__ __forceinline__ float log10_r(float x) { return log10f(x); }

template <typename R>
__device__ __noinline__ void spectrum_add(const StepArgs<R> &a, R delta, R eps, R w) {
  if (a.nbins <= 0) return;
  const R lo = (R)a.lg_lo, sc = (R)(a.lg_inv_span * a.nbins);
  R u = (log10_r(delta) - lo) * sc;
  if (u >= R(0) && u < R(a.nbins)) atomicAdd(a.spectrum + (int)u, (double)w);
  R v = (log10_r(eps) - lo) * sc;
  if (v >= R(0) && v < R(a.nbins)) atomicAdd(a.spectrum_energy + (int)v, (double)w);
}

// Upper bound of P_m(r1) over r1 for one sub-interval (Eq. (25)):
// with delta = r1^3, z = 2 delta / (3 chi (1 - delta)) and F1(z) <= g1(0)
// z^(1/3) (g1 = F1 z^(-1/3) decreases from g1(0) = 2.14953), the F1 term of
// P_m is at most 3 g1(0) (2/(3 chi))^(1/3) and the F2 term 3 max F2 =
// 3 x 0.60705, so
//   P_m <= alpha h sqrt3/(2 pi gamma) (5.6336 chi^(2/3) + 1.8212 chi)
// (the two bounds behind the time-step requirement of Sec. IV.H).  A factor
// 1.02 covers the tables' and this evaluation's rounding.
// Both bounds are evaluated in FP32 in either precision: a bound only has to
// lie above the probability, which the 2% margin keeps through FP32 rounding,
// and where FP32 underflows to 0 the probability is far below the smallest
// FP64 uniform as well.
template <typename R>
__device__ __forceinline__ R emit_bound(R chi, R gamma, R h) {
  // chi^(2/3) by the hardware base-2 logarithm and exponential (a few parts
  // in 1e7, far inside the 2% margin; chi = 0 gives 0, as it should)
  const float c = (float)chi, c23 = exp2f(0.6666667f * __log2f(c));
  return (R)(float(1.02 * kAlpha * kSqrt3Over2Pi) * (float)h / (float)gamma * (5.6336f * c23 + 1.8212f * c));
}

// Upper bound of P_p(de) over de for one sub-interval (Eq. (30)):
// P_p <= alpha h sqrt3/(2pi) (chi/eps) F2(z_p), and z_p >= z_min = 8/(3 chi)
// at de = 1/2, where F2 decreases beyond its maximum 0.60705 at z = 0.4169.
// Beyond 0.42, F2(z) = z K_{2/3}(z) lies below the first two terms of the
// asymptotic series of K_{2/3}, whose next term is negative:
//   F2(z) <= sqrt(pi z / 2) e^(-z) (1 + 7/(72 z)),
// which costs one exponential instead of a table evaluation.  A factor 1.02
// covers this evaluation's rounding.
template <typename R>
__device__ __forceinline__ R pair_bound(R chig, R eps, R h) {
  if (!(chig > R(0)) || !(eps > R(0))) return R(0);
  const float c = (float)chig, zmin = (8.0f / 3.0f) / c;
  float f2 = 0.6071f;
  if (zmin > 0.42f) f2 = sqrtf(float(kPi / 2) * zmin) * __expf(-zmin) * (1.0f + float(7.0 / 72.0) / zmin);
  return (R)(float(1.02 * kAlpha * kSqrt3Over2Pi) * (float)h * (c / (float)eps) * f2);
}

// Id of a product: child_id of the parent, keeping the parent's ensemble
// bits.  kind = product species | (sample << 8).
template <typename R>
__device__ __forceinline__ uint64_t product_id(const StepArgs<R> &a, uint64_t parent, unsigned step, unsigned sub,
                                               unsigned kind) {
  const uint64_t mix = child_id(parent, step, sub, kind, a.seed);
  return (parent & a.ens_mask) | (mix & ~a.ens_mask);
}

// Append a finished particle to its store (warp-aggregated slot reservation).
// Outcome bits of append / emit, added to the caller's counters: passing the
// counters themselves by reference would keep them in local memory.
constexpr unsigned kOutAbsorbed = 1u, kOutOverflow = 2u;

template <typename R>
__device__ __forceinline__ void count_outcome(const StepArgs<R> &a, unsigned r) {
  count_rare(a, kCntAbsorbed, r & kOutAbsorbed);
  count_rare(a, kCntOverflow, (r & kOutOverflow) >> 1);
}

template <typename R>
__device__ __noinline__ unsigned append(const StepArgs<R> &a, int sp, Pt<R> &q) {
  int cell = finish_cell(a, q);
  if (cell < 0) return kOutAbsorbed;
  unsigned mask = __activemask();
  // lanes appending to the same species share one atomic
  unsigned peers = __match_any_sync(mask, sp);
  int leader = __ffs(peers) - 1;
  int rank = __popc(peers & ((1u << (threadIdx.x & 31)) - 1u));
  unsigned long long base = 0;
  if ((int)(threadIdx.x & 31) == leader)
    base = (unsigned long long)atomicAdd((unsigned long long *)a.count + sp,
                                         (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  long long slot = (long long)base + rank;
  if (slot >= a.cap[sp]) {
    atomicOr(a.status, kStCapacity);
    return kOutOverflow;
  }
  store(a, sp, slot, q, cell, true);
  return 0;
}

// Queue a product for the rest of the step (same_step), or append it now.
// q.id is the parent's id on entry; the product's own id is product_id(q.id,
// step, sub, kind), formed here for an append and by the product pass for a
// queued product.
template <typename R>
__device__ __noinline__ unsigned emit(const StepArgs<R> &a, int pass, int sp, Pt<R> &q, unsigned step, unsigned sub,
                                      unsigned kind, R trem, V3<R> E, V3<R> B) {
  if (a.same_step && trem > R(0)) {
    // lanes queueing products in this pass share one atomic
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(a.pend_count + pass + 1, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
    if ((long long)slot >= a.pend_cap) {
      atomicOr(a.status, kStCapacity);
      return kOutOverflow;
    }
    Pend<R> *r = (Pend<R> *)a.pend[(pass + 1) & 1] + slot;
    r->off[0] = q.off[0]; r->off[1] = q.off[1]; r->off[2] = q.off[2];
    r->w = q.w; r->p = q.p; r->trem = trem; r->E = E; r->B = B;
    r->ci[0] = q.ci[0]; r->ci[1] = q.ci[1]; r->ci[2] = q.ci[2];
    r->sp = sp; r->parent = q.id; r->sub = sub; r->kind = kind;
    return 0;
  }
  q.id = product_id(a, q.id, step, sub, kind);
  return append(a, sp, q);
}

// Photons emitted by the lanes of one warp, held in shared memory until the
// warp is converged again: emitting lanes are few and seldom together, so
// queueing each product (a record written to shared memory) and emitting the
// queue at once lets the lanes share the atomic of emit / append instead of
// each paying its round trip while the rest of the warp waits.
constexpr unsigned kWarpQueue = 32;
template <typename R> struct WarpQueue {
  unsigned count;
  Pend<R> rec[kWarpQueue];
};

template <typename R>
__device__ __forceinline__ unsigned queue_emit(const StepArgs<R> &a, WarpQueue<R> *wq, int sp, const Pt<R> &q,
                                               unsigned step, unsigned sub, unsigned kind, R trem, V3<R> E,
                                               V3<R> B) {
  const unsigned slot = atomicAdd(&wq->count, 1u);
  if (slot >= kWarpQueue) {
    Pt<R> d = q;
    return emit(a, 0, sp, d, step, sub, kind, trem, E, B);   // full: emit now
  }
  Pend<R> *r = wq->rec + slot;
  r->off[0] = q.off[0]; r->off[1] = q.off[1]; r->off[2] = q.off[2];
  r->w = q.w; r->p = q.p; r->trem = trem; r->E = E; r->B = B;
  r->ci[0] = q.ci[0]; r->ci[1] = q.ci[1]; r->ci[2] = q.ci[2];
  r->sp = sp; r->parent = q.id; r->sub = sub; r->kind = kind;
  return 0;
}

// Emit a warp's queued products; every lane of the warp calls this.
template <typename R>
__device__ __noinline__ void flush_queue(const StepArgs<R> &a, WarpQueue<R> *wq, unsigned step) {
  __syncwarp();
  const unsigned n = min(wq->count, kWarpQueue);
  for (unsigned k = threadIdx.x & 31; k < n; k += 32) {
    const Pend<R> r = wq->rec[k];
    Pt<R> q;
    q.off[0] = r.off[0]; q.off[1] = r.off[1]; q.off[2] = r.off[2];
    q.ci[0] = r.ci[0]; q.ci[1] = r.ci[1]; q.ci[2] = r.ci[2];
    q.p = r.p; q.w = r.w; q.id = r.parent;
    count_outcome(a, emit(a, 0, r.sp, q, step, r.sub, r.kind, r.trem, r.E, r.B));
  }
  const unsigned lane = threadIdx.x & 31;
  __syncwarp();
  if (lane == 0) wq->count = 0;
  __syncwarp();
}

// Generator factors (Sec. VI) for the emission: N_g samples of the modified
// generator in sub-interval s (sample 0 is the parent's own draw r1, r2);
// each accepted sample makes a photon carrying delta = r1^3 of the parent's
// momentum before its recoil, kept with probability 1/f_g (a KEEP draw),
// with weight w f_g / N_g.  The parent's recoil is left to the caller.
struct SampleCounts {
  unsigned made = 0, gt1 = 0, out = 0;   // products made, P > 1 draws, outcome bits
};

template <typename R>
__device__ __noinline__ SampleCounts emit_samples(const StepArgs<R> &a, int pass, const Pt<R> &q, R r1, R r2, R pm,
                                                  R chi, R g, R h, int s, int n, unsigned step, V3<R> E, V3<R> B) {
  SampleCounts c;
  for (int j = 0; j < a.emit_ng; ++j) {
    R a1 = r1, a2 = r2, pmj = pm;
    if (j > 0) {
      draw2(q.id, step, (unsigned)s, kEmit | ((unsigned)j << 8), a.seed, a1, a2);
      pmj = prob_emit(a.tab, a1, chi, g, h);
      if (pmj > R(1)) {
        c.gt1++;
        if (a.pm_strict) atomicOr(a.status, kStPmGt1);
      }
    }
    if (!(a2 < pmj)) continue;
    if (a.emit_keep < R(1)) {
      R u, v;
      draw2(q.id, step, (unsigned)s, kKeep | ((unsigned)j << 8), a.seed, u, v);
      if (!(u < a.emit_keep)) continue;
    }
    const R delta = a1 * a1 * a1;
    Pt<R> ph = q;
    ph.p = {delta * q.p.x, delta * q.p.y, delta * q.p.z};
    ph.w = q.w * a.emit_wf;
    c.made++;
    if (a.nbins > 0) spectrum_add(a, delta, sqrt_r(dot(ph.p, ph.p)), ph.w);
    c.out |= emit(a, pass, kPhoton, ph, step, (unsigned)s, kPhoton | ((unsigned)j << 8), R(n - 1 - s) * h, E, B);
  }
  return c;
}

// The same for the pair generator: each accepted sample makes an electron
// with r1 of the photon momentum and a positron with 1 - r1, kept with
// probability 1/f_g, with weight w f_g / N_g.  The photon's own conversion
// (sample 0) is left to the caller.
template <typename R>
__device__ __noinline__ SampleCounts pair_samples(const StepArgs<R> &a, int pass, const Pt<R> &q, R r1, R r2, R pp,
                                                  R chig, R eps, R h, int s, int n, unsigned step, V3<R> E, V3<R> B) {
  SampleCounts c;
  const R trem = R(n - 1 - s) * h;
  for (int j = 0; j < a.pair_ng; ++j) {
    R a1 = r1, a2 = r2, ppj = pp;
    if (j > 0) {
      draw2(q.id, step, (unsigned)s, kPair | ((unsigned)j << 8), a.seed, a1, a2);
      ppj = prob_pair(a.tab, a1, chig, eps, h);
      if (ppj > R(1)) {
        c.gt1++;
        if (a.pm_strict) atomicOr(a.status, kStPmGt1);
      }
    }
    if (!(a2 < ppj)) continue;
    if (a.pair_keep < R(1)) {
      R u, v;
      draw2(q.id, step, (unsigned)s, kKeep | ((unsigned)j << 8) | (1u << 16), a.seed, u, v);
      if (!(u < a.pair_keep)) continue;
    }
    Pt<R> el = q, po = q;
    el.p = {a1 * q.p.x, a1 * q.p.y, a1 * q.p.z};
    const R c1 = R(1) - a1;
    po.p = {c1 * q.p.x, c1 * q.p.y, c1 * q.p.z};
    el.w = po.w = q.w * a.pair_wf;
    c.made++;
    c.out |= emit(a, pass, kElectron, el, step, (unsigned)s, kElectron | ((unsigned)j << 8), trem, E, B);
    c.out |= emit(a, pass, kPositron, po, step, (unsigned)s, kPositron | ((unsigned)j << 8), trem, E, B);
  }
  return c;
}

// Electron, positron or ion: the adaptive sub-interval loop (Sec. IV.H) of
// Boris push and modified emission generator (Sec. IV.G); ions are pushed only.
// massive_begin returns the step's number of sub-intervals (Eq. (28)) and
// loads the id when the generator will draw; massive_sub takes sub-interval
// s of n, each of length h.
template <typename R>
__device__ __forceinline__ int massive_begin(const StepArgs<R> &a, int sp, Pt<R> &q, R t_span, V3<R> E, V3<R> B,
                                             const uint64_t *idp) {
  const R m = a.mass[sp];
  const bool qed = (sp != kIon) && a.emission_on;
  if (qed && idp) q.id = __ldg(idp);
  int n = 1, capped = 0;
  if (qed) {
    R g0;
    if constexpr (sizeof(R) == 4) {
      R igm;
      lorentz(q.p, a.inv_mass[sp], a.inv_mass[sp] * a.inv_mass[sp], g0, igm);
    } else {
      g0 = sqrt_r(R(1) + dot(q.p, q.p) / (m * m));
    }
    n = nsub_lepton(t_span, g0, heff_lepton(q.p, g0, E, B), a.kappa, a.nsub_max, capped);
    count_rare(a, kCntCapped, (unsigned)capped);
  }
  return n;
}

template <typename R, bool EXT>
__device__ __forceinline__ void massive_sub(const StepArgs<R> &a, int pass, int sp, Pt<R> &q, const V3<R> &E,
                                            const V3<R> &B, Cnt &cnt, unsigned step, int s, int n, R h,
                                            WarpQueue<R> *wq = nullptr) {
  const R qc = a.charge[sp], m = a.mass[sp];
  const bool qed = (sp != kIon) && a.emission_on;
  boris(q.p, E, B, qc, m, h);
  R g, im;
  lorentz(q.p, a.inv_mass[sp], a.inv_mass[sp] * a.inv_mass[sp], g, im);
  move(a, q, V3<R>{q.p.x * im, q.p.y * im, q.p.z * im}, h);
  if (!qed) return;
  cnt.sub_l++;
  R chi = chi_lepton(q.p, g, E, B);
  R r1, r2;
  draw2(q.id, step, (unsigned)s, kEmit, a.seed, r1, r2);
  if (EXT && a.generator != 0) {
    // the unmodified generators of Sec. IV.F
    R delta, pe;
    bool fire;
    if (a.generator == 1) {
      delta = r1;                                   // r2 < P(r1)
      pe = prob_alternative(a.tab, r1, chi, g, h);
      fire = r2 < pe;
    } else {
      pe = std_total(a.std_lnw, chi, g, h);        // r1 < W(1), W(delta)/W(1) = r2
      if (sizeof(R) == 8) {
        // FP64: W(1) at the particle's chi where the interpolated table
        // (good to better than 1e-6) could decide otherwise, and delta at
        // the particle's chi from the panel quadrature
        if (fabs_r(r1 - pe) <= R(1e-5) * pe)
          pe = R(kAlpha) * h / g * (R)std_total_exact((const double *)a.tab, (double)chi);
        fire = r1 < pe;
        delta = fire ? (R)std_delta_exact((const double *)a.tab, (double)chi, (double)r2) : R(0);
      } else {
        fire = r1 < pe;
        delta = fire ? std_delta(a.tab, a.std_cdf, a.std_lnw, chi, r2) : R(0);
      }
    }
    if (pe > R(1)) {
      count_rare(a, kCntPmGt1, 1u);
      if (a.pm_strict) atomicOr(a.status, kStPmGt1);
    }
    if (fire) {
      Pt<R> ph = q;
      ph.p = {delta * q.p.x, delta * q.p.y, delta * q.p.z};
      const R omd = R(1) - delta;
      q.p = {omd * q.p.x, omd * q.p.y, omd * q.p.z};
      cnt.emis++;
      cnt.made_ph++;
      if (a.nbins > 0) spectrum_add(a, delta, sqrt_r(dot(ph.p, ph.p)), q.w);
      count_outcome(a, emit(a, pass, kPhoton, ph, step, (unsigned)s, kPhoton, R(n - 1 - s) * h, E, B));
    }
    return;
  }
  // P_m(r1) <= emit_bound <= r2: no emission, whatever r1 (and the bound
  // is below 1, so P_m is too); the generator factors reuse (r1, r2)
  if (!(EXT && (a.emit_ng > 1 || a.emit_keep < R(1))) && r2 >= emit_bound(chi, g, h)) return;
  R pm = prob_emit(a.tab, r1, chi, g, h);
  if (pm > R(1)) {
    count_rare(a, kCntPmGt1, 1u);
    if (a.pm_strict) atomicOr(a.status, kStPmGt1);
  }
  if (EXT && (a.emit_ng > 1 || a.emit_keep < R(1))) {
    // generator factors: products from N_g samples, kept with 1/f_g
    const SampleCounts sc = emit_samples(a, pass, q, r1, r2, pm, chi, g, h, s, n, step, E, B);
    cnt.made_ph += sc.made;
    count_rare(a, kCntPmGt1, sc.gt1);
    count_outcome(a, sc.out);
    if (r2 < pm) {
      const R omd = R(1) - r1 * r1 * r1;
      q.p = {omd * q.p.x, omd * q.p.y, omd * q.p.z};
      cnt.emis++;
    }
  } else if (r2 < pm) {
    // photon along p with delta of it; the parent keeps (1 - delta)
    R delta = r1 * r1 * r1;
    Pt<R> ph = q;
    ph.p = {delta * q.p.x, delta * q.p.y, delta * q.p.z};
    R omd = R(1) - delta;
    q.p = {omd * q.p.x, omd * q.p.y, omd * q.p.z};
    cnt.emis++;
    cnt.made_ph++;
    if (a.nbins > 0) spectrum_add(a, delta, sqrt_r(dot(ph.p, ph.p)), q.w);
    if (wq) count_outcome(a, queue_emit(a, wq, kPhoton, ph, step, (unsigned)s, kPhoton, R(n - 1 - s) * h, E, B));
    else count_outcome(a, emit(a, pass, kPhoton, ph, step, (unsigned)s, kPhoton, R(n - 1 - s) * h, E, B));
  }
}

template <typename R, bool EXT>
__device__ __forceinline__ void advance_massive(const StepArgs<R> &a, int pass, int sp, Pt<R> &q, R t_span,
                                                V3<R> E, V3<R> B, Cnt &cnt, const uint64_t *idp, unsigned step,
                                                bool deposit_later = false, WarpQueue<R> *wq = nullptr) {
  // start position (scalars: arrays handed to the deposit would live in
  // local memory for the whole loop)
  const int cs0 = q.ci[0], cs1 = q.ci[1], cs2 = q.ci[2];
  const R os0 = q.off[0], os1 = q.off[1], os2 = q.off[2];
  const R qc = a.charge[sp];
  const int n = massive_begin(a, sp, q, t_span, E, B, idp);
  const R h = t_span / R(n);
  for (int s = 0; s < n; ++s) massive_sub<R, EXT>(a, pass, sp, q, E, B, cnt, step, s, n, h, wq);
  if (a.deposit && qc != R(0) && !deposit_later) {
    const int cs[3] = {cs0, cs1, cs2};
    const R os[3] = {os0, os1, os2};
    const Pt<R> fin = q;
    deposit(a, cs, os, fin, qc * q.w);
  }
}

// Photon: straight flight with the pair generator (Sec. V.A) in the same
// sub-interval loop.  Returns false when the photon converted into a pair.
// idp: where to load the id from when a draw needs it (nullptr: q.id is set).
template <typename R, bool EXT>
__device__ __forceinline__ bool advance_photon(const StepArgs<R> &a, int pass, Pt<R> &q, R t_span, V3<R> E,
                                               V3<R> B, Cnt &cnt, const uint64_t *idp, R chi_star, unsigned step) {
  R eps, ie;
  photon_norm(q.p, eps, ie);
  const V3<R> dir = {q.p.x * ie, q.p.y * ie, q.p.z * ie};
  const R hg = heff_photon(dir, E, B);
  const R chig = eps * hg;
  int n = 1, capped = 0;
  if (a.pairs_on) {
    n = nsub_photon(t_span, hg, a.kappa, a.nsub_max, capped);
    count_rare(a, kCntCapped, (unsigned)capped);
  }
  const R h = t_span / R(n);
  // No draw can make a pair when P_p is below the smallest uniform: below
  // chi_star (uncapped) by the bound of photon_chi_star, else by pair_bound.
  bool may_pair = a.pairs_on;
  R bound = R(0);
  if (may_pair) {
    if (!capped && chig < chi_star) may_pair = false;
    else {
      bound = pair_bound(chig, eps, h);
      may_pair = bound >= r2_floor(h);
    }
  }
  // the generator factors draw further samples from the same (r1, r2)
  const bool plain = !(EXT && (a.pair_ng > 1 || a.pair_keep < R(1)));
  if (may_pair && idp) q.id = __ldg(idp);
  for (int s = 0; s < n; ++s) {
    move(a, q, dir, h);
    if (!a.pairs_on) continue;
    cnt.sub_g++;
    if (!may_pair) continue;
    R r1, r2;
    draw2(q.id, step, (unsigned)s, kPair, a.seed, r1, r2);
    // P_p(r1) <= bound <= r2: no pair, whatever r1 (and bound < 1, so P_p < 1)
    if (plain && r2 >= bound) continue;
    R pp = prob_pair(a.tab, r1, chig, eps, h);
    if (pp > R(1)) {
      count_rare(a, kCntPpGt1, 1u);
      if (a.pm_strict) atomicOr(a.status, kStPmGt1);
    }
    if (EXT && (a.pair_ng > 1 || a.pair_keep < R(1))) {
      // generator factors: pairs from N_g samples, kept with 1/f_g
      const SampleCounts sc = pair_samples(a, pass, q, r1, r2, pp, chig, eps, h, s, n, step, E, B);
      cnt.made_pair += sc.made;
      count_rare(a, kCntPpGt1, sc.gt1);
      count_outcome(a, sc.out);
      if (r2 < pp) {
        cnt.pairs++;
        return false;
      }
    } else if (r2 < pp) {
      // electron takes r1 of the photon momentum, positron 1 - r1
      Pt<R> el = q, po = q;
      el.p = {r1 * q.p.x, r1 * q.p.y, r1 * q.p.z};
      R r1c = R(1) - r1;
      po.p = {r1c * q.p.x, r1c * q.p.y, r1c * q.p.z};
      cnt.pairs++;
      cnt.made_pair++;
      R trem = R(n - 1 - s) * h;
      count_outcome(a, emit(a, pass, kElectron, el, step, (unsigned)s, kElectron, trem, E, B) |
                           emit(a, pass, kPositron, po, step, (unsigned)s, kPositron, trem, E, B));
      return false;
    }
  }
  return true;
}

// Bounded grid barrier (all blocks are co-resident: cooperative launch).
// Gives up after `limit` polls of ~64 ns (the default: ~1 s), sets the
// timeout status and returns false.
constexpr long long kBarrierPolls = 1ll << 24;

__device__ bool grid_barrier(unsigned *bar, int *status, long long limit = kBarrierPolls) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    unsigned g = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u) + 1u;
    ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        __nanosleep(64);
        if (++it > limit) {
          atomicOr(status, kStTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void flush(const Cnt &c, unsigned long long *g) {
  const unsigned v[10] = {c.emis, c.pairs, c.sub_l, c.sub_g, c.psteps[0], c.psteps[1], c.psteps[2],
                          c.psteps[3], c.made_ph, c.made_pair};
  const int slot[10] = {kCntEmissions, kCntPairs, kCntSubLepton, kCntSubPhoton, kCntSpeciesSteps,
                        kCntSpeciesSteps + 1, kCntSpeciesSteps + 2, kCntSpeciesSteps + 3, kCntPhotonsMade,
                        kCntPairsMade};
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    unsigned long long x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(g + slot[k], x);
  }
}

// ----- the start points of the cell-block pass (second store buffer) -------
// The start point of a record advanced by the cell-block pass (offsets and
// cell: all the deposit needs of it), kept in the store's second buffer.
__device__ __forceinline__ void keep_start(const StepArgs<float> &a, int sp, long long i, const Pt<float> &q,
                                           int cell) {
  ((float4 *)a.pos_scratch[sp])[i] = make_float4(q.off[0], q.off[1], q.off[2], __int_as_float(cell));
}
__device__ __forceinline__ void keep_start(const StepArgs<double> &a, int sp, long long i, const Pt<double> &q,
                                           int cell) {
  double2 *P2 = (double2 *)a.pos_scratch[sp] + 2 * i;
  P2[0] = make_double2(q.off[0], q.off[1]);
  P2[1] = make_double2(q.off[2], (double)cell);
}
__device__ __forceinline__ void load_start(const StepArgs<float> &a, int sp, long long i, float *off, int &cell) {
  const float4 v = __ldg((const float4 *)a.pos_scratch[sp] + i);
  off[0] = v.x; off[1] = v.y; off[2] = v.z;
  cell = __float_as_int(v.w);
}
__device__ __forceinline__ void load_start(const StepArgs<double> &a, int sp, long long i, double *off, int &cell) {
  const double2 *P = (const double2 *)a.pos_scratch[sp] + 2 * i;
  const double2 p0 = __ldg(P), p1 = __ldg(P + 1);
  off[0] = p0.x; off[1] = p0.y; off[2] = p1.x;
  cell = (int)p1.y;
}
template <typename R>
__device__ __forceinline__ void decode_cell(const StepArgs<R> &a, int cell, int *ci) {
  const unsigned row = fast_div((unsigned)cell, a.div_m[0], a.div_l[0]);
  const unsigned slab = fast_div((unsigned)cell, a.div_m[1], a.div_l[1]);
  ci[0] = cell - (int)row * a.n[0];
  ci[1] = (int)row - (int)slab * a.n[1];
  ci[2] = (int)slab;
}
template <typename R>
__device__ __forceinline__ int block_of_cell(const StepArgs<R> &a, int cell) {
  int ci[3];
  decode_cell(a, cell, ci);
  return ci[0] / kBlockCells + a.nb[0] * (ci[1] / kBlockCells + a.nb[1] * (ci[2] / kBlockCells));
}


// Pairs from the vacuum (Sec. V.B), once per step after the particles: in
// every cell the field at the centre (CIC of the Yee mesh there, or the
// analytic field at the step's time) gives
//   P_S = E^2 exp(-pi/E) V_cell dt / (4 pi^3)   (Compton units, E = |E|);
// with r < P_S an electron and a positron at rest are appended at one
// uniform point of the cell.  The cell index keys the draws: (r, u_x) from
// counter (step, 0, SCHWINGER, seed), (u_y, u_z) from (step, 1, ...).
template <typename R>
__global__ void __launch_bounds__(256) k_schwinger(const StepArgs<R> a) {
  __shared__ StepConst kc;
  if (threadIdx.x < (int)(sizeof(StepConst) / 8))
    ((unsigned long long *)&kc)[threadIdx.x] = ((const unsigned long long *)a.step_const)[threadIdx.x];
  __syncthreads();
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const R vol = R(a.dd[0] * a.dd[1] * a.dd[2]);
  unsigned pairs = 0, gt1 = 0;
  for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < ncell;
       cidx += (long long)gridDim.x * blockDim.x) {
    const unsigned cell = (unsigned)cidx;
    const unsigned row = fast_div(cell, a.div_m[0], a.div_l[0]);
    const unsigned slab = fast_div(cell, a.div_m[1], a.div_l[1]);
    Pt<R> q;
    q.ci[0] = (int)(cell - row * a.n[0]);
    q.ci[1] = (int)(row - slab * a.n[1]);
    q.ci[2] = (int)slab;
    q.off[0] = q.off[1] = q.off[2] = R(0.5);
    V3<R> E, B;
    if (a.field_mode == kFieldGrid) gather_grid(a, q, E, B);
    else field_analytic(a, kc, q, E, B);
    const R em = sqrt_r(E.x * E.x + E.y * E.y + E.z * E.z);
    if (!(em > R(0))) continue;
    const R ps = em * em * exp_r(-R(kPi) / em) / R(4.0 * kPi * kPi * kPi) * vol * a.dt;
    gt1 += ps > R(1);
    R r, ux;
    draw2((uint64_t)cell, kc.step, 0u, kSchwinger, a.seed, r, ux);
    if (!(r < ps)) continue;
    R uy, uz;
    draw2((uint64_t)cell, kc.step, 1u, kSchwinger, a.seed, uy, uz);
    Pt<R> el = q;
    el.off[0] = ux; el.off[1] = uy; el.off[2] = uz;
    el.p = {R(0), R(0), R(0)};
    el.w = a.schwinger_w;
    Pt<R> po = el;
    el.id = child_id((uint64_t)cell, kc.step, 0u, kElectron | kSchwingerKind, a.seed);
    po.id = child_id((uint64_t)cell, kc.step, 0u, kPositron | kSchwingerKind, a.seed);
    count_outcome(a, append(a, kElectron, el) | append(a, kPositron, po));
    ++pairs;
  }
  count_rare(a, kCntSchwinger, pairs);
  count_rare(a, kCntSchwingerGt1, gt1);
}

// Yee mesh: the largest |value| of each field component this step (a
// bound on every gathered |E| and |B|), reduced per warp and merged by
// atomicMax on the bit patterns (monotonic for non-negative values).
__device__ __forceinline__ unsigned long long abs_bits(float v) { return __float_as_uint(fabsf(v)); }
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

template <typename R> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using T = double2; static constexpr int n = 2; };
__device__ __forceinline__ unsigned long long abs_bits_max(const float4 &v) {
  const unsigned long long a = max(abs_bits(v.x), abs_bits(v.y)), b = max(abs_bits(v.z), abs_bits(v.w));
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long abs_bits_max(const double2 &v) {
  const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
  return a > b ? a : b;
}

// max |component| of each of the six mesh arrays (as ordered bit patterns of
// non-negative values), 16-byte loads where the array allows.
template <typename R>
__global__ void __launch_bounds__(256) k_grid_max(const StepArgs<R> a) {
  using V = typename Vec16<R>::T;
  constexpr int kV = Vec16<R>::n;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  for (int c = 0; c < 6; ++c) {
    const R *f = c < 3 ? a.E[c] : a.B[c - 3];
    unsigned long long m = 0;
    long long head = 0;
    if (((uintptr_t)f & 15) == 0) {
      const V *fv = (const V *)f;
      const long long nv = ncell / kV;
      for (long long i = t0; i < nv; i += stride) {
        const unsigned long long b = abs_bits_max(__ldg(fv + i));
        m = b > m ? b : m;
      }
      head = nv * kV;
    }
    for (long long i = head + t0; i < ncell; i += stride) {
      const unsigned long long b = abs_bits(__ldg(f + i));
      m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
      m = x > m ? x : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(a.grid_max + c, m);
  }
}

// The per-step field constants, formed once per step in FP64 by one thread.
// Ensemble mode: every thread of the one block also evaluates the fields
// of its ensembles at the step's time (FP64, stored in the context precision).
template <typename R>
__global__ void k_step_constants(const StepArgs<R> a) {
  Clock *clk = (Clock *)a.clock;
  const double t = clk->t;
  if (a.field_mode == kFieldEnsemble) {
    for (int e = threadIdx.x; e < a.n_ens; e += blockDim.x) {
      const double *q = a.ens_table + (size_t)e * QED_ENS_STRIDE;
      double sn, cs;
      sincos(q[1] * t + q[2], &sn, &cs);
      const double E[3] = {q[3] + q[0] * cs, q[4] + q[0] * sn, q[5]};
      R *f = a.ens_field + (size_t)e * kEnsFieldStride;
      for (int c = 0; c < 3; ++c) {
        f[c] = (R)E[c];
        f[3 + c] = (R)q[6 + c];
      }
      f[6] = (R)(sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]) +
                 sqrt(q[6] * q[6] + q[7] * q[7] + q[8] * q[8]));
      f[7] = R(0);
    }
  }
  __syncthreads();   // every thread has read the clock
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    step_constants(a, *(StepConst *)a.step_const);
    clk->t = t + a.dt_d;   // the next step starts dt later
    clk->step += 1;
  }
}

// Pass 0 of one particle family.  PHOTON: the photon store; otherwise
// electrons, positrons and ions.  Resident blocks per SM set the register
// budget: the photon path is light enough for four 256-thread blocks.
template <typename R, bool PHOTON> struct Pass0Occ;
template <> struct Pass0Occ<float, false> { static constexpr int blocks = 3; };
template <> struct Pass0Occ<double, false> { static constexpr int blocks = 1; };

// Analytic fields (not ensembles): e-, e+ and ions with lanes refilled one
// particle at a time.  A particle takes its own number of sub-intervals, so a lane that
// has finished takes the next particle while the others are still in their
// loops, instead of idling until the longest loop of the warp ends.  Warps
// take indices 32 at a time from the pass's work counter; every lane runs
// sub-interval after sub-interval of whichever particle it holds.
template <typename R, bool EXT>
__device__ __forceinline__ void massive_lanes(const StepArgs<R> &a, const StepConst &kc, Cnt &cnt,
                                              const long long *ns, long long total) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  bool has = false;
  int sp = kElectron, n = 1, s = 0, cell = 0;
  long long i = 0;
  Pt<R> q;
  V3<R> E, B;
  R h = R(0);
  long long qb = 0, qe = 0;   // the warp's batch of indices [qb, qe), warp-uniform
  bool dry = false;           // the work counter has run past the end
  for (;;) {
    for (;;) {
      const unsigned need = __ballot_sync(0xffffffffu, !has);
      if (!need || dry) break;
      if (qb >= qe) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(a.work_massive, 32ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        qb = (long long)b;
        qe = min(qb + 32, total);
        if (qb >= total) {
          dry = true;
          break;
        }
      }
      const long long avail = qe - qb;
      const int rank = __popc(need & below);
      if (!has && rank < avail) {
        long long it = qb + rank;
        sp = kElectron;
        if (it >= ns[kElectron]) {
          it -= ns[kElectron];
          sp = kPositron;
          if (it >= ns[kPositron]) { it -= ns[kPositron]; sp = kIon; }
        }
        i = it;
        load(a, sp, i, q, cell);
        if (cell >= 0) {
          cnt.psteps[sp]++;
          const unsigned row = fast_div((unsigned)cell, a.div_m[0], a.div_l[0]);
          const unsigned slab = fast_div((unsigned)cell, a.div_m[1], a.div_l[1]);
          q.ci[0] = cell - (int)row * a.n[0];
          q.ci[1] = (int)row - (int)slab * a.n[1];
          q.ci[2] = (int)slab;
          const uint64_t *idp = a.id[sp] + i;
          if (EXT && a.field_mode == kFieldEnsemble) {
            q.id = __ldg(idp);
            idp = nullptr;
            field_ensemble(a, q.id, E, B);
          } else {
            field_analytic(a, kc, q, E, B);
          }
          const R probe = (E.x + E.y + E.z + B.x + B.y + B.z) * R(0) + (q.p.x + q.p.y + q.p.z) * R(0);
          if (!(probe == R(0))) {
            count_rare(a, kCntNonfinite, 1u);
            atomicOr(a.status, kStNonfinite);
          }
          n = massive_begin(a, sp, q, a.dt, E, B, idp);
          h = a.dt / R(n);
          s = 0;
          has = true;
        }
      }
      qb += min((long long)__popc(need), avail);
    }
    if (!__any_sync(0xffffffffu, has)) break;
    if (has) {
      massive_sub<R, EXT>(a, 0, sp, q, E, B, cnt, kc.step, s, n, h);
      if (++s == n) {
        const int nc = finish_cell(a, q);
        if (nc < 0) count_rare(a, kCntAbsorbed, 1u);
        store(a, sp, i, q, nc, false);
        has = false;
      }
    }
  }
}

template <typename R, bool PHOTON, bool EXT>
__global__ void __launch_bounds__(256, (Pass0Occ<R, PHOTON>::blocks)) k_pass0(const StepArgs<R> a) {
  Cnt cnt;
  __shared__ long long ns[4];
  __shared__ StepConst kc;
  if (threadIdx.x < (int)(sizeof(StepConst) / 8))
    ((unsigned long long *)&kc)[threadIdx.x] = ((const unsigned long long *)a.step_const)[threadIdx.x];
  __shared__ long long nb0[4];
  // an overflowing append leaves count above the capacity: never read past it
  if (threadIdx.x < 4) {
    ns[threadIdx.x] = min(a.nstart[threadIdx.x], a.cap[threadIdx.x]);
    // records in cell-block order are advanced by k_blocks; this kernel takes the rest
    const unsigned *bs = a.blk_start[threadIdx.x];
    nb0[threadIdx.x] = (!PHOTON && bs) ? min((long long)bs[a.nblk], ns[threadIdx.x]) : 0;
    ns[threadIdx.x] -= nb0[threadIdx.x];
  }
  __syncthreads();
  const long long total = PHOTON ? ns[kPhoton] : ns[kElectron] + ns[kPositron] + ns[kIon];
  // (ensembles order their leptons by estimated sub-interval count instead,
  // and measured faster with whole-particle loops)
  if (!PHOTON && a.field_mode != kFieldGrid && a.field_mode != kFieldEnsemble) {
    massive_lanes<R, EXT>(a, kc, cnt, ns, total);
    flush(cnt, a.counters);
    return;
  }
  auto body = [&](long long it) {
    int sp = kPhoton;
    long long i = it;
    if (!PHOTON) {
      sp = kElectron;
      if (i >= ns[kElectron]) {
        i -= ns[kElectron];
        sp = kPositron;
        if (i >= ns[kPositron]) { i -= ns[kPositron]; sp = kIon; }
      }
      i += nb0[sp];
    }
    Pt<R> q;
    int cell;
    load(a, sp, i, q, cell);
    if (cell < 0) return;
    cnt.psteps[sp]++;
    const unsigned row = fast_div((unsigned)cell, a.div_m[0], a.div_l[0]);
    const unsigned slab = fast_div((unsigned)cell, a.div_m[1], a.div_l[1]);
    q.ci[0] = cell - (int)row * a.n[0];
    q.ci[1] = (int)row - (int)slab * a.n[1];
    q.ci[2] = (int)slab;
    V3<R> E, B;
    const uint64_t *idp = a.id[sp] + i;
    if (a.field_mode == kFieldGrid) {
      gather_grid(a, q, E, B);
    } else if (EXT && a.field_mode == kFieldEnsemble) {
      q.id = __ldg(idp);
      idp = nullptr;
      field_ensemble(a, q.id, E, B);
    } else {
      field_analytic(a, kc, q, E, B);
    }
    // a NaN or an infinity in any input makes this sum NaN or infinite
    const R probe = (E.x + E.y + E.z + B.x + B.y + B.z) * R(0) + (q.p.x + q.p.y + q.p.z) * R(0);
    if (!(probe == R(0))) {
      count_rare(a, kCntNonfinite, 1u);
      atomicOr(a.status, kStNonfinite);
    }
    bool alive = true;
    if (PHOTON) alive = advance_photon<R, EXT>(a, 0, q, a.dt, E, B, cnt, idp, (R)*a.chi_star, kc.step);
    else advance_massive<R, EXT>(a, 0, sp, q, a.dt, E, B, cnt, idp, kc.step);
    int nc = alive ? finish_cell(a, q) : -1;
    if (alive && nc < 0) count_rare(a, kCntAbsorbed, 1u);
    // a photon's momentum never changes: its momentum record is rewritten
    // only when the cell changed or the photon died
    if (PHOTON && nc == cell) store_pos(a, sp, i, q);
    else store(a, sp, i, q, nc, false);
  };
  // Static: grid-stride over rows of 256.  Work stealing (chunk > 0): blocks
  // take chunks of consecutive particles from a shared counter, so blocks
  // that drew cheap particles take more.  One loop, one copy of the body.
  __shared__ long long wb;
  const bool dyn = a.chunk > 0;
  long long next = (long long)blockIdx.x * blockDim.x;
  for (;;) {
    long long lo, hi;
    if (dyn) {
      __syncthreads();   // everyone has read the previous chunk's start
      if (threadIdx.x == 0) wb = (long long)atomicAdd(a.work_massive, (unsigned long long)a.chunk);
      __syncthreads();
      lo = wb;
      hi = min(lo + a.chunk, total);
    } else {
      lo = next;
      hi = min(lo + (long long)blockDim.x, total);
      next += (long long)gridDim.x * blockDim.x;
    }
    if (lo >= total) break;
    for (long long it = lo + threadIdx.x; it < hi; it += blockDim.x) body(it);
  }
  flush(cnt, a.counters);
}

// ----- photon pass 0 with per-thread asynchronous staging -----------------
// Photons are most of the particles of a cascade and their step is short, so
// memory latency dominates.  Each thread streams its own photons (grid-stride
// order) through kStages private shared-memory slots with cp.async: the
// records of the next kStages-1 photons are in flight while the current one
// is computed.  A thread only reads what it copied itself, so no barrier and
// no spin-wait is involved (cp.async.wait_group is a hardware wait).
constexpr int kPhotonThreads = 256;
// slots per thread: three 32-byte FP32 records, two 64-byte FP64 records
template <typename R> struct PhotonStages { static constexpr int n = sizeof(R) == 4 ? 3 : 2; };

template <typename R> struct Half;
template <> struct Half<float> { using T = float4; };
template <> struct Half<double> { struct alignas(16) T { double2 a, b; }; };

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename R> struct PhotonOcc { static constexpr int blocks = sizeof(R) == 4 ? 3 : 2; };

template <typename R, bool EXT>
__global__ void __launch_bounds__(kPhotonThreads, PhotonOcc<R>::blocks) k_photons(const StepArgs<R> a) {
  using T = typename Half<R>::T;
  constexpr int kChunks = sizeof(T) / 16;
  constexpr int kStages = PhotonStages<R>::n;
  // [stage][pos | mom][thread]: consecutive threads read consecutive slots
  __shared__ __align__(16) T slot[kStages][2][kPhotonThreads];
  __shared__ StepConst kc;
  Cnt cnt;
  if (threadIdx.x < (int)(sizeof(StepConst) / 8))
    ((unsigned long long *)&kc)[threadIdx.x] = ((const unsigned long long *)a.step_const)[threadIdx.x];
  __syncthreads();
  const long long n = min(a.nstart[kPhoton], a.cap[kPhoton]);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const T *gpos = (const T *)a.pos[kPhoton];
  const T *gmom = (const T *)a.mom[kPhoton];
  const R chi_star = (R)*a.chi_star;
  auto issue = [&](long long k) {
    const long long i = i0 + k * stride;
    if (i < n) {
      const int st = (int)(k % kStages);
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        cp_async16((char *)&slot[st][0][threadIdx.x] + 16 * c, (const char *)(gpos + i) + 16 * c);
        cp_async16((char *)&slot[st][1][threadIdx.x] + 16 * c, (const char *)(gmom + i) + 16 * c);
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < kStages - 1; ++k) issue(k);
  for (long long k = 0;; ++k) {
    const long long i = i0 + k * stride;
    if (i >= n) break;
    issue(k + kStages - 1);
    cp_wait<kStages - 1>();
    const int st = (int)(k % kStages);
    Pt<R> q;
    int cell;
    unpack(slot[st][0][threadIdx.x], slot[st][1][threadIdx.x], q, cell);
    if (cell < 0) continue;
    cnt.psteps[kPhoton]++;
    const unsigned row = fast_div((unsigned)cell, a.div_m[0], a.div_l[0]);
    const unsigned slab = fast_div((unsigned)cell, a.div_m[1], a.div_l[1]);
    q.ci[0] = cell - (int)row * a.n[0];
    q.ci[1] = (int)row - (int)slab * a.n[1];
    q.ci[2] = (int)slab;
    bool alive = true;
    R eps, ie;
    photon_norm(q.p, eps, ie);
    R hmax = sizeof(R) == 4 ? (R)kc.hmax_f : (R)kc.hmax;
    bool one = kc.one_interval;
    if (EXT && a.field_mode == kFieldEnsemble) {
      // the bound of the photon's own ensemble: |E| + |B| at this step
      q.id = __ldg(a.id[kPhoton] + i);
      const unsigned long long e = a.ens_shift >= 64 ? 0ull : (unsigned long long)(q.id >> a.ens_shift);
      hmax = e < (unsigned long long)a.n_ens ? __ldg(a.ens_field + e * kEnsFieldStride + 6) * R(1.00001) : R(0);
      one = a.dt * hmax <= R(0.999) * a.kappa * R(130.0 * kTwoPi);   // N = 1 for every H <= hmax
    }
    if (!a.pairs_on || (one && eps * hmax < R(0.99999) * chi_star)) {
      // This photon cannot pair in this step (chi_g <= eps hmax < chi*) and
      // takes one sub-interval: its step is the straight flight of
      // advance_photon with N = 1, without evaluating the field.
      if (!(q.p.x * R(0) + q.p.y * R(0) + q.p.z * R(0) == R(0))) {
        count_rare(a, kCntNonfinite, 1u);
        atomicOr(a.status, kStNonfinite);
      }
      move(a, q, V3<R>{q.p.x * ie, q.p.y * ie, q.p.z * ie}, a.dt);
      if (a.pairs_on) cnt.sub_g++;
    } else {
      V3<R> E, B;
      const uint64_t *idp = a.id[kPhoton] + i;
      if (a.field_mode == kFieldGrid) {
        gather_grid(a, q, E, B);
      } else if (EXT && a.field_mode == kFieldEnsemble) {
        idp = nullptr;                  // q.id was loaded for the bound above
        field_ensemble(a, q.id, E, B);
      } else {
        field_analytic(a, kc, q, E, B);
      }
      const R probe = (E.x + E.y + E.z + B.x + B.y + B.z) * R(0) + (q.p.x + q.p.y + q.p.z) * R(0);
      if (!(probe == R(0))) {
        count_rare(a, kCntNonfinite, 1u);
        atomicOr(a.status, kStNonfinite);
      }
      alive = advance_photon<R, EXT>(a, 0, q, a.dt, E, B, cnt, idp, chi_star, kc.step);
    }
    const int nc = alive ? finish_cell(a, q) : -1;
    if (alive && nc < 0) count_rare(a, kCntAbsorbed, 1u);
    // a photon's momentum never changes: its momentum record is rewritten
    // only when the cell changed or the photon died
    if (nc == cell) store_pos(a, kPhoton, i, q);
    else store(a, kPhoton, i, q, nc, false);
  }
  cp_wait<0>();
  flush(cnt, a.counters);
}

// Grid mode: electrons, positrons and ions in cell-block order.  Blocks take
// cell blocks by work stealing; the particles of a cell block deposit their
// current into a shared-memory tile covering the block and the deposit
// stencil's reach, which is then added to the global current with one atomic
// per non-zero tile node.
// Work items of the cell-block kernels: kBlockChunk consecutive records of
// one species in cell-block order (the sorted prefix of each store).
struct BlockItems {
  long long nsort[3], nitem[3];
  unsigned items;
};

// The families of the cell-block pass: electrons and positrons (LEPTONS),
// or ions alone, whose step has no event generator and is compiled without
// it.  FP32 runs four blocks per SM (64 registers): measured on the 512^3
// cascade, the pass took 4.38 ms per step at four blocks (the e-/e+ kernel
// spilling 68 B) and 4.80 at three (80 registers); before the gather took
// its interpolating form, three blocks had been best (8.43 ms, against 9.10
// at two and 8.70 at four).
template <typename R>
__device__ __forceinline__ BlockItems block_items(const StepArgs<R> &a, const long long *ns, bool ions) {
  BlockItems b;
  const int fam[3] = {kElectron, kPositron, kIon};
  b.items = 0;
  for (int f = 0; f < 3; ++f) {
    const int sp = fam[f];
    const bool mine = ions ? sp == kIon : sp != kIon;
    b.nsort[f] = (mine && a.blk_start[sp]) ? min((long long)a.blk_start[sp][a.nblk], ns[sp]) : 0;
    b.nitem[f] = (b.nsort[f] + kBlockChunk - 1) / kBlockChunk;
    b.items += (unsigned)b.nitem[f];
  }
  return b;
}

// Electrons and positrons of one work item with lanes refilled in groups: a
// lane holds one particle through its sub-interval loop (Sec. IV.H); once at
// least k lanes of the warp have finished, the warp takes that many new
// records from the item at once, so that their loads and field gathers are
// issued together, and every lane then takes its next sub-interval.
template <typename R, bool EXT>
__device__ __forceinline__ void blocks_refill(const StepArgs<R> &a, int sp, long long lo, int total, int *next,
                                              Cnt &cnt, unsigned step, int k) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  bool has = false, dry = false;
  Pt<R> q;
  V3<R> E, B;
  int n = 1, s = 0;
  R h = R(0);
  long long i = 0;
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, !has);
    if (!dry && (__popc(idle) >= k || idle == 0xffffffffu)) {
      const int want = __popc(idle);
      int base = 0;
      if (lane == 0) base = atomicAdd(next, want);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base + want >= total) dry = true;
      const int rank = __popc(idle & below);
      if (!has && base + rank < total) {
        i = lo + base + rank;
        int cell;
        load(a, sp, i, q, cell);
        if (cell >= 0) {
          if (a.deposit) keep_start(a, sp, i, q, cell);
          cnt.psteps[sp]++;
          decode_cell(a, cell, q.ci);
          gather_grid(a, q, E, B);
          const R probe = (E.x + E.y + E.z + B.x + B.y + B.z) * R(0) + (q.p.x + q.p.y + q.p.z) * R(0);
          if (!(probe == R(0))) {
            count_rare(a, kCntNonfinite, 1u);
            atomicOr(a.status, kStNonfinite);
          }
          n = massive_begin(a, sp, q, a.dt, E, B, a.id[sp] + i);
          h = a.dt / R(n);
          s = 0;
          has = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, has)) {
      if (dry) break;
      continue;
    }
    if (has) {
      massive_sub<R, EXT>(a, 0, sp, q, E, B, cnt, step, s, n, h);
      if (++s == n) {
        const int nc = finish_cell(a, q);
        if (nc < 0) count_rare(a, kCntAbsorbed, 1u);
        store(a, sp, i, q, nc, false);
        has = false;
      }
    }
  }
}

template <typename R, bool IONS> struct BlocksOcc { static constexpr int blocks = sizeof(R) == 4 ? 4 : 2; };

// Grid mode: electrons, positrons (IONS = false) or ions (IONS = true) in
// cell-block order, advanced in work items taken by work stealing; warps
// take 32 records at a time inside an item, so fast warps take more.  The
// current is deposited afterwards by k_deposit_blocks, from the start point
// each thread leaves in the store's second buffer (free between
// compactions): keeping the Esirkepov stencil out of this kernel keeps its
// code within the instruction cache.
template <typename R, bool EXT, bool IONS>
__global__ void __launch_bounds__(256, (BlocksOcc<R, IONS>::blocks)) k_blocks(const StepArgs<R> a) {
  __shared__ int blk;
  __shared__ int next;
  __shared__ long long ns[4];
  // e-/e+: each warp's queue of emitted photons (ions emit nothing)
  __shared__ WarpQueue<R> queues[IONS ? 1 : 8];
  WarpQueue<R> *wq = IONS ? nullptr : queues + (threadIdx.x >> 5);
  if (wq && (threadIdx.x & 31) == 0) wq->count = 0;
  Cnt cnt;
  const unsigned step = ((const StepConst *)a.step_const)->step;
  if (threadIdx.x < 4) ns[threadIdx.x] = min(a.nstart[threadIdx.x], a.cap[threadIdx.x]);
  __syncthreads();
  const BlockItems bi = block_items(a, ns, IONS);
  const int fam[3] = {kElectron, kPositron, kIon};
  const int lane = threadIdx.x & 31;
  unsigned *work = IONS ? a.work + 4 : a.work;
  for (;;) {
    if (threadIdx.x == 0) {
      blk = (int)atomicAdd(work, 1u);
      next = 0;
    }
    __syncthreads();
    unsigned item = (unsigned)blk;
    if (item >= bi.items) break;
    int f = 0;
    while (item >= bi.nitem[f]) { item -= (unsigned)bi.nitem[f]; ++f; }
    const int sp = IONS ? (int)kIon : fam[f];
    const long long lo = (long long)item * kBlockChunk, hi = min(lo + kBlockChunk, bi.nsort[f]);
    const int total = (int)(hi - lo);
    if (!IONS && a.refill_lanes > 0) {
      blocks_refill<R, EXT>(a, sp, lo, total, &next, cnt, step, a.refill_lanes);
      __syncthreads();   // blk and next are reused by the next item
      continue;
    }
    for (;;) {
      int base = 0;
      if (lane == 0) base = atomicAdd(&next, 32);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (wq) {
        __syncwarp();   // every lane's queued records are visible
        if (wq->count >= kWarpQueue - 8) flush_queue(a, wq, step);
      }
      if (base >= total) break;
      const int pos = base + lane;
      if (pos >= total) continue;
      const long long i = lo + pos;
      Pt<R> q;
      int cell;
      load(a, sp, i, q, cell);
      if (cell < 0) continue;
      if (a.deposit) keep_start(a, sp, i, q, cell);
      cnt.psteps[sp]++;
      const unsigned row = fast_div((unsigned)cell, a.div_m[0], a.div_l[0]);
      const unsigned slab = fast_div((unsigned)cell, a.div_m[1], a.div_l[1]);
      q.ci[0] = cell - (int)row * a.n[0];
      q.ci[1] = (int)row - (int)slab * a.n[1];
      q.ci[2] = (int)slab;
      V3<R> E, B;
      gather_grid(a, q, E, B);
      const R probe = (E.x + E.y + E.z + B.x + B.y + B.z) * R(0) + (q.p.x + q.p.y + q.p.z) * R(0);
      if (!(probe == R(0))) {
        count_rare(a, kCntNonfinite, 1u);
        atomicOr(a.status, kStNonfinite);
      }
      advance_massive<R, EXT>(a, 0, sp, q, a.dt, E, B, cnt, a.id[sp] + i, step, true, wq);
      const int nc = finish_cell(a, q);
      if (nc < 0) count_rare(a, kCntAbsorbed, 1u);
      store(a, sp, i, q, nc, false);
    }
    __syncthreads();   // blk and next are reused by the next item
  }
  if (wq) flush_queue(a, wq, step);   // the queue outlives the work items
  // every live record this block advanced was counted in psteps
  unsigned long long mine = cnt.psteps[kElectron] + cnt.psteps[kPositron] + cnt.psteps[kIon];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.counters + kCntBlockSteps, mine);
  flush(cnt, a.counters);
}

// The Esirkepov deposit of the records k_blocks advanced: start from the
// second buffer, end from the store.  One work item is one cell block: the
// e-, e+ and ion records of the sorted prefixes that belong to it deposit
// into a shared-memory tile covering the block and a halo of H cells each
// side (the current reduced per block in shared memory, as the paper's GPU
// code does, Appendix C), which is flushed once, with one global atomic per
// non-zero node.  A particle whose stencil leaves the tile (it has drifted
// farther since the last sort), every particle of a cell block too sparse to
// pay for zeroing and flushing a tile, and every particle with H = 0 add
// their current straight to J.  Blocks claim a.deposit_grab (1 .. 32)
// consecutive cell blocks at a time, so that every resident block gets
// several claims, and skip the empty ones.  A warp whose lanes all move
// within their cells takes the short form of the stencil: along each axis
// the shapes cover the cell's two nodes and the current crosses one edge,
// so each component has 4 terms instead of 18.
template <typename R> struct DepositOcc { static constexpr int blocks = sizeof(R) == 4 ? 4 : 2; };

// Add to a shared-memory value without reading the sum back (a reduction:
// no register waits on the result).  The address is a shared-window byte
// address: the tile's is formed once, and each term adds a constant to it.
__device__ __forceinline__ void red_shared(unsigned addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void red_shared(unsigned addr, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// The same, predicated on v != 0 (no branch: the zero terms of a move's
// support just do not add).
__device__ __forceinline__ void red_shared_nz(unsigned addr, float v) {
  asm volatile("{\n .reg .pred nz;\n setp.ne.f32 nz, %1, 0f00000000;\n @nz red.shared.add.f32 [%0], %1;\n}"
               ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void red_shared_nz(unsigned addr, double v) {
  asm volatile("{\n .reg .pred nz;\n setp.ne.f64 nz, %1, 0d0000000000000000;\n @nz red.shared.add.f64 [%0], %1;\n}"
               ::"r"(addr), "d"(v) : "memory");
}

// o: shared byte address of the tile node (cs) of the first component.
template <typename R, int T>
__device__ __forceinline__ void deposit_in_cell(const StepArgs<R> &a, unsigned o, const R *os, const R *oe, R qw) {
  constexpr int TT = T * T, TTT = TT * T;
  R A[3][2], D[3][2], pref[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R m = R(0.5) * (os[c] + oe[c]);
    A[c][0] = R(1) - m;
    A[c][1] = m;
    D[c][0] = os[c] - oe[c];
    D[c][1] = oe[c] - os[c];
    pref[c] = -qw * a.jscale[c] * D[c][0];
  }
  const R r12 = R(1.0 / 12.0);
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      red_shared(o + sizeof(R) * (k * TT + j * T), pref[0] * fma_r(A[1][j], A[2][k], r12 * D[1][j] * D[2][k]));
      red_shared(o + sizeof(R) * (TTT + k * TT + j), pref[1] * fma_r(A[0][j], A[2][k], r12 * D[0][j] * D[2][k]));
      red_shared(o + sizeof(R) * (2 * TTT + k * T + j), pref[2] * fma_r(A[0][j], A[1][k], r12 * D[0][j] * D[1][k]));
    }
}

template <typename R, int HALO>
__global__ void __launch_bounds__(256, DepositOcc<R>::blocks) k_deposit_blocks(const StepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char dep_smem[];
  R *jt = (R *)dep_smem;
  const unsigned jt_s = (unsigned)__cvta_generic_to_shared(jt);
  constexpr int halo = HALO;
  constexpr int T = tile_nodes(HALO), TT = T * T, TTT = TT * T;
  __shared__ unsigned grab, nonempty;
  __shared__ long long ns[4];
  __shared__ long long rlo[3], rn[3];       // per family: first record and count in the current cell block
  // wrapped global offsets of the tile's node rows: x index, y x nx, z x nx ny
  __shared__ long long gofs[3][kMaxTileNodes];
  if (threadIdx.x < 4) ns[threadIdx.x] = min(a.nstart[threadIdx.x], a.cap[threadIdx.x]);
  __syncthreads();
  const int fam[3] = {kElectron, kPositron, kIon};
  long long nsort[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const int sp = fam[f];
    nsort[f] = (a.blk_start[sp] && a.charge[sp] != R(0)) ? min((long long)a.blk_start[sp][a.nblk], ns[sp]) : 0;
  }
  const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
  // a tile pays for itself when the block holds a record per 64 of its values
  const long long tile_min = halo > 0 ? (3ll * TTT) / 64 : (1ll << 62);
  unsigned in_tile = 0;
  for (;;) {
    if (threadIdx.x == 0) grab = atomicAdd(a.work + 1, (unsigned)a.deposit_grab);
    __syncthreads();
    const unsigned base = grab;
    if (base >= (unsigned)a.nblk) break;
    if (threadIdx.x < 32) {
      const unsigned b = base + threadIdx.x;
      bool any = false;
      if ((int)threadIdx.x < a.deposit_grab && b < (unsigned)a.nblk)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          if (nsort[f] == 0) continue;
          const unsigned *st = a.blk_start[fam[f]];
          any |= min((long long)st[b + 1], nsort[f]) > min((long long)st[b], nsort[f]);
        }
      const unsigned m = __ballot_sync(0xffffffffu, any);
      if (threadIdx.x == 0) nonempty = m;
    }
    __syncthreads();
    for (unsigned m = nonempty; m; m &= m - 1) {
      const int bl = (int)base + __ffs(m) - 1;
      const int bc[3] = {bl % a.nb[0], (bl / a.nb[0]) % a.nb[1], bl / (a.nb[0] * a.nb[1])};
      int torg[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) torg[c] = bc[c] * kBlockCells - halo;
      if (threadIdx.x < 3) {
        const int f = threadIdx.x;
        long long lo = 0, hi = 0;
        if (nsort[f]) {
          const unsigned *st = a.blk_start[fam[f]];
          lo = min((long long)st[bl], nsort[f]);
          hi = min((long long)st[bl + 1], nsort[f]);
        }
        rlo[f] = lo;
        rn[f] = hi - lo;
      }
      __syncthreads();
      const long long total = rn[0] + rn[1] + rn[2];
      const bool tile = total >= tile_min;
      if (tile) {
        if (threadIdx.x < 3 * T) {
          const int c = threadIdx.x / T, k = threadIdx.x % T;
          const long long stride = c == 0 ? 1 : (c == 1 ? nx : nxy);
          gofs[c][k] = (long long)wrapi(torg[c] + k, a.n[c]) * stride;
        }
        using V = typename Vec16<R>::T;
        constexpr int kV = Vec16<R>::n, nv = (3 * TTT) / kV;
        for (int t = threadIdx.x; t < nv; t += blockDim.x) ((V *)jt)[t] = V{};
        for (int t = nv * kV + threadIdx.x; t < 3 * TTT; t += blockDim.x) jt[t] = R(0);
        __syncthreads();
      }
      // the block's records of each family are in cell order: lane l of a
      // warp takes record l x rows + k of one family, so that the lanes'
      // stencils lie in cells far apart and their shared-memory additions
      // seldom meet on one node, and a warp holds one family (ions, which
      // seldom leave their cells, then take the short form together)
      const long long rows0 = (rn[0] + 31) / 32, rows1 = (rn[1] + 31) / 32, rows2 = (rn[2] + 31) / 32;
      const long long rows01 = rows0 + rows1;
      for (long long t = threadIdx.x; t < 32 * (rows01 + rows2); t += blockDim.x) {
        const long long w = t >> 5;
        const int f = w < rows0 ? 0 : (w < rows01 ? 1 : 2);
        const long long rows_f = f == 0 ? rows0 : (f == 1 ? rows1 : rows2);
        const long long u = (t & 31) * rows_f + (w - (f == 0 ? 0 : (f == 1 ? rows0 : rows01)));
        const bool have = u < rn[f];
        const int sp = fam[f];
        const long long i = rlo[f] + (have ? u : 0);
        Pt<R> q1;
        R os[3];
        int c0, c1;
        load_start(a, sp, i, os, c0);
        load(a, sp, i, q1, c1);
        const bool live = have && c0 >= 0 && c1 >= 0;
        int cs[3], ce[3];
        decode_cell(a, live ? c0 : 0, cs);
        decode_cell(a, live ? c1 : 0, ce);
        // the end cell unwrapped next to the start (a step moves < 1 cell)
        bool inside = tile, incell = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          int dc = ce[c] - cs[c];
          const R disp = R(dc) + q1.off[c] - os[c];
          if (disp >= R(1)) dc -= a.n[c];
          else if (disp <= R(-1)) dc += a.n[c];
          q1.ci[c] = cs[c] + dc;
          incell &= dc == 0;
          // nodes cs - 1 .. cs + 2 cover every stencil of a move below one cell
          const int b0 = cs[c] - 1 - torg[c];
          inside &= b0 >= 0 && b0 + 3 < T;
        }
        const R qw = a.charge[sp] * q1.w;
        const unsigned act = __activemask();
        if (__all_sync(act, !live || (inside && incell))) {
          if (live) {
            deposit_in_cell<R, T>(a, jt_s + (unsigned)sizeof(R) * ((cs[2] - torg[2]) * TT + (cs[1] - torg[1]) * T +
                                                                   (cs[0] - torg[0])),
                                  os, q1.off, qw);
            ++in_tile;
          }
          continue;
        }
        if (!live) continue;
        if (!inside) {
          // drifted out of the tile since the sort: listed, and deposited
          // after this kernel by full warps (k_deposit_drift); a sparse
          // block without a tile deposits its records here
          if (tile && a.drift) {
            const unsigned slot = atomicAdd(a.work + 5, 1u);
            if ((long long)slot < a.drift_cap) {
              a.drift[slot] = ((unsigned long long)sp << 62) | (unsigned long long)i;
              continue;
            }
          }
          deposit(a, cs, os, q1, qw);
          continue;
        }
        EsirTerms<R> et;
        if (!esir_terms(a, cs, os, q1, qw, et)) {
          atomicOr(a.status, kStCourant);
          continue;
        }
        const unsigned o = jt_s + (unsigned)sizeof(R) * ((cs[2] - torg[2] + et.lo[2]) * TT +
                                                         (cs[1] - torg[1] + et.lo[1]) * T + (cs[0] - torg[0] + et.lo[0]));
        esir_apply(et, [&](int c, int i, int j, int k, R v) {
          red_shared_nz(o + (unsigned)sizeof(R) * (c * TTT + k * TT + j * T + i), v);
        });
        ++in_tile;
      }
      __syncthreads();
      if (tile) {
        for (int t = threadIdx.x; t < 3 * TTT; t += blockDim.x) {
          const R v = jt[t];
          if (v == R(0)) continue;
          const int c = t / TTT, r = t - c * TTT;
          const int tk = r / TT, r2 = r - tk * TT;
          const int tj = r2 / T, ti = r2 - tj * T;
          atomicAdd(a.J[c] + gofs[2][tk] + gofs[1][tj] + gofs[0][ti], v);
        }
        __syncthreads();   // the tile, rlo and rn are reused by the next cell block
      }
    }
  }
  unsigned long long v = in_tile;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.counters + kCntTileDeposits, v);
}

// The listed records that drifted out of their block's tile: the
// Esirkepov current of each straight into J, by full warps.
template <typename R>
__global__ void __launch_bounds__(256) k_deposit_drift(const StepArgs<R> a) {
  const long long n = min((long long)a.work[5], a.drift_cap);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const unsigned long long d = a.drift[k];
    const int sp = (int)(d >> 62);
    const long long i = (long long)(d & ((1ull << 62) - 1));
    Pt<R> q1;
    R os[3];
    int c0, c1;
    load_start(a, sp, i, os, c0);
    load(a, sp, i, q1, c1);
    int cs[3], ce[3];
    decode_cell(a, c0, cs);
    decode_cell(a, c1, ce);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      int dc = ce[c] - cs[c];
      const R disp = R(dc) + q1.off[c] - os[c];
      if (disp >= R(1)) dc -= a.n[c];
      else if (disp <= R(-1)) dc += a.n[c];
      q1.ci[c] = cs[c] + dc;
    }
    deposit(a, cs, os, q1, a.charge[sp] * q1.w);
  }
}

// Dynamic shared memory of the deposit kernel for a tile halo.
template <typename R> size_t deposit_smem(int halo) {
  return halo > 0 ? 3 * sizeof(R) * (size_t)tile_nodes(halo) * tile_nodes(halo) * tile_nodes(halo) : 0;
}

// The deposit kernel of a tile halo (the tile edge is a compile-time constant).
template <typename R> const void *deposit_kernel(int halo) {
  switch (halo) {
    case 0: return (const void *)k_deposit_blocks<R, 0>;
    case 1: return (const void *)k_deposit_blocks<R, 1>;
    case 2: return (const void *)k_deposit_blocks<R, 2>;
    case 3: return (const void *)k_deposit_blocks<R, 3>;
    default: return (const void *)k_deposit_blocks<R, 4>;
  }
}

// Passes 1, 2, ...: products evolving for the rest of the step.  All blocks
// are co-resident (cooperative launch) and meet at a bounded grid barrier
// between passes; pass p reads the buffer filled in pass p-1.
template <typename R, bool EXT>
__global__ void __launch_bounds__(256, 2) k_products(const StepArgs<R> a) {
  Cnt cnt;
  const R chi_star = (R)*a.chi_star;
  const unsigned step = ((const StepConst *)a.step_const)->step;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int pass = 1; pass <= kMaxPass; ++pass) {
    if (pass > 1 && !grid_barrier(a.barrier, a.status)) break;
    const long long n = (long long)*((volatile unsigned long long *)(a.pend_count + pass));
    if (n == 0) break;
    if (pass == kMaxPass) { atomicOr(a.status, kStTimeout); break; }
    const long long lim = n < a.pend_cap ? n : a.pend_cap;
    const Pend<R> *buf = (const Pend<R> *)a.pend[pass & 1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += stride) {
      const Pend<R> r = buf[i];
      Pt<R> q;
      q.off[0] = r.off[0]; q.off[1] = r.off[1]; q.off[2] = r.off[2];
      q.ci[0] = r.ci[0]; q.ci[1] = r.ci[1]; q.ci[2] = r.ci[2];
      q.p = r.p; q.w = r.w;
      q.id = product_id(a, r.parent, step, r.sub, r.kind);
      bool alive = true;
      if (r.sp == kPhoton) alive = advance_photon<R, EXT>(a, pass, q, r.trem, r.E, r.B, cnt, nullptr, chi_star, step);
      else advance_massive<R, EXT>(a, pass, r.sp, q, r.trem, r.E, r.B, cnt, nullptr, step);
      if (alive) {
        Pt<R> fin = q;   // a copy: q itself stays in registers
        count_outcome(a, append(a, r.sp, fin));
      }
    }
  }
  flush(cnt, a.counters);
}

template <typename R, bool EXT>
int launch(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  StepArgs<R> a{};
  for (int sp = 0; sp < 4; ++sp) {
    const Store &st = c->st[sp];
    a.pos[sp] = st.pos[st.cur];
    a.mom[sp] = st.mom[st.cur];
    a.pos_scratch[sp] = st.pos[st.cur ^ 1];
    a.id[sp] = st.id[st.cur];
    a.cap[sp] = st.cap;
    a.charge[sp] = (R)c->species.charge[sp];
    a.mass[sp] = (R)c->species.mass[sp];
    a.inv_mass[sp] = c->species.mass[sp] > 0.0 ? (R)(1.0 / c->species.mass[sp]) : R(0);
  }
  a.count = c->d_count;
  a.nstart = c->d_nstart;
  a.pend[0] = c->pend[0];
  a.pend[1] = c->pend[1];
  a.pend_count = c->d_pend_count;
  a.pend_cap = c->pend_cap;
  fast_div_magic((unsigned)c->grid.n[0], a.div_m[0], a.div_l[0]);
  fast_div_magic((unsigned)(c->grid.n[0] * c->grid.n[1]), a.div_m[1], a.div_l[1]);
  for (int k = 0; k < 3; ++k) {
    a.n[k] = c->grid.n[k];
    a.periodic[k] = c->grid.periodic[k];
    a.d[k] = (R)c->grid.d[k];
    a.inv_d[k] = (R)(1.0 / c->grid.d[k]);
    a.dd[k] = c->grid.d[k];
    a.x0[k] = c->grid.x0[k];
  }
  a.field_mode = c->grid.field_mode;
  for (int k = 0; k < 16; ++k) a.fp[k] = c->grid.fp[k];
  a.ens_shift = c->par.ens_bits > 0 ? 64 - c->par.ens_bits : 64;
  a.ens_mask = c->par.ens_bits > 0 ? ~0ull << (64 - c->par.ens_bits) : 0ull;
  a.n_ens = c->n_ens;
  a.ens_table = c->d_ens;
  a.ens_field = (R *)c->d_ens_field;
  a.ens_hmax = c->ens_hmax;
  {
    const double efg = c->par.emit_fg > 1.0 ? c->par.emit_fg : 1.0;
    const double pfg = c->par.pair_fg > 1.0 ? c->par.pair_fg : 1.0;
    a.emit_ng = c->par.emit_ng > 1 ? c->par.emit_ng : 1;
    a.pair_ng = c->par.pair_ng > 1 ? c->par.pair_ng : 1;
    a.emit_keep = (R)(1.0 / efg);
    a.pair_keep = (R)(1.0 / pfg);
    a.emit_wf = (R)(efg / (double)a.emit_ng);
    a.pair_wf = (R)(pfg / (double)a.pair_ng);
  }
  a.schwinger = c->par.schwinger_on;
  a.schwinger_w = (R)c->par.schwinger_weight;
  a.generator = c->par.generator;
  a.std_cdf = (const R *)c->d_std_cdf;
  a.std_lnw = (const R *)c->d_std_lnw;
  a.chunk = c->tune.work_chunk;
  a.work_massive = c->d_pend_count + kWorkSlot;
  a.clock = c->d_clock;
  a.dt_d = dt;
  if (a.field_mode == kFieldGrid) {
    for (int k = 0; k < 3; ++k) {
      a.E[k] = (const R *)f->E[k];
      a.B[k] = (const R *)f->B[k];
      a.J[k] = (R *)f->J[k];
    }
  }
  a.deposit = (a.field_mode == kFieldGrid) && c->par.deposit_on;
  a.deposit_halo = c->tune.deposit_halo;
  a.refill_lanes = c->tune.refill_lanes;
  a.dt = (R)dt;
  {
    const double vol = c->grid.d[0] * c->grid.d[1] * c->grid.d[2];
    for (int k = 0; k < 3; ++k) a.jscale[k] = (R)(c->grid.d[k] / dt / vol);
  }
  a.kappa = (R)c->par.kappa;
  a.nsub_max = c->par.nsub_max;
  a.emission_on = c->par.emission_on;
  a.pairs_on = c->par.pairs_on;
  a.same_step = c->par.same_step_children;
  a.pm_strict = c->par.pm_strict;
  a.seed = c->par.seed;
  a.tab = (const R *)c->d_tables;
  a.chi_star = c->d_chi_star;
  a.nblk = c->nblk;
  for (int k = 0; k < 3; ++k) a.nb[k] = c->nb[k];
  for (int sp = 0; sp < 4; ++sp)
    a.blk_start[sp] = (c->sorted && c->nblk > 0 && !c->key_ensembles && sp != kPhoton && c->st[sp].cap > 0)
                          ? c->d_blk_start + (size_t)sp * (c->nblk + 1) : nullptr;
  a.work = (unsigned *)(c->d_pend_count + kMaxPass + 2);
  a.drift = c->d_drift;
  a.drift_cap = c->drift_cap;
  a.step_const = c->d_step_const;
  a.counters = c->d_counters;
  a.spectrum = c->d_spec;
  a.spectrum_energy = c->d_spec_e;
  a.nbins = c->par.nbins;
  a.lg_lo = c->par.lg_lo;
  a.lg_inv_span = 1.0 / (c->par.lg_hi - c->par.lg_lo);
  a.status = c->d_status;
  a.barrier = c->d_barrier;

  // the step starts with its resets (counts, J) on the stream
  qed_mark(c, QED_STAGE_BEGIN, s);
  if (cudaMemcpyAsync(c->d_nstart, c->d_count, 4 * sizeof(long long), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return QED_ERR_CUDA;
  if (cudaMemsetAsync(c->d_pend_count, 0, sizeof(unsigned long long) * (kMaxPass + 5), s) !=
      cudaSuccess)
    return QED_ERR_CUDA;
  if (a.deposit) {
    size_t nc = (size_t)a.n[0] * a.n[1] * a.n[2];
    for (int k = 0; k < 3; ++k)
      if (cudaMemsetAsync(a.J[k], 0, nc * sizeof(R), s) != cudaSuccess) return QED_ERR_CUDA;
  }
  // the mesh maxima: from the field update of the step before, within one
  // qed_step call, else read off the fields
  const bool have_max = a.field_mode == kFieldGrid && c->grid_max_ready;
  c->grid_max_ready = 0;
  if (have_max && fold_grid_max(c, s) != QED_OK) return QED_ERR_CUDA;
  a.grid_max = a.field_mode == kFieldGrid ? c->d_grid_max : nullptr;
  a.eps_star_out = a.field_mode == kFieldGrid ? c->d_eps_star : nullptr;
  if (a.grid_max && !have_max && cudaMemsetAsync(c->d_grid_max, 0, sizeof(unsigned long long) * 6, s) != cudaSuccess)
    return QED_ERR_CUDA;
  void *args[] = {(void *)&a};
  cudaError_t e = cudaSuccess;
  if (c->ev_start) cudaEventRecord(c->ev_start, s);
  if (a.grid_max && !have_max) {
    c->launches += 1;
    e = cudaLaunchKernel((const void *)k_grid_max<R>, dim3(c->num_sms * 4), dim3(256), args, 0, s);
  }
  c->launches += 3;
  if (e == cudaSuccess)
    e = cudaLaunchKernel((const void *)k_step_constants<R>, dim3(1),
                       dim3(a.field_mode == kFieldEnsemble ? 256 : 32), args, 0, s);
  qed_mark(c, QED_STAGE_CONSTANTS, s);
  // concurrent: the e-/e+/ion pass runs on the side stream beside the
  // photon pass (fork after the step constants, join before the products)
  const bool conc = c->tune.concurrent && c->side && !a.blk_start[kElectron];
  if (e == cudaSuccess && conc) {
    e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if (e == cudaSuccess)
      e = cudaLaunchKernel((const void *)k_pass0<R, false, EXT>, dim3(c->num_sms * c->tune.massive_blocks_per_sm),
                           dim3(256), args, 0, c->side);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
  }
  if (e == cudaSuccess)
    e = cudaLaunchKernel((const void *)k_photons<R, EXT>, dim3(c->num_sms * c->tune.photon_blocks_per_sm),
                         dim3(kPhotonThreads), args, 0, s);
  if (c->ev_photon) cudaEventRecord(c->ev_photon, s);
  qed_mark(c, QED_STAGE_PHOTONS, s);
  if (e == cudaSuccess && a.blk_start[kElectron]) {
    c->launches += 1;
    e = cudaLaunchKernel((const void *)k_blocks<R, EXT, false>, dim3(c->blocks_cells), dim3(256), args, 0, s);
    if (e == cudaSuccess && a.blk_start[kIon]) {
      c->launches += 1;
      e = cudaLaunchKernel((const void *)k_blocks<R, EXT, true>, dim3(c->blocks_cells_ions), dim3(256), args, 0, s);
    }
    qed_mark(c, QED_STAGE_BLOCKS, s);
    if (e == cudaSuccess && a.deposit) {
      c->launches += 1;
      const void *kern = deposit_kernel<R>(a.deposit_halo);
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, deposit_smem<R>(a.deposit_halo)) !=
              cudaSuccess ||
          per_sm < 1)
        return QED_ERR_CUDA;
      // claims of 1 .. 32 cell blocks: eight or more per resident block
      const long long per = (long long)c->nblk / (8ll * per_sm * c->num_sms);
      a.deposit_grab = (int)(per < 1 ? 1 : (per > 32 ? 32 : per));
      e = cudaLaunchKernel(kern, dim3(per_sm * c->num_sms), dim3(256), args, deposit_smem<R>(a.deposit_halo), s);
      if (e == cudaSuccess && a.drift) {
        c->launches += 1;
        e = cudaLaunchKernel((const void *)k_deposit_drift<R>, dim3(c->num_sms * 4), dim3(256), args, 0, s);
      }
    }
  } else {
    qed_mark(c, QED_STAGE_BLOCKS, s);
  }
  qed_mark(c, QED_STAGE_DEPOSIT, s);
  if (e == cudaSuccess && conc) e = cudaStreamWaitEvent(s, c->ev_join, 0);
  else if (e == cudaSuccess)
    e = cudaLaunchKernel((const void *)k_pass0<R, false, EXT>, dim3(c->num_sms * c->tune.massive_blocks_per_sm),
                         dim3(256), args, 0, s);
  qed_mark(c, QED_STAGE_MASSIVE, s);
  if (e == cudaSuccess && a.same_step) {
    c->launches += 1;
    e = cudaLaunchCooperativeKernel((const void *)k_products<R, EXT>, dim3(c->blocks_products), dim3(256), args, 0, s);
  }
  qed_mark(c, QED_STAGE_PRODUCTS, s);
  if (e == cudaSuccess && a.schwinger) {
    c->launches += 1;
    e = cudaLaunchKernel((const void *)k_schwinger<R>, dim3(c->num_sms * 8), dim3(256), args, 0, s);
  }
  qed_mark(c, QED_STAGE_SCHWINGER, s);
  if (c->ev_stop) cudaEventRecord(c->ev_stop, s);
  return e == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}


template <typename R, bool EXT>
int step_blocks(qed_ctx *c) {
  int a = 0, b = 0, p = 0, g = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g, k_blocks<R, EXT, false>, 256, 0) != cudaSuccess || g < 1)
    return QED_ERR_CUDA;
  c->blocks_cells = g * c->num_sms;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g, k_blocks<R, EXT, true>, 256, 0) != cudaSuccess || g < 1)
    return QED_ERR_CUDA;
  c->blocks_cells_ions = g * c->num_sms;
  for (int h = 1; h <= kMaxDepositHalo; ++h)
    if (cudaFuncSetAttribute(deposit_kernel<R>(h), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)deposit_smem<R>(h)) != cudaSuccess)
      return QED_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_photons<R, EXT>, qed::kPhotonThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pass0<R, false, EXT>, 256, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, k_products<R, EXT>, 256, 0) != cudaSuccess ||
      a < 1 || b < 1 || p < 1)
    return QED_ERR_CUDA;
  c->blocks_photon = a * c->num_sms;
  c->blocks_massive = b * c->num_sms;
  c->blocks_products = p * c->num_sms;   // co-resident: the barrier needs every block running
  return QED_OK;
}

// Occupancy limits of the photon and the e-/e+/ion passes (blocks per SM).
template <typename R, bool EXT>
int max_blocks(int *photon, int *massive) {
  cudaError_t e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(photon, k_photons<R, EXT>, kPhotonThreads, 0);
  cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(massive, k_pass0<R, false, EXT>, 256, 0);
  return (e1 == cudaSuccess && e2 == cudaSuccess && *photon >= 1 && *massive >= 1) ? QED_OK : QED_ERR_CUDA;
}

}  // namespace
}  // namespace qed
