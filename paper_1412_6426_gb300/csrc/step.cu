// The particle step: field gather, Boris push, adaptive event generator with
// photon emission and pair creation, append of products, Esirkepov deposit.
//
// One persistent launch per step (all species).  Pass 0 advances every
// particle alive at the start of the step by dt, with the fields taken once
// at its start position (Sec. IV.H: no re-interpolation inside the step).
// Products created in sub-interval s of an N-interval loop carry the time
// left, (N-1-s) h, and the parent's frozen fields into a product buffer;
// passes 1, 2, ... (separated by a bounded grid barrier) advance them for that
// time, and so on until no products are left.  Finished products are appended
// to their species stores.  Dead particles keep their slot (cell = -1) until
// the next compaction.
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

// A product waiting to evolve for the rest of the step.
template <typename R> struct Pend {
  R off[3];
  R w;
  V3<R> p;
  R trem;
  V3<R> E, B;
  int ci[3];
  int sp;
  uint64_t id;
};

struct Cnt {
  unsigned long long sub_l = 0, sub_g = 0, psteps = 0;
  unsigned emis = 0, pairs = 0, pm1 = 0, pp1 = 0, capped = 0, absorbed = 0, overflow = 0, nonfin = 0;
};

// ----- store access --------------------------------------------------------
__device__ __forceinline__ void load(const StepArgs<float> &a, int sp, long long i, Pt<float> &q,
                                     int &cell) {
  float4 P = __ldg((const float4 *)a.pos[sp] + i);
  float4 M = __ldg((const float4 *)a.mom[sp] + i);
  q.off[0] = P.x; q.off[1] = P.y; q.off[2] = P.z; q.w = P.w;
  q.p = {M.x, M.y, M.z};
  cell = __float_as_int(M.w);
  q.id = __ldg(a.id[sp] + i);
}
__device__ __forceinline__ void load(const StepArgs<double> &a, int sp, long long i, Pt<double> &q,
                                     int &cell) {
  const double2 *P = (const double2 *)a.pos[sp] + 2 * i;
  const double2 *M = (const double2 *)a.mom[sp] + 2 * i;
  double2 p0 = __ldg(P), p1 = __ldg(P + 1), m0 = __ldg(M), m1 = __ldg(M + 1);
  q.off[0] = p0.x; q.off[1] = p0.y; q.off[2] = p1.x; q.w = p1.y;
  q.p = {m0.x, m0.y, m1.x};
  cell = (int)m1.y;
  q.id = __ldg(a.id[sp] + i);
}
__device__ __forceinline__ void store(const StepArgs<float> &a, int sp, long long i,
                                      const Pt<float> &q, int cell, bool with_id) {
  ((float4 *)a.pos[sp])[i] = make_float4(q.off[0], q.off[1], q.off[2], q.w);
  ((float4 *)a.mom[sp])[i] = make_float4(q.p.x, q.p.y, q.p.z, __int_as_float(cell));
  if (with_id) a.id[sp][i] = q.id;
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

// ----- fields --------------------------------------------------------------
__device__ __forceinline__ void sincos_2pi_frac(double cycles, float &s, float &c) {
  double f = cycles - rint(cycles);
  sincospif((float)(2.0 * f), &s, &c);
}
__device__ __forceinline__ void sincos_2pi_frac(double cycles, double &s, double &c) {
  double f = cycles - rint(cycles);
  sincospi(2.0 * f, &s, &c);
}

// Analytic fields at the particle position and time a.t (modes of qed.h).
template <typename R>
__device__ void field_analytic(const StepArgs<R> &a, const Pt<R> &q, V3<R> &E, V3<R> &B) {
  E = {R(0), R(0), R(0)};
  B = {R(0), R(0), R(0)};
  if (a.field_mode == kFieldUniform) {
    E = {R(a.fp[0]), R(a.fp[1]), R(a.fp[2])};
    B = {R(a.fp[3]), R(a.fp[4]), R(a.fp[5])};
  } else if (a.field_mode == kFieldRotatingE) {
    R s, c;
    sincos_2pi_frac(a.fp[1] * a.t * (1.0 / kTwoPi), s, c);
    E = {R(a.fp[0]) * c, R(a.fp[0]) * s, R(0)};
  } else if (a.field_mode == kFieldGaussianLP) {
    // zeta: distance travelled past the focus along -x; eta: retarded time.
    // The carrier phase is formed in FP64 and reduced to one cycle.
    double xa = a.x0[0] + ((double)q.ci[0] + (double)q.off[0]) * a.dd[0];
    double zeta_d = a.fp[4] - xa;
    double eta_d = (a.t - a.fp[7]) - zeta_d;
    R y = R(a.x0[1] - a.fp[5]) + (R(q.ci[1]) + q.off[1]) * a.d[1];
    R z = R(a.x0[2] - a.fp[6]) + (R(q.ci[2]) + q.off[2]) * a.d[2];
    R w = R(a.fp[1]), w0 = R(a.fp[2]), tau = R(a.fp[3]);
    R zeta = R(zeta_d), eta = R(eta_d);
    R zr = R(0.5) * w * w0 * w0;
    R rz = zeta / zr;
    R wz2 = w0 * w0 * (R(1) + rz * rz);
    R r2 = y * y + z * z;
    R invR = zeta / (zeta * zeta + zr * zr);
    R gouy = atan(rz);
    R extra = -R(0.5) * w * r2 * invR + gouy + R(a.fp[8]);
    double cycles = a.fp[1] * eta_d * (1.0 / kTwoPi) + (double)extra * (1.0 / kTwoPi);
    R s, c;
    sincos_2pi_frac(cycles, s, c);
    R env = exp_r(R(-2.0 * 0.6931471805599453) * eta * eta / (tau * tau));
    R amp = R(a.fp[0]) * sqrt_r(w0 * w0 / wz2) * exp_r(-r2 / wz2) * env;
    E.y = amp * c;
    B.z = -E.y;
  }
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// CIC gather of one staggered component (stagger sx, sy, sz in {0, 1/2}).
template <typename R>
__device__ __forceinline__ R cic(const R *__restrict__ f, const StepArgs<R> &a, const int *ci,
                                 const R *off, int sx, int sy, int sz) {
  int b[3];
  R fr[3];
  const int sg[3] = {sx, sy, sz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R v = sg[c] ? off[c] - R(0.5) : off[c];
    int bb = ci[c];
    if (v < R(0)) { v += R(1); bb -= 1; }
    b[c] = bb;
    fr[c] = v;
  }
  int i0 = wrapi(b[0], a.n[0]), i1 = wrapi(b[0] + 1, a.n[0]);
  int j0 = wrapi(b[1], a.n[1]), j1 = wrapi(b[1] + 1, a.n[1]);
  int k0 = wrapi(b[2], a.n[2]), k1 = wrapi(b[2] + 1, a.n[2]);
  long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
  R acc = R(0);
  acc += (R(1) - fr[0]) * (R(1) - fr[1]) * (R(1) - fr[2]) * __ldg(f + k0 * nxy + j0 * nx + i0);
  acc += fr[0] * (R(1) - fr[1]) * (R(1) - fr[2]) * __ldg(f + k0 * nxy + j0 * nx + i1);
  acc += (R(1) - fr[0]) * fr[1] * (R(1) - fr[2]) * __ldg(f + k0 * nxy + j1 * nx + i0);
  acc += fr[0] * fr[1] * (R(1) - fr[2]) * __ldg(f + k0 * nxy + j1 * nx + i1);
  acc += (R(1) - fr[0]) * (R(1) - fr[1]) * fr[2] * __ldg(f + k1 * nxy + j0 * nx + i0);
  acc += fr[0] * (R(1) - fr[1]) * fr[2] * __ldg(f + k1 * nxy + j0 * nx + i1);
  acc += (R(1) - fr[0]) * fr[1] * fr[2] * __ldg(f + k1 * nxy + j1 * nx + i0);
  acc += fr[0] * fr[1] * fr[2] * __ldg(f + k1 * nxy + j1 * nx + i1);
  return acc;
}

template <typename R>
__device__ void gather_grid(const StepArgs<R> &a, const Pt<R> &q, V3<R> &E, V3<R> &B) {
  E.x = cic(a.E[0], a, q.ci, q.off, 1, 0, 0);
  E.y = cic(a.E[1], a, q.ci, q.off, 0, 1, 0);
  E.z = cic(a.E[2], a, q.ci, q.off, 0, 0, 1);
  B.x = cic(a.B[0], a, q.ci, q.off, 0, 1, 1);
  B.y = cic(a.B[1], a, q.ci, q.off, 1, 0, 1);
  B.z = cic(a.B[2], a, q.ci, q.off, 1, 1, 0);
}

// ----- Esirkepov deposit (linear shape) ------------------------------------
template <typename R>
__device__ void deposit(const StepArgs<R> &a, const int *cs, const R *os, const Pt<R> &q, R qw) {
  R S0[3][4], dS[3][4];
  int base[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    base[c] = cs[c] - 1;
    R ua = R(1) + os[c];
    R ub = R(q.ci[c] - cs[c] + 1) + q.off[c];
    if (!(fabs(ub - ua) < R(1))) { atomicOr(a.status, kStCourant); return; }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      R s0 = R(1) - fabs(ua - R(m));
      R s1 = R(1) - fabs(ub - R(m));
      s0 = s0 > R(0) ? s0 : R(0);
      s1 = s1 > R(0) ? s1 : R(0);
      S0[c][m] = s0;
      dS[c][m] = s1 - s0;
    }
  }
  const R inv_vol = a.inv_d[0] * a.inv_d[1] * a.inv_d[2];
  const R pref[3] = {-qw * a.d[0] / a.dt * inv_vol, -qw * a.d[1] / a.dt * inv_vol,
                     -qw * a.d[2] / a.dt * inv_vol};
  long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
  int I[4], Jj[4], K[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    I[m] = wrapi(base[0] + m, a.n[0]);
    Jj[m] = wrapi(base[1] + m, a.n[1]);
    K[m] = wrapi(base[2] + m, a.n[2]);
  }
  const R third = R(1.0 / 3.0);
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 4; ++j) {
      R acc = R(0);
      R wyz = S0[1][j] * S0[2][k] + R(0.5) * dS[1][j] * S0[2][k] + R(0.5) * S0[1][j] * dS[2][k] +
              third * dS[1][j] * dS[2][k];
      for (int i = 0; i < 4; ++i) {
        acc += pref[0] * dS[0][i] * wyz;
        if (acc != R(0)) atomicAdd(a.J[0] + K[k] * nxy + Jj[j] * nx + I[i], acc);
      }
    }
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 4; ++i) {
      R acc = R(0);
      R wxz = S0[0][i] * S0[2][k] + R(0.5) * dS[0][i] * S0[2][k] + R(0.5) * S0[0][i] * dS[2][k] +
              third * dS[0][i] * dS[2][k];
      for (int j = 0; j < 4; ++j) {
        acc += pref[1] * dS[1][j] * wxz;
        if (acc != R(0)) atomicAdd(a.J[1] + K[k] * nxy + Jj[j] * nx + I[i], acc);
      }
    }
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < 4; ++i) {
      R acc = R(0);
      R wxy = S0[0][i] * S0[1][j] + R(0.5) * dS[0][i] * S0[1][j] + R(0.5) * S0[0][i] * dS[1][j] +
              third * dS[0][i] * dS[1][j];
      for (int k = 0; k < 4; ++k) {
        acc += pref[2] * dS[2][k] * wxy;
        if (acc != R(0)) atomicAdd(a.J[2] + K[k] * nxy + Jj[j] * nx + I[i], acc);
      }
    }
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
    if (a.periodic[c]) q.ci[c] = wrapi(q.ci[c], a.n[c]);
    else if (q.ci[c] < 0 || q.ci[c] >= a.n[c]) return -1;
  }
  return (q.ci[2] * a.n[1] + q.ci[1]) * a.n[0] + q.ci[0];
}

template <typename R>
__device__ void spectrum_add(const StepArgs<R> &a, R delta, R eps, R w) {
  if (a.nbins <= 0) return;
  double u = (log10((double)delta) - a.lg_lo) * a.lg_inv_span * a.nbins;
  if (u >= 0.0 && u < a.nbins) atomicAdd(a.spectrum + (int)u, (double)w);
  double v = (log10((double)eps) - a.lg_lo) * a.lg_inv_span * a.nbins;
  if (v >= 0.0 && v < a.nbins) atomicAdd(a.spectrum_energy + (int)v, (double)w);
}

// Append a finished particle to its store (warp-aggregated slot reservation).
template <typename R>
__device__ void append(const StepArgs<R> &a, int sp, Pt<R> &q, Cnt &cnt) {
  int cell = finish_cell(a, q);
  if (cell < 0) { cnt.absorbed++; return; }
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
    cnt.overflow++;
    return;
  }
  store(a, sp, slot, q, cell, true);
}

// Queue a product for the rest of the step (same_step), or append it now.
template <typename R>
__device__ void emit(const StepArgs<R> &a, int pass, int sp, Pt<R> &q, R trem, V3<R> E, V3<R> B,
                     Cnt &cnt) {
  if (a.same_step && trem > R(0)) {
    unsigned long long slot = atomicAdd(a.pend_count + pass + 1, 1ull);
    if ((long long)slot >= a.pend_cap) {
      atomicOr(a.status, kStCapacity);
      cnt.overflow++;
      return;
    }
    Pend<R> *r = (Pend<R> *)a.pend[(pass + 1) & 1] + slot;
    r->off[0] = q.off[0]; r->off[1] = q.off[1]; r->off[2] = q.off[2];
    r->w = q.w; r->p = q.p; r->trem = trem; r->E = E; r->B = B;
    r->ci[0] = q.ci[0]; r->ci[1] = q.ci[1]; r->ci[2] = q.ci[2];
    r->sp = sp; r->id = q.id;
  } else {
    append(a, sp, q, cnt);
  }
}

// Advance one particle by t_span with frozen fields.  Returns false when the
// particle was converted (photon -> pair).  The caller applies boundaries.
template <typename R>
__device__ bool advance(const StepArgs<R> &a, int pass, int sp, Pt<R> &q, R t_span, V3<R> E,
                        V3<R> B, Cnt &cnt) {
  const int cs[3] = {q.ci[0], q.ci[1], q.ci[2]};
  const R os[3] = {q.off[0], q.off[1], q.off[2]};
  bool alive = true;
  if (sp != kPhoton) {
    const R qc = a.charge[sp], m = a.mass[sp];
    const bool qed = (sp != kIon) && a.emission_on;
    int n = 1, capped = 0;
    if (qed) {
      R g0 = sqrt_r(R(1) + dot(q.p, q.p) / (m * m));
      n = nsub_lepton(t_span, g0, heff_lepton(q.p, g0, E, B), a.kappa, a.nsub_max, capped);
      cnt.capped += capped;
    }
    const R h = t_span / R(n);
    for (int s = 0; s < n; ++s) {
      boris(q.p, E, B, qc, m, h);
      R g = sqrt_r(R(1) + dot(q.p, q.p) / (m * m));
      R im = R(1) / (m * g);
      move(a, q, V3<R>{q.p.x * im, q.p.y * im, q.p.z * im}, h);
      if (!qed) continue;
      cnt.sub_l++;
      R chi = chi_lepton(q.p, g, E, B);
      R r1, r2;
      draw2(q.id, a.step, (unsigned)s, kEmit, a.seed, r1, r2);
      R pm = prob_emit(a.tab, r1, chi, g, h);
      if (pm > R(1)) {
        cnt.pm1++;
        if (a.pm_strict) atomicOr(a.status, kStPmGt1);
      }
      if (r2 < pm) {
        // photon along p with delta of it; the parent keeps (1 - delta)
        R delta = r1 * r1 * r1;
        Pt<R> ph = q;
        ph.p = {delta * q.p.x, delta * q.p.y, delta * q.p.z};
        ph.id = child_id(q.id, a.step, (unsigned)s, kPhoton, a.seed);
        R omd = R(1) - delta;
        q.p = {omd * q.p.x, omd * q.p.y, omd * q.p.z};
        cnt.emis++;
        spectrum_add(a, delta, sqrt_r(dot(ph.p, ph.p)), q.w);
        emit(a, pass, kPhoton, ph, R(n - 1 - s) * h, E, B, cnt);
      }
    }
    if (a.deposit && qc != R(0)) deposit(a, cs, os, q, qc * q.w);
  } else {
    const R eps = sqrt_r(dot(q.p, q.p));
    V3<R> dir = {R(0), R(0), R(0)};
    if (eps > R(0)) dir = {q.p.x / eps, q.p.y / eps, q.p.z / eps};
    const R hg = heff_photon(dir, E, B);
    const R chig = eps * hg;
    int n = 1, capped = 0;
    if (a.pairs_on) {
      n = nsub_photon(t_span, hg, a.kappa, a.nsub_max, capped);
      cnt.capped += capped;
    }
    const R h = t_span / R(n);
    for (int s = 0; s < n; ++s) {
      move(a, q, dir, h);
      if (!a.pairs_on) continue;
      cnt.sub_g++;
      R r1, r2;
      draw2(q.id, a.step, (unsigned)s, kPair, a.seed, r1, r2);
      R pp = prob_pair(a.tab, r1, chig, eps, h);
      if (pp > R(1)) {
        cnt.pp1++;
        if (a.pm_strict) atomicOr(a.status, kStPmGt1);
      }
      if (r2 < pp) {
        // electron takes r1 of the photon momentum, positron 1 - r1
        Pt<R> el = q, po = q;
        el.p = {r1 * q.p.x, r1 * q.p.y, r1 * q.p.z};
        R r1c = R(1) - r1;
        po.p = {r1c * q.p.x, r1c * q.p.y, r1c * q.p.z};
        el.id = child_id(q.id, a.step, (unsigned)s, kElectron, a.seed);
        po.id = child_id(q.id, a.step, (unsigned)s, kPositron, a.seed);
        cnt.pairs++;
        R trem = R(n - 1 - s) * h;
        emit(a, pass, kElectron, el, trem, E, B, cnt);
        emit(a, pass, kPositron, po, trem, E, B, cnt);
        alive = false;
        break;
      }
    }
  }
  return alive;
}

// Bounded grid barrier (all blocks are co-resident: cooperative launch).
// Gives up after ~1 s, sets the timeout status and returns false.
__device__ bool grid_barrier(unsigned *bar, int *status) {
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
        if (++it > (1ll << 24)) {
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
  unsigned long long v[kNumCounters] = {c.emis, c.pairs, c.sub_l, c.sub_g, c.pm1, c.pp1, c.capped,
                                         c.absorbed, c.overflow, c.nonfin, c.psteps};
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    unsigned long long x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(g + k, x);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_step(const StepArgs<R> a) {
  Cnt cnt;
  __shared__ long long ns[4];
  // an overflowing append leaves count above the capacity: never read past it
  if (threadIdx.x < 4) ns[threadIdx.x] = min(a.nstart[threadIdx.x], a.cap[threadIdx.x]);
  __syncthreads();
  const long long total = ns[0] + ns[1] + ns[2] + ns[3];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += stride) {
    int sp = 0;
    long long i = it;
    while (i >= ns[sp]) { i -= ns[sp]; ++sp; }
    Pt<R> q;
    int cell;
    load(a, sp, i, q, cell);
    if (cell < 0) continue;
    cnt.psteps++;
    q.ci[0] = cell % a.n[0];
    q.ci[1] = (cell / a.n[0]) % a.n[1];
    q.ci[2] = cell / (a.n[0] * a.n[1]);
    V3<R> E, B;
    if (a.field_mode == kFieldGrid) gather_grid(a, q, E, B);
    else field_analytic(a, q, E, B);
    if (!(isfinite(E.x) && isfinite(E.y) && isfinite(E.z) && isfinite(B.x) && isfinite(B.y) &&
          isfinite(B.z) && isfinite(q.p.x) && isfinite(q.p.y) && isfinite(q.p.z))) {
      cnt.nonfin++;
      atomicOr(a.status, kStNonfinite);
    }
    bool alive = advance(a, 0, sp, q, a.dt, E, B, cnt);
    int nc = alive ? finish_cell(a, q) : -1;
    if (alive && nc < 0) cnt.absorbed++;
    store(a, sp, i, q, nc, false);
  }
  if (a.same_step) {
    for (int pass = 1; pass <= kMaxPass; ++pass) {
      if (!grid_barrier(a.barrier, a.status)) break;
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
        q.p = r.p; q.w = r.w; q.id = r.id;
        if (advance(a, pass, r.sp, q, r.trem, r.E, r.B, cnt)) append(a, r.sp, q, cnt);
      }
    }
  }
  flush(cnt, a.counters);
}

template <typename R>
int launch(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  StepArgs<R> a{};
  for (int sp = 0; sp < 4; ++sp) {
    const Store &st = c->st[sp];
    a.pos[sp] = st.pos[st.cur];
    a.mom[sp] = st.mom[st.cur];
    a.id[sp] = st.id[st.cur];
    a.cap[sp] = st.cap;
    a.charge[sp] = (R)c->species.charge[sp];
    a.mass[sp] = (R)c->species.mass[sp];
  }
  a.count = c->d_count;
  a.nstart = c->d_nstart;
  a.pend[0] = c->pend[0];
  a.pend[1] = c->pend[1];
  a.pend_count = c->d_pend_count;
  a.pend_cap = c->pend_cap;
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
  a.t = c->time;
  if (a.field_mode == kFieldGrid) {
    for (int k = 0; k < 3; ++k) {
      a.E[k] = (const R *)f->E[k];
      a.B[k] = (const R *)f->B[k];
      a.J[k] = (R *)f->J[k];
    }
  }
  a.deposit = (a.field_mode == kFieldGrid) && c->par.deposit_on;
  a.dt = (R)dt;
  a.kappa = (R)c->par.kappa;
  a.nsub_max = c->par.nsub_max;
  a.emission_on = c->par.emission_on;
  a.pairs_on = c->par.pairs_on;
  a.same_step = c->par.same_step_children;
  a.pm_strict = c->par.pm_strict;
  a.seed = c->par.seed;
  a.step = (unsigned)c->step;
  a.tab = (const R *)c->d_tables;
  a.counters = c->d_counters;
  a.spectrum = c->d_spec;
  a.spectrum_energy = c->d_spec_e;
  a.nbins = c->par.nbins;
  a.lg_lo = c->par.lg_lo;
  a.lg_inv_span = 1.0 / (c->par.lg_hi - c->par.lg_lo);
  a.status = c->d_status;
  a.barrier = c->d_barrier;

  if (cudaMemcpyAsync(c->d_nstart, c->d_count, 4 * sizeof(long long), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return QED_ERR_CUDA;
  if (cudaMemsetAsync(c->d_pend_count, 0, sizeof(unsigned long long) * (kMaxPass + 2), s) !=
      cudaSuccess)
    return QED_ERR_CUDA;
  if (a.deposit) {
    size_t nc = (size_t)a.n[0] * a.n[1] * a.n[2];
    for (int k = 0; k < 3; ++k)
      if (cudaMemsetAsync(a.J[k], 0, nc * sizeof(R), s) != cudaSuccess) return QED_ERR_CUDA;
  }
  void *args[] = {(void *)&a};
  cudaError_t e;
  if (c->ev_start) cudaEventRecord(c->ev_start, s);
  c->launches += 1;
  if (a.same_step)
    e = cudaLaunchCooperativeKernel((const void *)k_step<R>, dim3(c->step_blocks), dim3(256), args, 0, s);
  else
    e = cudaLaunchKernel((const void *)k_step<R>, dim3(c->step_blocks), dim3(256), args, 0, s);
  if (c->ev_stop) cudaEventRecord(c->ev_stop, s);
  return e == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

}  // namespace
}  // namespace qed

int qed_step_kernel_blocks(qed_ctx *c) {
  int per_sm = 0;
  cudaError_t e = c->prec == 64
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qed::k_step<double>, 256, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qed::k_step<float>, 256, 0);
  if (e != cudaSuccess || per_sm < 1) return QED_ERR_CUDA;
  c->step_blocks = per_sm * c->num_sms;
  return QED_OK;
}

int qed_launch_step(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  return c->prec == 64 ? qed::launch<double>(c, f, dt, s) : qed::launch<float>(c, f, dt, s);
}

size_t qed_pend_bytes(int prec) {
  return prec == 64 ? sizeof(qed::Pend<double>) : sizeof(qed::Pend<float>);
}
