// Rate-table build (FP64, on the device, once at init).
//
// The emission density Eq. (24) and the pair density Eq. (30) need the
// synchrotron functions F1(z) = z int_z^inf K_{5/3} and F2(z) = z K_{2/3}(z)
// (Sec. IV.E).  Following the tabulation the paper recommends (Sec. IV.F),
// g1 = F1 z^{-1/3} and g2 = F2 z^{-1/3} are fitted per sub-interval of each
// binade of z by Chebyshev interpolation at D+1 nodes and stored as monomial
// coefficients in t in [-1,1] (layout in qed_device.cuh, Tab<R>).
#include <cmath>

#include "qed_internal.h"

namespace qed {
namespace {

// F1 and F2 at x > 0 from K_nu(x) = int_0^inf exp(-x cosh u) cosh(nu u) du and
// int_x^inf K_nu = int_0^inf exp(-x cosh u) cosh(nu u)/cosh(u) du, summed with
// the trapezoidal rule (exponentially convergent for these even, analytic
// integrands).  The step resolves the exp(-x u^2/2) core at large x.
__device__ void syn_quadrature(double x, double &f1, double &f2) {
  double h = fmin(1.0 / 16.0, 0.45 / sqrt(x));
  double peak = asinh(0.6666666666666666 / x);
  double a = 0.5 * exp(-x), b = a;
  for (int k = 1; k < 4000000; ++k) {
    double u = k * h;
    double ch = cosh(u);
    double e = exp(-x * ch);
    double ta = e * cosh(1.6666666666666667 * u) / ch;
    double tb = e * cosh(0.6666666666666666 * u);
    a += ta;
    b += tb;
    if (u > peak && ta < 1e-19 * a && tb < 1e-19 * b) break;
  }
  f1 = x * h * a;
  f2 = x * h * b;
}

template <typename R>
__global__ void k_tab_nodes(double *nodes) {
  using C = Tab<R>;
  const int total = C::NB * C::S * C::NC;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int k = i % C::NC;
  int s = (i / C::NC) % C::S;
  int b = i / (C::NC * C::S);
  int e = b + C::EMIN;
  double t = cos(3.141592653589793 * (k + 0.5) / C::NC);
  double z = ldexp(1.0 + (s + 0.5 * (t + 1.0)) / C::S, e);
  double f1, f2;
  syn_quadrature(z, f1, f2);
  double c = cbrt(z);
  double sc = e >= 0 ? exp(z) : 1.0;
  nodes[i] = f1 / c * sc;
  nodes[total + i] = f2 / c * sc;
}

template <typename R>
__global__ void k_tab_coefs(const double *nodes, R *tab) {
  using C = Tab<R>;
  const int per = C::NB * C::S;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    double g23 = tgamma(2.0 / 3.0);
    tab[0] = (R)(cbrt(4.0) * g23);          // g1(0) = 2^{2/3} Gamma(2/3)
    tab[1] = (R)(g23 / cbrt(2.0));          // g2(0) = 2^{-1/3} Gamma(2/3)
    tab[2] = (R)(3.141592653589793 / sqrt(3.0));
    tab[3] = (R)0;
  }
  if (i >= 2 * per) return;
  int f = i / per, bs = i % per;
  const double *v = nodes + f * per * C::NC + bs * C::NC;
  // Chebyshev coefficients a_j = (2/n) sum_k v_k T_j(t_k), a_0 halved
  double a[C::NC];
  for (int j = 0; j < C::NC; ++j) {
    double acc = 0.0;
    for (int k = 0; k < C::NC; ++k) acc += v[k] * cos(3.141592653589793 * j * (k + 0.5) / C::NC);
    a[j] = 2.0 * acc / C::NC;
  }
  a[0] *= 0.5;
  // monomial form: sum_j a_j T_j(t), T_{j+1} = 2 t T_j - T_{j-1}
  double mono[C::NC], tm1[C::NC], t0[C::NC], t1[C::NC];
  for (int j = 0; j < C::NC; ++j) { mono[j] = 0.0; tm1[j] = 0.0; t0[j] = 0.0; }
  t0[0] = 1.0;
  mono[0] += a[0];
  if (C::NC > 1) {
    for (int j = 0; j < C::NC; ++j) tm1[j] = t0[j];
    for (int j = 0; j < C::NC; ++j) t0[j] = 0.0;
    t0[1] = 1.0;
    for (int j = 0; j < C::NC; ++j) mono[j] += a[1] * t0[j];
    for (int n = 2; n < C::NC; ++n) {
      for (int j = 0; j < C::NC; ++j) t1[j] = (j > 0 ? 2.0 * t0[j - 1] : 0.0) - tm1[j];
      for (int j = 0; j < C::NC; ++j) { tm1[j] = t0[j]; t0[j] = t1[j]; mono[j] += a[n] * t1[j]; }
    }
  }
  R *out = tab + C::kHeader + f * per * C::NC + bs * C::NC;
  for (int j = 0; j < C::NC; ++j) out[j] = (R)mono[j];
}

template <typename R>
int build_into(qed_ctx *c, R *dst, cudaStream_t s) {
  using C = Tab<R>;
  const int total = C::NB * C::S * C::NC;
  double *nodes = nullptr;
  if (cudaMallocAsync(&nodes, sizeof(double) * 2 * total, s) != cudaSuccess) return QED_ERR_CUDA;
  c->launches += 2;
  k_tab_nodes<R><<<(total + 127) / 128, 128, 0, s>>>(nodes);
  k_tab_coefs<R><<<(2 * C::NB * C::S + 127) / 128, 128, 0, s>>>(nodes, dst);
  cudaError_t err = cudaGetLastError();
  cudaFreeAsync(nodes, s);
  return err == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

template <typename R>
int build(qed_ctx *c, cudaStream_t s) {
  return build_into<R>(c, (R *)c->d_tables, s);
}

// Standard event generator tables (Sec. IV.F), in FP64: for each chi_j the
// cumulative W(s^3) = int_0^s 3 t^2 G(t^3, chi_j) dt over the s grid, by
// 8-point Gauss-Legendre per cell (the integrand is smooth in s: it is the
// modified generator's 3 r1^2 G(r1^3)), normalised by W(1), and ln W(1).
__constant__ double kGL8x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                                0.7966664774136267,  0.9602898564975363};
__constant__ double kGL8w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                0.2223810344533745, 0.1012285362903763};

template <typename R>
__global__ void __launch_bounds__(256) k_std_rows(const double *tab64, R *cdf, R *lnw) {
  constexpr int NI = kStdCols - 1;          // cells per row
  constexpr int PER = NI / 256;             // cells per thread (consecutive)
  static_assert(NI % 256 == 0, "cells per row");
  __shared__ double part[256];
  const int j = blockIdx.x;
  const double chi = exp(kStdLnChiLo + j * kStdDLn);
  double cell[PER], mine = 0.0;
  for (int k = 0; k < PER; ++k) {
    const int i = threadIdx.x * PER + k;
    const double a = (double)i / NI, b = (double)(i + 1) / NI, m = 0.5 * (a + b), r = 0.5 * (b - a);
    double acc = 0.0;
    for (int q = 0; q < 8; ++q)
      acc += kGL8w[q] * prob_emit<double>(tab64, m + r * kGL8x[q], chi, 1.0, 1.0 / kAlpha);
    cell[k] = r * acc;
    mine += cell[k];
  }
  part[threadIdx.x] = mine;
  __syncthreads();
  // inclusive scan of the per-thread sums (Hillis-Steele)
  for (int o = 1; o < 256; o <<= 1) {
    const double v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0.0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const double total = part[255];
  double run = part[threadIdx.x] - mine;
  R *row = cdf + (size_t)j * kStdCols;
  if (threadIdx.x == 0) row[0] = R(0);
  for (int k = 0; k < PER; ++k) {
    run += cell[k];
    const int i = threadIdx.x * PER + k + 1;
    row[i] = i == NI ? R(1) : (R)(run / total);
  }
  if (threadIdx.x == 0) lnw[j] = (R)log(total);
}

template <typename R>
int build_standard(qed_ctx *c, cudaStream_t s) {
  const double *tab64 = nullptr;
  double *tmp = nullptr;
  if (c->prec == 64) {
    tab64 = (const double *)c->d_tables;
  } else {
    // a temporary FP64 synchrotron table, used only to fill the standard generator's table
    if (cudaMallocAsync(&tmp, sizeof(double) * Tab<double>::kSize, s) != cudaSuccess) return QED_ERR_CUDA;
    int rc = build_into<double>(c, tmp, s);
    if (rc != QED_OK) {
      cudaFreeAsync(tmp, s);
      return rc;
    }
    tab64 = tmp;
  }
  c->launches += 1;
  k_std_rows<R><<<kStdRows, 256, 0, s>>>(tab64, (R *)c->d_std_cdf, (R *)c->d_std_lnw);
  cudaError_t err = cudaGetLastError();
  if (tmp) cudaFreeAsync(tmp, s);
  return err == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

}  // namespace
}  // namespace qed

int qed_build_tables(qed_ctx *c, cudaStream_t s) {
  return c->prec == 64 ? qed::build<double>(c, s) : qed::build<float>(c, s);
}

int qed_build_standard_tables(qed_ctx *c, cudaStream_t s) {
  return c->prec == 64 ? qed::build_standard<double>(c, s) : qed::build_standard<float>(c, s);
}
