// Yee FDTD field update (Appendix C; Yee 1966), symmetrised in time as the
// paper does for its PIC loop (Appendix A): B half step, E full step with the
// deposited current, B half step, so E and B are both known at integer steps.
// Compton units: dB/dt = -curl E, dE/dt = curl B - 4 pi alpha J.  Periodic.
#include "qed_internal.h"

namespace qed {
namespace {

struct Mesh {
  int nx, ny, nz;
};

__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// One thread per cell; blocks of 32 x 8 cells in the x-y plane, blockIdx.z =
// k, so the cell's indices come from the launch (no division) and each warp
// reads 32 consecutive x.
__device__ __forceinline__ bool cell_ijk(const Mesh &m, int &i, int &j, int &k) {
  i = blockIdx.x * 32 + threadIdx.x;
  j = blockIdx.y * 8 + threadIdx.y;
  k = blockIdx.z;
  return i < m.nx && j < m.ny;
}

// |v| as ordered bits (the mesh maxima's encoding: FP32 bits zero-extended,
// FP64 bits; non-negative values order as their bits).
__device__ __forceinline__ unsigned long long abs_bits(float v) { return __float_as_uint(fabsf(v)); }
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

// Per component, the largest |value| the block wrote, into mx[0..2] of one
// of kMaxStripes stripes of 6 (atomicMax of the bits; blocks spread over
// the stripes, so that the atomics do not queue on three addresses);
// every thread of the block calls this.
template <typename R>
__device__ __forceinline__ void block_max3(bool in, R a, R b, R c, unsigned long long *mx) {
  __shared__ unsigned long long wm[8][3];
  unsigned long long m[3] = {in ? abs_bits(a) : 0ull, in ? abs_bits(b) : 0ull, in ? abs_bits(c) : 0ull};
  const int t = threadIdx.y * blockDim.x + threadIdx.x, warp = t >> 5;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, m[q], o);
      m[q] = x > m[q] ? x : m[q];
    }
    if ((t & 31) == 0) wm[warp][q] = m[q];
  }
  __syncthreads();
  if (t < 3) {
    unsigned long long v = 0;
    for (int w = 0; w < (int)(blockDim.x * blockDim.y) / 32; ++w) v = wm[w][t] > v ? wm[w][t] : v;
    const unsigned stripe = (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) % kMaxStripes;
    if (v) atomicMax(mx + 6 * stripe + t, v);
  }
}

// The maxima of the stripes, into out[0..5].
__global__ void k_max_fold(const unsigned long long *stripes, unsigned long long *out) {
  const int q = threadIdx.x;
  if (q >= 6) return;
  unsigned long long v = 0;
  for (int s = 0; s < kMaxStripes; ++s) v = stripes[6 * s + q] > v ? stripes[6 * s + q] : v;
  out[q] = v;
}

// B -= h * curl E   (curl E at the B positions, forward differences); with
// mx, the largest |B| of each component written goes to mx[0..2].
template <typename R>
__global__ void __launch_bounds__(256) k_yee_b(const R *__restrict__ Ex, const R *__restrict__ Ey,
                                               const R *__restrict__ Ez, R *Bx, R *By, R *Bz, Mesh m, R h_dx,
                                               R h_dy, R h_dz, unsigned long long *mx) {
  int i, j, k;
  const bool in = cell_ijk(m, i, j, k);
  R bx = R(0), by = R(0), bz = R(0);
  if (in) {
    const long long nx = m.nx, nxy = (long long)m.nx * m.ny;
    const long long c = k * nxy + j * nx + i;
    const long long ip = c - i + wrap_up(i, m.nx);
    const long long jp = c + (long long)(wrap_up(j, m.ny) - j) * nx;
    const long long kp = c + (long long)(wrap_up(k, m.nz) - k) * nxy;
    R ex = Ex[c], ey = Ey[c], ez = Ez[c];
    bx = Bx[c] - (h_dy * (Ez[jp] - ez) - h_dz * (Ey[kp] - ey));
    by = By[c] - (h_dz * (Ex[kp] - ex) - h_dx * (Ez[ip] - ez));
    bz = Bz[c] - (h_dx * (Ey[ip] - ey) - h_dy * (Ex[jp] - ex));
    Bx[c] = bx;
    By[c] = by;
    Bz[c] = bz;
  }
  if (mx) block_max3(in, bx, by, bz, mx);
}

// E += dt * (curl B - 4 pi alpha J)   (curl B at the E positions, backward
// differences); the largest |E| of each component written goes to mx[0..2].
template <typename R>
__global__ void __launch_bounds__(256) k_yee_e(R *Ex, R *Ey, R *Ez, const R *__restrict__ Bx,
                                               const R *__restrict__ By, const R *__restrict__ Bz,
                                               const R *__restrict__ Jx, const R *__restrict__ Jy,
                                               const R *__restrict__ Jz, Mesh m, R t_dx, R t_dy, R t_dz,
                                               R t_src, unsigned long long *mx) {
  int i, j, k;
  const bool in = cell_ijk(m, i, j, k);
  R ex = R(0), ey = R(0), ez = R(0);
  if (in) {
    const long long nx = m.nx, nxy = (long long)m.nx * m.ny;
    const long long c = k * nxy + j * nx + i;
    const long long im = c - i + wrap_dn(i, m.nx);
    const long long jm = c + (long long)(wrap_dn(j, m.ny) - j) * nx;
    const long long km = c + (long long)(wrap_dn(k, m.nz) - k) * nxy;
    R bx = Bx[c], by = By[c], bz = Bz[c];
    ex = Ex[c] + (t_dy * (bz - Bz[jm]) - t_dz * (by - By[km]) - t_src * Jx[c]);
    ey = Ey[c] + (t_dz * (bx - Bx[km]) - t_dx * (bz - Bz[im]) - t_src * Jy[c]);
    ez = Ez[c] + (t_dx * (by - By[im]) - t_dy * (bx - Bx[jm]) - t_src * Jz[c]);
    Ex[c] = ex;
    Ey[c] = ey;
    Ez[c] = ez;
  }
  if (mx) block_max3(in, ex, ey, ez, mx);
}

template <typename R>
int yee(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  Mesh m{c->grid.n[0], c->grid.n[1], c->grid.n[2]};
  if (m.nz > 65535) return QED_ERR_ARG;
  const dim3 blocks((m.nx + 31) / 32, (m.ny + 7) / 8, m.nz), threads(32, 8);
  const double *d = c->grid.d;
  R *E[3], *B[3], *J[3];
  for (int k = 0; k < 3; ++k) {
    E[k] = (R *)f->E[k];
    B[k] = (R *)f->B[k];
    J[k] = (R *)f->J[k];
  }
  const double h = 0.5 * dt;
  // the new fields' maxima, for the next step of the same qed_step call
  unsigned long long *mx = c->d_grid_max_next;
  if (cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 6 * kMaxStripes, s) != cudaSuccess) return QED_ERR_CUDA;
  c->launches += 3;
  k_yee_b<R><<<blocks, threads, 0, s>>>(E[0], E[1], E[2], B[0], B[1], B[2], m, (R)(h / d[0]), (R)(h / d[1]),
                                         (R)(h / d[2]), nullptr);
  k_yee_e<R><<<blocks, threads, 0, s>>>(E[0], E[1], E[2], B[0], B[1], B[2], J[0], J[1], J[2], m, (R)(dt / d[0]),
                                     (R)(dt / d[1]), (R)(dt / d[2]), (R)(dt * 4.0 * 3.141592653589793 * kAlpha),
                                     mx);
  k_yee_b<R><<<blocks, threads, 0, s>>>(E[0], E[1], E[2], B[0], B[1], B[2], m, (R)(h / d[0]), (R)(h / d[1]),
                                         (R)(h / d[2]), mx + 3);
  if (cudaGetLastError() != cudaSuccess) return QED_ERR_CUDA;
  c->grid_max_ready = 1;
  return QED_OK;
}

}  // namespace

int fold_grid_max(qed_ctx *c, cudaStream_t s) {
  c->launches += 1;
  k_max_fold<<<1, 32, 0, s>>>(c->d_grid_max_next, c->d_grid_max);
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}
}  // namespace qed

int qed_launch_yee(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  return c->prec == 64 ? qed::yee<double>(c, f, dt, s) : qed::yee<float>(c, f, dt, s);
}
