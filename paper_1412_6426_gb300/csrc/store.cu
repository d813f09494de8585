// Particle store: conversion from/to absolute FP64 positions, live counts,
// and stable removal of dead particles (tiled stream compaction).
#include <cmath>

#include "qed_internal.h"

namespace qed {
namespace {

struct alignas(16) D4 { double2 a, b; };  // 32-byte FP64 record half

template <typename R> struct Rec;
template <> struct Rec<float> { using T = float4; };
template <> struct Rec<double> { using T = D4; };

__device__ __forceinline__ void put(float4 *pos, float4 *mom, long long i, const double *off, double w,
                                    const double *p, int cell) {
  pos[i] = make_float4((float)off[0], (float)off[1], (float)off[2], (float)w);
  mom[i] = make_float4((float)p[0], (float)p[1], (float)p[2], __int_as_float(cell));
}
__device__ __forceinline__ void put(D4 *pos, D4 *mom, long long i, const double *off, double w,
                                    const double *p, int cell) {
  D4 P, M;
  P.a = make_double2(off[0], off[1]);
  P.b = make_double2(off[2], w);
  M.a = make_double2(p[0], p[1]);
  M.b = make_double2(p[2], (double)cell);
  pos[i] = P;
  mom[i] = M;
}
__device__ __forceinline__ int cell_of(const float4 &m) { return __float_as_int(m.w); }
__device__ __forceinline__ int cell_of(const D4 &m) { return (int)m.b.y; }
__device__ __forceinline__ void set_cell_dead(float4 &m) { m.w = __int_as_float(-1); }
__device__ __forceinline__ void set_cell_dead(D4 &m) { m.b.y = -1.0; }

struct Lattice {
  int n[3], periodic[3];
  double d[3], x0[3];
};

template <typename R>
__global__ void k_set(typename Rec<R>::T *pos, typename Rec<R>::T *mom, uint64_t *ids, long long *count,
                      int sp, Lattice L, const double *x, const double *p, const double *w,
                      const uint64_t *id, long long n, unsigned long long *counters) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) count[sp] = n;
  if (i >= n) return;
  double off[3];
  int ci[3];
  bool dead = false;
  for (int c = 0; c < 3; ++c) {
    double u = (x[3 * i + c] - L.x0[c]) / L.d[c];
    double f = floor(u);
    double o = u - f;
    long long k = (long long)f;
    if (o >= 1.0) { o -= 1.0; k += 1; }
    if (L.periodic[c]) {
      k %= L.n[c];
      if (k < 0) k += L.n[c];
    } else if (k < 0 || k >= L.n[c]) {
      dead = true;
    }
    ci[c] = (int)k;
    off[c] = o;
  }
  int cell = dead ? -1 : (ci[2] * L.n[1] + ci[1]) * L.n[0] + ci[0];
  if (dead) atomicAdd(counters + kCntAbsorbed, 1ull);
  const double pp[3] = {p[3 * i], p[3 * i + 1], p[3 * i + 2]};
  put(pos, mom, i, off, w[i], pp, cell);
  ids[i] = id[i];
}

__device__ __forceinline__ void get(const float4 &P, const float4 &M, double *off, double &w, double *p) {
  off[0] = P.x; off[1] = P.y; off[2] = P.z; w = P.w;
  p[0] = M.x; p[1] = M.y; p[2] = M.z;
}
__device__ __forceinline__ void get(const D4 &P, const D4 &M, double *off, double &w, double *p) {
  off[0] = P.a.x; off[1] = P.a.y; off[2] = P.b.x; w = P.b.y;
  p[0] = M.a.x; p[1] = M.a.y; p[2] = M.b.x;
}

template <typename R>
__global__ void k_get(const typename Rec<R>::T *pos, const typename Rec<R>::T *mom, const uint64_t *ids,
                      Lattice L, double *x, double *p, double *w, uint64_t *id, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename Rec<R>::T P = pos[i], M = mom[i];
  double off[3], pp[3], ww;
  get(P, M, off, ww, pp);
  int cell = cell_of(M);
  int ci[3] = {cell % L.n[0], (cell / L.n[0]) % L.n[1], cell / (L.n[0] * L.n[1])};
  for (int c = 0; c < 3; ++c) {
    x[3 * i + c] = L.x0[c] + ((double)ci[c] + off[c]) * L.d[c];
    p[3 * i + c] = pp[c];
  }
  w[i] = ww;
  id[i] = ids[i];
}

// ----- compaction ----------------------------------------------------------
// Tiles of kCompactTile records, processed in rounds of 256 consecutive
// records so that loads stay coalesced and the output keeps the input order.
// Optionally the live records are split into two classes, class 1 placed
// after class 0 (each class in input order): photons whose momentum is below
// eps_star cannot convert to pairs in the analytic field of the run, and
// gathering them lets whole warps take the photon kernel's short path.
// Layout of tiles: [0] records scanned, [1] live total, [2 + t] class-0
// count/offset of tile t, [2 + maxt + t] the same for class 1.
__device__ __forceinline__ float p2_of(const float4 &m) { return m.x * m.x + m.y * m.y + m.z * m.z; }
__device__ __forceinline__ double p2_of(const D4 &m) { return m.a.x * m.a.x + m.a.y * m.a.y + m.b.x * m.b.x; }

template <typename T>
__device__ __forceinline__ int record_class(const T &m, double eps2) {
  if (cell_of(m) < 0) return -1;
  return (double)p2_of(m) < eps2 ? 1 : 0;
}

template <typename T>
__global__ void k_tile_count(const T *mom, const long long *count, int sp, long long cap, long long *tiles,
                             long long maxt, const double *eps_star) {
  __shared__ unsigned wsum[2][8];
  const long long n = min(count[sp], cap);  // count exceeds cap after an overflow
  const double e = eps_star ? *eps_star : 0.0;
  const double eps2 = e * e;
  if (blockIdx.x == 0 && threadIdx.x == 0) tiles[0] = n;
  const long long ntiles = (n + kCompactTile - 1) / kCompactTile;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    unsigned c0 = 0, c1 = 0;
    for (int r = 0; r < kCompactTile / 256; ++r) {
      long long i = t * kCompactTile + r * 256 + threadIdx.x;
      const int cls = i < n ? record_class(mom[i], eps2) : -1;
      c0 += cls == 0;
      c1 += cls == 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
      c0 += __shfl_xor_sync(0xffffffffu, c0, o);
      c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    }
    if ((threadIdx.x & 31) == 0) {
      wsum[0][threadIdx.x >> 5] = c0;
      wsum[1][threadIdx.x >> 5] = c1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned s0 = 0, s1 = 0;
      for (int k = 0; k < 8; ++k) { s0 += wsum[0][k]; s1 += wsum[1][k]; }
      tiles[2 + t] = s0;
      tiles[2 + maxt + t] = s1;
    }
    __syncthreads();
  }
}

// Exclusive scans of the tile counts of class 0, then class 1 (continuing
// after the class-0 total), in one block; writes the live total.
__global__ void k_tile_scan(long long *tiles, long long *count, int sp, long long maxt) {
  __shared__ long long part[1024];
  __shared__ long long carry;
  const long long n = tiles[0];
  const long long ntiles = (n + kCompactTile - 1) / kCompactTile;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int cls = 0; cls < 2; ++cls) {
    long long *arr = tiles + 2 + cls * maxt;
    for (long long base = 0; base < ntiles; base += 1024) {
      long long i = base + threadIdx.x;
      long long v = i < ntiles ? arr[i] : 0;
      part[threadIdx.x] = v;
      __syncthreads();
      for (int o = 1; o < 1024; o <<= 1) {
        long long add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
      }
      if (i < ntiles) arr[i] = carry + part[threadIdx.x] - v;
      __syncthreads();
      if (threadIdx.x == 1023) carry += part[1023];
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    count[sp] = carry;
    tiles[1] = carry;
  }
}

template <typename T>
__global__ void k_tile_scatter(const T *pos, const T *mom, const uint64_t *id, T *pos2, T *mom2,
                               uint64_t *id2, const long long *tiles, long long maxt, const double *eps_star) {
  __shared__ unsigned wcount[2][8];
  const long long n = tiles[0];
  const double e = eps_star ? *eps_star : 0.0;
  const double eps2 = e * e;
  const long long ntiles = (n + kCompactTile - 1) / kCompactTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long long out[2] = {tiles[2 + t], tiles[2 + maxt + t]};
    for (int r = 0; r < kCompactTile / 256; ++r) {
      long long i = t * kCompactTile + r * 256 + threadIdx.x;
      const int cls = i < n ? record_class(mom[i], eps2) : -1;
      const unsigned b0 = __ballot_sync(0xffffffffu, cls == 0);
      const unsigned b1 = __ballot_sync(0xffffffffu, cls == 1);
      if (lane == 0) {
        wcount[0][warp] = __popc(b0);
        wcount[1][warp] = __popc(b1);
      }
      __syncthreads();
      unsigned before[2] = {0, 0}, all[2] = {0, 0};
      for (int k = 0; k < 8; ++k)
        for (int c = 0; c < 2; ++c) {
          before[c] += k < warp ? wcount[c][k] : 0u;
          all[c] += wcount[c][k];
        }
      if (cls >= 0) {
        const unsigned b = cls ? b1 : b0;
        long long o = out[cls] + before[cls] + __popc(b & ((1u << lane) - 1u));
        pos2[o] = pos[i];
        mom2[o] = mom[i];
        id2[o] = id[i];
      }
      out[0] += all[0];
      out[1] += all[1];
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void k_count_live(const T *mom, const long long *count, int sp, long long cap, long long *live) {
  const long long n = min(count[sp], cap);
  unsigned long long mine = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    mine += cell_of(mom[i]) >= 0;
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd((unsigned long long *)live + sp, mine);
}


// ----- counting sort: by cell block (grid mode) or by sub-interval count ----
// Counting sort of the live records by key: the 8x8x8 cell block of the
// record (grid mode), or for independent ensembles the number of
// sub-intervals the adaptive event generator will take for the record's next
// step, estimated from its momentum and its ensemble's field bound, so that
// the lanes of a warp run loops of about equal length: histogram, one-block
// exclusive scan into the per-species key starts, scatter through per-key
// cursors.  Dead records are dropped.  Lanes of a warp that land on the same
// key share one atomic.
struct BlockGeom {
  int n[3], nb[3];
  unsigned div_m[2];       // cell / n0 and cell / (n0 n1) by multiply-shift
  int div_l[2];
  int nkeys;
  int per_block;           // keys per cell block: 1, or one per cell (kBlockVolume)
  int nsub_key;            // 1: key = estimated sub-intervals (ensembles)
  int ens_shift;           // ensemble = id >> ens_shift (64: ensemble 0)
  int n_ens;
  const float *ens_h;      // per ensemble: |E0| + |Eu| + |Bu|
  float dt, kappa, mass;
  // photons on the Yee mesh: those that may pair (|p| >= eps*) by cell
  // block, so that their field gathers hit cached lines; the others, which
  // take the straight flight, after them (key nkeys - 1)
  int photon_split;
  const double *eps_star;
};

// The key of a cell: its cell block, and with one key per cell its place in
// the block (x fastest), so that the records of a block are in cell order
// and a warp's 32 consecutive records sit in a few neighbouring cells.
__device__ __forceinline__ int block_of(int cell, const BlockGeom &g) {
  const unsigned row = fast_div((unsigned)cell, g.div_m[0], g.div_l[0]);
  const unsigned slab = fast_div((unsigned)cell, g.div_m[1], g.div_l[1]);
  const int i = cell - (int)row * g.n[0], j = (int)row - (int)slab * g.n[1], k = (int)slab;
  const int b = (i / kBlockCells) + g.nb[0] * ((j / kBlockCells) + g.nb[1] * (k / kBlockCells));
  if (g.per_block == 1) return b;
  return b * kBlockVolume + (i % kBlockCells) + kBlockCells * ((j % kBlockCells) + kBlockCells * (k % kBlockCells));
}

// Sub-intervals of Eq. (28) with the ensemble's bound |E0| + |Eu| + |Bu| in
// place of H_eff, in FP32: the key only orders the records, so an estimate
// will do.
__device__ __forceinline__ int nsub_key(uint64_t id, float p2, const BlockGeom &g) {
  const unsigned long long e = g.ens_shift >= 64 ? 0ull : (unsigned long long)(id >> g.ens_shift);
  if (e >= (unsigned long long)g.n_ens || !(g.mass > 0.f)) return 0;
  const float H = __ldg(g.ens_h + e);
  if (!(H > 0.f)) return 0;
  const float gamma = sqrtf(1.f + p2 / (g.mass * g.mass));
  const float dtq = g.kappa * 137.f * fminf(0.67f * cbrtf(gamma) / cbrtf(H * H), 2.f / H);
  const float n = ceilf(g.dt / dtq);
  return n < (float)(g.nkeys - 1) ? (int)n : g.nkeys - 1;
}

template <typename T>
__device__ __forceinline__ int key_of(int cell, uint64_t id, const T &m, const BlockGeom &g) {
  if (g.nsub_key) return nsub_key(id, (float)p2_of(m), g);
  if (g.photon_split) {
    const double e = *g.eps_star;
    if ((double)p2_of(m) < e * e) return g.nkeys - 1;
  }
  return block_of(cell, g);
}

// Two of block_atomic_add at once: both atomics are issued before either
// result is read.
__device__ __forceinline__ void block_atomic_add2(unsigned *ctr, const int *key, const bool *on, unsigned *out) {
  const int lane = threadIdx.x & 31;
  unsigned peers[2] = {0u, 0u}, base[2] = {0u, 0u};
  int leader[2] = {0, 0};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const unsigned mask = __ballot_sync(0xffffffffu, on[r]);
    if (on[r]) {
      peers[r] = __match_any_sync(mask, key[r]);
      leader[r] = __ffs(peers[r]) - 1;
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (on[r] && lane == leader[r]) base[r] = atomicAdd(ctr + key[r], (unsigned)__popc(peers[r]));
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (on[r]) out[r] = __shfl_sync(peers[r], base[r], leader[r]) + __popc(peers[r] & ((1u << lane) - 1u));
}

__device__ __forceinline__ unsigned block_atomic_add(unsigned *ctr, int key, bool on) {
  const unsigned mask = __ballot_sync(0xffffffffu, on);
  if (!on) return 0;
  const unsigned peers = __match_any_sync(mask, key);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(ctr + key, (unsigned)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// Two records per thread and iteration (i and i + stride), their loads and
// atomics issued together, so that their latencies overlap.
template <typename T>
__global__ void k_blk_hist(const T *mom, const uint64_t *id, const long long *count, int sp, long long cap,
                           BlockGeom g, unsigned *hist) {
  const long long n = min(count[sp], cap);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += 2 * stride) {
    int cell[2] = {-1, -1};
    uint64_t pid[2] = {0, 0};
    T M[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const long long i = base + r * stride + threadIdx.x;
      if (i < n) {
        M[r] = mom[i];
        cell[r] = cell_of(M[r]);
        if (g.nsub_key) pid[r] = id[i];
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const bool live = cell[r] >= 0;
      block_atomic_add(hist, live ? key_of(cell[r], pid[r], M[r], g) : 0, live);
    }
  }
}

// Exclusive scan of the histogram in three launches of 1024-thread blocks,
// each thread taking kScanRun consecutive keys: the sum of each part of
// kScanPart keys, an exclusive scan of those sums, then each part scanned
// again with its offset.  Writes the scatter cursor of every key, the first
// record of every cell block, the end of the last and the total
// (count[sp]).
constexpr int kScanBlock = 1024, kScanRun = 16, kScanPart = kScanBlock * kScanRun;

// The kScanRun keys of this thread (zero past n), by 16-byte loads where
// they lie inside the histogram.
__device__ __forceinline__ void load_run(const unsigned *h, long long first, int n, unsigned *v) {
  if (first + kScanRun <= n) {
#pragma unroll
    for (int q = 0; q < kScanRun / 4; ++q) {
      const uint4 u = ((const uint4 *)(h + first))[q];
      v[4 * q] = u.x; v[4 * q + 1] = u.y; v[4 * q + 2] = u.z; v[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kScanRun; ++q) v[q] = first + q < n ? h[first + q] : 0u;
  }
}

// Exclusive scan of one value per thread over a 1024-thread block; *total
// receives the block's sum.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned *warp_tot, unsigned *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;   // inclusive over the warps
  }
  __syncthreads();
  *total = warp_tot[31];
  const unsigned excl = x - v + (warp > 0 ? warp_tot[warp - 1] : 0u);
  __syncthreads();   // warp_tot is reused by the caller's next scan
  return excl;
}

// A species with no records skips the histogram's zeroing and scan (its
// starts are all zero): the histogram then holds another species' cursors.
__global__ void k_zero_hist(unsigned *hist, long long n, const long long *count, int sp) {
  if (count[sp] <= 0) return;
  const long long nv = n / 4, stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride)
    ((uint4 *)hist)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (long long i = 4 * nv + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) hist[i] = 0u;
}

__global__ void k_blk_sums(const unsigned *hist, int n, unsigned *part, const long long *count, int sp) {
  __shared__ unsigned wt[32];
  if (count[sp] <= 0) {
    if (threadIdx.x == 0) part[blockIdx.x] = 0u;
    return;
  }
  unsigned v[kScanRun], sum = 0;
  load_run(hist, (long long)blockIdx.x * kScanPart + (long long)threadIdx.x * kScanRun, n, v);
#pragma unroll
  for (int q = 0; q < kScanRun; ++q) sum += v[q];
  unsigned total;
  block_exclusive_scan(sum, wt, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Each thread scans a run of consecutive sums in turn (their total first,
// then the runs' exclusive scan across the block, then the run itself).
__global__ void k_blk_scan_parts(unsigned *part, int nparts, unsigned *start, int nstart, long long *count, int sp) {
  __shared__ unsigned wt[32];
  const int run = (nparts + kScanBlock - 1) / kScanBlock;
  const int lo = min(nparts, (int)threadIdx.x * run), hi = min(nparts, lo + run);
  unsigned sum = 0;
  for (int i = lo; i < hi; ++i) sum += part[i];
  unsigned total;
  unsigned e = block_exclusive_scan(sum, wt, &total);
  for (int i = lo; i < hi; ++i) {
    const unsigned v = part[i];
    part[i] = e;
    e += v;
  }
  if (threadIdx.x == 0) {
    start[nstart] = total;
    count[sp] = total;
  }
}

// The scatter cursor of every key, and the first record of every cell block
// (the first key of the block; keys past nblk x per_block each start an
// entry of their own).
__global__ void k_blk_scan_out(unsigned *hist, int n, const unsigned *part, unsigned *start, int per_block,
                               int nmain, int nblk, const long long *count, int sp) {
  __shared__ unsigned wt[32];
  const long long first = (long long)blockIdx.x * kScanPart + (long long)threadIdx.x * kScanRun;
  if (count[sp] <= 0) {
    for (int q = 0; q < kScanRun; ++q) {
      const long long i = first + q;
      if (i < n) {
        if (i >= nmain) start[nblk + (i - nmain)] = 0u;
        else if (i % per_block == 0) start[i / per_block] = 0u;
      }
    }
    return;
  }
  unsigned v[kScanRun], sum = 0;
  load_run(hist, first, n, v);
#pragma unroll
  for (int q = 0; q < kScanRun; ++q) sum += v[q];
  unsigned total;
  unsigned e = block_exclusive_scan(sum, wt, &total) + part[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kScanRun; ++q) {
    const long long i = first + q;
    if (i < n) {
      if (i >= nmain) start[nblk + (i - nmain)] = e;
      else if (i % per_block == 0) start[i / per_block] = e;
    }
    const unsigned x = v[q];
    v[q] = e;   // becomes the scatter cursor
    e += x;
  }
  if (first + kScanRun <= n) {
#pragma unroll
    for (int q = 0; q < kScanRun / 4; ++q)
      ((uint4 *)(hist + first))[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < kScanRun; ++q)
      if (first + q < n) hist[first + q] = v[q];
  }
}

template <typename T>
__global__ void k_blk_scatter(const T *pos, const T *mom, const uint64_t *id, T *pos2, T *mom2, uint64_t *id2,
                              const long long *count, int sp, long long cap, BlockGeom g, unsigned *cursor) {
  const long long n = min(count[sp], cap);   // records before the sort (the total goes elsewhere)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += 2 * stride) {
    // two records per thread (i and i + stride): all their loads first,
    // then both cursor atomics, then the stores
    int cell[2] = {-1, -1}, key[2] = {0, 0};
    bool live[2];
    T M[2], P[2];
    uint64_t pid[2] = {0, 0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const long long i = base + r * stride + threadIdx.x;
      if (i < n) {
        M[r] = mom[i];
        P[r] = pos[i];
        pid[r] = id[i];
        cell[r] = cell_of(M[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      live[r] = cell[r] >= 0;
      if (live[r]) key[r] = key_of(cell[r], pid[r], M[r], g);
    }
    unsigned o[2] = {0u, 0u};
    block_atomic_add2(cursor, key, live, o);
#pragma unroll
    for (int r = 0; r < 2; ++r)
      if (live[r]) {
        pos2[o[r]] = P[r];
        mom2[o[r]] = M[r];
        id2[o[r]] = pid[r];
      }
  }
}

template <typename R>
int sort_blocks(qed_ctx *c, int sp, cudaStream_t s) {
  using T = typename Rec<R>::T;
  Store &st = c->st[sp];
  if (st.cap == 0 || c->nblk == 0) return QED_OK;
  BlockGeom g;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = c->grid.n[k];
    g.nb[k] = c->nb[k];
  }
  fast_div_magic((unsigned)g.n[0], g.div_m[0], g.div_l[0]);
  fast_div_magic((unsigned)(g.n[0] * g.n[1]), g.div_m[1], g.div_l[1]);
  // photons by cell block only: most fly straight without a gather, and the
  // finer order did not pay for its larger histogram
  g.per_block = (c->key_ensembles || sp == kPhoton) ? 1 : c->blk_keys;
  const int nmain = c->nblk * g.per_block;
  g.nkeys = nmain;
  g.nsub_key = c->key_ensembles;
  g.ens_shift = c->par.ens_bits > 0 ? 64 - c->par.ens_bits : 64;
  g.n_ens = c->n_ens;
  g.ens_h = c->d_ens_h;
  g.dt = (float)c->last_dt;
  g.kappa = (float)c->par.kappa;
  g.mass = (sp == kIon || !c->par.emission_on) ? 0.f : (float)c->species.mass[sp];
  g.photon_split = sp == kPhoton && !c->key_ensembles;
  g.eps_star = c->d_eps_star;
  if (g.photon_split) g.nkeys = nmain + 1;
  const int cur = st.cur, nxt = cur ^ 1;
  unsigned *start = g.photon_split ? c->d_phot_start : c->d_blk_start + (size_t)sp * (c->nblk + 1);
  k_zero_hist<<<c->num_sms * 4, 256, 0, s>>>(c->d_blk_cursor, (long long)g.nkeys + 1, c->d_count, sp);
  const int grid = c->num_sms * 8;
  c->launches += 4;
  k_blk_hist<T><<<grid, 256, 0, s>>>((const T *)st.mom[cur], st.id[cur], c->d_count, sp, (long long)st.cap, g,
                                     c->d_blk_cursor);
  // the record count to scatter is read on the device: the histogram keeps it
  // total -> [4 + sp]; the block sums go to the spare words after the cursors
  const int nparts = (g.nkeys + kScanPart - 1) / kScanPart;
  unsigned *part = c->d_blk_cursor + (g.nkeys + 2);
  const int nstart = c->nblk + (g.nkeys - nmain);
  c->launches += 2;
  k_blk_sums<<<nparts, kScanBlock, 0, s>>>(c->d_blk_cursor, g.nkeys, part, c->d_count, sp);
  k_blk_scan_parts<<<1, kScanBlock, 0, s>>>(part, nparts, start, nstart, c->d_count + 4, sp);
  k_blk_scan_out<<<nparts, kScanBlock, 0, s>>>(c->d_blk_cursor, g.nkeys, part, start, g.per_block, nmain, c->nblk,
                                              c->d_count, sp);
  k_blk_scatter<T><<<grid, 256, 0, s>>>((const T *)st.pos[cur], (const T *)st.mom[cur], st.id[cur],
                                        (T *)st.pos[nxt], (T *)st.mom[nxt], st.id[nxt], c->d_count, sp,
                                        (long long)st.cap, g, c->d_blk_cursor);
  if (cudaGetLastError() != cudaSuccess) return QED_ERR_CUDA;
  // the live count becomes the store size
  if (cudaMemcpyAsync(c->d_count + sp, c->d_count + 4 + sp, sizeof(long long), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return QED_ERR_CUDA;
  st.cur = nxt;
  return QED_OK;
}

// ----- thinning (Sec. VI): global even redistribution per group --------------
// Three passes over one species: (1) per group (ensemble, or the species)
// the live count N and weight W; (2) where N > L, each record survives with
// probability L/N (its own uniform, purpose THIN, counter = the step just
// taken) and the survivors' weight W' is summed; (3) where N > L and W' > 0
// the others die and the survivors' weights are multiplied by W/W'.  The
// decision of pass 2 is drawn again in pass 3 from the same stream.
struct ThinArgs {
  int ens_shift;           // 64: one group
  int groups;
  long long limit;
  const double *ens;       // ensemble table (thin_scale in column 9) or null
  unsigned seed;
  const void *clock;       // {double t; long long step}, already advanced
  unsigned long long *n;   // [groups]
  double *w, *wsurv;       // [groups]
  unsigned long long *thinned;
};

__device__ __forceinline__ double weight_of(const float4 &P) { return (double)P.w; }
__device__ __forceinline__ double weight_of(const D4 &P) { return P.b.y; }
__device__ __forceinline__ void set_weight(float4 &P, double w) { P.w = (float)w; }
__device__ __forceinline__ void set_weight(D4 &P, double w) { P.b.y = w; }

__device__ __forceinline__ int group_of(uint64_t id, const ThinArgs &t) {
  const unsigned long long e = t.ens_shift >= 64 ? 0ull : (unsigned long long)(id >> t.ens_shift);
  return e < (unsigned long long)t.groups ? (int)e : -1;
}

// Limit of group g: the species limit, times the ensemble's thin_scale when positive.
__device__ __forceinline__ long long group_limit(int g, const ThinArgs &t) {
  long long L = t.limit;
  if (t.ens) {
    const double sc = t.ens[(size_t)g * QED_ENS_STRIDE + 9];
    if (sc > 0.0) L = (long long)floor((double)L * sc);
  }
  return L;
}

__device__ __forceinline__ bool thin_survives(uint64_t id, const ThinArgs &t, long long L, unsigned long long N) {
  const unsigned step = (unsigned)(((const long long *)t.clock)[1] - 1);
  const uint4 o = philox4x32_10(make_uint4(step, 0u, kThin, t.seed), make_uint2((unsigned)id, (unsigned)(id >> 32)));
  const double u = uniform_pair(o.x, o.y, (double *)nullptr);
  return u < (double)L / (double)N;
}

constexpr int kThinShared = 2048;   // groups accumulated in shared memory first

// Lanes with the same group add their values with one atomic per group.
__device__ __forceinline__ void group_add(int g, bool on, double w, unsigned long long *n, double *wsum) {
  const unsigned mask = __ballot_sync(0xffffffffu, on);
  if (!on) return;
  const unsigned peers = __match_any_sync(mask, g);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  double tot = 0.0;
  for (unsigned m = peers; m; m &= m - 1) tot += __shfl_sync(peers, w, __ffs(m) - 1);
  if (lane == leader) {
    if (n) atomicAdd(n + g, (unsigned long long)__popc(peers));
    atomicAdd(wsum + g, tot);
  }
}

// Per-block partial sums in shared memory (up to kThinShared groups), then
// one global atomic per non-empty group and block.
struct ThinShared {
  unsigned long long n[kThinShared];
  double w[kThinShared];
};

__device__ __forceinline__ void thin_shared_zero(ThinShared &sh, int groups) {
  for (int k = threadIdx.x; k < groups; k += blockDim.x) {
    sh.n[k] = 0;
    sh.w[k] = 0.0;
  }
  __syncthreads();
}

__device__ __forceinline__ void thin_shared_flush(ThinShared &sh, int groups, unsigned long long *n, double *w) {
  __syncthreads();
  for (int k = threadIdx.x; k < groups; k += blockDim.x) {
    if (n && sh.n[k]) atomicAdd(n + k, sh.n[k]);
    if (sh.w[k] != 0.0) atomicAdd(w + k, sh.w[k]);
  }
}

// A thread's running sums for the group of its last particles, added to the
// block's shared sums when the group changes: a species without ensembles
// (one group), or an ensemble stored contiguously, costs one shared atomic
// per thread instead of one per particle.
struct GroupRun {
  int g = -1;
  unsigned long long n = 0;
  double w = 0.0;
  __device__ __forceinline__ void flush(ThinShared &sh, bool count) {
    if (g < 0) return;
    if (count) atomicAdd(&sh.n[g], n);
    atomicAdd(&sh.w[g], w);
  }
  __device__ __forceinline__ void add(ThinShared &sh, bool count, int gi, double wi) {
    if (gi != g) {
      flush(sh, count);
      g = gi;
      n = 0;
      w = 0.0;
    }
    n += 1;
    w += wi;
  }
};

template <typename T>
__global__ void k_thin_count(const T *pos, const T *mom, const uint64_t *id, const long long *count, int sp,
                             long long cap, ThinArgs t) {
  __shared__ ThinShared sh;
  const bool priv = t.groups <= kThinShared;
  if (priv) thin_shared_zero(sh, t.groups);
  const long long n = min(count[sp], cap);
  const long long stride = (long long)gridDim.x * blockDim.x;
  GroupRun run;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    int g = -1;
    double w = 0.0;
    if (i < n && cell_of(mom[i]) >= 0) {
      g = t.ens_shift >= 64 ? 0 : group_of(id[i], t);   // one group: the id is not needed
      w = weight_of(pos[i]);
    }
    if (priv) {
      if (g >= 0) run.add(sh, true, g, w);
    } else {
      group_add(g, g >= 0, w, t.n, t.w);
    }
  }
  if (priv) {
    run.flush(sh, true);
    thin_shared_flush(sh, t.groups, t.n, t.w);
  }
}

// One group at or below its limit: nothing to mark or apply.
__device__ __forceinline__ bool thin_nothing(const ThinArgs &t) {
  return t.groups == 1 && (long long)t.n[0] <= group_limit(0, t);
}

template <typename T>
__global__ void k_thin_mark(const T *pos, const T *mom, const uint64_t *id, const long long *count, int sp,
                            long long cap, ThinArgs t) {
  if (thin_nothing(t)) return;
  __shared__ ThinShared sh;
  const bool priv = t.groups <= kThinShared;
  if (priv) thin_shared_zero(sh, t.groups);
  const long long n = min(count[sp], cap);
  const long long stride = (long long)gridDim.x * blockDim.x;
  GroupRun run;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    int g = -1;
    double w = 0.0;
    if (i < n && cell_of(mom[i]) >= 0) {
      const uint64_t pid = id[i];
      g = group_of(pid, t);
      if (g >= 0) {
        const unsigned long long N = t.n[g];
        const long long L = group_limit(g, t);
        if ((long long)N > L && thin_survives(pid, t, L, N)) w = weight_of(pos[i]);
        else g = -1;
      }
    }
    if (priv) {
      if (g >= 0) run.add(sh, false, g, w);
    } else {
      group_add(g, g >= 0, w, nullptr, t.wsurv);
    }
  }
  if (priv) {
    run.flush(sh, false);
    thin_shared_flush(sh, t.groups, nullptr, t.wsurv);
  }
}

template <typename T>
__global__ void k_thin_apply(T *pos, T *mom, const uint64_t *id, const long long *count, int sp, long long cap,
                             ThinArgs t) {
  if (thin_nothing(t)) return;
  const long long n = min(count[sp], cap);
  unsigned long long removed = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    T M = mom[i];
    if (cell_of(M) < 0) continue;
    const uint64_t pid = id[i];
    const int g = group_of(pid, t);
    if (g < 0) continue;
    const unsigned long long N = t.n[g];
    const double ws = t.wsurv[g];
    const long long L = group_limit(g, t);
    if ((long long)N <= L || !(ws > 0.0)) continue;
    if (thin_survives(pid, t, L, N)) {
      T P = pos[i];
      set_weight(P, weight_of(P) * (t.w[g] / ws));
      pos[i] = P;
    } else {
      set_cell_dead(M);
      mom[i] = M;
      ++removed;
    }
  }
  for (int o = 16; o > 0; o >>= 1) removed += __shfl_xor_sync(0xffffffffu, removed, o);
  if ((threadIdx.x & 31) == 0 && removed) atomicAdd(t.thinned, removed);
}

template <typename R>
int thin(qed_ctx *c, int sp, cudaStream_t s) {
  using T = typename Rec<R>::T;
  Store &st = c->st[sp];
  const long long L = c->par.thin_limit[sp];
  if (st.cap == 0 || L <= 0 || !c->d_thin) return QED_OK;
  ThinArgs t;
  // groups are ensembles only in the ensemble field mode; elsewhere the id
  // bits only record lineage and the species is one group
  const bool by_ens = c->par.ens_bits > 0 && c->grid.field_mode == QED_FIELD_ENSEMBLE;
  t.ens_shift = by_ens ? 64 - c->par.ens_bits : 64;
  t.groups = by_ens ? c->n_ens : 1;
  t.limit = L;
  t.ens = by_ens ? c->d_ens : nullptr;
  t.seed = c->par.seed;
  t.clock = c->d_clock;
  t.n = (unsigned long long *)c->d_thin;
  t.w = (double *)(t.n + c->thin_groups);
  t.wsurv = t.w + c->thin_groups;
  t.thinned = c->d_counters + kCntThinned;
  if (cudaMemsetAsync(c->d_thin, 0, (size_t)c->thin_groups * 24, s) != cudaSuccess) return QED_ERR_CUDA;
  const int grid = c->num_sms * 8;
  const int cur = st.cur;
  c->launches += 3;
  k_thin_count<T><<<grid, 256, 0, s>>>((const T *)st.pos[cur], (const T *)st.mom[cur], st.id[cur], c->d_count, sp,
                                       (long long)st.cap, t);
  k_thin_mark<T><<<grid, 256, 0, s>>>((const T *)st.pos[cur], (const T *)st.mom[cur], st.id[cur], c->d_count, sp,
                                      (long long)st.cap, t);
  k_thin_apply<T><<<grid, 256, 0, s>>>((T *)st.pos[cur], (T *)st.mom[cur], st.id[cur], c->d_count, sp,
                                       (long long)st.cap, t);
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

Lattice lattice(const qed_ctx *c) {
  Lattice L;
  for (int k = 0; k < 3; ++k) {
    L.n[k] = c->grid.n[k];
    L.periodic[k] = c->grid.periodic[k];
    L.d[k] = c->grid.d[k];
    L.x0[k] = c->grid.x0[k];
  }
  return L;
}

template <typename R>
int set(qed_ctx *c, int sp, const double *x, const double *p, const double *w, const uint64_t *id,
        int64_t n, cudaStream_t s) {
  using T = typename Rec<R>::T;
  Store &st = c->st[sp];
  int blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  c->launches += 1;
  k_set<R><<<blocks, 256, 0, s>>>((T *)st.pos[st.cur], (T *)st.mom[st.cur], st.id[st.cur], c->d_count,
                                   sp, lattice(c), x, p, w, id, (long long)n, c->d_counters);
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

template <typename R>
int get(qed_ctx *c, int sp, double *x, double *p, double *w, uint64_t *id, int64_t n, cudaStream_t s) {
  using T = typename Rec<R>::T;
  Store &st = c->st[sp];
  if (n <= 0) return QED_OK;
  int blocks = (int)((n + 255) / 256);
  c->launches += 1;
  k_get<R><<<blocks, 256, 0, s>>>((const T *)st.pos[st.cur], (const T *)st.mom[st.cur], st.id[st.cur],
                                   lattice(c), x, p, w, id, (long long)n);
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

template <typename R>
int compact(qed_ctx *c, int sp, bool partition, cudaStream_t s) {
  using T = typename Rec<R>::T;
  Store &st = c->st[sp];
  if (st.cap == 0) return QED_OK;
  int cur = st.cur, nxt = cur ^ 1;
  long long maxtiles = (st.cap + kCompactTile - 1) / kCompactTile;
  const long long maxt = c->tile_cap / 2;
  int g = (int)(maxtiles < (long long)c->num_sms * 8 ? maxtiles : (long long)c->num_sms * 8);
  if (g < 1) g = 1;
  const double *eps = (partition && sp == kPhoton) ? c->d_eps_star : nullptr;
  c->launches += 3;
  k_tile_count<T><<<g, 256, 0, s>>>((const T *)st.mom[cur], c->d_count, sp, (long long)st.cap, c->d_tile,
                                    maxt, eps);
  k_tile_scan<<<1, 1024, 0, s>>>(c->d_tile, c->d_count, sp, maxt);
  k_tile_scatter<T><<<g, 256, 0, s>>>((const T *)st.pos[cur], (const T *)st.mom[cur], st.id[cur],
                                       (T *)st.pos[nxt], (T *)st.mom[nxt], st.id[nxt], c->d_tile, maxt, eps);
  if (cudaGetLastError() != cudaSuccess) return QED_ERR_CUDA;
  st.cur = nxt;
  return QED_OK;
}

template <typename R>
int count_live(qed_ctx *c, long long *d_live, cudaStream_t s) {
  using T = typename Rec<R>::T;
  if (cudaMemsetAsync(d_live, 0, 4 * sizeof(long long), s) != cudaSuccess) return QED_ERR_CUDA;
  for (int sp = 0; sp < 4; ++sp) {
    const Store &st = c->st[sp];
    if (st.cap == 0) continue;
    c->launches += 1;
    k_count_live<T><<<c->num_sms * 4, 256, 0, s>>>((const T *)st.mom[st.cur], c->d_count, sp,
                                                    (long long)st.cap, d_live);
  }
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

}  // namespace
}  // namespace qed

size_t qed_record_bytes(int prec) { return prec == 64 ? 2 * sizeof(qed::D4) : 2 * sizeof(float4); }

int qed_launch_set(qed_ctx *c, int sp, const double *x, const double *p, const double *w,
                   const uint64_t *id, int64_t n, cudaStream_t s) {
  return c->prec == 64 ? qed::set<double>(c, sp, x, p, w, id, n, s) : qed::set<float>(c, sp, x, p, w, id, n, s);
}

int qed_launch_get(qed_ctx *c, int sp, double *x, double *p, double *w, uint64_t *id, int64_t n,
                   cudaStream_t s) {
  return c->prec == 64 ? qed::get<double>(c, sp, x, p, w, id, n, s) : qed::get<float>(c, sp, x, p, w, id, n, s);
}

int qed_launch_compact(qed_ctx *c, int sp, bool partition, cudaStream_t s) {
  return c->prec == 64 ? qed::compact<double>(c, sp, partition, s) : qed::compact<float>(c, sp, partition, s);
}

int qed_launch_sort(qed_ctx *c, int sp, cudaStream_t s) {
  return c->prec == 64 ? qed::sort_blocks<double>(c, sp, s) : qed::sort_blocks<float>(c, sp, s);
}

int qed_launch_count_live(qed_ctx *c, long long *d_live, cudaStream_t s) {
  return c->prec == 64 ? qed::count_live<double>(c, d_live, s) : qed::count_live<float>(c, d_live, s);
}

int qed_launch_thin(qed_ctx *c, int sp, cudaStream_t s) {
  return c->prec == 64 ? qed::thin<double>(c, sp, s) : qed::thin<float>(c, sp, s);
}
