// qed_particles_read_static: read the live particles of one species into
// caller buffers without allocating any memory.
//
// Some callers cannot call cudaMalloc at the point where they want results:
// hosts that hand all device memory to their own pool allocator up front (a
// cudaMalloc behind the pool's back can fail or fragment it), and real-time
// loops that forbid allocation after start-up (an allocation can block on
// the driver for an unbounded time).  qed_particles_get may allocate a
// staging buffer (pageable host output) and compacts the store through the
// library's tile buffer; this variant keeps its tile counts and offsets in a
// fixed file-scope device array instead, writes straight into the caller's
// device or page-locked host buffers, and leaves the store as it is (dead
// records stay in place until the next compaction).
#include <mutex>

#include "qed_internal.h"

namespace {

// Largest store this entry point can scan: kReadStaticTiles tiles of
// qed::kCompactTile records (65536 * 2048 = 134,217,728 records).
constexpr long long kReadStaticTiles = 65536;
constexpr long long kReadStaticMaxRecords = kReadStaticTiles * qed::kCompactTile;

// The fixed scratch (512 KiB + 16 B), held by every GPU that loads the
// library until the process exits.  Layout: [0] records scanned, [1] live
// total, [2 + t] live records of tile t, then its exclusive output offset.
// Every slot a call reads is written earlier in the same call, so nothing
// has to start at zero; calls that overlap on the GPU share it and race.
static __device__ __align__(256) long long g_read_scratch[kReadStaticTiles + 2];

// Host-side device address of g_read_scratch, looked up once per device.
// In host code the name g_read_scratch is only a host-side stand-in, so the
// kernels are always given the address returned by cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
long long *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// The address of the scratch on device dev (the context's device), looked up
// with that device current; the caller's current device is restored.
int scratch_address(int dev, long long **out) {
  if (dev < 0 || dev >= kMaxDevices) return QED_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return QED_ERR_CUDA;
    }
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return QED_ERR_CUDA;
    }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_read_scratch);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return QED_ERR_CUDA;
    }
    g_scratch_addr[dev] = (long long *)p;
  }
  *out = g_scratch_addr[dev];
  return QED_OK;
}

struct alignas(16) Half64 { double2 a, b; };  // one 32-byte half of an FP64 record

__device__ __forceinline__ int live_cell(const float4 &m) { return __float_as_int(m.w); }
__device__ __forceinline__ int live_cell(const Half64 &m) { return (int)m.b.y; }

struct Geometry {
  int n[3];
  double d[3], x0[3];
};

template <typename T>
__global__ void k_read_count(const T *mom, long long n, long long *scr) {
  __shared__ unsigned wsum[8];
  if (blockIdx.x == 0 && threadIdx.x == 0) scr[0] = n;
  const long long ntiles = (n + qed::kCompactTile - 1) / qed::kCompactTile;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    unsigned mine = 0;
    for (int r = 0; r < qed::kCompactTile / 256; ++r) {
      long long i = t * qed::kCompactTile + r * 256 + threadIdx.x;
      mine += (i < n && live_cell(mom[i]) >= 0) ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned s = 0;
      for (int k = 0; k < 8; ++k) s += wsum[k];
      scr[2 + t] = s;
    }
    __syncthreads();
  }
}

__global__ void k_read_scan(long long *scr) {
  __shared__ long long part[1024];
  __shared__ long long carry;
  const long long ntiles = (scr[0] + qed::kCompactTile - 1) / qed::kCompactTile;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < ntiles; base += 1024) {
    long long i = base + threadIdx.x;
    long long v = i < ntiles ? scr[2 + i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      long long add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < ntiles) scr[2 + i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) scr[1] = carry;
}

__device__ __forceinline__ void unpack(const float4 &P, const float4 &M, double *off, double &w, double *p) {
  off[0] = P.x; off[1] = P.y; off[2] = P.z; w = P.w;
  p[0] = M.x; p[1] = M.y; p[2] = M.z;
}
__device__ __forceinline__ void unpack(const Half64 &P, const Half64 &M, double *off, double &w, double *p) {
  off[0] = P.a.x; off[1] = P.a.y; off[2] = P.b.x; w = P.b.y;
  p[0] = M.a.x; p[1] = M.a.y; p[2] = M.b.x;
}

// Stable scatter of the live records, converted to absolute FP64 positions.
template <typename T>
__global__ void k_read_scatter(const T *pos, const T *mom, const uint64_t *ids, Geometry g, const long long *scr,
                               double *x, double *p, double *w, uint64_t *id, long long max_n) {
  __shared__ unsigned wcount[8];
  const long long n = scr[0];
  const long long ntiles = (n + qed::kCompactTile - 1) / qed::kCompactTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long long out = scr[2 + t];
    for (int r = 0; r < qed::kCompactTile / 256; ++r) {
      long long i = t * qed::kCompactTile + r * 256 + threadIdx.x;
      T M;
      int cell = -1;
      if (i < n) {
        M = mom[i];
        cell = live_cell(M);
      }
      bool live = cell >= 0;
      unsigned b = __ballot_sync(0xffffffffu, live);
      if (lane == 0) wcount[warp] = __popc(b);
      __syncthreads();
      unsigned before = 0, all = 0;
      for (int k = 0; k < 8; ++k) {
        before += k < warp ? wcount[k] : 0u;
        all += wcount[k];
      }
      long long o = out + before + __popc(b & ((1u << lane) - 1u));
      if (live && o < max_n) {
        double off[3], pp[3], ww;
        unpack(pos[i], M, off, ww, pp);
        const int ci[3] = {cell % g.n[0], (cell / g.n[0]) % g.n[1], cell / (g.n[0] * g.n[1])};
        for (int c = 0; c < 3; ++c) {
          x[3 * o + c] = g.x0[c] + ((double)ci[c] + off[c]) * g.d[c];
          p[3 * o + c] = pp[c];
        }
        w[o] = ww;
        id[o] = ids[i];
      }
      out += all;
      __syncthreads();
    }
  }
}

// Device-usable alias of a caller pointer; nullptr for pageable host memory
// (which would need a staging allocation).
void *device_usable(void *ptr) {
  cudaPointerAttributes at;
  if (!ptr || cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return ptr;
  if (at.type == cudaMemoryTypeHost) {
    void *dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, ptr, 0) == cudaSuccess) return dp;
    cudaGetLastError();
  }
  return nullptr;
}

template <typename T>
int read_static(qed_ctx *c, int sp, long long n, long long *scr, double *x, double *p, double *w, uint64_t *id,
                long long max_n, cudaStream_t s) {
  const qed::Store &st = c->st[sp];
  Geometry g;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = c->grid.n[k];
    g.d[k] = c->grid.d[k];
    g.x0[k] = c->grid.x0[k];
  }
  long long ntiles = (n + qed::kCompactTile - 1) / qed::kCompactTile;
  int blocks = (int)(ntiles < (long long)c->num_sms * 8 ? (ntiles > 0 ? ntiles : 1) : (long long)c->num_sms * 8);
  c->launches += 3;
  k_read_count<T><<<blocks, 256, 0, s>>>((const T *)st.mom[st.cur], n, scr);
  k_read_scan<<<1, 1024, 0, s>>>(scr);
  k_read_scatter<T><<<blocks, 256, 0, s>>>((const T *)st.pos[st.cur], (const T *)st.mom[st.cur], st.id[st.cur], g,
                                           scr, x, p, w, id, max_n);
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

}  // namespace

extern "C" int qed_particles_read_static(qed_ctx *c, int sp, double *x, double *p, double *w, uint64_t *id,
                                         int64_t max_n, int64_t *n_out, void *stream) {
  if (!c || sp < 0 || sp >= QED_NSPECIES || !n_out || max_n < 0) return QED_ERR_ARG;
  *n_out = 0;
  // the stream, the store and the scratch all belong to the context's device
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return QED_ERR_CUDA;
  }
  if (cur != c->device) return QED_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  long long *scr = nullptr;
  int rc = scratch_address(c->device, &scr);
  if (rc != QED_OK) return rc;
  long long records = 0;
  if (cudaMemcpyAsync(&records, c->d_count + sp, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return QED_ERR_CUDA;
  if (records > c->st[sp].cap) records = c->st[sp].cap;
  if (records > kReadStaticMaxRecords) return QED_ERR_CAPACITY;
  double *dx = nullptr, *dp = nullptr, *dw = nullptr;
  uint64_t *di = nullptr;
  if (max_n > 0) {
    dx = (double *)device_usable(x);
    dp = (double *)device_usable(p);
    dw = (double *)device_usable(w);
    di = (uint64_t *)device_usable(id);
    if (!dx || !dp || !dw || !di) return QED_ERR_ARG;
  }
  rc = c->prec == 64 ? read_static<Half64>(c, sp, records, scr, dx, dp, dw, di, max_n, s)
                     : read_static<float4>(c, sp, records, scr, dx, dp, dw, di, max_n, s);
  if (rc != QED_OK) return rc;
  long long live = 0;
  int bits = 0;
  if (cudaMemcpyAsync(&live, scr + 1, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&bits, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return QED_ERR_CUDA;
  *n_out = live;
  // a device failure latches the context, as in qed_particles_get
  const int st = qed_latch_status(c, bits);
  if (st != QED_OK) return st;
  return live > max_n ? QED_ERR_ARG : QED_OK;
}
