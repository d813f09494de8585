// Philox4x32-10 on the GPU: the library's device generator (qed_device.cuh)
// next to cuRAND's curand_Philox4x32_10, an independent implementation, on
// the same (counter, key) pairs.  Reads lines "c0 c1 c2 c3 k0 k1" from stdin
// and prints, per line, the library's four words then cuRAND's four.
#include <cstdio>
#include <vector>

#include <curand_kernel.h>

#include "qed_device.cuh"

__global__ void k_both(const uint4 *ctr, const uint2 *key, int n, uint4 *lib, uint4 *ref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lib[i] = qed::philox4x32_10(ctr[i], key[i]);
  ref[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

int main() {
  std::vector<uint4> c;
  std::vector<uint2> k;
  unsigned v[6];
  while (std::scanf("%u %u %u %u %u %u", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6) {
    c.push_back(make_uint4(v[0], v[1], v[2], v[3]));
    k.push_back(make_uint2(v[4], v[5]));
  }
  const int n = (int)c.size();
  if (n == 0) return 0;
  uint4 *dc, *dl, *dr;
  uint2 *dk;
  if (cudaMalloc(&dc, n * sizeof(uint4)) != cudaSuccess || cudaMalloc(&dl, n * sizeof(uint4)) != cudaSuccess ||
      cudaMalloc(&dr, n * sizeof(uint4)) != cudaSuccess || cudaMalloc(&dk, n * sizeof(uint2)) != cudaSuccess)
    return 2;
  cudaMemcpy(dc, c.data(), n * sizeof(uint4), cudaMemcpyHostToDevice);
  cudaMemcpy(dk, k.data(), n * sizeof(uint2), cudaMemcpyHostToDevice);
  k_both<<<(n + 255) / 256, 256>>>(dc, dk, n, dl, dr);
  std::vector<uint4> l(n), r(n);
  if (cudaMemcpy(l.data(), dl, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(r.data(), dr, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess)
    return 3;
  for (int i = 0; i < n; ++i)
    std::printf("%u %u %u %u %u %u %u %u\n", l[i].x, l[i].y, l[i].z, l[i].w, r[i].x, r[i].y, r[i].z, r[i].w);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dl);
  cudaFree(dr);
  return 0;
}
