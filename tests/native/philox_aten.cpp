// Philox4x32-10 outputs from PyTorch's ATen engine (an implementation of the
// generator written independently of this project), for the known-answer
// pin of the oracle's generator.  Reads lines "c0 c1 c2 c3 k0 k1" (decimal)
// from stdin and prints the four output words of each.  The engine is keyed
// by its seed (k0 | k1 << 32); its counter starts at (offset, subsequence) =
// (c0 | c1 << 32, c2 | c3 << 32), and its first four outputs are the block
// of that counter.
#include <ATen/core/PhiloxRNGEngine.h>

#include <cstdint>
#include <cstdio>

int main() {
  unsigned long long c[4], k[2];
  while (std::scanf("%llu %llu %llu %llu %llu %llu", &c[0], &c[1], &c[2], &c[3], &k[0], &k[1]) == 6) {
    const uint64_t seed = k[0] | (k[1] << 32);
    const uint64_t subsequence = c[2] | (c[3] << 32);
    const uint64_t offset = c[0] | (c[1] << 32);
    at::philox_engine e(seed, subsequence, offset);
    uint32_t o[4];
    for (int j = 0; j < 4; ++j) o[j] = e();
    std::printf("%u %u %u %u\n", o[0], o[1], o[2], o[3]);
  }
  return 0;
}
