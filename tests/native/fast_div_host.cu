// Host check of the library's multiply-shift division (qed_internal.h):
// for each divisor d on the command line, fast_div_magic(d) gives (m, l),
// and (umulhi(n, m) + n) >> l must equal n / d for every n < 2^31.  The
// program tries every n below 2^16 and in the top 2^16 below 2^31, the
// multiples of d and their neighbours near both ends, and 2^20 values from
// a 64-bit linear congruential sequence; it prints the number of misses.
#include <cstdio>
#include <cstdlib>
#include <cstdint>

#include "qed_internal.h"

// CUDA's __umulhi(a, b): the high 32 bits of the 64-bit product
static unsigned umulhi(unsigned a, unsigned b) { return (unsigned)(((uint64_t)a * b) >> 32); }

int main(int argc, char **argv) {
  long misses = 0, tried = 0;
  for (int k = 1; k < argc; ++k) {
    const unsigned d = (unsigned)strtoul(argv[k], nullptr, 10);
    unsigned m;
    int l;
    qed::fast_div_magic(d, m, l);
    auto check = [&](uint64_t n) {
      if (n >= (1ull << 31)) return;
      ++tried;
      const unsigned q = (umulhi((unsigned)n, m) + (unsigned)n) >> l;
      if (q != (unsigned)(n / d)) ++misses;
    };
    for (uint64_t n = 0; n < (1u << 16); ++n) check(n), check((1ull << 31) - 1 - n);
    for (uint64_t j = 1; j < 64; ++j) {
      const uint64_t a = j * d, b = ((1ull << 31) / d - j) * d;
      for (int e = -1; e <= 1; ++e) check(a + e), check(b + e);
    }
    uint64_t x = 0x9E3779B97F4A7C15ull ^ d;
    for (int i = 0; i < (1 << 20); ++i) {
      x = x * 6364136223846793005ull + 1442695040888963407ull;
      check(x >> 33);
    }
  }
  printf("%ld %ld\n", misses, tried);
  return 0;
}
