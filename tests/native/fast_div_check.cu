// Host check of the multiply-shift division used to unravel node indices:
// floor(x / d) for every divisor 1..4100, divisors next to powers of two up
// to 2^31 - 1, and dividends spread over [0, 2^31) including both ends.
// Prints "ok" and exits 0, or prints the first mismatch and exits 1.
#include <cstdio>
#include <cstdint>

#include "../../paper_1712_06091_gb300/csrc/adr_common.cuh"

static int check(unsigned d) {
  unsigned mul;
  int shr;
  adr::fast_div_params(d, mul, shr);
  uint64_t state = 0x9e3779b97f4a7c15ull ^ d;
  const unsigned edge[] = {0u, 1u, d - 1u, d, d + 1u, 2u * d - 1u, 0x7ffffffeu, 0x7fffffffu};
  for (int t = 0; t < 4096 + 8; ++t) {
    unsigned x;
    if (t < 8) {
      x = edge[t] & 0x7fffffffu;
    } else {
      state = state * 6364136223846793005ull + 1442695040888963407ull;
      x = (unsigned)(state >> 33);   // 31 random bits
    }
    const unsigned got = adr::fast_div(x, mul, shr), want = x / d;
    if (got != want) {
      std::printf("mismatch: %u / %u = %u, got %u\n", x, d, want, got);
      return 1;
    }
  }
  return 0;
}

int main() {
  for (unsigned d = 1; d <= 4100; ++d)
    if (check(d)) return 1;
  for (int l = 12; l <= 31; ++l)
    for (long long o = -3; o <= 3; ++o) {
      const long long d = (1ll << l) + o;
      if (d >= 1 && d <= 0x7fffffffll && check((unsigned)d)) return 1;
    }
  std::printf("ok\n");
  return 0;
}
