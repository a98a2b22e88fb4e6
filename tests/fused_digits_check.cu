// Host driver for tests/test_fused_digits.py: prints the fused kernel's constants and the
// balanced digits its host-callable helpers give for the fixed-point values the test passes,
// for both digit shapes (11 digits of 5 bits, 9 digits of 6 bits).  No GPU is touched.
//   stdin: "c" (constants: beta, digits, max sets, max modes, chunk bytes, bias of the 11-digit
//          shape), "c9" (beta, digits, max modes, bias of the 9-digit shape, the digit count
//          chosen for 1489 and 1490 positions), or "d <int64>" / "d9 <int64>" (the digits of
//          that value in the 11- / 9-digit shape, most significant first).
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "zp_fused.h"

template <int NDIG>
static void print_digits(long long x) {
  const long long y = x + zp::fused_bias<NDIG>();
  const int beta = zp::fused_beta(NDIG);
  for (int t = 0; t < NDIG; ++t) {
    const int f = zp::fused_digit_field<NDIG>(y, t);
    std::printf("%d%c", t == 0 ? f : f - (1 << (beta - 1)), t + 1 < NDIG ? ' ' : '\n');
  }
}

int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (std::strcmp(op, "c") == 0) {
      std::printf("%d %d %d %" PRId64 " %u %lld\n", zp::kFusedBeta, zp::kFusedDigits, zp::kFusedMaxSets,
                  (int64_t)zp::kFusedMaxModes, zp::kFusedBChunk, zp::fused_bias());
    } else if (std::strcmp(op, "c9") == 0) {
      std::printf("%d %d %" PRId64 " %lld %d %d\n", zp::fused_beta(zp::kFusedDigitsShort), zp::kFusedDigitsShort,
                  (int64_t)zp::kFusedMaxModesShort, zp::fused_bias<zp::kFusedDigitsShort>(),
                  zp::fused_digits_for(zp::kFusedMaxModesShort), zp::fused_digits_for(zp::kFusedMaxModesShort + 1));
    } else if (op[0] == 'd') {
      long long x = 0;
      if (std::scanf("%lld", &x) != 1) return 1;
      if (std::strcmp(op, "d9") == 0) print_digits<zp::kFusedDigitsShort>(x);
      else print_digits<zp::kFusedDigits>(x);
    }
  }
  return 0;
}
