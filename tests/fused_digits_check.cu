// Host driver for tests/test_fused_digits.py: prints the fused kernel's constants and the
// balanced digits its host-callable helpers give for the fixed-point values the test passes.
// No GPU is touched.
//   stdin: "c" (constants: beta, digits, max sets, max modes, chunk bytes, bias) or
//          "d <int64>" (the digits of that value, most significant first).
#include <cinttypes>
#include <cstdio>

#include "zp_fused.h"

int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (op[0] == 'c') {
      std::printf("%d %d %d %" PRId64 " %u %lld\n", zp::kFusedBeta, zp::kFusedDigits, zp::kFusedMaxSets,
                  (int64_t)zp::kFusedMaxModes, zp::kFusedBChunk, zp::fused_bias());
    } else if (op[0] == 'd') {
      long long x = 0;
      if (std::scanf("%lld", &x) != 1) return 1;
      const long long y = x + zp::fused_bias();
      for (int t = 0; t < zp::kFusedDigits; ++t) {
        const int f = zp::fused_digit_field(y, t);
        std::printf("%d%c", t == 0 ? f : f - (1 << (zp::kFusedBeta - 1)), t + 1 < zp::kFusedDigits ? ' ' : '\n');
      }
    }
  }
  return 0;
}
