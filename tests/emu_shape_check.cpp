// Host driver for tests/test_emu_shape.py: prints the emulated-float64 GEMM's shape choice for
// each "K mn_tiles sms" line on stdin as "ok beta s KC kc_per_batch k_batches split paired planes
// plane_split", and for each "d beta s X" line the slice digits of X read off the biased word
// (most significant first).
#include <cstdio>
#include <cstring>

#include "zp_emu_shape.h"

int main() {
  char tok[32];
  while (std::scanf("%31s", tok) == 1) {
    if (std::strcmp(tok, "d") == 0) {
      int beta = 0, s = 0;
      long long x = 0;
      if (std::scanf("%d %d %lld", &beta, &s, &x) != 3) return 1;
      const long long y = x + zp::slice_bias(beta, s);
      for (int t = 0; t < s; ++t) std::printf("%d%c", zp::slice_digit(y, beta, s, s - 1 - t), t + 1 < s ? ' ' : '\n');
      continue;
    }
    long long K = 0, tiles = 0;
    int sms = 0;
    if (std::sscanf(tok, "%lld", &K) != 1 || std::scanf("%lld %d", &tiles, &sms) != 2) return 1;
    zp::EmuShape e;
    const bool ok = zp::choose_emu_shape(K, tiles, sms, &e);
    std::printf("%d %d %d %d %d %d %d %d %d %d\n", ok ? 1 : 0, e.sp.beta, e.sp.s, e.KC, e.kc_per_batch, e.k_batches,
                e.split, e.paired ? 1 : 0, e.planes, e.plane_split);
  }
  return 0;
}
