// Host driver for tests/test_emu_shape.py: prints the emulated-float64 GEMM's shape choice for
// each "K mn_tiles sms" line on stdin as "ok beta s KC kc_per_batch k_batches split paired planes plane_split".
#include <cstdio>

#include "zp_emu_shape.h"

int main() {
  long long K = 0, tiles = 0;
  int sms = 0;
  while (std::scanf("%lld %lld %d", &K, &tiles, &sms) == 3) {
    zp::EmuShape e;
    const bool ok = zp::choose_emu_shape(K, tiles, sms, &e);
    std::printf("%d %d %d %d %d %d %d %d %d %d\n", ok ? 1 : 0, e.sp.beta, e.sp.s, e.KC, e.kc_per_batch, e.k_batches,
                e.split, e.paired ? 1 : 0, e.planes, e.plane_split);
  }
  return 0;
}
