// Host driver for tests/test_join_round.py: for each "H L ls e2" line on stdin prints the bits
// of join_to_double(H, L, ls, e2) and of the 128-bit reference int128_to_double of the same
// integer, as two hexadecimal words.  No GPU is touched.
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "zp_emu_device.cuh"

int main() {
  long long H = 0, L = 0;
  int ls = 0, e2 = 0;
  while (std::scanf("%lld %lld %d %d", &H, &L, &ls, &e2) == 4) {
    const double a = zp::join_to_double(H, L, ls, e2);
    const double b = zp::int128_to_double((__int128)((unsigned __int128)(__int128)H << ls) + (__int128)L, e2);
    unsigned long long ba, bb;
    std::memcpy(&ba, &a, 8);
    std::memcpy(&bb, &b, 8);
    std::printf("%016llx %016llx\n", ba, bb);
  }
  return 0;
}
