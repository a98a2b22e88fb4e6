// Shape of the float64-emulating tensor-core GEMM (host logic, no device code): slice widths
// and the cut of K into batches whose float32 sums of digit products stay exact integers.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

namespace zp {

// K values per chunk of the slice products' operands (bf16, 128-byte rows).
constexpr int kSliceBK = 64;

struct SliceParams {
  int beta = 6, s = 9;
};

// Slice widths, fewest slice pairs (s (s+1) / 2) first, all with beta * s >= 54 bits.
constexpr int kSliceOpts = 4;
constexpr int kSliceBeta[kSliceOpts] = {7, 6, 5, 4};
constexpr int kSliceS[kSliceOpts] = {8, 9, 11, 14};

#if defined(__CUDACC__)
#define ZP_SLICE_HD __host__ __device__
#else
#define ZP_SLICE_HD
#endif

// The balanced base-2^beta digits of a fixed-point X (s digits, the s - 1 low ones in
// [-2^(beta-1), 2^(beta-1)), the top one what remains) read off the biased word
// Y = X + slice_bias(beta, s): low digit p (least significant first) is Y's beta-bit field p minus
// 2^(beta-1), the top digit Y >> (beta (s - 1)).
ZP_SLICE_HD constexpr long long slice_bias(int beta, int s) {
  long long b = 0;
  for (int p = 0; p < s - 1; ++p) b += (1ll << (beta - 1)) << (beta * p);
  return b;
}
ZP_SLICE_HD constexpr int slice_digit(long long y, int beta, int s, int p) {
  return p == s - 1 ? (int)(y >> (beta * p)) : (int)((y >> (beta * p)) & ((1ll << beta) - 1)) - (1 << (beta - 1));
}

// Largest number of K chunks (kSliceBK values) one batch may hold with slice option o: with
// |a_1| <= 2^beta and |a_t| <= 2^(beta-1) for t >= 2 (each later digit cuts a remainder of at
// most 1/2), diagonal d sums K * (2 * 2^beta * 2^(beta-1) + (d-3) * 2^(2 beta - 2)) at most,
// largest at d = s + 1: K * 2^(2 beta) * (1 + (s-2)/4), which must stay below 2^24.
inline int max_batch_chunks(int o) {
  const double per_k = std::ldexp(1.0, 2 * kSliceBeta[o]) * (1.0 + (kSliceS[o] - 2) / 4.0);
  return (int)std::floor((16777216.0 - 1.0) / (per_k * kSliceBK));
}

// How K is cut: slice option, chunks per batch, batches, and the recombination's Horner split.
struct EmuShape {
  SliceParams sp;
  int KC = 0;            // K chunks
  int kc_per_batch = 0;  // chunks per K batch
  int k_batches = 1;
  int split = 0;         // diagonals in the first Horner chain
  // Paired diagonals: one GEMM launch forms the sums of two neighbouring diagonals (d, d + 1)
  // and stores T_d 2^beta + T_(d+1) as one int32 (when that cannot overflow), so ceil(s / 2)
  // planes of sums cross memory instead of s.  Plane q holds diagonals (2q - s % 2, 2q + 1 -
  // s % 2) (0-based; a diagonal -1 is empty), and consecutive planes differ by 2^(2 beta).
  bool paired = false;
  int planes = 0;       // planes of sums (s, or ceil(s / 2) when paired)
  int plane_split = 0;  // planes in the first Horner chain
};

// Largest |sum of digit products| of one diagonal over `chunks` K chunks (the bound of
// max_batch_chunks) with slice option o.
inline double diagonal_bound(int o, int chunks) {
  return std::ldexp(1.0, 2 * kSliceBeta[o]) * (1.0 + (kSliceS[o] - 2) / 4.0) * kSliceBK * chunks;
}

// A large output (M x N tiles filling the GPU twice) takes one K batch with the fewest slice
// pairs that K allows, since every batch adds a full set of int32 sums to write and read.  A
// small output is cut along K into about enough batches to fill two tiles per SM, with the
// fewest-pair width whose batch length allows it.  Beyond one batch, or when no width allows
// one, the batch count is kept within 1024.  The recombination adds the batches' sums (below
// k_batches * 2^24) and runs two int64 Horner chains; the split keeps both within 63 bits.
inline bool choose_emu_shape(int64_t K, int64_t mn_tiles, int sms, EmuShape* e) {
  constexpr int BK = kSliceBK;
  const int KC = (int)((K + BK - 1) / BK);
  e->KC = KC;
  const int64_t target = 2 * (int64_t)sms;
  int o = -1, cpb = 0;
  if (mn_tiles >= target) {
    for (int i = 0; i < kSliceOpts && o < 0; ++i)
      if (KC <= max_batch_chunks(i)) {
        o = i;
        cpb = KC;
      }
  } else {
    const int want = (int)std::min<int64_t>(KC, (target + mn_tiles - 1) / mn_tiles);
    const int need = (KC + want - 1) / want;
    for (int i = 0; i < kSliceOpts && o < 0; ++i) {
      const int c = std::min(max_batch_chunks(i), need);
      if ((KC + c - 1) / c <= 1024) {
        o = i;
        cpb = c;
      }
    }
  }
  for (int i = 0; i < kSliceOpts && o < 0; ++i) {
    const int mx = max_batch_chunks(i);
    if ((KC + mx - 1) / mx <= 1024) {
      o = i;
      cpb = mx;
    }
  }
  if (o < 0) return false;
  e->sp.beta = kSliceBeta[o];
  e->sp.s = kSliceS[o];
  e->kc_per_batch = cpb;
  e->k_batches = (KC + cpb - 1) / cpb;
  int tb = 24;  // bits of |sum over batches of T_d|
  while ((1ll << (tb - 24)) < e->k_batches) ++tb;
  const int beta = e->sp.beta, s = e->sp.s;
  e->split = std::min(s, (62 - tb) / beta + 1);
  // The second chain holds s - split diagonals: tb + beta (s - split - 1) + 1 bits.
  if (s > e->split && tb + beta * (s - e->split - 1) + 1 > 63) return false;
  e->planes = s;
  e->plane_split = e->split;
  // Pairs: |T_d 2^beta + T_(d+1)| <= bound (2^beta + 1) must stay below 2^31 in every batch;
  // a plane summed over the batches then has tp = 31 + ceil(log2 k_batches) bits, and each
  // Horner step of the recombination shifts by 2 beta.
  if (diagonal_bound(o, cpb) * (std::ldexp(1.0, beta) + 1.0) < 2147483648.0) {
    const int planes = (s + 1) / 2;
    const int tp = tb + 7;
    const int psplit = std::min(planes, (62 - tp) / (2 * beta) + 1);
    if (psplit >= 1 && (planes == psplit || tp + 2 * beta * (planes - psplit - 1) + 1 <= 63)) {
      e->paired = true;
      e->planes = planes;
      e->plane_split = psplit;
    }
  }
  return true;
}

}  // namespace zp
