// Device helpers of the float64-emulating tensor-core contractions (error-free slicing of
// Ozaki et al., written from its definition): power-of-two scale exponents, fixed-point
// conversion from a float64's bits, and the exact integer recombination's final rounding.
// Integer-pipe arithmetic throughout: GB300's float64 pipe is the scarce one.
#pragma once

#include <cstdint>

namespace zp {

// Row exponent marking a row that holds an infinity or a NaN: its slices are zero and every
// output that involves it is NaN.
constexpr int kNonFiniteRow = 1 << 20;

// Exponent e with 2^e > |x| for the largest |x| given as its float64 bits with the sign
// cleared (positive doubles order like their bit patterns, infinities and NaNs above all
// finite values); 0 for zero, -1022 for subnormals, kNonFiniteRow for a non-finite row.
__device__ __forceinline__ int scale_exponent(unsigned long long max_abs_bits) {
  if (max_abs_bits == 0) return 0;
  const int ef = (int)(max_abs_bits >> 52);
  if (ef == 0x7ff) return kNonFiniteRow;
  return ef ? ef - 1022 : -1022;
}

// X = round-half-even(z * 2^shift) for shift = beta * s - e, i.e. x = z 2^(-e) in [-1, 1] as a
// fixed-point integer with beta * s fraction bits (|X| <= 2^(beta s) <= 2^56), from z's bits.
__device__ __forceinline__ long long to_fixed(double z, int shift) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(z);
  const int ef = (int)((b >> 52) & 0x7ff);
  const unsigned long long frac = b & 0xfffffffffffffull;
  const unsigned long long m = ef ? (frac | (1ull << 52)) : frac;  // |z| = m 2^(max(ef,1) - 1075)
  const int sh = (ef ? ef : 1) - 1075 + shift;
  unsigned long long mag;
  if (sh >= 0) {
    mag = m << sh;  // |z| < 2^e keeps this below 2^(beta s)
  } else if (sh <= -64) {
    mag = 0;  // m 2^sh < 2^-11
  } else {
    const int r = -sh;
    mag = m >> r;
    const unsigned long long rem = m & ((1ull << r) - 1);
    const unsigned long long half = 1ull << (r - 1);
    if (rem > half || (rem == half && (mag & 1))) ++mag;
  }
  return (b >> 63) ? -(long long)mag : (long long)mag;
}

// Leading zero bits of a 64-bit word (64 for zero), on the device and on the host.
__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// float64 with the given bit pattern, on the device and on the host.
__host__ __device__ __forceinline__ double double_of_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// Correctly rounded float64 of N * 2^e2 (round half to even), N a signed 128-bit integer.
// The mantissa and exponent are assembled on the integer pipe; results outside the normal
// range go through ldexp.
__host__ __device__ __forceinline__ double int128_to_double(__int128 N, int e2) {
  if (N == 0) return 0.0;
  const bool neg = N < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)0 - (unsigned __int128)N : (unsigned __int128)N;
  const unsigned long long hi = (unsigned long long)(M >> 64), lo = (unsigned long long)M;
  const int nbits = hi ? 128 - clz64(hi) : 64 - clz64(lo);
  unsigned long long mant;
  if (nbits <= 53) {
    mant = lo << (53 - nbits);
  } else {
    const int r = nbits - 53;
    const unsigned __int128 q = M >> r;
    mant = (unsigned long long)q;
    const unsigned __int128 rem = M - (q << r);
    const unsigned __int128 half = (unsigned __int128)1 << (r - 1);
    if (rem > half || (rem == half && (mant & 1))) ++mant;
  }
  int ex = nbits - 1 + e2;  // N 2^e2 = (mant / 2^52) 2^ex
  if (mant == (1ull << 53)) {
    mant >>= 1;
    ++ex;
  }
  if (ex < -1022 || ex > 1023) {
    const double v = ldexp((double)mant, ex - 52);
    return neg ? -v : v;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(ex + 1023) << 52) |
                                  (mant & 0xfffffffffffffull);
  return double_of_bits(bits);
}

// Correctly rounded float64 of (H 2^ls + L) 2^e2 (round half to even), the join of the
// recombination's two Horner chains, with 64-bit operations only: the part of L above bit ls
// is carried into H, the sign is taken off (|N| = MH 2^ls + ML, 0 <= ML < 2^ls), and the
// 53-bit mantissa with its rounding bits is cut from MH and ML.  Values of fewer than 54
// bits, |H| of 2^62 or more, shifts outside 1..62 and results outside the normal range take
// the 128-bit path.
__host__ __device__ __forceinline__ double join_to_double(long long H, long long L, int ls, int e2) {
  if (ls >= 1 && ls <= 62 && (H >> 62) == (H >> 63)) {
    const unsigned long long lr = (unsigned long long)L & ((1ull << ls) - 1);
    const long long hc = H + (L >> ls);
    const bool neg = hc < 0;
    const unsigned long long mh = neg ? (unsigned long long)(-(hc + (lr != 0 ? 1 : 0))) : (unsigned long long)hc;
    const unsigned long long ml = neg && lr != 0 ? (1ull << ls) - lr : lr;
    const int nb = 64 - clz64(mh);
    const int r = nb + ls - 53;  // bits below the mantissa
    if (mh != 0 && r >= 1) {
      unsigned long long mant;
      bool up;
      if (r >= ls) {
        const int rs = r - ls;  // bits of MH below the mantissa, 0..11
        mant = mh >> rs;
        if (rs == 0) {
          const unsigned long long half = 1ull << (ls - 1);
          up = ml > half || (ml == half && (mant & 1));
        } else {
          const unsigned long long rem = mh & ((1ull << rs) - 1), half = 1ull << (rs - 1);
          up = rem > half || (rem == half && (ml != 0 || (mant & 1)));
        }
      } else {
        mant = (mh << (ls - r)) | (ml >> r);
        const unsigned long long rem = ml & ((1ull << r) - 1), half = 1ull << (r - 1);
        up = rem > half || (rem == half && (mant & 1));
      }
      mant += up ? 1 : 0;
      int ex = nb + ls - 1 + e2;  // |N| 2^e2 lies in [2^ex, 2^(ex+1))
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++ex;
      }
      if (ex >= -1022 && ex <= 1023) {
        const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(ex + 1023) << 52) |
                                        (mant & 0xfffffffffffffull);
        return double_of_bits(bits);
      }
    }
  }
  return int128_to_double((__int128)((unsigned __int128)(__int128)H << ls) + (__int128)L, e2);
}

// Horner step acc * 2^beta + t in two's-complement int64 (the true value fits; see `split`).
__device__ __forceinline__ long long horner(long long acc, int beta, long long t) {
  return (long long)(((unsigned long long)acc << beta) + (unsigned long long)t);
}

}  // namespace zp
