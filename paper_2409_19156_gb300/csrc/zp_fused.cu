// Fused float64-accurate Zernike series for up to 16 coefficient sets: the basis is built on
// chip and fed straight to the tensor cores; no basis value, digit or partial sum is written
// to global memory.
//
//   F[p, s] = sum_j Z_j(p) C[j, s],   s < 16,
//
// contracted by error-free slicing (Ozaki et al., a published scheme, written here from its
// definition): every Z_j(p) is scaled by 2^-e_p (e_p = 1 for 0 <= r <= 1, where |Z| <= 1;
// else from a first pass over the point's modes), truncated to a fixed-point integer and cut
// into D balanced base-2^beta digits a_1..a_D (integers of at most beta + 1 bits, exact in
// bfloat16): D = 11 digits of 5 bits (55 fraction bits) for contractions of up to 5041
// positions, D = 9 of 6 bits (54 bits) for up to 1489; the coefficients are rounded to the same
// fixed point and cut the same way per set (b_1..b_D, scale 2^-e_s).
// Then Z C = 2^(e_p + e_s) sum_d T_d 2^(-beta d) with T_d = sum_{t+u=d} sum_j a_t b_u, kept for
// d <= D + 1 (the dropped pairs weigh below about 2^-(beta D) of the scales).
//
// One persistent CTA per SM works through 128-point tiles:
//  - warps 0-11 (three threads per point, each walking one of three streams of |m| columns:
//    more independent float64 chains per scheduler than two streams give) run the float64
//    recursion of Sec. 2 (Algorithm 1's column order within a stream, cos/sin(m theta) by
//    angle addition between consecutive columns), form each value, cut it into its D digits
//    on the integer pipe and write them into D digit tiles in shared memory (the tensor
//    core's 64-byte swizzled K-major layout, 32 K values per stage, two stages, the streams'
//    8-value units interleaved along K);
//  - warp 12 issues the tcgen05 MMAs: per K step and A digit t, one MMA of N = 16 D against
//    the coefficient digit tile shifted by t blocks of 16 rows (zero blocks in front), so that
//    every MMA adds a_t b_u into the TMEM columns of diagonal t + u for all u at once; every
//    diagonal sum is an integer below 2^24 (the position limits above), hence exact in float32;
//  - the warps of streams 0 and 1, after producing a tile, take the previous tile's D x 16
//    diagonal sums out of TMEM, recombine them exactly in integers (two Horner chains joined
//    into 128 bits) and round once to float64.
// The K order of the contraction is the plan's slot order with every column padded to a
// multiple of 8 positions (so a column's steps fill whole 16-byte operand units in unrolled
// straight-line code), and the coefficient digits are prepared per call in that order
// (fused_coeff_kernel).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "zp_api_common.h"
#include "zp_device.cuh"
#include "zp_emu_device.cuh"
#include "zp_fused.h"
#include "zp_ptx.cuh"
#include "zp_series_internal.h"

namespace zp {
namespace {

constexpr int FM = 128;             // points per tile (TMEM lanes)
constexpr int FBK = 32;             // K values per stage (64-byte bf16 rows)
constexpr int FNS = kFusedMaxSets;  // sets per digit block (rows of a B block, TMEM columns)
constexpr uint32_t kRowBytes = 64;
constexpr uint32_t kASlice = FM * kRowBytes;                 // one digit tile of A: 8 KB
constexpr uint32_t kBBlock = FNS * kRowBytes;                // one digit block of B: 1 KB
constexpr int kStages = 2;
constexpr int kAccStride = 256;                              // two accumulators in 512 columns
// Warps 0 .. 4 kStreams - 1 produce (warp w: point rows 32 (w % 4) .. + 31, stream w / 4); the
// warps of streams 0 and 1 also drain the accumulator of the previous tile (warp w: its rows,
// sets 8 (w / 4) .. + 7); the last warp issues MMAs.
constexpr int kStreams = kFusedStreams;
constexpr int kProducerWarps = 4 * kStreams, kMmaWarp = kProducerWarps;
constexpr int kDrainWarps = 8;
constexpr int kThreads = 32 * (kProducerWarps + 1);  // 416
constexpr uint32_t kAux = 2048;

// The digit shape of a launch: NDIG digits of Beta bits per value (11 x 5 for contractions of
// up to 5041 positions, 9 x 6 for up to 1489).  A stage holds NDIG digit tiles of A and
// 2 NDIG - 1 blocks of B (NDIG - 1 zero blocks, then the coefficient digits); the accumulator
// holds NDIG diagonal blocks of 16 sets; the drain's first Horner chain takes Split diagonals.
template <int NDIG>
struct FK {
  static constexpr int Beta = fused_beta(NDIG);
  static constexpr uint32_t ABytes = NDIG * kASlice;
  static constexpr uint32_t BPadBytes = (2 * NDIG - 1) * kBBlock;
  static constexpr uint32_t BCopyOffset = (NDIG - 1) * kBBlock;
  static constexpr uint32_t BCopyBytes = NDIG * kBBlock;
  static constexpr uint32_t StageBytes = ABytes + BPadBytes;
  static constexpr int AccCols = NDIG * FNS;
  static constexpr int Split = NDIG == kFusedDigits ? 5 : 4;
  static constexpr long long Bias = fused_bias<NDIG>();
  static constexpr uint32_t Smem = kStages * StageBytes + 1024 + kAux;
  static_assert(BPadBytes % 1024 == 0 && ABytes % 1024 == 0, "1024-byte aligned operand tiles");
  static_assert(Smem <= 232448, "shared memory per CTA");
  static_assert(AccCols <= kAccStride, "accumulator fits its TMEM half");
  static_assert(BCopyBytes <= kFusedBChunk, "a chunk's digit blocks fit its stride");
  // Both Horner chains stay within int64: diagonal sums below 2^24, Beta bits per step.
  static_assert(24 + Beta * (Split - 1) + 1 <= 63 && 24 + Beta * (NDIG - Split - 1) + 1 <= 63, "Horner chains");
};

__device__ unsigned int g_fused_error = 0;  // set when a bounded wait gives up

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Digit t >= 1 of two biased words as one word of two bf16 (value 0 low): the unsigned Beta-bit
// fields f placed under the bfloat16 pattern of 128 (0x4300 | f is exactly 128 + f for f < 128),
// then one packed subtraction of 128 + 2^(Beta-1) leaves the balanced digit f - 2^(Beta-1) in
// each half (exact).
template <int NDIG, int T>
__device__ __forceinline__ uint32_t digit_pair_low(long long Y0, long long Y1) {
  constexpr int B = FK<NDIG>::Beta;
  static_assert(T >= 1 && T < NDIG, "unsigned digit fields");
  constexpr int s = B * (NDIG - 1 - T);  // bit position of the field
  constexpr uint32_t mask = (1u << B) - 1u;
  uint32_t a, b;
  if constexpr (s + B <= 32) {
    a = (uint32_t)Y0 >> s;
    b = s >= 16 ? (uint32_t)Y1 >> (s - 16) : (uint32_t)Y1 << (16 - s);
  } else {
    a = (uint32_t)(Y0 >> s);
    b = (uint32_t)(Y1 >> s) << 16;
  }
  const uint32_t w = (a & mask) | (b & (mask << 16)) | 0x43004300u;
  __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&w);
  constexpr unsigned short sub = (unsigned short)(0x4300u | (1u << (B - 1)));  // 128 + 2^(B-1)
  v = __hsub2(v, __nv_bfloat162(__nv_bfloat16_raw{sub}, __nv_bfloat16_raw{sub}));
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Digit 0 (signed, at most 2^Beta + 1 in magnitude) of two biased words, by the float32 magic
// sum.
template <int NDIG>
__device__ __forceinline__ uint32_t digit_pair_top(long long Y0, long long Y1) {
  const uint32_t f0 = __float_as_uint(__int_as_float(0x4B400000 + fused_digit_field<NDIG>(Y0, 0)) - 12582912.0f);
  const uint32_t f1 = __float_as_uint(__int_as_float(0x4B400000 + fused_digit_field<NDIG>(Y1, 0)) - 12582912.0f);
  return __byte_perm(f0, f1, 0x7632);
}

template <int NDIG, int T = 1>
__device__ __forceinline__ void digit_pair_lows(long long Y0, long long Y1, uint32_t (&w)[NDIG]) {
  if constexpr (T < NDIG) {
    w[T] = digit_pair_low<NDIG, T>(Y0, Y1);
    digit_pair_lows<NDIG, T + 1>(Y0, Y1, w);
  }
}

// All NDIG digits of two biased words Y = X + bias, joined per digit (value 0 low).
template <int NDIG>
__device__ __forceinline__ void digit_pair_biased(long long Y0, long long Y1, uint32_t (&w)[NDIG]) {
  w[0] = digit_pair_top<NDIG>(Y0, Y1);
  digit_pair_lows<NDIG>(Y0, Y1, w);
}

// Two values' digits joined per digit into one 32-bit word of two bf16 (value 0 low).
template <int NDIG>
__device__ __forceinline__ void digit_pair(long long X0, long long X1, uint32_t (&w)[NDIG]) {
  digit_pair_biased<NDIG>(X0 + FK<NDIG>::Bias, X1 + FK<NDIG>::Bias, w);
}

struct Barriers {
  uint64_t full[kStages];   // producer warps (one arrival each)
  uint64_t bfull[kStages];  // coefficient digit copy (1 arrival + bytes)
  uint64_t empty[kStages];  // MMA commit
  uint64_t tfull[2];        // MMA commit after a tile's last stage
  uint64_t tempty[2];       // draining warps after draining the accumulator (8 arrivals)
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};
static_assert(sizeof(Barriers) <= kAux, "barrier block");

// Bounded wait by one lane of the warp; the others learn the outcome by a shuffle.  Roles that
// mostly wait for the producers (the epilogue) poll with a sleep in between.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int lane,
                                          bool sleepy = false) {
  bool ok = true;
  if (lane == 0) ok = sleepy ? ptx::mbar_wait_sleepy(bar, parity, abort_flag, 500) : ptx::mbar_wait(bar, parity, abort_flag);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// z * 2^shift truncated toward zero to an int64 (|z| 2^shift < 2^55, z finite), from z's bits
// on the integer pipe: the float64 -> int64 conversion instruction issues on GB300's float64
// pipe, the one this kernel is bound by.  Truncation instead of rounding leaves an error below
// 2^-shift per value (one unit of the last of the 55 fraction bits).
__device__ __forceinline__ long long to_fixed_trunc(double z, int shift) {
  const uint32_t hi = (uint32_t)__double2hiint(z), lo = (uint32_t)__double2loint(z);
  const int ef = (int)((hi >> 20) & 0x7ffu);
  const int sh = ef - 1075 + shift;  // |z| 2^shift = m 2^sh with m the 53-bit significand
  const unsigned long long m = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
  unsigned long long mag = sh >= 0 ? (m << (sh & 63)) : (m >> (-sh < 63 ? -sh : 63));
  mag = ef == 0 ? 0ull : mag;  // zero (and subnormals, far below the last fraction bit)
  return (hi >> 31) ? -(long long)mag : (long long)mag;
}

__device__ __forceinline__ void fail(volatile int* abort_flag) {
  *abort_flag = 1;
  atomicOr(&g_fused_error, 1u);
}

// Values the fused kernel contracts: VK_Z the basis Z (the forward series), VK_DTHETA its
// theta-derivative (m R times the other angular factor, negated for cos), VK_DRHO its
// rho-derivative (dR/drho times the angular factor, the recursion's derivative lane).  The
// two derivative series give the adjoint's point gradients: grad_r = sum_s G (dZ/dr C).
constexpr int VK_Z = kFusedZ, VK_DTHETA = kFusedDTheta, VK_DRHO = kFusedDRho;

// The float64 walk of one point over every column of its plan (Sec. 2 recursion, rescaled as
// in the plan's tables: Q_N = (A_N rho^2 - B_N) Q_{N-1} - Q_{N-2}, R = W0_N Q_N; for VK_DRHO
// also Q'_N = (A_N rho^2 - B_N) Q'_{N-1} + 2 A_N rho Q_{N-1} - Q'_{N-2}), calling emit(value)
// for every output slot in the plan's slot order: Q_N cos/sin(m theta), Q_N times the
// derivative of cos/sin(m theta), or Q'_N cos/sin(m theta) -- the values the kernel digitises
// (the weight W0_N travels with the coefficients).  Used for the row scale of points off the
// unit disc, so written for clarity: seeds from powers, angles from sincos.
template <int VK, typename Emit>
__device__ __forceinline__ void walk_point(const FusedInst& d, double rho, double th, Emit&& emit) {
  const double u = rho * rho;
  for (int c = 0; c < d.n_cols; ++c) {
    const Column col = d.cols[c];
    const int m = col.m;
    double cm = 1.0, sm = 0.0;
    if (m != 0) sincos((double)m * th, &sm, &cm);
    // Angular factors of a cos and of a sin output.
    const double fc = VK == VK_DTHETA ? -(double)m * sm : cm;
    const double fs = VK == VK_DTHETA ? (double)m * cm : sm;
    const double* h = d.table + (size_t)col.table_row * kRow;
    const uint2* st = d.steps + col.table_row + kHeaderRows;
    const int32_t* sp = d.slot_ptr + col.slot_base;
    // Seeds Q_{-1} = 0, Q_{-2} = -rho^m (and their rho-derivatives) with (A_0, B_0) = (0, 0),
    // (A_1, B_1) = (m + 2, m + 1) from the column header.
    double S = 0.0, T = -pow_uint(rho, m);
    double Sd = 0.0, Td = m > 0 ? -(double)m * pow_uint(rho, m - 1) : 0.0;
    for (int N = 0; N < col.n_steps; ++N) {
      const double* row = h + (size_t)(kHeaderRows + N) * kRow;
      const double A = N >= 2 ? row[0] : (N == 1 ? h[4] : 0.0);
      const double B = N >= 2 ? row[1] : (N == 1 ? h[8] : 0.0);
      const double g = fma(A, u, -B);
      const double qd = fma(g, Sd, fma(2.0 * A * rho, S, -Td));
      const double q = fma(g, S, -T);
      Td = Sd;
      Sd = qd;
      T = S;
      S = q;
      const double v = VK == VK_DRHO ? qd : q;
      const uint32_t info = st[N].x;
      uint32_t cnt = info & 0xffu, flags = info >> 8;
      if (cnt == 0) continue;
      if (cnt == kStepIrregular) {
        for (int s = sp[N]; s < sp[N + 1]; ++s) {
          const uint32_t code = (uint32_t)__ldg(d.slot_idx + s);
          emit(v * ((code >> 31) ? fs : fc));
        }
      } else {
        for (; cnt > 0; --cnt, flags >>= 1) emit(v * ((flags & 1u) ? fs : fc));
      }
    }
  }
}

// Item `it` of the launch: instance and first point.
__device__ __forceinline__ void item_of(const FusedArgs& a, int64_t it, int& inst, int64_t& p0) {
  if (a.items) {
    const FusedItem w = a.items[it];
    inst = w.inst;
    p0 = (int64_t)w.tile * FM;
  } else {
    inst = 0;
    p0 = it * FM;
  }
}

__device__ __forceinline__ const FusedInst& inst_of(const FusedArgs& a, int inst) {
  return a.insts ? a.insts[inst] : a.single;
}

// Drains accumulator `acc` of a finished tile for this thread's row and 8 sets (h): NDIG diagonal
// sums per output out of TMEM, recombined exactly (two Horner chains joined into 128 bits) and
// rounded once to float64.
template <int NDIG>
__device__ __forceinline__ void drain_tile(const FusedInst& d, int64_t p0, uint32_t tmem_base, uint32_t acc, uint32_t q,
                                           uint32_t row, int h, int ep) {
  using K = FK<NDIG>;
  const int64_t p = p0 + row;
  long long hi[8] = {}, lo[8] = {};
#pragma unroll
  for (int db = 0; db < NDIG; ++db) {
    uint32_t v[8];
    ptx::tmem_ld_32x32b_x8(tmem_base + ((q * 32u) << 16) + acc * kAccStride + (uint32_t)(db * FNS + h * 8), v);
    ptx::tmem_ld_wait(v);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const long long tv = (long long)__float2int_rn(__uint_as_float(v[i]));
      if (db < K::Split) hi[i] = horner(hi[i], K::Beta, tv);
      else lo[i] = horner(lo[i], K::Beta, tv);
    }
  }
  if (p >= d.P) return;
  const int e_base = ep - K::Beta * (NDIG + 1);
  if (d.dot_out) {
    // Row sum over this thread's 8 sets of G times the series; the point's two halves are added
    // onto the zeroed output (two addends: the same float64 sum in either order).
    const double* grow = d.gdot + p * d.S;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (h * 8 + i >= d.S) break;
      const int ec = d.cexp[h * 8 + i];
      const double v = (ep == kNonFiniteRow || ec == kNonFiniteRow)
                           ? __longlong_as_double(0x7ff8000000000000ll)
                           : join_to_double(hi[i], lo[i], K::Beta * (NDIG - K::Split), e_base + ec);
      acc = fma(grow[h * 8 + i], v, acc);
    }
    atomicAdd(d.dot_out + p, acc);
    return;
  }
  if (!d.out) return;
  double* orow = d.out + p * d.S;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (h * 8 + i >= d.S) break;
    const int ec = d.cexp[h * 8 + i];
    orow[h * 8 + i] = (ep == kNonFiniteRow || ec == kNonFiniteRow)
                          ? __longlong_as_double(0x7ff8000000000000ll)
                          : join_to_double(hi[i], lo[i], K::Beta * (NDIG - K::Split), e_base + ec);
  }
}

template <int VK, int NDIG>
__global__ void __launch_bounds__(kThreads, 1) fused_emu_kernel(FusedArgs a) {
  using K = FK<NDIG>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  Barriers* bar = reinterpret_cast<Barriers*>(smem + kStages * K::StageBytes);
  volatile int* abort_flag = &bar->abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      ptx::mbar_init(&bar->full[i], kProducerWarps);
      ptx::mbar_init(&bar->bfull[i], 1);
      ptx::mbar_init(&bar->empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&bar->tfull[i], 1);
      ptx::mbar_init(&bar->tempty[i], kDrainWarps);
    }
    ptx::mbar_init(&bar->drain, 1);
    bar->abort_flag = 0;
    ptx::fence_barrier_init();
  }
  // The zero blocks in front of each stage's coefficient digits (never overwritten).
  for (uint32_t i = threadIdx.x; i < kStages * K::BCopyOffset / 16; i += kThreads) {
    const uint32_t st = i / (K::BCopyOffset / 16), o = i % (K::BCopyOffset / 16);
    reinterpret_cast<uint4*>(smem + st * K::StageBytes + K::ABytes)[o] = make_uint4(0u, 0u, 0u, 0u);
  }
  ptx::fence_proxy_async_smem();
  if (warp == kMmaWarp) {
    ptx::tmem_alloc(&bar->tmem_base, 2 * kAccStride);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = bar->tmem_base;

  if (warp < kProducerWarps) {
    // ------------------------------------------------------- producers (and accumulator drain)
    const uint32_t q = (uint32_t)(warp & 3);          // TMEM lane quadrant of this warp
    const uint32_t row = q * 32 + (uint32_t)lane;     // point row of the tile (TMEM lane)
    const int strm = warp >> 2;                       // column stream of this thread
    int stage = 0;
    uint32_t sphase = 0;
    uint32_t b_issued0 = 0u, b_issued1 = 0u;  // coefficient copies issued per stage (warp 0, lane 0)
    static_assert(kStages == 2, "two stages");
    bool ok = true;
    int64_t local = 0;
    // The previous tile, drained after this thread produced the next one.
    int prev_inst = -1, prev_ep = 0;
    int64_t prev_p0 = 0;
    auto drain_prev = [&]() -> bool {
      if (strm >= 2) return true;  // streams 0 and 1 drain
      const uint32_t pacc = (uint32_t)((local - 1) & 1), puse = (uint32_t)(((local - 1) >> 1) & 1);
      if (!warp_wait(&bar->tfull[pacc], puse, abort_flag, lane)) return false;
      ptx::tc_fence_after();
      drain_tile<NDIG>(inst_of(a, prev_inst), prev_p0, tmem_base, pacc, q, row, strm, prev_ep);
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&bar->tempty[pacc]);
      return true;
    };
    for (int64_t it = blockIdx.x; it < a.n_items && ok; it += gridDim.x, ++local) {
      int ii;
      int64_t p0;
      item_of(a, it, ii, p0);
      const FusedInst& d = inst_of(a, ii);
      const int64_t p = p0 + row;
      const bool valid = p < d.P;
      const double rho = valid ? d.r[p] : 0.0, th = valid ? d.theta[p] : 0.0;
      // Row exponent: on the unit disc |R| <= 1, so |Q cos/sin| <= 1 / w_N < 2^ep_disc; elsewhere
      // the point's largest digitised value decides (both threads of the point walk all of its
      // columns for it).
      int ep = d.ep_disc;
      if (!(rho >= 0.0 && rho <= 1.0 && isfinite(th))) {
        unsigned long long mx = 0;
        bool bad = false;
        walk_point<VK>(d, rho, th, [&](double z) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(z) & 0x7fffffffffffffffull;
          mx = b > mx ? b : mx;
          bad |= !isfinite(z);
        });
        ep = bad ? kNonFiniteRow : scale_exponent(mx);
      }
      const bool zero_row = ep == kNonFiniteRow;
      const int shift = K::Beta * NDIG - (zero_row ? 0 : ep);

      int unit = 0;  // this stream's next unit; its global unit is kStreams unit + strm
      uint32_t w[NDIG][4];
      uint8_t* sA = smem + stage * K::StageBytes;
      // This stream's next unit in shared memory (its byte offset within digit tile 0), opening
      // the stage at the stream's first unit in it (slot below kStreams: the stream's previous
      // unit lies in the stage before): waiting for the stage to be free, stream 0 starting its
      // coefficient copy (every stream has a unit in every stage).  -1 when a bounded wait gave up.
      auto open_unit = [&]() -> int {
        const int g = kStreams * unit + strm;  // global unit
        const int slot = g & 3;                 // unit slot within the stage (0..3)
        if (slot < kStreams) {
          if (!warp_wait(&bar->empty[stage], sphase ^ 1u, abort_flag, lane)) return -1;
          sA = smem + stage * K::StageBytes;
          if (warp == 0 && lane == 0) {
            const int kc = g >> 2;
            ptx::mbar_arrive_expect_tx(&bar->bfull[stage], K::BCopyBytes);
            ptx::bulk_g2s(sA + K::ABytes + K::BCopyOffset, d.bdig + (size_t)kc * kFusedBChunk, K::BCopyBytes,
                          &bar->bfull[stage]);
            if (stage == 0) ++b_issued0;
            else ++b_issued1;
          }
        }
        return (int)ptx::sw_offset_b16<kRowBytes>(row, (uint32_t)(slot * 8));
      };
      // The unit is written: hand the stage to the MMA warp after the stream's last unit in it
      // (slot 4 - kStreams or later: the stream's next unit lies in the next stage).
      auto finish_unit = [&]() {
        const int slot = (kStreams * unit + strm) & 3;
        ++unit;
        if (slot >= 4 - kStreams) {
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&bar->full[stage]);
          if (++stage == kStages) {
            stage = 0;
            sphase ^= 1u;
          }
        }
      };
      auto store_unit = [&]() -> bool {
        const int off = open_unit();
        if (off < 0) return false;
#pragma unroll
        for (int t = 0; t < NDIG; ++t)
          *reinterpret_cast<uint4*>(sA + t * kASlice + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
        finish_unit();
        return true;
      };
      // Digits of two consecutive K values into word `word` of the unit (word 0..3): per digit,
      // the two values' bf16 patterns joined into one 32-bit word.
      auto put_pair_const = [&](auto word_c, double z0, double z1) {
        constexpr int word = decltype(word_c)::value;
        const long long Y0 = (zero_row ? 0 : to_fixed_trunc(z0, shift)) + K::Bias;
        const long long Y1 = (zero_row ? 0 : to_fixed_trunc(z1, shift)) + K::Bias;
        uint32_t pw[NDIG];
        digit_pair_biased<NDIG>(Y0, Y1, pw);
#pragma unroll
        for (int t = 0; t < NDIG; ++t) w[t][word] = pw[t];
      };
      // The walk of this stream's columns (Sec. 2 recursion in the plan's rescaled form, Algorithm
      // 1's column order within the stream).  The recursion runs uniformly from the seeds
      // q_{-2} = -rho^m, q_{-1} = 0 with (A_0, B_0) = (0, 0) and (A_1, B_1) = ((m+2), (m+1)), so
      // unrolled steps need no cases; cos/sin(m theta) and rho^m advance by one or two columns
      // by angle addition and products.
      const double u = rho * rho;
      double s1, c1;
      sincos(th, &s1, &c1);
      const double c2 = fma(c1, c1, -s1 * s1), s2 = 2.0 * s1 * c1;
      // Three streams deal the columns out about three |m| apart: steps of 3 theta too (a step
      // of 4 as two of 2).  The walk starts from the state of m = 0 (cos = 1, sin = 0, rho^0 = 1).
      const double c3 = fma(c2, c1, -s2 * s1), s3 = fma(s2, c1, c2 * s1), r3 = u * rho;
      double cm = 1.0, sm = 0.0, pm = 1.0;
      double pm1 = 0.0;  // rho^(m-1) for the derivative lane's seed (VK_DRHO)
      int m_prev = 0;
      const int ncs = d.ncols_s[strm];
      int scol0 = 0;
      for (int sp = 0; sp < strm; ++sp) scol0 += d.ncols_s[sp];
      const int32_t* scol = d.scols + scol0;
      for (int ci = 0; ci < ncs && ok; ++ci) {
        const int c = scol[ci];
        const Column col = d.cols[c];
        const int m = col.m;
        if (m == m_prev + 1) {
          const double cn = fma(cm, c1, -sm * s1);
          sm = fma(sm, c1, cm * s1);
          cm = cn;
          if constexpr (VK == VK_DRHO) pm1 = pm;
          pm *= rho;
        } else if (m == m_prev + 2) {
          const double cn = fma(cm, c2, -sm * s2);
          sm = fma(sm, c2, cm * s2);
          cm = cn;
          if constexpr (VK == VK_DRHO) pm1 = pm * rho;
          pm *= u;
        } else if (m == m_prev + 3) {
          const double cn = fma(cm, c3, -sm * s3);
          sm = fma(sm, c3, cm * s3);
          cm = cn;
          if constexpr (VK == VK_DRHO) pm1 = pm * u;
          pm *= r3;
        } else if (m != m_prev) {
          cm = 1.0;
          sm = 0.0;
          if (m != 0) sincos((double)m * th, &sm, &cm);
          pm = pow_uint(rho, m);
          if constexpr (VK == VK_DRHO) pm1 = m > 0 ? pow_uint(rho, m - 1) : 0.0;
        }
        m_prev = m;
        // Angular factors of a cos and of a sin output (their theta-derivatives for VK_DTHETA).
        const double fcos = VK == VK_DTHETA ? -(double)m * sm : cm;
        const double fsin = VK == VK_DTHETA ? (double)m * cm : sm;
        const double* h = d.table + (size_t)col.table_row * kRow;
        const int n_steps = col.n_steps;
        const int4 fc = d.fcols[c];
        const int kind = fc.x & 255;
        const double fa = (fc.x >> 8) & 1 ? fsin : fcos, fb = (fc.x >> 9) & 1 ? fsin : fcos;
        // VK_DRHO walks the value lane times 2 rho (seed -2 rho^(m+1)): with u = rho^2,
        // dQ_N/drho = 2 rho dQ_N/du and dQ_N/du = A_N Q_{N-1} + g_N dQ_{N-1}/du - dQ_{N-2}/du, so
        // the derivative lane Q'_N = g_N Q'_{N-1} + A_N (2 rho Q_{N-1}) - Q'_{N-2} takes A_N from
        // the table with no product by rho per step.  Its seeds: Q'_{-1} = 0, Q'_{-2} = -m rho^(m-1).
        double S = 0.0, T = VK == VK_DRHO ? -pm * (2.0 * rho) : -pm;
        double Sd = 0.0, Td = VK == VK_DRHO ? -(double)m * pm1 : 0.0;
        // The recursion coefficient g_N = A_N rho^2 - B_N of step N < n_steps.
        auto coef = [&](int N, double& A) -> double {
          const double* rw = h + (size_t)(kHeaderRows + N) * kRow;
          A = N >= 2 ? rw[0] : (N == 1 ? h[4] : 0.0);
          const double B = N >= 2 ? rw[1] : (N == 1 ? h[8] : 0.0);
          return fma(A, u, -B);
        };
        // One recursion step N < n_steps: Q_N, or Q'_N for VK_DRHO (S, T then hold 2 rho Q).
        auto step = [&](int N) -> double {
          double A;
          const double g = coef(N, A);
          if constexpr (VK == VK_DRHO) {
            const double qd = fma(g, Sd, fma(A, S, -Td));
            Td = Sd;
            Sd = qd;
          }
          const double qv = fma(g, S, -T);
          T = S;
          S = qv;
          return VK == VK_DRHO ? Sd : qv;
        };
        // The recursion is linear in its seeds: walked from the seeds times an angular factor f
        // it gives Q_N f directly, one FMA per output instead of a product after the step (the
        // derivative lane of VK_DRHO needs Q_N itself and keeps the products).  Steps past the
        // column's end (the padding of its last unit) are not walked: a zero value's digits are
        // zero words.
        constexpr bool kScaled = VK != VK_DRHO;
        if (kind == kFusedKindTwo) {
          // Two outputs per step: four steps fill one unit.
          double Sa = 0.0, Ta = -pm * fa, Sb = 0.0, Tb = -pm * fb;
          for (int N0 = 0; N0 < n_steps && ok; N0 += 4) {
            auto one = [&](auto ic) {
              constexpr int i = decltype(ic)::value;
              if (i == 0 || N0 + i < n_steps) {
                if constexpr (kScaled) {
                  double A;
                  const double g = coef(N0 + i, A);
                  const double qa = fma(g, Sa, -Ta), qb = fma(g, Sb, -Tb);
                  Ta = Sa;
                  Sa = qa;
                  Tb = Sb;
                  Sb = qb;
                  put_pair_const(ic, qa, qb);
                } else {
                  const double qv = step(N0 + i);
                  put_pair_const(ic, qv * fa, qv * fb);
                }
              } else {
#pragma unroll
                for (int t = 0; t < NDIG; ++t) w[t][i] = 0u;
              }
            };
            one(std::integral_constant<int, 0>{});
            one(std::integral_constant<int, 1>{});
            one(std::integral_constant<int, 2>{});
            one(std::integral_constant<int, 3>{});
            ok = store_unit();
          }
        } else if (kind == kFusedKindOne) {
          // One output per step: eight steps fill one unit.  m = 0: the angular factor is 1 (its
          // theta-derivative 0).
          const double f1 = m == 0 ? (VK == VK_DTHETA ? 0.0 : 1.0) : fa;
          double Sa = 0.0, Ta = -pm * f1;
          auto out = [&](int N) -> double {
            if constexpr (kScaled) {
              double A;
              const double qa = fma(coef(N, A), Sa, -Ta);
              Ta = Sa;
              Sa = qa;
              return qa;
            } else {
              return step(N) * f1;
            }
          };
          for (int N0 = 0; N0 < n_steps && ok; N0 += 8) {
            auto two = [&](auto ic) {
              constexpr int i = decltype(ic)::value;
              if (i == 0 || N0 + 2 * i < n_steps) {
                const double z0 = out(N0 + 2 * i);
                const double z1 = N0 + 2 * i + 1 < n_steps ? out(N0 + 2 * i + 1) : 0.0;
                put_pair_const(ic, z0, z1);
              } else {
#pragma unroll
                for (int t = 0; t < NDIG; ++t) w[t][i] = 0u;
              }
            };
            two(std::integral_constant<int, 0>{});
            two(std::integral_constant<int, 1>{});
            two(std::integral_constant<int, 2>{});
            two(std::integral_constant<int, 3>{});
            ok = store_unit();
          }
        } else {
          // Any other step pattern: outputs one at a time in slot order, each pair of values
          // written into the open unit as one 32-bit word per digit.
          const uint2* st = d.steps + col.table_row + kHeaderRows;
          const int32_t* sp = d.slot_ptr + col.slot_base;
          int kin = 0, off = 0;  // K position within the open unit, its byte offset
          double pending = 0.0;
          bool have = false;
          auto emit = [&](double z) {
            if (!have) {
              pending = z;
              have = true;
              return;
            }
            have = false;
            if (!ok) return;
            if (kin == 0) {
              off = open_unit();
              if (off < 0) {
                ok = false;
                return;
              }
            }
            uint32_t pw[NDIG];
            digit_pair<NDIG>(zero_row ? 0 : to_fixed_trunc(pending, shift), zero_row ? 0 : to_fixed_trunc(z, shift), pw);
#pragma unroll
            for (int t = 0; t < NDIG; ++t) *reinterpret_cast<uint32_t*>(sA + t * kASlice + off + kin * 2) = pw[t];
            kin += 2;
            if (kin == 8) {
              kin = 0;
              finish_unit();
            }
          };
          for (int N = 0; N < n_steps; ++N) {
            const double qv = step(N);
            const uint32_t info = st[N].x;
            uint32_t cnt = info & 0xffu, flags = info >> 8;
            if (cnt == 0) continue;
            if (cnt == kStepIrregular) {
              for (int sl = sp[N]; sl < sp[N + 1]; ++sl) emit(qv * (((uint32_t)__ldg(d.slot_idx + sl) >> 31) ? fsin : fcos));
            } else {
              for (; cnt > 0; --cnt, flags >>= 1) emit(qv * ((flags & 1u) ? fsin : fcos));
            }
          }
          if (have) emit(0.0);
          while (kin != 0) emit(0.0), emit(0.0);
        }
      }
      // Zero units up to the tile's unit count (the same for every stream, whole stages).
#pragma unroll
      for (int t = 0; t < NDIG; ++t) w[t][0] = w[t][1] = w[t][2] = w[t][3] = 0u;
      const int my_units = (d.units - strm + kStreams - 1) / kStreams;
      while (ok && unit < my_units) ok = store_unit();
      // Drain the previous tile's accumulator now that this one is on its way.
      if (ok && prev_inst >= 0) ok = drain_prev();
      if (!ok) {
        fail(abort_flag);
        break;
      }
      prev_inst = ii;
      prev_p0 = p0;
      prev_ep = ep;
    }
    if (ok && prev_inst >= 0 && !drain_prev()) fail(abort_flag);
    // Every coefficient copy this CTA issued has landed before the CTA may exit (a wait that
    // ignores the abort flag, still bounded).
    if (warp == 0 && lane == 0) {
      int never = 0;
      if (b_issued0 && !ptx::mbar_wait(&bar->bfull[0], (b_issued0 - 1u) & 1u, &never)) atomicOr(&g_fused_error, 1u);
      if (b_issued1 && !ptx::mbar_wait(&bar->bfull[1], (b_issued1 - 1u) & 1u, &never)) atomicOr(&g_fused_error, 1u);
    }
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(FM, K::AccCols);
      int stage = 0;
      uint32_t phase = 0;
      int64_t local = 0;
      for (int64_t it = blockIdx.x; it < a.n_items && !*abort_flag; it += gridDim.x, ++local) {
        int ii;
        int64_t p0;
        item_of(a, it, ii, p0);
        const int KC = inst_of(a, ii).KC;
        const uint32_t acc = (uint32_t)(local & 1), use = (uint32_t)((local >> 1) & 1);
        if (!ptx::mbar_wait_sleepy(&bar->tempty[acc], use ^ 1u, abort_flag, 200)) {
          fail(abort_flag);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * kAccStride;
        bool ok = true;
        for (int kc = 0; kc < KC; ++kc) {
          if (!ptx::mbar_wait_sleepy(&bar->full[stage], phase, abort_flag, 200) ||
              !ptx::mbar_wait(&bar->bfull[stage], phase, abort_flag)) {
            fail(abort_flag);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t sA = ptx::smem_u32(smem + stage * K::StageBytes);
          const uint32_t sB = sA + K::ABytes;
#pragma unroll
          for (int ks = 0; ks < FBK / 16; ++ks) {
#pragma unroll
            for (int t = 0; t < NDIG; ++t) {
              // A digit t+1 times the coefficient digits shifted down by t blocks: block
              // (t+1) + u - 2 of the accumulator (diagonal t+1+u) receives a_{t+1} b_u.
              const uint64_t adesc = ptx::sw_kmajor_desc<kRowBytes>(sA + t * kASlice + ks * 32);
              const uint64_t bdesc = ptx::sw_kmajor_desc<kRowBytes>(sB + (NDIG - 1 - t) * kBBlock + ks * 32);
              ptx::mma_bf16(d_tmem, adesc, bdesc, idesc, (kc == 0 && ks == 0 && t == 0) ? 0u : 1u);
            }
          }
          ptx::mma_commit(&bar->empty[stage]);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        ptx::mma_commit(&bar->tfull[acc]);
      }
      // Every MMA this thread issued has completed before TMEM is released (a wait that
      // ignores the abort flag, still bounded).
      ptx::mma_commit(&bar->drain);
      int never = 0;
      if (!ptx::mbar_wait(&bar->drain, 0u, &never)) atomicOr(&g_fused_error, 1u);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 2 * kAccStride);
  }
}

// The recursion weight W0_N of mode j (the plan's table): the fused kernel digitises Q_N trig and
// contracts it with W0_N C[j][s].
__device__ __forceinline__ double mode_weight(const FusedInst& d, int64_t j) {
  const Column col = d.cols[d.mode_col[j]];
  return d.table[((size_t)col.table_row + kHeaderRows + d.mode_N[j]) * kRow + 3];
}

// Set scale exponents: cexp[s] = e with 2^e > max_j |W0_N(j) C[j][s]| (kNonFiniteRow for a set
// holding an infinity or a NaN), one block per instance, sets past S get 0.
__global__ void __launch_bounds__(256) fused_cexp_kernel(FusedArgs a, int64_t n_inst) {
  __shared__ unsigned long long red[FNS][8];
  const int64_t inst = blockIdx.x;
  if (inst >= n_inst) return;
  const FusedInst& d = inst_of(a, (int)inst);
  unsigned long long mx[FNS];
#pragma unroll
  for (int s = 0; s < FNS; ++s) mx[s] = 0;
  for (int64_t j = threadIdx.x; j < d.J; j += blockDim.x) {
    const double wj = mode_weight(d, j);
#pragma unroll
    for (int s = 0; s < FNS; ++s) {
      if (s < d.S) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(wj * d.coeffs[j * d.S + s]) & 0x7fffffffffffffffull;
        mx[s] = b > mx[s] ? b : mx[s];
      }
    }
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int s = 0; s < FNS; ++s) {
    unsigned long long v = mx[s];
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (lane == 0) red[s][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < FNS) {
    unsigned long long v = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v = red[threadIdx.x][w] > v ? red[threadIdx.x][w] : v;
    d.cexp[threadIdx.x] = (int)threadIdx.x < d.S ? scale_exponent(v) : 0;
  }
}

// Coefficient digits in the fused layout's K order (the plan's slot order, each column padded to
// a multiple of 8 positions): thread = (chunk, set, group of 8 positions); the
// 8 values' NDIG digits are written as one 16-byte unit into each digit block's row for the set.
template <int NDIG>
__global__ void __launch_bounds__(256) fused_coeff_kernel(FusedArgs a, const int32_t* chunk_inst, int64_t n_chunks) {
  using K = FK<NDIG>;
  const int64_t total = n_chunks * FNS * (FBK / 8);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i / (FNS * (FBK / 8));
    const int s = (int)((i / (FBK / 8)) % FNS);
    const int q = (int)(i % (FBK / 8));
    const int inst = chunk_inst ? chunk_inst[g] : 0;
    const FusedInst& d = inst_of(a, inst);
    const int64_t kc = g - d.kc_base;
    const int ec = s < d.S ? d.cexp[s] : 0;
    const bool use = s < d.S && ec != kNonFiniteRow;
    long long X[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t k = kc * FBK + q * 8 + e;
      X[e] = 0;
      const int32_t slot = (use && k < d.Kp) ? __ldg(d.kperm + k) : -1;
      if (slot >= 0) {
        const int64_t j = (int64_t)((uint32_t)__ldg(d.slot_idx + slot) & 0x7fffffffu);
        X[e] = to_fixed(mode_weight(d, j) * d.coeffs[j * d.S + s], K::Beta * NDIG - ec);
      }
    }
    uint32_t w[NDIG][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t pw[NDIG];
      digit_pair<NDIG>(X[2 * e], X[2 * e + 1], pw);
#pragma unroll
      for (int t = 0; t < NDIG; ++t) w[t][e] = pw[t];
    }
    uint8_t* chunk = d.bdig + (size_t)kc * kFusedBChunk;
#pragma unroll
    for (int t = 0; t < NDIG; ++t)
      *reinterpret_cast<uint4*>(chunk + ptx::sw_offset_b16<kRowBytes>((uint32_t)(t * FNS + s), (uint32_t)(q * 8))) =
          make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
}

}  // namespace

int fused_ep_for(const zp_plan* plan, int vk) {
  int m_max = 0, n_max = 0;
  for (const Column& c : plan->cols) {
    m_max = std::max(m_max, c.m);
    n_max = std::max(n_max, c.m + 2 * (c.n_steps - 1));
  }
  const int64_t bound = vk == kFusedDTheta ? m_max : (vk == kFusedDRho ? (int64_t)n_max * n_max : 1);
  int extra = 0;
  while ((int64_t(1) << extra) < bound) ++extra;
  return plan->fused_ep + extra;
}

namespace {
template <int NDIG>
cudaError_t fused_set_smem() {
  constexpr int smem = (int)FK<NDIG>::Smem;
  cudaError_t e = cudaFuncSetAttribute(fused_emu_kernel<VK_Z, NDIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_emu_kernel<VK_DTHETA, NDIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_emu_kernel<VK_DRHO, NDIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

template <int NDIG>
void fused_launch_ndig(const FusedArgs& a, int64_t n_inst, const int32_t* chunk_inst, int64_t n_chunks, int sms,
                       cudaStream_t stream, int vk, bool coeff_digits) {
  constexpr uint32_t smem = FK<NDIG>::Smem;
  if (coeff_digits) {
    fused_cexp_kernel<<<(unsigned)n_inst, 256, 0, stream>>>(a, n_inst);
    const int64_t threads = n_chunks * FNS * (FBK / 8);
    fused_coeff_kernel<NDIG><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, 8 * (int64_t)sms)),
                               256, 0, stream>>>(a, chunk_inst, n_chunks);
  }
  const unsigned grid = (unsigned)std::min<int64_t>(a.n_items, sms);
  if (vk == kFusedDTheta) fused_emu_kernel<VK_DTHETA, NDIG><<<grid, kThreads, smem, stream>>>(a);
  else if (vk == kFusedDRho) fused_emu_kernel<VK_DRHO, NDIG><<<grid, kThreads, smem, stream>>>(a);
  else fused_emu_kernel<VK_Z, NDIG><<<grid, kThreads, smem, stream>>>(a);
}
}  // namespace

zp_status fused_launch(const FusedArgs& a, int64_t n_inst, const int32_t* chunk_inst, int64_t n_chunks,
                       cudaStream_t stream, int vk, bool coeff_digits) {
  if (a.n_items == 0) return ZP_OK;
  if (vk != kFusedZ && vk != kFusedDTheta && vk != kFusedDRho) return set_error(ZP_ERR_INVALID_ARG, "fused value kind");
  if (a.ndig != kFusedDigits && a.ndig != kFusedDigitsShort) return set_error(ZP_ERR_INVALID_ARG, "fused digit count");
  static DeviceMemo<int> sms_memo;
  int sms = 0;
  ZP_TRY(sms_memo.get(&sms, [](int* x) -> zp_status {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(x, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = fused_set_smem<kFusedDigits>();
    if (e == cudaSuccess) e = fused_set_smem<kFusedDigitsShort>();
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "fused kernel set-up");
  }));
  if (a.ndig == kFusedDigitsShort)
    fused_launch_ndig<kFusedDigitsShort>(a, n_inst, chunk_inst, n_chunks, sms, stream, vk, coeff_digits);
  else
    fused_launch_ndig<kFusedDigits>(a, n_inst, chunk_inst, n_chunks, sms, stream, vk, coeff_digits);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "fused series launch");
}

namespace {
// The single-instance descriptor of a plan's fused layout (value kind Z; no output set).
FusedInst single_inst(const zp_plan* plan, const double* r, const double* theta, int64_t P, const double* coeffs,
                      int64_t S) {
  FusedInst d;
  d.cols = plan->dev.cols;
  d.table = plan->dev.table;
  d.steps = plan->dev.split_step;
  d.slot_ptr = plan->dev.slot_ptr;
  d.slot_idx = plan->dev.slot_idx;
  d.mode_col = plan->dev.mode_col;
  d.mode_N = plan->dev.mode_N;
  d.fcols = plan->dev.fused_col;
  d.scols = (const int32_t*)(plan->dev.fused_col + plan->cols.size());
  for (int st = 0; st < kFusedStreams; ++st) d.ncols_s[st] = plan->fused_ncols[st];
  d.units = plan->fused_units;
  d.ep_disc = plan->fused_ep;
  d.kperm = plan->dev.fused_kperm;
  d.Kp = plan->fused_kpad;
  d.n_cols = (int32_t)plan->cols.size();
  d.KC = (int32_t)((plan->fused_kpad + FBK - 1) / FBK);
  d.kc_base = 0;
  d.J = plan->n_modes;
  d.P = P;
  d.S = S;
  d.r = r;
  d.theta = theta;
  d.coeffs = coeffs;
  return d;
}
}  // namespace

zp_status fused_series_eval(const zp_plan* plan, const double* r, const double* theta, int64_t P, const double* coeffs,
                            int64_t S, double* out, cudaStream_t stream) {
  if (S > kFusedMaxSets || plan->fused_kpad > kFusedMaxModes)
    return set_error(ZP_ERR_UNSUPPORTED, "fused series: at most 16 sets and 5041 padded modes");
  FusedArgs a;
  FusedInst& d = a.single;
  d = single_inst(plan, r, theta, P, coeffs, S);
  d.out = out;
  ScratchBuffer buf;
  const size_t bbytes = (size_t)d.KC * kFusedBChunk;
  ZP_TRY(buf.alloc(bbytes + 256, stream));
  d.bdig = (uint8_t*)buf.ptr;
  d.cexp = (int*)((uint8_t*)buf.ptr + bbytes);
  a.n_items = (P + FM - 1) / FM;
  a.ndig = fused_digits_for(plan->fused_kpad);
  return fused_launch(a, 1, nullptr, d.KC, stream);
}

zp_status fused_point_grads(const zp_plan* plan, const double* r, const double* theta, int64_t P, const double* coeffs,
                            int64_t S, const double* G, double* grad_r, double* grad_theta, cudaStream_t stream) {
  if (S > kFusedMaxSets || plan->fused_kpad > kFusedMaxModes)
    return set_error(ZP_ERR_UNSUPPORTED, "fused series: at most 16 sets and 5041 padded modes");
  if (P == 0 || (!grad_r && !grad_theta)) return ZP_OK;
  FusedArgs a;
  FusedInst& d = a.single;
  d = single_inst(plan, r, theta, P, coeffs, S);
  d.gdot = G;
  ScratchBuffer buf;
  const size_t bbytes = (size_t)d.KC * kFusedBChunk;
  ZP_TRY(buf.alloc(bbytes + 256, stream));
  d.bdig = (uint8_t*)buf.ptr;
  d.cexp = (int*)((uint8_t*)buf.ptr + bbytes);
  a.n_items = (P + FM - 1) / FM;
  a.ndig = fused_digits_for(plan->fused_kpad);
  bool digits = true;  // the coefficient digits once, for the first pass
  for (int k = 0; k < 2; ++k) {
    double* g = k == 0 ? grad_theta : grad_r;
    if (!g) continue;
    const cudaError_t e = cudaMemsetAsync(g, 0, (size_t)P * sizeof(double), stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    const int vk = k == 0 ? kFusedDTheta : kFusedDRho;
    d.dot_out = g;
    d.ep_disc = fused_ep_for(plan, vk);
    ZP_TRY(fused_launch(a, 1, nullptr, d.KC, stream, vk, digits));
    digits = false;
  }
  return ZP_OK;
}

zp_status fused_error_word(unsigned int* value, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_fused_error, sizeof(unsigned int));
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyFromSymbol");
  if (reset) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_fused_error, &zero, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyToSymbol");
  }
  return ZP_OK;
}

}  // namespace zp
