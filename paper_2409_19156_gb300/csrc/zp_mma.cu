// Split-precision Zernike series on the fifth-generation tensor cores (tcgen05 + TMEM).
//
//   F[p, s] = sum_j Z_j(p) C[j, s],   Z from the float64 per-column recursion (zp_walk.cu),
// contracted as BF16x3 (Z = Zh + Zl, C = Ch + Cl in bfloat16, F ~ Zh Ch + Zh Cl + Zl Ch with
// float32 accumulation) or TF32 (one product of TF32-rounded operands).
//
// Two kernels per slab of point tiles, back to back on the caller's stream:
//  (A) split_basis_kernel: one thread per point walks every |m| column (the recursion of
//      Sec. 2 in float64, Algorithm 1's order), rotates cos/sin(m theta) by angle addition
//      from column to column, splits each Z into bfloat16 hi/lo (or TF32), packs 8 (4)
//      consecutive K values in registers and writes each 16-byte unit straight to its place
//      in the tensor core's swizzled K-major layout in a scratch buffer.
//      The K order of the contraction is the plan's slot order (column by column), so a
//      thread's outputs are consecutive in K; the coefficient rows are permuted to match.
//  (B) split_gemm_kernel: persistent, warp-specialised tcgen05 GEMM on CTA pairs (clusters
//      of two): in each CTA warp 0 streams its 128 points' A chunks and half of each B (sets x
//      K) chunk into its own shared-memory ring with bulk copies and mbarrier transaction
//      counts; warp 1 of the even CTA issues tcgen05.mma.cta_group::2 (M = 256 points across
//      the pair, N = 256 sets, K = 16 per instruction) into one of two TMEM accumulators in
//      each CTA; warps 2-5 of each CTA drain its other accumulator (tcgen05.ld) to float32
//      rows of F while the next tile accumulates; warp 6 passes barrier signals between the
//      pair.  A single-CTA form (M = 128) runs when pairs cannot.
// The coefficients are split/permuted once per call by split_coeff_kernel.  The same GEMM with
// integer-valued bfloat16 slices is the float64-emulating contraction (KIND_SLICE, below).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <utility>
#include <vector>

#include "zp_device.cuh"
#include "zp_api_common.h"
#include "zp_ptx.cuh"
#include "zp_emu_device.cuh"
#include "zp_emu_shape.h"
#include "zp_fused.h"
#include "zp_series_internal.h"

namespace zp {
namespace {

constexpr int BM = 128;  // points per tile (TMEM lanes)
constexpr int BN = 256;  // coefficient sets per tile (TMEM columns per accumulator)
constexpr uint32_t kRingBytes = 192u << 10;  // shared-memory ring of operand stages
constexpr int kCoeffThreads = BN;

// Operand kinds of the GEMM: BF16x3 (hi/lo halves, three products), TF32 (one product),
// SLICE (one bf16 product of integer-valued slices, for the emulated-float64 contraction).
constexpr int KIND_BF16X3 = 0, KIND_TF32 = 1, KIND_SLICE = 2;

// Operand rows: BF16x3 keeps 64-byte rows in the 64-byte swizzle layout (a K chunk of 32
// values; hi + lo stages of 48 KB, 4 in the ring: with 128-byte rows and 2 stages of 96 KB the
// bulk copies' latency was exposed to the MMA issue, 8.6 against 8.2 ms at mixed_n32).  TF32
// and the slice products keep 128-byte rows (48 KB stages, 4 in the ring): with 64-byte rows
// a stage holds only two MMAs and the per-stage barrier work dominated (TF32 7.3 -> 8.9 ms).
template <int KIND>
struct Cfg {
  static constexpr uint32_t ROW = KIND == KIND_BF16X3 ? 64u : 128u;  // bytes per operand row
  static constexpr int BK = (int)ROW / (KIND == KIND_TF32 ? 4 : 2);  // K elements per row
  static constexpr int PARTS = KIND == KIND_BF16X3 ? 2 : 1;          // hi (+ lo)
  static constexpr uint32_t A_PART = BM * ROW;                       // one 128-row K chunk
  static constexpr uint32_t B_PART = BN * ROW;
  static constexpr uint32_t A_CHUNK = A_PART * PARTS;
  static constexpr uint32_t B_CHUNK = B_PART * PARTS;
  static constexpr int KSTEPS = (int)ROW / 32;  // MMA K-steps per chunk (16 bf16 or 8 tf32 = 32 bytes each)
};

__device__ unsigned int g_split_error = 0;  // set when a bounded wait gives up

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float of a float64 by truncating its significand (integer pipe: the float64 pipe is the
// scarce one).  Relative error below 2^-23; magnitudes under the float normal range give a
// signed zero, finite ones above it infinity; infinities and NaNs are kept.  The split
// operands carry 16 (BF16x3) or 11 (TF32) significant bits, so truncation is harmless.
__device__ __forceinline__ float float_of_double(double x) {
  return __uint_as_float(trunc_float_bits((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x)));
}

// Two floats rounded to bfloat16 (nearest even) in one 32-bit word, `lo` in the low half.
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

struct BasisArgs {
  const Column* cols;
  int n_cols;
  const double* table;
  const uint2* steps;  // per table row: slot count and sin flags, float32 weight
  const int32_t* slot_ptr;
  const int32_t* slot_idx;
  const double* r;
  const double* theta;
  int64_t P;
  int64_t mt_base;  // first point tile of this slab
  int KC;           // K chunks
  uint8_t* A;       // slab scratch: [tiles][KC][A_CHUNK]
};

// Register packing of consecutive K values into one 16-byte unit of the swizzled layout:
// each push shifts the 128-bit chain w[3]:w[2]:w[1]:w[0] right by one element (two for
// push32) and inserts the new element(s) at the top, so after a full unit w[0] holds the
// first element.
struct Pack16 {
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  __device__ __forceinline__ void push16(uint32_t v) {
    w[0] = __funnelshift_r(w[0], w[1], 16);
    w[1] = __funnelshift_r(w[1], w[2], 16);
    w[2] = __funnelshift_r(w[2], w[3], 16);
    w[3] = __funnelshift_r(w[3], v, 16);
  }
  __device__ __forceinline__ void push32(uint32_t v) {
    w[0] = w[1];
    w[1] = w[2];
    w[2] = w[3];
    w[3] = v;
  }
  __device__ __forceinline__ void store(uint8_t* dst) const {
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
};

// No shared memory or barriers: each thread owns two rows of the 128-point tile (rows t and
// t + 64), packs 8 bf16 (or 4 tf32) consecutive K values of each row in registers and writes
// every 16-byte unit straight to its place in the swizzled chunk (measured faster than
// staging whole chunks in shared memory for bulk stores).  With two points per thread (TF32)
// the table and slot loads are shared and the float64 pipe gets two independent recursions;
// BF16x3 keeps one point per thread (measured faster: its hi/lo split and packing add
// integer work per value that the second point does not amortise).
template <bool TF32>
__host__ __device__ constexpr int basis_ppt() {
  return TF32 ? 2 : 1;
}
template <bool TF32>
__host__ __device__ constexpr int basis_threads() {
  return BM / basis_ppt<TF32>();
}

template <bool TF32>
__device__ __forceinline__ void split_basis_tile(const BasisArgs& a, int64_t tile);

// One CTA per point tile of the slab (grid-stride if the grid is smaller).
template <bool TF32>
__global__ void __launch_bounds__(basis_threads<TF32>()) split_basis_kernel(BasisArgs a, int64_t tiles) {
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) split_basis_tile<TF32>(a, tile);
}

template <bool TF32>
__device__ __forceinline__ void split_basis_tile(const BasisArgs& a, int64_t tile) {
  using C = Cfg<TF32 ? KIND_TF32 : KIND_BF16X3>;
  constexpr int UNIT = TF32 ? 4 : 8;  // K values per 16-byte unit
  constexpr int Q = basis_ppt<TF32>();
  uint32_t rowi[Q];
  double rho[Q], u[Q], s1[Q], c1[Q], cm[Q], sm[Q], pm[Q], T[Q], S[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rowi[i] = threadIdx.x + (uint32_t)i * basis_threads<TF32>();
    const int64_t p = (a.mt_base + tile) * BM + rowi[i];
    const bool valid = p < a.P;
    rho[i] = valid ? a.r[p] : 0.0;
    const double th = valid ? a.theta[p] : 0.0;
    u[i] = rho[i] * rho[i];
    sincos(th, &s1[i], &c1[i]);
    cm[i] = 1.0;
    sm[i] = 0.0;
    pm[i] = 1.0;
  }
  int m_prev = 0;
  uint8_t* gA = a.A + (size_t)tile * a.KC * C::A_CHUNK;
  int k = 0;
  Pack16 hi[Q], lo[Q];

  // Writes the unit that value k - 1 completed.
  auto flush = [&]() {
    const int k0 = k - UNIT;
    uint8_t* chunk = gA + (size_t)(k0 / C::BK) * C::A_CHUNK;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if constexpr (TF32) {
        hi[i].store(chunk + ptx::sw_offset_b32<C::ROW>(rowi[i], (uint32_t)(k0 % C::BK)));
      } else {
        const uint32_t off = ptx::sw_offset_b16<C::ROW>(rowi[i], (uint32_t)(k0 % C::BK));
        hi[i].store(chunk + off);
        lo[i].store(chunk + C::A_PART + off);
      }
    }
  };
  // One value at K position k.
  auto push1 = [&](const float (&z)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if constexpr (TF32) {
        hi[i].push32(__float_as_uint(to_tf32(z[i])));
      } else {
        const uint32_t h = bf16x2_bits(z[i], 0.0f) & 0xffffu;
        const uint32_t l = bf16x2_bits(z[i] - __uint_as_float(h << 16), 0.0f) & 0xffffu;
        hi[i].push16(h);
        lo[i].push16(l);
      }
    }
    if (++k % UNIT == 0) flush();
  };
  // BF16x3: two values at K positions k and k + 1, converted in pairs (the same roundings
  // as two single pushes).
  auto push2 = [&](const float (&z0)[Q], const float (&z1)[Q]) {
    uint32_t h2[Q], l2[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      h2[i] = bf16x2_bits(z0[i], z1[i]);
      l2[i] = bf16x2_bits(z0[i] - __uint_as_float(h2[i] << 16), z1[i] - __uint_as_float(h2[i] & 0xffff0000u));
    }
    if ((k & (UNIT - 1)) == UNIT - 1) {  // the first value completes a unit
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        hi[i].push16(h2[i] & 0xffffu);
        lo[i].push16(l2[i] & 0xffffu);
      }
      ++k;
      flush();
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        hi[i].push16(h2[i] >> 16);
        lo[i].push16(l2[i] >> 16);
      }
      ++k;
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        hi[i].push32(h2[i]);
        lo[i].push32(l2[i]);
      }
      k += 2;
      if ((k & (UNIT - 1)) == 0) flush();
    }
  };

  for (int c = 0; c < a.n_cols; ++c) {
    const Column col = a.cols[c];
    const int m = col.m;
    const double* h = a.table + (size_t)col.table_row * kRow;
    float cf[Q], sf[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (m == m_prev + 1) {
        const double cn = fma(cm[i], c1[i], -sm[i] * s1[i]);
        const double sn = fma(sm[i], c1[i], cm[i] * s1[i]);
        cm[i] = cn;
        sm[i] = sn;
        pm[i] *= rho[i];
      } else if (m != m_prev) {
        const int64_t p = (a.mt_base + tile) * BM + rowi[i];
        const double th = p < a.P ? a.theta[p] : 0.0;
        sincos((double)m * th, &sm[i], &cm[i]);
        pm[i] = pow_uint(rho[i], m);
      }
      cf[i] = float_of_double(cm[i]);
      sf[i] = float_of_double(sm[i]);
      T[i] = pm[i];
      S[i] = pm[i] * fma(h[4], u[i], -h[8]);  // R_{m+2}^m = rho^m ((m+2) rho^2 - (m+1))
    }
    m_prev = m;
    const uint2* st = a.steps + col.table_row + kHeaderRows;
    const int32_t* sp = a.slot_ptr + col.slot_base;
    // Outputs of step N: value qv times the weight, times cos or sin per slot.  Per value
    // the float64 pipe sees only the two recursion FMAs; the weight and the angular factor
    // are applied in float32 (converted on the integer pipe).
    auto emit = [&](const double (&qv)[Q], uint2 info, int N) {
      float Rf[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) Rf[i] = float_of_double(qv[i]) * __uint_as_float(info.y);
      uint32_t cnt = info.x & 0xffu, flags = info.x >> 8;
      if (cnt == kStepIrregular) {
        for (int s = sp[N]; s < sp[N + 1]; ++s) {
          const uint32_t code = (uint32_t)__ldg(a.slot_idx + s);
          float z[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) z[i] = Rf[i] * ((code >> 31) ? sf[i] : cf[i]);
          push1(z);
        }
        return;
      }
      if constexpr (!TF32) {
        for (; cnt >= 2; cnt -= 2, flags >>= 2) {
          float z0[Q], z1[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            z0[i] = Rf[i] * ((flags & 1u) ? sf[i] : cf[i]);
            z1[i] = Rf[i] * ((flags & 2u) ? sf[i] : cf[i]);
          }
          push2(z0, z1);
        }
      }
      for (; cnt > 0; --cnt, flags >>= 1) {
        float z[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) z[i] = Rf[i] * ((flags & 1u) ? sf[i] : cf[i]);
        push1(z);
      }
    };
    // Step N's recursion value is formed before step N - 1's outputs are emitted, so the
    // float64 latency of the recursion overlaps the conversions, products and packing.
    double qp[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) qp[i] = T[i];
    uint2 ip = st[0];
    if (col.n_steps > 1) {
      const uint2 in = st[1];
      emit(qp, ip, 0);
#pragma unroll
      for (int i = 0; i < Q; ++i) qp[i] = S[i];
      ip = in;
      for (int N = 2; N < col.n_steps; ++N) {
        const double2 AB = *reinterpret_cast<const double2*>(h + (size_t)(kHeaderRows + N) * kRow);
        const uint2 inN = st[N];
        double q[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const double g = fma(AB.x, u[i], -AB.y);
          q[i] = fma(g, S[i], -T[i]);
          T[i] = S[i];
          S[i] = q[i];
        }
        emit(qp, ip, N - 1);
#pragma unroll
        for (int i = 0; i < Q; ++i) qp[i] = q[i];
        ip = inN;
      }
    }
    emit(qp, ip, col.n_steps - 1);
  }
  const float zeros[Q] = {};
  while (k % C::BK != 0) push1(zeros);
}

struct CoeffArgs {
  const double* coeffs;  // [J][S]
  const int32_t* slot_idx;
  int64_t J, S;
  int KC;
  uint8_t* B;  // [NT][KC][B_CHUNK]
};

template <bool TF32>
__global__ void __launch_bounds__(kCoeffThreads) split_coeff_kernel(CoeffArgs a) {
  using C = Cfg<TF32 ? KIND_TF32 : KIND_BF16X3>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const int nt = blockIdx.x / a.KC, kc = blockIdx.x % a.KC;
  const uint32_t t = threadIdx.x;
  const int64_t s = (int64_t)nt * BN + t;
  for (int kk = 0; kk < C::BK; ++kk) {
    const int64_t kg = (int64_t)kc * C::BK + kk;
    double v = 0.0;
    if (kg < a.J && s < a.S) {
      const int64_t j = (int64_t)((uint32_t)__ldg(a.slot_idx + kg) & 0x7fffffffu);
      v = a.coeffs[j * a.S + s];
    }
    const float f = (float)v;
    if constexpr (TF32) {
      *reinterpret_cast<float*>(smem + ptx::sw_offset_b32<C::ROW>(t, kk)) = to_tf32(f);
    } else {
      const __nv_bfloat16 hi = __float2bfloat16_rn(f);
      const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
      const uint32_t off = ptx::sw_offset_b16<C::ROW>(t, kk);
      *reinterpret_cast<__nv_bfloat16*>(smem + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(smem + C::B_PART + off) = lo;
    }
  }
  __syncthreads();
  uint4* dst = reinterpret_cast<uint4*>(a.B + ((size_t)nt * a.KC + kc) * C::B_CHUNK);
  const uint4* src = reinterpret_cast<const uint4*>(smem);
  for (uint32_t i = t; i < C::B_CHUNK / 16; i += kCoeffThreads) dst[i] = src[i];
}

struct GemmArgs {
  const uint8_t* A;  // slab: [tiles][KC][A_CHUNK] (slice 0 for KIND_SLICE)
  const uint8_t* B;  // [NT][KC][B_CHUNK] (slice 0 for KIND_SLICE)
  float* F;          // [P][S] (KIND_SLICE: int32 values)
  int64_t P, S;
  int64_t mt_base;
  int64_t m_tiles;  // tiles in this slab
  int n_tiles;      // NT
  int KC;
  // KIND_SLICE: the tile's K runs over npairs slice pairs (t, u) with t + u = npairs - 1
  // (0-based), KC chunks each; A slice t starts a_slice_stride bytes after slice t-1, B likewise.
  int npairs = 1;
  int64_t a_slice_stride = 0;
  int64_t b_slice_stride = 0;
  // KIND_SLICE split over K: k batch kb covers K chunks [kb * kc_per_batch, min(KC, ...)) and
  // writes its sums t_batch_stride elements after batch kb - 1 (kc_per_batch 0: one batch).
  int k_batches = 1;
  int kc_per_batch = 0;
  int64_t t_batch_stride = 0;
  // KIND_SLICE with paired diagonals (npairs unused): the tile is 128 points x 128 sets and
  // covers the diagonals dp and dp + 1 (0-based; dp = -1 leaves only diagonal 0).  B holds per
  // (set tile, K chunk) all s_slices slices of 128 rows back to back (128 rows x 128 bytes each),
  // so that one N = 256 MMA of A slice t against slices (dp - t, dp + 1 - t) adds into both
  // diagonals' accumulators (TMEM columns 0-127 and 128-255); A slice dp + 1 meets only B slice
  // 0 (an N = 128 MMA into columns 128-255).  The epilogue stores T_dp 2^beta + T_(dp+1) as one
  // int32 (the host checks that it cannot overflow).
  int paired = 0;
  int dp = 0;
  int beta = 0;
  int s_slices = 0;
  int nb = 128;  // paired: sets per tile = rows of a slice block (a multiple of 16; below 128 single CTAs only)
};

// Threads of the GEMM kernel: producer, MMA and 4 epilogue warps, plus, for a CTA pair, one
// warp whose thread passes barrier signals between the pair's two CTAs.
template <int CG>
constexpr int gemm_threads() {
  return CG == 2 ? 224 : 192;
}

// One CTA's shared-memory stage: its A chunk and its share of the B chunk's rows (all of them
// for a single CTA, half for each CTA of a pair).
template <int KIND, int CG>
struct Stage {
  using C = Cfg<KIND>;
  static constexpr uint32_t B_PART = (uint32_t)(BN / CG) * C::ROW;
  static constexpr uint32_t B_CHUNK = B_PART * C::PARTS;
  static constexpr uint32_t BYTES = C::A_CHUNK + B_CHUNK;
  static constexpr int COUNT = (int)(kRingBytes / BYTES);
  static constexpr uint32_t SMEM = COUNT * BYTES + 1024 /*align*/ + 256 /*barriers*/;
};

// Persistent GEMM over output tiles; every operand chunk comes from global memory into the
// CTA's own shared memory by a plain bulk copy.  CG = 1: one CTA per 128-point tile.  CG = 2:
// a cluster of two CTAs per 256-point tile, multiplied by cta_group::2 MMAs that the even CTA
// issues: each CTA loads its own 128 points' A chunk and half of the B chunk's rows, the MMA
// reads both CTAs' halves, and each CTA's tensor memory receives its own points' accumulators,
// so a B chunk crosses L2 once per pair instead of once per CTA.  The pair's signals are remote
// mbarrier arrives: the odd CTA's relay thread reports its landed chunks to the even CTA, the
// even CTA's forwarder thread passes the MMA completions (stage free, accumulator ready) to the
// odd one, and the odd CTA's epilogue warps report drained accumulators to the even one.
template <int KIND, int CG>
__global__ void __launch_bounds__(gemm_threads<CG>(), 1) split_gemm_kernel(GemmArgs a) {
  using C = Cfg<KIND>;
  using S = Stage<KIND, CG>;
  constexpr bool TF32 = KIND == KIND_TF32;
  constexpr bool PAIR = CG == 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::COUNT * S::BYTES);
  uint64_t* empty = full + S::COUNT;
  uint64_t* tmem_full = empty + S::COUNT;
  uint64_t* tmem_empty = tmem_full + 2;
  uint64_t* drain = tmem_empty + 2;
  uint32_t* tmem_base_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_base_slot + 1);
  volatile int* never = abort_flag + 1;  // stays 0: waits that must not be cut short by an abort

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = PAIR ? ptx::cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int64_t cid = blockIdx.x / CG, nclusters = gridDim.x / CG;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S::COUNT; ++i) {
      // The pair's even CTA also counts the relay's arrive for the odd CTA's half.
      ptx::mbar_init(&full[i], PAIR && leader ? 2 : 1);
      ptx::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&tmem_full[i], 1);
      ptx::mbar_init(&tmem_empty[i], 4 * CG);  // one arrive per epilogue warp of each CTA
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    *never = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      ptx::tmem_alloc_pair(tmem_base_slot, 512);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(tmem_base_slot, 512);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  if constexpr (PAIR) {
    ptx::cluster_sync();  // both CTAs' barriers exist before any remote arrive
  } else {
    __syncthreads();
  }
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_base_slot;

  // Tile t: k batch t / per_batch, then group of CG point tiles and set tile, set tile fastest.
  const int64_t groups_n = a.n_tiles;
  const int64_t groups_m = (a.m_tiles + CG - 1) / CG;
  const int64_t per_batch = groups_m * groups_n;
  const int64_t total = per_batch * a.k_batches;
  const int kcb = a.kc_per_batch > 0 ? a.kc_per_batch : a.KC;
  // K chunks [kc0, kc0 + nkc) of tile t.
  auto k_range = [&](int64_t t, int& kc0, int& nkc) {
    const int kb = (int)(t / per_batch);
    kc0 = kb * kcb;
    nkc = (kc0 + kcb < a.KC ? kc0 + kcb : a.KC) - kc0;
  };
  // Operand chunks of tile t: per slice pair (or per A slice with paired diagonals) nkc chunks.
  auto n_items = [&](int nkc) { return (KIND == KIND_SLICE && a.paired ? a.dp + 2 : a.npairs) * nkc; };
  // This CTA's point tile of tile t, slab-local (past the slab's last tile for the odd CTA of a
  // half-filled last group: that CTA loads the last tile instead and stores nothing).
  auto own_mtile = [&](int64_t t) { return ((t % per_batch) / groups_n) * CG + (int64_t)rank; };
  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(&g_split_error, 1u);
  };

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t t = cid; t < total && !*abort_flag; t += nclusters) {
        const int64_t mt_own = own_mtile(t);
        const int64_t mt = mt_own < a.m_tiles ? mt_own : a.m_tiles - 1;
        const int nt = (int)((t % per_batch) % groups_n);
        int kc0, nkc;
        k_range(t, kc0, nkc);
        const uint8_t* gA0 = a.A + (size_t)mt * a.KC * C::A_CHUNK;
        const uint8_t* gB0 = a.B + (size_t)nt * a.KC * C::B_CHUNK;
        const int items = n_items(nkc);
        for (int kk = 0; kk < items; ++kk) {
          if (!ptx::mbar_wait<PAIR>(&empty[stage], phase ^ 1u, abort_flag)) {
            fail();
            break;
          }
          const int ts = kk / nkc, kc = kc0 + kk % nkc;  // A slice ts
          const uint8_t* gA = gA0 + (size_t)ts * a.a_slice_stride + (size_t)kc * C::A_CHUNK;
          uint8_t* sA = smem + stage * S::BYTES;
          uint8_t* sB = sA + C::A_CHUNK;
          if (KIND == KIND_SLICE && a.paired) {
            // B slices (dp - ts, dp + 1 - ts), or slice 0 alone for ts = dp + 1 (an N = 128
            // MMA); a pair's CTAs hold one slice each, or one half of slice 0's rows each.
            const bool both = ts <= a.dp;
            const uint32_t blk_bytes = (uint32_t)a.nb * C::ROW;
            const uint8_t* blk = a.B + (((size_t)nt * a.KC + kc) * a.s_slices + (both ? a.dp - ts : 0)) * blk_bytes;
            const uint32_t b_bytes = (both ? 2 * blk_bytes : blk_bytes) / CG;
            ptx::mbar_arrive_expect_tx(&full[stage], C::A_CHUNK + b_bytes);
            ptx::bulk_g2s(sA, gA, C::A_CHUNK, &full[stage]);
            ptx::bulk_g2s(sB, blk + rank * b_bytes, b_bytes, &full[stage]);
          } else {
            // Rows [rank BN / CG, (rank + 1) BN / CG) of each part of the chunk.
            const uint8_t* gc = gB0 + (size_t)(a.npairs - 1 - ts) * a.b_slice_stride + (size_t)kc * C::B_CHUNK;
            ptx::mbar_arrive_expect_tx(&full[stage], S::BYTES);
            ptx::bulk_g2s(sA, gA, C::A_CHUNK, &full[stage]);
            if constexpr (C::PARTS == 1 || !PAIR) {
              ptx::bulk_g2s(sB, gc + rank * S::B_PART, S::B_CHUNK, &full[stage]);
            } else {
#pragma unroll
              for (int part = 0; part < C::PARTS; ++part)
                ptx::bulk_g2s(sB + part * S::B_PART, gc + part * C::B_PART + rank * S::B_PART, S::B_PART,
                              &full[stage]);
            }
          }
          if (++stage == S::COUNT) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      constexpr uint32_t idesc = TF32 ? ptx::idesc_tf32_f32(BM * CG, BN) : ptx::idesc_bf16_f32(BM * CG, BN);
      // Paired slice tiles: N = 2 nb (both diagonals) or nb (the second alone).
      const uint32_t idesc_pair = ptx::idesc_bf16_f32(BM * CG, KIND == KIND_SLICE && a.paired ? 2 * a.nb : BN);
      const uint32_t idesc_half = ptx::idesc_bf16_f32(BM * CG, KIND == KIND_SLICE && a.paired ? a.nb : BN / 2);
      auto mma = [&](uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
        if constexpr (TF32) {
          if constexpr (PAIR) ptx::mma_tf32_pair(d, ad, bd, id, acc);
          else ptx::mma_tf32(d, ad, bd, id, acc);
        } else {
          if constexpr (PAIR) ptx::mma_bf16_pair(d, ad, bd, id, acc);
          else ptx::mma_bf16(d, ad, bd, id, acc);
        }
      };
      auto commit = [&](uint64_t* bar) {
        if constexpr (PAIR) ptx::mma_commit_pair(bar);
        else ptx::mma_commit(bar);
      };
      int stage = 0;
      uint32_t phase = 0;
      int64_t local = 0;
      for (int64_t t = cid; t < total && !*abort_flag; t += nclusters, ++local) {
        const uint32_t acc = (uint32_t)(local & 1);
        const uint32_t acc_phase = (uint32_t)((local >> 1) & 1);
        if (!ptx::mbar_wait<PAIR>(&tmem_empty[acc], acc_phase ^ 1u, abort_flag)) {
          fail();
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        int kc0, nkc;
        k_range(t, kc0, nkc);
        bool ok = true;
        const int items = n_items(nkc);
        for (int kk = 0; kk < items; ++kk) {
          if (!ptx::mbar_wait<PAIR>(&full[stage], phase, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t sA = ptx::smem_u32(smem + stage * S::BYTES);
          const uint32_t sB = sA + C::A_CHUNK;
          // Paired slice tiles: A slice dp + 1 meets B slice 0 only (diagonal dp + 1, N = 128).
          const bool half = KIND == KIND_SLICE && a.paired && kk / nkc > a.dp;
#pragma unroll
          for (int ks = 0; ks < C::KSTEPS; ++ks) {
            const uint32_t koff = ks * 32;
            const uint32_t first = (kk == 0 && ks == 0) ? 0u : 1u;
            if constexpr (KIND == KIND_BF16X3) {
              const uint64_t ah = ptx::sw_kmajor_desc<C::ROW>(sA + koff);
              const uint64_t al = ptx::sw_kmajor_desc<C::ROW>(sA + C::A_PART + koff);
              const uint64_t bh = ptx::sw_kmajor_desc<C::ROW>(sB + koff);
              const uint64_t bl = ptx::sw_kmajor_desc<C::ROW>(sB + S::B_PART + koff);
              mma(d_tmem, ah, bh, idesc, first);
              mma(d_tmem, ah, bl, idesc, 1u);
              mma(d_tmem, al, bh, idesc, 1u);
            } else {
              mma(half ? d_tmem + (uint32_t)a.nb : d_tmem, ptx::sw_kmajor_desc<C::ROW>(sA + koff),
                  ptx::sw_kmajor_desc<C::ROW>(sB + koff),
                  half ? idesc_half : (KIND == KIND_SLICE && a.paired ? idesc_pair : idesc), first);
            }
          }
          commit(&empty[stage]);
          if (++stage == S::COUNT) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        commit(&tmem_full[acc]);
      }
      // Every MMA issued here completes before the CTA (and a pair's peer, whose shared and
      // tensor memory those MMAs use) moves on to leave.
      commit(drain);
      if (!ptx::mbar_wait(drain, 0u, never)) atomicOr(&g_split_error, 1u);
    }
  } else if (PAIR && warp == 6) {
    // Pair signals, in the same order as the MMA thread's waits and commits.  Even CTA: each
    // stage the MMAs freed and each accumulator they filled is passed to the odd CTA.  Odd CTA:
    // each of its landed chunks is reported to the even CTA's full barrier.
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t local = 0;
      for (int64_t t = cid; t < total && !*abort_flag; t += nclusters, ++local) {
        int kc0, nkc;
        k_range(t, kc0, nkc);
        const int items = n_items(nkc);
        bool ok = true;
        for (int kk = 0; kk < items; ++kk) {
          uint64_t* bar = leader ? &empty[stage] : &full[stage];
          if (!ptx::mbar_wait(bar, phase, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          ptx::mbar_arrive_remote(ptx::mapa_shared(bar, leader ? 1u : 0u));
          if (++stage == S::COUNT) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (leader) {
          const uint32_t acc = (uint32_t)(local & 1);
          if (!ptx::mbar_wait(&tmem_full[acc], (uint32_t)((local >> 1) & 1), abort_flag)) {
            fail();
            break;
          }
          ptx::mbar_arrive_remote(ptx::mapa_shared(&tmem_full[acc], 1u));
        }
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    // Epilogue: warp & 3 selects the TMEM lane quadrant it may access.
    const uint32_t q = (uint32_t)(warp & 3);
    const uint32_t row = q * 32 + lane;
    const uint32_t empty_remote = PAIR && !leader ? ptx::mapa_shared(&tmem_empty[0], 0u) : 0u;
    int64_t local = 0;
    for (int64_t t = cid; t < total; t += nclusters, ++local) {
      const uint32_t acc = (uint32_t)(local & 1);
      const uint32_t acc_phase = (uint32_t)((local >> 1) & 1);
      // One lane per warp polls the barrier; the shuffle hands its answer to the warp.
      bool ok = true;
      if (lane == 0) ok = ptx::mbar_wait<PAIR>(&tmem_full[acc], acc_phase, abort_flag);
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
        fail();
        break;
      }
      ptx::tc_fence_after();
      const int64_t mt_own = own_mtile(t);
      const int nt = (int)((t % per_batch) % groups_n);
      const int64_t p = (a.mt_base + mt_own) * BM + row;
      const bool store = mt_own < a.m_tiles && p < a.P;
      const bool paired = KIND == KIND_SLICE && a.paired;
      const int tile_cols = paired ? a.nb : BN;
      const int64_t col0 = (int64_t)nt * tile_cols;
      float* frow = a.F + (t / per_batch) * a.t_batch_stride + p * a.S;
      const bool vec = (a.S % 4) == 0;
      const uint32_t tacc = tmem_base + ((q * 32u) << 16) + acc * BN;
#pragma unroll 1
      for (int c0 = 0; c0 < tile_cols; c0 += 32) {
        uint32_t v[32];
        if (paired) {
          // T_(dp+1) in columns nb .. 2 nb - 1, T_dp (none for dp = -1) in columns 0 .. nb - 1
          // (a narrow tile reads past them into columns it does not store).
          ptx::tmem_ld_32x32b_x32(tacc + (uint32_t)a.nb + (uint32_t)c0, v);
          ptx::tmem_ld_wait(v);
          if (a.dp >= 0) {
            uint32_t h[32];
            ptx::tmem_ld_32x32b_x32(tacc + (uint32_t)c0, h);
            ptx::tmem_ld_wait(h);
            const int scale = 1 << a.beta;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              v[i] = (uint32_t)(__float2int_rn(__uint_as_float(h[i])) * scale + __float2int_rn(__uint_as_float(v[i])));
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = (uint32_t)__float2int_rn(__uint_as_float(v[i]));
          }
        } else {
          ptx::tmem_ld_32x32b_x32(tacc + (uint32_t)c0, v);
          ptx::tmem_ld_wait(v);
          if constexpr (KIND == KIND_SLICE) {
            // Slice products sum to integers below 2^24 (exact in float32): store them as int32.
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = (uint32_t)__float2int_rn(__uint_as_float(v[i]));
          }
        }
        if (store) {
          const int64_t cbase = col0 + c0;
          const int64_t cend = a.S < col0 + tile_cols ? a.S : col0 + tile_cols;  // this tile's columns only
          if (vec && cbase + 32 <= cend) {
            float4* dst = reinterpret_cast<float4*>(frow + cbase);
#pragma unroll
            for (int i = 0; i < 8; ++i)
              __stcs(dst + i, make_float4(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]),
                                          __uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3])));
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (cbase + i < cend) frow[cbase + i] = __uint_as_float(v[i]);
          }
        }
      }
      // The warp's loads of this accumulator are done: one arrive per warp (remote for the odd
      // CTA of a pair, whose accumulators the even CTA's MMAs fill).
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR && !leader) ptx::mbar_arrive_remote(empty_remote + acc * (uint32_t)sizeof(uint64_t));
        else ptx::mbar_arrive(&tmem_empty[acc]);
      }
    }
  }
  ptx::tc_fence_before();
  if constexpr (PAIR) {
    ptx::cluster_sync();  // no CTA of a pair leaves while its peer may still signal it
  } else {
    __syncthreads();
  }
  if (warp == 1) {
    ptx::tc_fence_after();
    if constexpr (PAIR) ptx::tmem_dealloc_pair(tmem_base, 512);
    else ptx::tmem_dealloc(tmem_base, 512);
  }
}

// ------------------------------------------------------------ stacked-diagonal slice products
// For a narrow B (at most 16 sets, the adjoints' grad_C = Z G): one launch forms the sums of
// every diagonal at once, so that A's slices cross HBM once instead of once per plane launch.
// Per 32-value K chunk a stage holds A's s slices (128 rows x 64 bytes each, 64-byte swizzle)
// and B's chunk as 2s - 1 blocks of 16 rows: s - 1 zero blocks, then slices 0 .. s-1.  The MMA
// of A slice t against the s blocks that start at block s - 1 - t (N = 16 s) adds a_t b_(j-t)
// into column block j for every j >= t (zeros below), so column block j accumulates diagonal
// j (0-based) and one MMA per A slice and K step covers every slice pair of the kept diagonals.
constexpr int kStkNB = 16;                          // sets per tile (rows of a B block)
constexpr uint32_t kStkRow = 64;                    // bytes per operand row
constexpr int kStkBK = (int)kStkRow / 2;            // K values per chunk
constexpr int kStkMaxS = 11;                        // slices (two stages must fit)
constexpr uint32_t kStkASlice = BM * kStkRow;       // 8 KB
constexpr uint32_t kStkBBlock = kStkNB * kStkRow;   // 1 KB
constexpr int kStkStages = 2;
__host__ __device__ constexpr uint32_t stk_stage_bytes(int s) {
  return (uint32_t)s * kStkASlice + (uint32_t)(2 * s - 1) * kStkBBlock;
}
constexpr uint32_t kStkSmem = kStkStages * stk_stage_bytes(kStkMaxS) + 1024 /*align*/ + 256 /*barriers*/;
static_assert(kStkSmem <= 232448, "shared memory per CTA");
static_assert(kStkNB * kStkMaxS <= 256, "an accumulator fits half of the tensor memory");

struct StackedArgs {
  const uint8_t* A;  // [m_tiles][KC][s][kStkASlice]
  const uint8_t* B;  // [KC][2s - 1][kStkBBlock]
  int* T;            // diagonal d of K batch kb at T + kb * batch_stride + d * diag_stride, [rows][N]
  int64_t rows, N;
  int64_t m_tiles;
  int KC, s, k_batches, kc_per_batch;
  int64_t diag_stride, batch_stride;
};

// Persistent: warp 0 loads the stages (one thread, plain bulk copies), warp 1 issues the MMAs,
// warps 2-5 store the diagonal sums of finished tiles as int32 (every sum is an integer below
// 2^24, exact in float32).  Tile t = (K batch t / m_tiles, point tile t % m_tiles).
__global__ void __launch_bounds__(192, 1) stacked_slice_gemm_kernel(StackedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const int s = a.s;
  const uint32_t a_bytes = (uint32_t)s * kStkASlice, b_bytes = (uint32_t)(2 * s - 1) * kStkBBlock;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStkStages * stk_stage_bytes(kStkMaxS));
  uint64_t* empty = full + kStkStages;
  uint64_t* tmem_full = empty + kStkStages;
  uint64_t* tmem_empty = tmem_full + 2;
  uint64_t* drain = tmem_empty + 2;
  uint32_t* tmem_base_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_base_slot + 1);
  volatile int* never = abort_flag + 1;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStkStages; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&tmem_full[i], 1);
      ptx::mbar_init(&tmem_empty[i], 4);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    *never = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_base_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_base_slot;

  const int64_t total = a.m_tiles * a.k_batches;
  auto k_range = [&](int64_t t, int& kc0, int& nkc) {
    kc0 = (int)(t / a.m_tiles) * a.kc_per_batch;
    nkc = (kc0 + a.kc_per_batch < a.KC ? kc0 + a.kc_per_batch : a.KC) - kc0;
  };
  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(&g_split_error, 1u);
  };

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
        const int64_t mt = t % a.m_tiles;
        int kc0, nkc;
        k_range(t, kc0, nkc);
        bool ok = true;
        for (int kc = kc0; kc < kc0 + nkc; ++kc) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          uint8_t* sA = smem + stage * stage_bytes;
          ptx::mbar_arrive_expect_tx(&full[stage], stage_bytes);
          ptx::bulk_g2s(sA, a.A + ((size_t)mt * a.KC + kc) * a_bytes, a_bytes, &full[stage]);
          ptx::bulk_g2s(sA + a_bytes, a.B + (size_t)kc * b_bytes, b_bytes, &full[stage]);
          if (++stage == kStkStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = ptx::idesc_bf16_f32(BM, kStkNB * s);
      int stage = 0;
      uint32_t phase = 0;
      int64_t local = 0;
      for (int64_t t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++local) {
        const uint32_t acc = (uint32_t)(local & 1);
        if (!ptx::mbar_wait(&tmem_empty[acc], (uint32_t)((local >> 1) & 1) ^ 1u, abort_flag)) {
          fail();
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * 256u;
        int kc0, nkc;
        k_range(t, kc0, nkc);
        bool ok = true;
        for (int kk = 0; kk < nkc; ++kk) {
          if (!ptx::mbar_wait(&full[stage], phase, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t sA = ptx::smem_u32(smem + stage * stage_bytes);
          const uint32_t sB = sA + a_bytes;
          for (int ts = 0; ts < s; ++ts) {
#pragma unroll
            for (int ks = 0; ks < (int)kStkRow / 32; ++ks) {
              const uint32_t first = (kk == 0 && ts == 0 && ks == 0) ? 0u : 1u;
              ptx::mma_bf16(d_tmem, ptx::sw_kmajor_desc<kStkRow>(sA + (uint32_t)ts * kStkASlice + ks * 32u),
                            ptx::sw_kmajor_desc<kStkRow>(sB + (uint32_t)(s - 1 - ts) * kStkBBlock + ks * 32u), idesc,
                            first);
            }
          }
          ptx::mma_commit(&empty[stage]);
          if (++stage == kStkStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        ptx::mma_commit(&tmem_full[acc]);
      }
      // Every MMA issued here completes before the CTA leaves.
      ptx::mma_commit(drain);
      if (!ptx::mbar_wait(drain, 0u, never)) atomicOr(&g_split_error, 1u);
    }
  } else {
    // Epilogue: warp & 3 selects the TMEM lane quadrant it may access.
    const uint32_t q = (uint32_t)(warp & 3);
    const uint32_t row = q * 32 + lane;
    const bool vec = a.N == kStkNB;
    int64_t local = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++local) {
      const uint32_t acc = (uint32_t)(local & 1);
      bool ok = true;
      if (lane == 0) ok = ptx::mbar_wait(&tmem_full[acc], (uint32_t)((local >> 1) & 1), abort_flag);
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
        fail();
        break;
      }
      ptx::tc_fence_after();
      const int64_t p = (t % a.m_tiles) * BM + row;
      const bool store = p < a.rows;
      int* trow = a.T + (t / a.m_tiles) * a.batch_stride + p * a.N;
      const uint32_t tacc = tmem_base + ((q * 32u) << 16) + acc * 256u;
#pragma unroll 1
      for (int d = 0; d < s; ++d) {
        uint32_t v[8], w[8];
        ptx::tmem_ld_32x32b_x8(tacc + (uint32_t)(d * kStkNB), v);
        ptx::tmem_ld_wait(v);
        ptx::tmem_ld_32x32b_x8(tacc + (uint32_t)(d * kStkNB + 8), w);
        ptx::tmem_ld_wait(w);
        if (store) {
          int x[16];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            x[i] = __float2int_rn(__uint_as_float(v[i]));
            x[8 + i] = __float2int_rn(__uint_as_float(w[i]));
          }
          int* dst = trow + d * a.diag_stride;
          if (vec) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              __stcs(reinterpret_cast<int4*>(dst) + i, make_int4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]));
          } else {
            for (int i = 0; i < (int)a.N; ++i) dst[i] = x[i];
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tmem_empty[acc]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 512);
  }
}

// Optional per-phase timing: CUDA events recorded on the launching stream around every
// launch, summed per phase after the stream is synchronised.
struct PhaseTimer {
  float* ms = nullptr;  // [3]: coefficient split, basis split, GEMM (NULL: no timing)
  cudaStream_t stream = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[3];
  void begin(int phase, cudaEvent_t* start, cudaStream_t on) {
    *start = nullptr;
    if (!ms) return;
    cudaEventCreate(start);
    cudaEventRecord(*start, on);
    (void)phase;
  }
  void end(int phase, cudaEvent_t start, cudaStream_t on) {
    if (!ms) return;
    cudaEvent_t stop;
    cudaEventCreate(&stop);
    cudaEventRecord(stop, on);
    ev[phase].emplace_back(start, stop);
  }
  zp_status finish() {
    if (!ms) return ZP_OK;
    cudaError_t e = cudaStreamSynchronize(stream);
    for (int i = 0; i < 3; ++i) {
      ms[i] = 0.0f;
      for (auto& pr : ev[i]) {
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pr.first, pr.second);
        ms[i] += t;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
      ev[i].clear();
    }
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "phase timing");
  }
};

// Launch geometry of the persistent GEMM: one CTA per SM (the ring fills most of the
// shared memory).
struct GemmShape {
  int sms = 0;
  int pairs = 0;  // CTA pairs that can be resident at once (0: pairs cannot run)
};

// CTA pairs of split_gemm_kernel<KIND, 2> that fit on the GPU at once (one per two SMs when
// the GPCs allow it), after raising the kernel's shared-memory limit.
template <int KIND>
int max_pairs() {
  using S = Stage<KIND, 2>;
  if (cudaFuncSetAttribute(split_gemm_kernel<KIND, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(2);
  lc.blockDim = dim3(gemm_threads<2>());
  lc.dynamicSmemBytes = S::SMEM;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, split_gemm_kernel<KIND, 2>, &lc) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int KIND>
zp_status gemm_shape(GemmShape* g) {
  static DeviceMemo<GemmShape> memo;
  return memo.get(g, [](GemmShape* x) -> zp_status {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(split_gemm_kernel<KIND, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Stage<KIND, 1>::SMEM) != cudaSuccess) {
      cudaGetLastError();
      return set_error(ZP_ERR_CUDA, "cudaFuncSetAttribute(split_gemm_kernel)");
    }
    x->pairs = max_pairs<KIND>();
    return ZP_OK;
  });
}

// CTA pairs are used unless ZP_GEMM_CTA_PAIRS=0 (read at every launch).
inline bool pairs_enabled() {
  const char* v = std::getenv("ZP_GEMM_CTA_PAIRS");
  return !(v && v[0] == '0');
}

// The stacked-diagonal slice products for narrow B (ZP_EMU_STACKED=0 turns them off, for
// comparison with the paired plane launches).
inline bool stacked_enabled() {
  const char* v = std::getenv("ZP_EMU_STACKED");
  return !(v && v[0] == '0');
}

zp_status launch_stacked(const StackedArgs& sa, int sms, cudaStream_t stream) {
  static DeviceMemo<int> attr;
  int set = 0;
  ZP_TRY(attr.get(&set, [](int* x) -> zp_status {
    const cudaError_t e =
        cudaFuncSetAttribute(stacked_slice_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStkSmem);
    *x = 1;
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaFuncSetAttribute");
  }));
  const int64_t total = sa.m_tiles * sa.k_batches;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(total, sms));
  stacked_slice_gemm_kernel<<<grid, 192, kStkSmem, stream>>>(sa);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "stacked_slice_gemm_kernel launch");
}

// Persistent launch over `tiles` point tiles x NT set tiles (x K batches): CTA pairs over
// 256-point tiles when they can run and there are two point tiles or more, else one CTA per
// SM over 128-point tiles.
template <int KIND>
zp_status launch_gemm(const GemmArgs& ga, int64_t tiles, int NT, const GemmShape& g, cudaStream_t stream) {
  const int64_t kb = ga.k_batches > 0 ? ga.k_batches : 1;
  cudaError_t e;
  // Narrow paired slice tiles (fewer than 128 sets) run on single CTAs: a pair splits B's rows.
  const bool narrow = KIND == KIND_SLICE && ga.paired && ga.nb < BN / 2;
  if (g.pairs > 0 && tiles >= 2 && !narrow && pairs_enabled()) {
    const int64_t groups = (tiles + 1) / 2 * NT * kb;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(2 * std::min<int64_t>(groups, g.pairs)));
    lc.blockDim = dim3(gemm_threads<2>());
    lc.dynamicSmemBytes = Stage<KIND, 2>::SMEM;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    e = cudaLaunchKernelEx(&lc, split_gemm_kernel<KIND, 2>, ga);
  } else {
    const unsigned grid = (unsigned)std::min<int64_t>(tiles * NT * kb, g.sms);
    split_gemm_kernel<KIND, 1><<<grid, gemm_threads<1>(), Stage<KIND, 1>::SMEM, stream>>>(ga);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "split_gemm_kernel launch");
}

template <bool TF32>
zp_status run_split(const zp_plan* plan, const double* r, const double* theta, int64_t P, const double* coeffs,
                    int64_t S, float* out, cudaStream_t stream, float* phase_ms, const SplitScratch* preset) {
  PhaseTimer timer;
  timer.ms = phase_ms;
  timer.stream = stream;
  cudaEvent_t ev0;
  constexpr int KIND = TF32 ? KIND_TF32 : KIND_BF16X3;
  using C = Cfg<KIND>;
  const int64_t J = plan->n_modes;
  const int KC = (int)((J + C::BK - 1) / C::BK);
  const int64_t MT = (P + BM - 1) / BM;
  const int NT = (int)((S + BN - 1) / BN);
  const size_t tile_bytes = (size_t)KC * C::A_CHUNK;
  const size_t b_bytes = (size_t)NT * KC * C::B_CHUNK;
  ScratchBuffer bbuf, abuf;
  uint8_t* A = nullptr;
  uint8_t* B = nullptr;
  // A basis wave: the point tiles whose CTAs are resident at once.  The basis kernel is
  // latency-bound per CTA, so a launch that ends with a part-filled wave takes nearly as long as
  // a full one; slabs are therefore whole waves where the scratch allows.
  GemmShape gs;
  ZP_TRY(gemm_shape<KIND>(&gs));
  int per_sm = 0;
  static DeviceMemo<int> basis_per_sm;
  ZP_TRY(basis_per_sm.get(&per_sm, [](int* x) -> zp_status {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(x, split_basis_kernel<TF32>, basis_threads<TF32>(), 0) !=
        cudaSuccess) {
      cudaGetLastError();
      *x = 1;
    }
    // The coefficient kernel's shared memory limit, set once per device.
    const cudaError_t e = cudaFuncSetAttribute(split_coeff_kernel<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(Cfg<TF32 ? KIND_TF32 : KIND_BF16X3>::B_CHUNK + 1024));
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaFuncSetAttribute(split_coeff_kernel)");
  }));
  const int64_t wave = (int64_t)std::max(per_sm, 1) * gs.sms;
  int64_t slab = 0;
  if (preset) {
    // Caller-provided scratch: the B tiles first, then as many point tiles as fit.
    if (preset->b_bytes < b_bytes || preset->a_bytes < tile_bytes)
      return set_error(ZP_ERR_INVALID_ARG, "split scratch too small for this problem");
    A = preset->a;
    B = preset->b;
    const int64_t fit = (int64_t)(preset->a_bytes / tile_bytes);
    slab = std::min<int64_t>(MT, fit >= wave ? fit / wave * wave : fit);
  } else {
    // Slabs of about 512 MB of split basis, rounded to whole waves (at least one, at most 4 GB),
    // run back to back on the caller's stream.  (Running the float64 basis of slab i+1 on a
    // second stream beside the GEMM of slab i was measured slower on GB300: the GEMM is
    // sensitive to the basis kernel's extra L2 write traffic.)
    const int64_t cap = (int64_t)((512ull << 20) / tile_bytes);
    const int64_t hard = std::max<int64_t>(1, (int64_t)((4ull << 30) / tile_bytes));
    int64_t want = std::max<int64_t>(1, (cap + wave / 2) / wave) * wave;
    if (want > hard) want = hard >= gs.sms ? hard / gs.sms * gs.sms : hard;
    slab = std::max<int64_t>(1, std::min<int64_t>(MT, want));
    ZP_TRY(bbuf.alloc(b_bytes, stream));
    ZP_TRY(abuf.alloc((size_t)slab * tile_bytes, stream));
    A = (uint8_t*)abuf.ptr;
    B = (uint8_t*)bbuf.ptr;
  }

  const uint32_t coeff_smem = C::B_CHUNK + 1024;
  cudaError_t e;

  CoeffArgs ca{coeffs, plan->dev.slot_idx, J, S, KC, B};
  timer.begin(0, &ev0, stream);
  split_coeff_kernel<TF32><<<(unsigned)(NT * KC), kCoeffThreads, coeff_smem, stream>>>(ca);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "split_coeff_kernel launch");
  timer.end(0, ev0, stream);

  for (int64_t mt0 = 0; mt0 < MT; mt0 += slab) {
    const int64_t tiles = std::min<int64_t>(slab, MT - mt0);
    BasisArgs ba{plan->dev.cols, (int)plan->cols.size(), plan->dev.table, plan->dev.split_step, plan->dev.slot_ptr,
                 plan->dev.slot_idx,
                 r, theta, P, mt0, KC, A};
    timer.begin(1, &ev0, stream);
    split_basis_kernel<TF32><<<(unsigned)tiles, basis_threads<TF32>(), 0, stream>>>(ba, tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "split_basis_kernel launch");
    timer.end(1, ev0, stream);
    GemmArgs ga{A, B, out, P, S, mt0, tiles, NT, KC};
    timer.begin(2, &ev0, stream);
    ZP_TRY(launch_gemm<KIND>(ga, tiles, NT, gs, stream));
    timer.end(2, ev0, stream);
  }
  return timer.finish();
}

// ---------------------------------------------------------------------------------------
// Float64-accurate GEMM emulated on the tensor cores (Ozaki-style error-free slicing, a
// published scheme):  C[m][n] = sum_k A(m, k) B(n, k)  for float64 A, B.  Rows of A and of B
// are scaled by powers of two into [-1, 1], rounded to fixed point with beta * s >= 54
// fraction bits and cut into s balanced digits of beta bits, x = sum_t a_t 2^(-beta t) (small
// integers, exact in bfloat16).  For each slice diagonal d = t + u the GEMM sums all pairs
// (t, u) along a concatenated K into float32; with K cut into batches short enough, every
// partial sum is an integer below 2^24, hence exact, and is stored as int32.  The batches'
// sums are added and C = sigma_m sigma_n sum_d 2^(-beta d) T_d is formed exactly in integers
// and rounded once to float64.  Pairs with t + u > s + 1 are dropped (their total is below
// 2^(-beta s) of the scales).  Slicing and recombination run on the integer pipe: GB300's
// float64 pipe issues at 1/64 of its float32 rate.

static_assert(Cfg<KIND_SLICE>::BK == kSliceBK, "slice chunk width shared with zp_emu_shape.h");

// A float64 operand read with strides: X(row, k) = x[row * sr + k * sk].
struct Operand {
  const double* x;
  int64_t sr, sk;
};

// Largest |X(row, k)| of every row as float64 bits with the sign cleared (positive doubles
// order like their bit patterns), combined over K ranges by atomicMax into bits[row] (zeroed
// first).  Grid y = K range of k_per_block.  ROWS_FAST: thread = row (coalesced when
// sr == 1); otherwise warp = row, lanes across K (coalesced when sk == 1).
template <bool ROWS_FAST>
__global__ void row_absmax_kernel(Operand X, int64_t rows, int64_t K, int64_t k_per_block,
                                  unsigned long long* __restrict__ bits) {
  const int64_t k0 = (int64_t)blockIdx.y * k_per_block;
  const int64_t k1 = k0 + k_per_block < K ? k0 + k_per_block : K;
  unsigned long long mx = 0;
  // |x| as bits; four loads in flight per thread before their maxima are taken.
  auto mag = [&](int64_t row, int64_t k) {
    return (unsigned long long)__double_as_longlong(X.x[row * X.sr + k * X.sk]) & 0x7fffffffffffffffull;
  };
  auto max4 = [](unsigned long long a, unsigned long long b, unsigned long long c, unsigned long long d) {
    a = a > b ? a : b;
    c = c > d ? c : d;
    return a > c ? a : c;
  };
  if constexpr (ROWS_FAST) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    int64_t k = k0;
    for (; k + 3 < k1; k += 4) {
      const unsigned long long v = max4(mag(row, k), mag(row, k + 1), mag(row, k + 2), mag(row, k + 3));
      mx = v > mx ? v : mx;
    }
    for (; k < k1; ++k) {
      const unsigned long long v = mag(row, k);
      mx = v > mx ? v : mx;
    }
    if (mx) atomicMax(bits + row, mx);
  } else {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (row >= rows) return;
    int64_t k = k0 + lane;
    for (; k + 96 < k1; k += 128) {
      const unsigned long long v = max4(mag(row, k), mag(row, k + 32), mag(row, k + 64), mag(row, k + 96));
      mx = v > mx ? v : mx;
    }
    for (; k < k1; k += 32) {
      const unsigned long long v = mag(row, k);
      mx = v > mx ? v : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_down_sync(0xffffffffu, mx, off);
      mx = o > mx ? o : mx;
    }
    if (lane == 0 && mx) atomicMax(bits + row, mx);
  }
}

__global__ void row_exponent_kernel(const unsigned long long* __restrict__ bits, int64_t rows, int* __restrict__ expo) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < rows) expo[row] = scale_exponent(bits[row]);
}

// Power-of-two scale exponent of every row (2^e > max_k |X(row, k)|), with enough K ranges
// in flight to fill the GPU.  `bits` is scratch of `rows` words.
zp_status scale_rows(Operand X, int64_t rows, int64_t K, unsigned long long* bits, int* expo, cudaStream_t stream) {
  if (rows <= 0) return ZP_OK;
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)rows * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
  const bool rows_fast = X.sr == 1 || K < 32;
  const int64_t row_threads = rows_fast ? rows : rows * 32;
  const int64_t want = 152 * 1024;  // about the threads that fill the GPU (152 SMs x 1024)
  int64_t k_blocks = std::max<int64_t>(1, std::min<int64_t>((want + row_threads - 1) / row_threads, (K + 63) / 64));
  k_blocks = std::min<int64_t>(k_blocks, 65535);
  const int64_t kpb = (K + k_blocks - 1) / k_blocks;
  k_blocks = (K + kpb - 1) / kpb;
  const dim3 grid((unsigned)((row_threads + 255) / 256), (unsigned)k_blocks);
  if (rows_fast)
    row_absmax_kernel<true><<<grid, 256, 0, stream>>>(X, rows, K, kpb, bits);
  else
    row_absmax_kernel<false><<<grid, 256, 0, stream>>>(X, rows, K, kpb, bits);
  row_exponent_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, stream>>>(bits, rows, expo);
  e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "row scale launch");
}

// Cuts 8 fixed-point values X[0..7] (beta * s fraction bits) into s balanced base-2^beta digits
// and writes slice t's 16-byte unit of bf16 integers at `dst + t * slice_stride` (slice 0 the
// most significant).  The digits below the top one lie in [-2^(beta-1), 2^(beta-1)); they are
// the beta-bit fields f of the biased word Y = X + slice_bias(beta, s), minus 2^(beta-1), and the
// top digit is what is left of Y above them (|a_1| <= 2^beta): the same digits as cutting
// a = X mod 2^beta into that range and carrying.  A field (f < 128 for
// beta <= 7) under the bfloat16 pattern 0x4300 is exactly 128 + f, so one packed subtraction of
// 128 + 2^(beta-1) turns the fields of two values into their two digits (exact); the top digit
// goes through float32 (exact below 2^22).
__device__ __forceinline__ void cut_slices(const long long (&X)[8], int beta, int s, long long bias, uint8_t* dst,
                                           int64_t slice_stride) {
  const uint32_t mask = (1u << beta) - 1u;
  const uint32_t mask2 = mask | (mask << 16);
  const uint16_t sub_bits = (uint16_t)(0x4300u | (1u << (beta - 1)));  // bfloat16 128 + 2^(beta-1)
  const __nv_bfloat162 sub(__nv_bfloat16_raw{sub_bits}, __nv_bfloat16_raw{sub_bits});
  long long Y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) Y[q] = X[q] + bias;
  for (int p = 0; p < s - 1; ++p) {  // field p: slice s - 1 - p
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t f = (((uint32_t)Y[2 * i] & 0xffffu) | ((uint32_t)Y[2 * i + 1] << 16)) & mask2;
      __nv_bfloat162 v;
      const uint32_t pat = f | 0x43004300u;
      v = *reinterpret_cast<const __nv_bfloat162*>(&pat);
      v = __hsub2(v, sub);
      w[i] = *reinterpret_cast<const uint32_t*>(&v);
      Y[2 * i] >>= beta;
      Y[2 * i + 1] >>= beta;
    }
    *reinterpret_cast<uint4*>(dst + (size_t)(s - 1 - p) * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t h0 = __float_as_uint(__int_as_float(0x4B400000 + (int)Y[2 * i]) - 12582912.0f);
    const uint32_t h1 = __float_as_uint(__int_as_float(0x4B400000 + (int)Y[2 * i + 1]) - 12582912.0f);
    w[i] = __byte_perm(h0, h1, 0x7632);
  }
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Slices of an operand's rows in the tensor core's K-major swizzled chunks (rows of ROW bytes,
// ROW / 2 K values): tile (row / ROWS) x K chunk kc at (tile * KC + kc) * chunk_stride bytes
// (ROWS * ROW for one slice per chunk, s times that when the slices of a chunk lie back to
// back), slice t a further t * slice_stride.  Thread = (row, group of 8 consecutive K): rows fastest when an operand's
// rows are contiguous (KFAST = false), K groups fastest when its K is (coalesced loads either
// way).  Rows past `rows` and K past `K` are zero.
template <int ROWS_T, bool KFAST, uint32_t ROW = Cfg<KIND_SLICE>::ROW>
__global__ void slice_rows_kernel(Operand X, int64_t rows, int64_t tiles, int64_t K, int KC,
                                  const int* __restrict__ expo, SliceParams sp, uint8_t* dst, int64_t slice_stride,
                                  int64_t chunk_stride, int rows_per_tile = 0) {
  constexpr int BK = (int)ROW / 2;
  const int ROWS = ROWS_T > 0 ? ROWS_T : rows_per_tile;  // ROWS_T = 0: a multiple of 16 given at launch
  const int64_t rows_pad = tiles * ROWS;
  const int64_t groups = (int64_t)KC * (BK / 8);
  const int64_t total = rows_pad * groups;
  const long long bias = slice_bias(sp.beta, sp.s);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t row, k0;
    if constexpr (KFAST && ROW == 64) {
      // Eight threads per (row pair, K chunk): rows 2j and 2j + 1 share a 128-byte line of the
      // 64-byte layout, so each slice's stores fill whole lines.
      const int64_t rest = i >> 3, sub = i & 7;
      row = 2 * (rest / KC) + (sub >> 2);
      k0 = (rest % KC) * BK + (sub & 3) * 8;
    } else {
      row = KFAST ? i / groups : i % rows_pad;
      k0 = (KFAST ? i % groups : i / rows_pad) * 8;
    }
    const bool valid = row < rows;
    const int ex = valid ? expo[row] : 0;
    const bool use = valid && ex != kNonFiniteRow;
    const int shift = sp.beta * sp.s - ex;
    long long x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (use && k0 + q < K) ? to_fixed(X.x[row * X.sr + (k0 + q) * X.sk], shift) : 0;
    const int64_t tile = row / ROWS;
    const uint32_t r = (uint32_t)(row % ROWS);
    const int kc = (int)(k0 / BK);
    uint8_t* d = dst + ((size_t)tile * KC + kc) * chunk_stride + ptx::sw_offset_b16<ROW>(r, (uint32_t)(k0 % BK));
    cut_slices(x, sp.beta, sp.s, bias, d, slice_stride);
  }
}

struct RecombineArgs {
  const int* T;            // [k_batches][ndiag][rows][N] int32 sums (planes of one or two diagonals)
  const long long* T64;    // or [ndiag][rows][N] int64 sums of all batches (then k_batches = 1)
  int64_t diag_stride;     // rows * N
  int64_t batch_stride;    // ndiag * rows * N
  int k_batches, ndiag, split;
  int beta;                // bits between consecutive planes (beta, or 2 beta for paired diagonals)
  int e_base;              // -beta_slice (s + 1): exponent of the last plane's unit
  const int* rexp;         // [rows]
  const int* cexp;         // [N]
  int64_t rows, N;
  double* C;               // row m at C + m * ldc
  int64_t ldc;
};

// VW consecutive diagonal sums (streaming loads), VW in {1, 2, 4}.
template <int VW>
__device__ __forceinline__ void load_sums(const int* p, long long (&t)[VW]) {
  if constexpr (VW == 4) {
    const int4 v = __ldcs(reinterpret_cast<const int4*>(p));
    t[0] = v.x, t[1] = v.y, t[2] = v.z, t[3] = v.w;
  } else if constexpr (VW == 2) {
    const int2 v = __ldcs(reinterpret_cast<const int2*>(p));
    t[0] = v.x, t[1] = v.y;
  } else {
    t[0] = __ldcs(p);
  }
}
template <int VW>
__device__ __forceinline__ void load_sums(const long long* p, long long (&t)[VW]) {
#pragma unroll
  for (int k = 0; k < VW; k += 2) {
    if (k + 1 < VW) {
      const longlong2 v = __ldcs(reinterpret_cast<const longlong2*>(p + k));
      t[k] = v.x, t[k + 1] = v.y;
    } else {
      t[k] = __ldcs(p + k);
    }
  }
}

// Sums the K batches' int32 diagonal sums of every element of a batch plane into int64 `acc`
// (zeroed by the caller), `per` batches per thread: many threads share a long batch list, and
// the integer atomics make the result exact and independent of their order.
__global__ void sum_batches_kernel(const int* __restrict__ T, int64_t batch_stride, int k_batches, int per,
                                   long long* __restrict__ acc) {
  const int64_t groups = (k_batches + per - 1) / per;
  const int64_t total = batch_stride * groups;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i % batch_stride;
    const int kb0 = (int)(i / batch_stride) * per;
    const int kb1 = kb0 + per < k_batches ? kb0 + per : k_batches;
    long long sum = 0;
    for (int kb = kb0; kb < kb1; ++kb) sum += __ldcs(T + kb * batch_stride + e);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + e), (unsigned long long)sum);
  }
}

// Number of consecutive outputs of one recombination thread (a 16-byte store per two).
constexpr int kRecombineWidth = 4;
// From this many K batches on, the batches are pre-summed in parallel before recombining.
constexpr int kPreReduceBatches = 8;

// C[m][n] = sigma_m sigma_n 2^e_base Nmn with Nmn = sum_q (sum_batches T_q) 2^(beta (ndiag-1-q))
// over the planes q (one diagonal each, or two when paired: then beta is twice the slice
// width), formed exactly: the first `split` planes in one int64 Horner chain, the rest in
// another, joined into 128 bits and rounded once.
// Block = row m of C (grid-stride), threads across n, VW consecutive outputs per thread.
// SH > 0: the Horner shift is the constant SH (= a.beta), so the 64-bit shifts compile to a
// fixed instruction pair instead of the general variable-shift sequence.
template <int VW, typename TT, int SH = 0>
__global__ void recombine_kernel(RecombineArgs a) {
  const TT* Tbase;
  if constexpr (sizeof(TT) == 8) {
    Tbase = a.T64;
  } else {
    Tbase = a.T;
  }
  const int hsh = SH > 0 ? SH : a.beta;
  const int lo_shift = hsh * (a.ndiag - a.split);
  const int e_base = a.e_base;
  // Vector path: VW-wide loads of T (its rows are VW-aligned when N is) and 16-byte stores of C.
  const bool vec =
      (a.N % VW) == 0 && (VW == 1 || ((a.ldc % 2) == 0 && ((uintptr_t)a.C % 16) == 0));
  for (int64_t m = blockIdx.x; m < a.rows; m += gridDim.x) {
    const bool row_bad = a.rexp[m] == kNonFiniteRow;
    const int em = a.rexp[m] + e_base;
    const TT* trow = Tbase + m * a.N;
    double* crow = a.C + m * a.ldc;
    if (vec) {
      for (int64_t n0 = (int64_t)threadIdx.x * VW; n0 < a.N; n0 += (int64_t)blockDim.x * VW) {
        long long hi[VW] = {}, lo[VW] = {};
        if (a.k_batches == 1) {
          // One batch: the diagonal loads are independent, unrolled so they are all in flight.
          const TT* tp = trow + n0;
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            if (q < a.ndiag) {
              long long t[VW];
              load_sums<VW>(tp, t);
              tp += a.diag_stride;
#pragma unroll
              for (int k = 0; k < VW; ++k) {
                if (q < a.split) hi[k] = horner(hi[k], hsh, t[k]);
                else lo[k] = horner(lo[k], hsh, t[k]);
              }
            }
          }
        } else {
          for (int q = 0; q < a.ndiag; ++q) {
            long long t[VW] = {};
            for (int kb = 0; kb < a.k_batches; ++kb) {
              long long v[VW];
              load_sums<VW>(trow + kb * a.batch_stride + q * a.diag_stride + n0, v);
#pragma unroll
              for (int k = 0; k < VW; ++k) t[k] += v[k];
            }
#pragma unroll
            for (int k = 0; k < VW; ++k) {
              if (q < a.split) hi[k] = horner(hi[k], hsh, t[k]);
              else lo[k] = horner(lo[k], hsh, t[k]);
            }
          }
        }
        double v[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          const int ec = a.cexp[n0 + k];
          v[k] = (row_bad || ec == kNonFiniteRow)
                     ? __longlong_as_double(0x7ff8000000000000ll)
                     : join_to_double(hi[k], lo[k], lo_shift, em + ec);
        }
        if constexpr (VW == 1) {
          __stcs(crow + n0, v[0]);
        } else {
#pragma unroll
          for (int k = 0; k < VW; k += 2)
            __stcs(reinterpret_cast<double2*>(crow + n0 + k), make_double2(v[k], v[k + 1]));
        }
      }
    } else {
      for (int64_t n = threadIdx.x; n < a.N; n += blockDim.x) {
        long long hi = 0, lo = 0;
        for (int q = 0; q < a.ndiag; ++q) {
          long long t = 0;
          for (int kb = 0; kb < a.k_batches; ++kb) t += trow[kb * a.batch_stride + q * a.diag_stride + n];
          if (q < a.split) hi = horner(hi, hsh, t);
          else lo = horner(lo, hsh, t);
        }
        crow[n] = (row_bad || a.cexp[n] == kNonFiniteRow)
                      ? __longlong_as_double(0x7ff8000000000000ll)
                      : join_to_double(hi, lo, lo_shift, em + a.cexp[n]);
      }
    }
  }
}

// recombine_kernel for one K batch (only) and the common plane shapes, with the plane count, the
// split of the Horner chains and the shift per plane fixed at compile time: the loops unroll
// completely and every shift is a constant.  4 consecutive outputs per thread (16-byte loads of
// each plane and of the column exponents, 16-byte stores); needs N % 4 == 0, an even ldc and
// a 16-byte aligned C.
template <int NPL, int SPLIT, int SH>
__global__ void __launch_bounds__(256) recombine_planes_kernel(RecombineArgs a) {
  constexpr int LS = SH * (NPL - SPLIT);
  for (int64_t m = blockIdx.x; m < a.rows; m += gridDim.x) {
    const int rx = a.rexp[m];
    const bool row_bad = rx == kNonFiniteRow;
    const int em = rx + a.e_base;
    const int* trow = a.T + m * a.N;
    double* crow = a.C + m * a.ldc;
    for (int64_t n0 = (int64_t)threadIdx.x * 4; n0 < a.N; n0 += (int64_t)blockDim.x * 4) {
      int4 v[NPL];
#pragma unroll
      for (int q = 0; q < NPL; ++q) v[q] = __ldcs(reinterpret_cast<const int4*>(trow + q * a.diag_stride + n0));
      const int4 ce = __ldg(reinterpret_cast<const int4*>(a.cexp + n0));
      double out[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        long long hi = 0, lo = 0;
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
          const int t = k == 0 ? v[q].x : (k == 1 ? v[q].y : (k == 2 ? v[q].z : v[q].w));
          if (q < SPLIT) hi = horner(hi, SH, t);
          else lo = horner(lo, SH, t);
        }
        const int ec = k == 0 ? ce.x : (k == 1 ? ce.y : (k == 2 ? ce.z : ce.w));
        out[k] = (row_bad || ec == kNonFiniteRow) ? __longlong_as_double(0x7ff8000000000000ll)
                                                  : join_to_double(hi, lo, LS, em + ec);
      }
      __stcs(reinterpret_cast<double2*>(crow + n0), make_double2(out[0], out[1]));
      __stcs(reinterpret_cast<double2*>(crow + n0 + 2), make_double2(out[2], out[3]));
    }
  }
}

// An emulated GEMM in progress: the B operand sliced once (all N rows), then A in slabs of
// row tiles, each slab: row scales, slices, one GEMM launch per slice diagonal (all pairs of
// the diagonal and all K batches), recombination into C.
struct EmuGemm {
  EmuShape sh;
  int64_t N = 0, K = 0, NT = 0;
  int nb = BN / 2;  // sets per tile of the paired layout
  int sms = 0;
  GemmShape gs;
  int64_t slab_tiles = 0;  // row tiles per slab
  int64_t recombine_blocks = 0;
  ScratchBuffer accbuf;  // int64 batch sums (runs with many K batches)
  ScratchBuffer bsl, cexp, asl, rexp, tbuf, maxbits;
  int64_t a_stride = 0, b_stride = 0;
  // Stacked-diagonal slice products (at most 16 sets, at most kStkMaxS slices): one launch per
  // slab over 32-value K chunks (KCs of them, kcb_s per K batch, kb_s batches); s planes.
  bool stacked = false;
  int KCs = 0, kcb_s = 0, kb_s = 0;
  int planes = 0;  // planes of sums written per K batch

  // Chooses the shape for M rows, slices B (B(n, k), n < N) and sizes the slab scratch.
  zp_status prepare(int64_t M, int64_t N_, int64_t K_, Operand B, cudaStream_t stream) {
    using C = Cfg<KIND_SLICE>;
    N = N_;
    K = K_;
    NT = (N + BN - 1) / BN;
    const int64_t MT = (M + BM - 1) / BM;
    ZP_TRY(gemm_shape<KIND_SLICE>(&gs));
    sms = gs.sms;
    // One resident wave of recombination blocks, grid-striding over the rows.
    int per_sm = 0;
    static DeviceMemo<int> recombine_per_sm;
    ZP_TRY(recombine_per_sm.get(&per_sm, [](int* x) -> zp_status {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(x, recombine_kernel<kRecombineWidth, int>, 256, 0) !=
          cudaSuccess) {
        cudaGetLastError();
        *x = 4;
      }
      return ZP_OK;
    }));
    recombine_blocks = (int64_t)std::max(per_sm, 1) * sms;
    if (!choose_emu_shape(K, MT * NT, sms, &sh))
      return set_error(ZP_ERR_UNSUPPORTED, "emulated float64 GEMM: contraction too long");
    // Paired diagonals: set tiles of nb (two diagonals share a tile's 2 nb accumulator columns):
    // 128, or for fewer sets the smallest multiple of 16 holding them all (a narrow tile: MMAs of
    // N = 2 nb, so that few sets do not pay for 256-column MMAs).
    if (sh.paired) {
      nb = N >= BN / 2 ? BN / 2 : (int)((N + 15) / 16 * 16);
      NT = (N + nb - 1) / nb;
    }
    planes = sh.planes;
    stacked = N <= kStkNB && sh.sp.s <= kStkMaxS && stacked_enabled();
    if (stacked) {
      NT = 1;
      KCs = (int)((K + kStkBK - 1) / kStkBK);
      kcb_s = 2 * sh.kc_per_batch;  // the same K values per batch as the 64-value chunks
      kb_s = (KCs + kcb_s - 1) / kcb_s;
      planes = sh.sp.s;
    }
    // Slab: int32 sums (k_batches x planes x rows x N x 4 B) within about 4 GB.
    const size_t t_tile = (size_t)sh.k_batches * planes * BM * N * sizeof(int);
    slab_tiles = std::max<int64_t>(1, std::min<int64_t>(MT, (int64_t)((4ull << 30) / t_tile)));
    a_stride = slab_tiles * sh.KC * (int64_t)C::A_CHUNK;
    b_stride = NT * sh.KC * (int64_t)C::B_CHUNK;
    // A paired B holds NT x KC x s blocks of nb rows; a stacked B KCs x (2s - 1) blocks of 16.
    const size_t b_stk = (size_t)KCs * (2 * sh.sp.s - 1) * kStkBBlock;
    ZP_TRY(bsl.alloc(stacked      ? b_stk
                     : sh.paired ? (size_t)NT * sh.KC * sh.sp.s * nb * C::ROW
                                 : (size_t)sh.sp.s * b_stride,
                     stream));
    ZP_TRY(cexp.alloc((size_t)N * sizeof(int), stream));
    ZP_TRY(asl.alloc(stacked ? (size_t)slab_tiles * KCs * sh.sp.s * kStkASlice : (size_t)sh.sp.s * a_stride, stream));
    ZP_TRY(rexp.alloc((size_t)slab_tiles * BM * sizeof(int), stream));
    ZP_TRY(tbuf.alloc((size_t)slab_tiles * t_tile, stream));
    if (sh.k_batches >= kPreReduceBatches)
      ZP_TRY(accbuf.alloc((size_t)planes * slab_tiles * BM * N * sizeof(long long), stream));
    ZP_TRY(maxbits.alloc((size_t)std::max<int64_t>(N, slab_tiles * BM) * sizeof(unsigned long long), stream));
    ZP_TRY(scale_rows(B, N, K, (unsigned long long*)maxbits.ptr, (int*)cexp.ptr, stream));
    const bool kfast = B.sk == 1 && B.sr != 1;
    if (stacked) {
      // Per 32-value K chunk: s - 1 zero blocks, then slices 0 .. s-1 of 16 rows.
      cudaError_t e = cudaMemsetAsync(bsl.ptr, 0, b_stk, stream);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
      const int64_t cs = (int64_t)(2 * sh.sp.s - 1) * kStkBBlock;
      uint8_t* b0 = (uint8_t*)bsl.ptr + (size_t)(sh.sp.s - 1) * kStkBBlock;
      if (kfast)
        slice_rows_kernel<kStkNB, true, kStkRow><<<1024, 256, 0, stream>>>(B, N, 1, K, KCs, (const int*)cexp.ptr,
                                                                           sh.sp, b0, kStkBBlock, cs);
      else
        slice_rows_kernel<kStkNB, false, kStkRow><<<1024, 256, 0, stream>>>(B, N, 1, K, KCs, (const int*)cexp.ptr,
                                                                            sh.sp, b0, kStkBBlock, cs);
    } else if (sh.paired) {
      // Per (set tile, K chunk): slices 0..s-1 of nb rows back to back.
      const int64_t blk = (int64_t)nb * C::ROW, cs = (int64_t)sh.sp.s * blk;
      if (kfast)
        slice_rows_kernel<0, true><<<1024, 256, 0, stream>>>(B, N, NT, K, sh.KC, (const int*)cexp.ptr, sh.sp,
                                                            (uint8_t*)bsl.ptr, blk, cs, nb);
      else
        slice_rows_kernel<0, false><<<1024, 256, 0, stream>>>(B, N, NT, K, sh.KC, (const int*)cexp.ptr, sh.sp,
                                                             (uint8_t*)bsl.ptr, blk, cs, nb);
    } else if (kfast) {
      slice_rows_kernel<BN, true><<<1024, 256, 0, stream>>>(B, N, NT, K, sh.KC, (const int*)cexp.ptr, sh.sp,
                                                           (uint8_t*)bsl.ptr, b_stride, C::B_CHUNK);
    } else {
      slice_rows_kernel<BN, false><<<1024, 256, 0, stream>>>(B, N, NT, K, sh.KC, (const int*)cexp.ptr, sh.sp,
                                                            (uint8_t*)bsl.ptr, b_stride, C::B_CHUNK);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "B slicing launch");
  }

  // C rows [0, rows) (rows <= slab_tiles * BM) = A rows [0, rows) times B^T.
  // a_rowmax: NULL, or the rows' largest |value| high words << 32 (formed by the producer of
  // A), which then replace the pass over A for the row scales.
  zp_status run_slab(int64_t rows, Operand A, double* Cout, int64_t ldc, cudaStream_t stream,
                     const unsigned long long* a_rowmax = nullptr) {
    using C = Cfg<KIND_SLICE>;
    const int64_t tiles = (rows + BM - 1) / BM;
    if (a_rowmax) {
      row_exponent_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, stream>>>(a_rowmax, rows, (int*)rexp.ptr);
      const cudaError_t e0 = cudaGetLastError();
      if (e0 != cudaSuccess) return cuda_error(e0, "row_exponent_kernel launch");
    } else {
      ZP_TRY(scale_rows(A, rows, K, (unsigned long long*)maxbits.ptr, (int*)rexp.ptr, stream));
    }
    if (stacked) return run_slab_stacked(rows, tiles, A, Cout, ldc, stream);
    if (A.sk == 1 && A.sr != 1)
      slice_rows_kernel<BM, true><<<2048, 256, 0, stream>>>(A, rows, tiles, K, sh.KC, (const int*)rexp.ptr, sh.sp,
                                                           (uint8_t*)asl.ptr, a_stride, C::A_CHUNK);
    else
      slice_rows_kernel<BM, false><<<2048, 256, 0, stream>>>(A, rows, tiles, K, sh.KC, (const int*)rexp.ptr, sh.sp,
                                                            (uint8_t*)asl.ptr, a_stride, C::A_CHUNK);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "A slicing launch");
    const int64_t trows = slab_tiles * BM;
    const int64_t diag_stride = trows * N, batch_stride = (int64_t)sh.planes * diag_stride;
    const int hsh = sh.paired ? 2 * sh.sp.beta : sh.sp.beta;
    for (int q = 0; q < sh.planes; ++q) {
      GemmArgs ga{(const uint8_t*)asl.ptr, (const uint8_t*)bsl.ptr,
                  (float*)tbuf.ptr + (size_t)q * diag_stride, rows, N, 0, tiles, (int)NT, sh.KC};
      if (sh.paired) {
        // Plane q: diagonals (2q - s % 2, 2q + 1 - s % 2), 0-based.
        ga.paired = 1;
        ga.nb = nb;
        ga.dp = 2 * q - (sh.sp.s & 1);
        ga.beta = sh.sp.beta;
        ga.s_slices = sh.sp.s;
      } else {
        ga.npairs = q + 1;  // diagonal q: pairs (t, q - t)
      }
      ga.a_slice_stride = a_stride;
      ga.b_slice_stride = b_stride;
      ga.k_batches = sh.k_batches;
      ga.kc_per_batch = sh.kc_per_batch;
      ga.t_batch_stride = batch_stride;
      ZP_TRY(launch_gemm<KIND_SLICE>(ga, tiles, (int)NT, gs, stream));
    }
    return recombine(rows, Cout, ldc, sh.k_batches, sh.planes, sh.plane_split, hsh, stream);
  }

  // The stacked-diagonal form of run_slab: A's slices in 64-byte rows, all s diagonals of a tile
  // by one launch, s planes of sums per K batch.
  zp_status run_slab_stacked(int64_t rows, int64_t tiles, Operand A, double* Cout, int64_t ldc, cudaStream_t stream) {
    const int sl = sh.sp.s;
    const int64_t cs = (int64_t)sl * kStkASlice;
    if (A.sk == 1 && A.sr != 1)
      slice_rows_kernel<BM, true, kStkRow><<<2048, 256, 0, stream>>>(A, rows, tiles, K, KCs, (const int*)rexp.ptr,
                                                                     sh.sp, (uint8_t*)asl.ptr, kStkASlice, cs);
    else
      slice_rows_kernel<BM, false, kStkRow><<<2048, 256, 0, stream>>>(A, rows, tiles, K, KCs, (const int*)rexp.ptr,
                                                                      sh.sp, (uint8_t*)asl.ptr, kStkASlice, cs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "A slicing launch");
    const int64_t diag_stride = slab_tiles * BM * N;
    StackedArgs sa{(const uint8_t*)asl.ptr, (const uint8_t*)bsl.ptr, (int*)tbuf.ptr, rows, N, tiles,
                   KCs, sl, kb_s, kcb_s, diag_stride, (int64_t)sl * diag_stride};
    ZP_TRY(launch_stacked(sa, sms, stream));
    return recombine(rows, Cout, ldc, kb_s, sl, sh.split, sh.sp.beta, stream);
  }

  // C rows [0, rows) from the int32 sums in tbuf: k_batches batches of ndiag planes (consecutive
  // planes hsh bits apart), the first `split` planes in the first Horner chain.
  zp_status recombine(int64_t rows, double* Cout, int64_t ldc, int k_batches, int ndiag, int split, int hsh,
                      cudaStream_t stream) {
    cudaError_t e = cudaSuccess;
    const int64_t diag_stride = slab_tiles * BM * N, batch_stride = (int64_t)ndiag * diag_stride;
    const int e_base = -sh.sp.beta * (sh.sp.s + 1);
    RecombineArgs ra{(const int*)tbuf.ptr, nullptr, diag_stride, batch_stride, k_batches, ndiag,
                     split, hsh, e_base,
                     (const int*)rexp.ptr, (const int*)cexp.ptr, rows, N, Cout, ldc};
    const unsigned rblocks = (unsigned)std::min<int64_t>(rows, recombine_blocks);
    if (k_batches >= kPreReduceBatches) {
      // Many K batches (a small output cut along a long K): the batches are first summed into
      // int64 planes by many threads, then recombined as one batch.
      if ((e = cudaMemsetAsync(accbuf.ptr, 0, (size_t)batch_stride * sizeof(long long), stream)) != cudaSuccess)
        return cuda_error(e, "cudaMemsetAsync");
      const int per = 8;
      const int64_t work = batch_stride * ((k_batches + per - 1) / per);
      sum_batches_kernel<<<(unsigned)std::min<int64_t>((work + 255) / 256, 8 * (int64_t)sms), 256, 0, stream>>>(
          (const int*)tbuf.ptr, batch_stride, k_batches, per, (long long*)accbuf.ptr);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "sum_batches_kernel launch");
      ra.T = nullptr;
      ra.T64 = (const long long*)accbuf.ptr;
      ra.k_batches = 1;
      recombine_kernel<kRecombineWidth, long long><<<rblocks, 256, 0, stream>>>(ra);
    } else {
      // The paired plane shapes of the four slice widths (planes, chains' split, shift per
      // plane) run fully unrolled; anything else takes the general kernel.
      const bool vec = ra.k_batches == 1 && (N % 4) == 0 && (ldc % 2) == 0 && ((uintptr_t)Cout % 16) == 0 &&
                       ((uintptr_t)cexp.ptr % 16) == 0;
      const int shape = vec ? ra.ndiag * 10000 + ra.split * 100 + ra.beta : 0;
      switch (shape) {
        case 50312: recombine_planes_kernel<5, 3, 12><<<rblocks, 256, 0, stream>>>(ra); break;
        case 40314: recombine_planes_kernel<4, 3, 14><<<rblocks, 256, 0, stream>>>(ra); break;
        case 60410: recombine_planes_kernel<6, 4, 10><<<rblocks, 256, 0, stream>>>(ra); break;
        case 70408: recombine_planes_kernel<7, 4, 8><<<rblocks, 256, 0, stream>>>(ra); break;
        default: recombine_kernel<kRecombineWidth, int><<<rblocks, 256, 0, stream>>>(ra); break;
      }
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "recombine_kernel launch");
  }
};

zp_status run_emulated_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                            const double* coeffs, int64_t S, double* out, cudaStream_t stream) {
  const int64_t J = plan->n_modes;
  EmuGemm g;
  // B(n = set s, k = mode j) = C[j][s].
  ZP_TRY(g.prepare(P, S, J, Operand{coeffs, 1, S}, stream));
  const int64_t slab_rows = g.slab_tiles * BM;
  ScratchBuffer zbuf;
  ZP_TRY(zbuf.alloc((size_t)J * slab_rows * sizeof(double), stream));
  for (int64_t p0 = 0; p0 < P; p0 += slab_rows) {
    const int64_t Ps = std::min<int64_t>(slab_rows, P - p0);
    ZP_TRY(launch_walk(plan, r + p0, theta + p0, Ps, 0, (double*)zbuf.ptr, nullptr, stream));
    // A(m = point p, k = mode j) = Z[j][p] of this slab.
    ZP_TRY(g.run_slab(Ps, Operand{(const double*)zbuf.ptr, 1, Ps}, out + (size_t)p0 * S, S, stream));
  }
  return ZP_OK;
}

}  // namespace

zp_status series_eval_emulated_fp64(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                                    const double* coeffs, int64_t S, double* out, cudaStream_t stream) {
  return run_emulated_fp64(plan, r, theta, P, coeffs, S, out, stream);
}

zp_status emulated_gemm_fp64(int64_t M, int64_t N, int64_t K, const double* A, int64_t a_sm, int64_t a_sk,
                             const double* B, int64_t b_sn, int64_t b_sk, double* C, int64_t ldc,
                             cudaStream_t stream, const unsigned long long* a_rowmax) {
  if (M <= 0 || N <= 0) return ZP_OK;
  if (K <= 0) {
    for (int64_t m = 0; m < M; ++m) {
      const cudaError_t e = cudaMemsetAsync(C + m * ldc, 0, (size_t)N * sizeof(double), stream);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    }
    return ZP_OK;
  }
  EmuGemm g;
  ZP_TRY(g.prepare(M, N, K, Operand{B, b_sn, b_sk}, stream));
  const int64_t slab_rows = g.slab_tiles * BM;
  for (int64_t m0 = 0; m0 < M; m0 += slab_rows) {
    const int64_t rows = std::min<int64_t>(slab_rows, M - m0);
    ZP_TRY(g.run_slab(rows, Operand{A + m0 * a_sm, a_sm, a_sk}, C + m0 * ldc, ldc, stream,
                      a_rowmax ? a_rowmax + m0 : nullptr));
  }
  return ZP_OK;
}

zp_status series_eval_split(const zp_plan* plan, const double* r, const double* theta, int64_t P,
                            const double* coeffs, int64_t S, zp_precision prec, float* out, cudaStream_t stream,
                            float* phase_ms, const SplitScratch* preset) {
  if (prec == ZP_PREC_TF32) return run_split<true>(plan, r, theta, P, coeffs, S, out, stream, phase_ms, preset);
  return run_split<false>(plan, r, theta, P, coeffs, S, out, stream, phase_ms, preset);
}

size_t split_scratch_bytes(zp_precision prec, int64_t n_modes, int64_t n_sets, size_t* b_bytes, size_t* tile_bytes) {
  const bool tf32 = prec == ZP_PREC_TF32;
  const int64_t bk = tf32 ? Cfg<KIND_TF32>::BK : Cfg<KIND_BF16X3>::BK;
  const size_t a_chunk = tf32 ? Cfg<KIND_TF32>::A_CHUNK : Cfg<KIND_BF16X3>::A_CHUNK;
  const size_t b_chunk = tf32 ? Cfg<KIND_TF32>::B_CHUNK : Cfg<KIND_BF16X3>::B_CHUNK;
  const int64_t KC = (n_modes + bk - 1) / bk;
  const int64_t NT = (n_sets + BN - 1) / BN;
  *b_bytes = (size_t)NT * KC * b_chunk;
  *tile_bytes = (size_t)KC * a_chunk;
  return *b_bytes + *tile_bytes;
}

namespace {
// Self-test of the bounded wait: one thread waits on an mbarrier that nothing ever arrives on;
// the wait gives up after limit_ns and records the timeout in the status word, exactly as the
// tensor-core kernels do.  No asynchronous copy or TMEM is involved, so giving up is safe.
__global__ void wait_selftest_kernel(uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    abort_flag = 0;
    ptx::fence_barrier_init();
    if (!ptx::mbar_wait(&bar, 0u, &abort_flag, limit_ns)) atomicOr(&g_split_error, 2u);
    ptx::mbar_arrive(&bar);  // complete the phase so the barrier is left in a finished state
  }
}
}  // namespace

zp_status wait_selftest(int32_t limit_ms, cudaStream_t stream) {
  wait_selftest_kernel<<<1, 32, 0, stream>>>((uint64_t)limit_ms * 1000000ull);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "wait_selftest_kernel launch");
}

zp_status split_error_word(unsigned int* value, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_split_error, sizeof(unsigned int));
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyFromSymbol");
  if (reset) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_split_error, &zero, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyToSymbol");
  }
  return ZP_OK;
}

}  // namespace zp

extern "C" zp_status zp_device_wait_selftest(int32_t limit_ms, void* stream) {
  zp::clear_error();
  if (limit_ms < 1 || limit_ms > 2000) return zp::set_error(ZP_ERR_INVALID_ARG, "limit_ms must be 1..2000");
  return zp::wait_selftest(limit_ms, (cudaStream_t)stream);
}

extern "C" zp_status zp_device_wait_status(int32_t reset) {
  zp::clear_error();
  unsigned int v = 0, f = 0;
  ZP_TRY(zp::split_error_word(&v, reset != 0));
  ZP_TRY(zp::fused_error_word(&f, reset != 0));
  if (v || f) return zp::set_error(ZP_ERR_TIMEOUT, "a bounded device wait in a tensor-core series kernel gave up");
  return ZP_OK;
}
