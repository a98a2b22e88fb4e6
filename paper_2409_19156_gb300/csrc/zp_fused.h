// Host-side interface of the fused float64-accurate series for few coefficient sets
// (zp_fused.cu): the basis is generated inside the tensor-core kernel and never written out.
#pragma once

#include <cstdint>

#include "zp_internal.h"

namespace zp {

constexpr int kFusedBeta = 5;       // bits per digit (the long-contraction shape)
constexpr int kFusedDigits = 11;    // digits per value: 55 fraction bits
constexpr int kFusedMaxSets = 16;   // coefficient sets per launch
// Longest contraction (K positions of the fused layout, padding included) whose diagonal sums
// stay exact integers in float32: K * 2^(2 beta) * (1 + (digits - 2) / 4) < 2^24.
constexpr int64_t kFusedMaxModes = 5041;
// Short contractions take 9 digits of 6 bits (54 fraction bits): K * 2^12 * (1 + 7 / 4) < 2^24
// for K <= 1489, and two digits fewer to cut, multiply and recombine per value.
constexpr int kFusedDigitsShort = 9;
constexpr int64_t kFusedMaxModesShort = 1489;
// Digits per value for a launch whose longest contraction has `kpad` positions.
inline int fused_digits_for(int64_t kpad) { return kpad <= kFusedMaxModesShort ? kFusedDigitsShort : kFusedDigits; }
// Bits per digit of the NDIG-digit shape.
__host__ __device__ constexpr int fused_beta(int ndig) { return ndig == kFusedDigitsShort ? 6 : kFusedBeta; }
// Bytes between consecutive 32-mode chunks of coefficient digits: room for 11 digit blocks of 16
// sets x 64 bytes (each row the tensor core's 64-byte swizzled K-major layout); the 9-digit shape
// uses the first 9 blocks of each chunk.
constexpr uint32_t kFusedBChunk = (uint32_t)kFusedDigits * kFusedMaxSets * 64u;

// Balanced base-2^beta digits of a fixed-point value X (|X| < 2^(beta NDIG)), most significant
// first: Y = X + fused_bias<NDIG>() holds, for the NDIG - 1 low positions, the unsigned fields
// f_t = d_t + 2^(beta-1) of the balanced digits d_t in [-2^(beta-1), 2^(beta-1)); the most
// significant digit is Y >> (beta (NDIG - 1)) itself (at most 2^beta + 1 in magnitude), so that
// X = sum_t d_t 2^(beta (NDIG - 1 - t)) with d_0 the top digit.
template <int NDIG = kFusedDigits>
__host__ __device__ constexpr long long fused_bias() {
  constexpr int beta = fused_beta(NDIG);
  long long b = 0;
  for (int t = 0; t < NDIG - 1; ++t) b += (long long)(1 << (beta - 1)) << (beta * t);
  return b;
}
// Digit t of the biased word Y: t = 0 the signed top digit, else the unsigned field.
template <int NDIG = kFusedDigits>
__host__ __device__ inline int fused_digit_field(long long Y, int t) {
  constexpr int beta = fused_beta(NDIG);
  return t == 0 ? (int)(Y >> (beta * (NDIG - 1)))
                : (int)((unsigned long long)(Y >> (beta * (NDIG - 1 - t))) & ((1u << beta) - 1u));
}

// One series instance of the fused kernel (device pointers).
struct FusedInst {
  const Column* cols = nullptr;
  const double* table = nullptr;
  const uint2* steps = nullptr;  // the plan's per-step slot counts and sin flags
  const int32_t* slot_ptr = nullptr;
  const int32_t* slot_idx = nullptr;
  const int32_t* mode_col = nullptr;  // column of every mode
  const int32_t* mode_N = nullptr;    // Jacobi degree of every mode
  const int4* fcols = nullptr;       // the plan's fused contraction layout per column
  const int32_t* scols = nullptr;    // columns of stream 0, then of stream 1 (walk order)
  const int32_t* kperm = nullptr;    // slot of every K position of that layout, -1 for padding
  int64_t Kp = 0;                    // K positions of that layout
  int32_t ncols_s[kFusedStreams] = {};  // columns per stream
  int32_t units = 0;                 // global 8-value units of the layout (stream s owns every kFusedStreams-th)
  int32_t ep_disc = 1;               // row scale exponent for points on the unit disc
  int32_t n_cols = 0;
  int32_t KC = 0;        // 32-position chunks of the contraction
  int64_t kc_base = 0;   // first chunk of this instance in the launch's chunk numbering
  int64_t J = 0, P = 0, S = 0;
  const double* r = nullptr;
  const double* theta = nullptr;
  const double* coeffs = nullptr;  // [J][S]
  uint8_t* bdig = nullptr;         // [KC][kFusedBChunk] coefficient digits (written per call)
  int* cexp = nullptr;             // [kFusedMaxSets] set scale exponents (written per call)
  double* out = nullptr;           // [P][S]
  // Instead of out: dot_out[p] += sum_s gdot[p][s] F[p][s] (two atomic adds per point onto a
  // zeroed array, one per half of the sets: the same sum in either order).
  const double* gdot = nullptr;    // [P][S]
  double* dot_out = nullptr;       // [P]
};

// Values a fused launch contracts with the coefficients: the basis Z (the series), its theta-
// derivative or its rho-derivative (the adjoint's point gradients as row sums of G times those
// series).
constexpr int kFusedZ = 0, kFusedDTheta = 1, kFusedDRho = 2;

// Row scale exponent of on-disc points for value kind vk: 2^e above every |value| of the plan on
// the unit disc (|R| <= 1, |dR/dtheta| <= m_max, |dR/drho| <= n_max^2 by Markov's inequality, each
// over the smallest weight W0_N).
int fused_ep_for(const zp_plan* plan, int vk);

// A 128-point tile of one instance.
struct FusedItem {
  int32_t inst;
  int32_t tile;
};

// Launch description: `insts` and `items` in device memory, or (both NULL) one instance
// passed by value whose tiles are the items in order.
struct FusedArgs {
  const FusedInst* insts = nullptr;
  const FusedItem* items = nullptr;
  int64_t n_items = 0;
  int ndig = kFusedDigits;  // digits per value: fused_digits_for(the largest instance's Kp)
  FusedInst single;
};

// Coefficient scales and digits of every instance (n_inst instances, chunk_inst[g] = instance of
// global chunk g, n_chunks chunks in total; chunk_inst NULL for the single-instance form; skipped
// when coeff_digits is false: a previous launch on the stream made them), then the fused kernel
// for value kind vk over all items: stream-ordered, no host synchronisation (capturable).
zp_status fused_launch(const FusedArgs& a, int64_t n_inst, const int32_t* chunk_inst, int64_t n_chunks,
                       cudaStream_t stream, int vk = kFusedZ, bool coeff_digits = true);

// F = Z C for one plan with S <= kFusedMaxSets and plan->fused_kpad <= kFusedMaxModes (scratch
// for the coefficient digits from the library's pool).
zp_status fused_series_eval(const zp_plan* plan, const double* r, const double* theta, int64_t P, const double* coeffs,
                            int64_t S, double* out, cudaStream_t stream);

// grad_theta[p] = sum_s G[p][s] (dZ/dtheta C)[p][s] and grad_r[p] likewise with dZ/drho (either
// may be NULL), by the fused kernel's derivative series: the adjoint's point gradients for
// S <= kFusedMaxSets and plan->fused_kpad <= kFusedMaxModes, without the [modes x points]
// matrix H = C G^T.
zp_status fused_point_grads(const zp_plan* plan, const double* r, const double* theta, int64_t P, const double* coeffs,
                            int64_t S, const double* G, double* grad_r, double* grad_theta, cudaStream_t stream);

// Reads and optionally clears the fused kernel's wait-status word (non-zero: a bounded wait
// gave up).
zp_status fused_error_word(unsigned int* value, bool reset);

}  // namespace zp
