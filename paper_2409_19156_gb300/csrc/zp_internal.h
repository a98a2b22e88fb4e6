// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "zernike_gb300.h"

namespace zp {

// Doubles per row of a column's recursion table.  Row layout (index N = Jacobi degree):
//   N >= 2: {A_N, B_N, 2 A_N, W0_N, W1_N, W2_N, W3_N, 0}
//   N = 0, 1: {0, 0, 0, W0, W1, W2, W3, 0} with W_k = k!
// Two header rows precede row N = 0 and hold the seed constants:
//   header[k]     = binom(m, k)                 (k = 0..3)  -> Taylor coefficients of rho^m
//   header[4 + k] = (m+2) binom(m+2, k)                      -> of (m+2) rho^(m+2)
//   header[8 + k] = (m+1) binom(m, k)                        -> of (m+1) rho^m
constexpr int kRow = 8;
constexpr int kHeaderRows = 2;

// One |m| column of a plan: the recursion walks N = 0 .. n_steps-1.
struct Column {
  int32_t m;          // |m| (the Jacobi alpha)
  int32_t n_steps;    // N_max + 1
  int32_t table_row;  // first header row of this column in the table (rows of kRow doubles)
  int32_t slot_base;  // index of (column, N = 0) in slot_ptr
};

// Step descriptor of the split-precision basis, one per table row (header rows unused):
//   .x = number of slots of the step | (sin flags of its first 24 slots << 8), or
//        kStepIrregular when the step has more than 24 slots (then slot_idx is read);
//   .y = bits of the float32 weight W0_N (the float64 value truncated toward zero).
constexpr uint32_t kStepIrregular = 255u;
constexpr int kStepMaxFlags = 24;
constexpr int kPlanSections = 9;

// Contraction layout of the fused float64-accurate series: the columns are dealt to
// kFusedStreams streams (that many producer threads per point); a column's outputs fill whole
// 8-value units (16-byte operand units, zero padded), and unit j of stream s is the global unit
// kFusedStreams j + s (four global units per 32-position stage).  Per column
// (int4): x = kind | (sin flag of the step's first output) << 8 | (of its second) << 9 (kind 1:
// every step has one output, kind 2: every step has two outputs in the same cos/sin order,
// kind 0: anything else), y = stream, z = first unit within the stream, w = number of outputs.
// The columns of stream 0, then of stream 1, ..., in walk order, follow the n_columns records.
constexpr int kFusedKindGeneric = 0, kFusedKindOne = 1, kFusedKindTwo = 2;
constexpr int kFusedStreams = 3;

// float32 bits of a float64 given as its high and low words, by truncating the significand:
// magnitudes below the float32 normal range give a signed zero, finite ones above it
// infinity; infinities are kept and NaNs stay NaNs (quiet).  Integer operations only.
__host__ __device__ inline uint32_t trunc_float_bits(uint32_t hi, uint32_t lo) {
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {
    // Bits 31..23 of t hold the low 9 exponent bits; subtracting 0x180 there rebiases
    // 1023 -> 127 for every exponent of the float32 normal range.
    const uint32_t t = (hi << 3) | (lo >> 29);
    return (t - 0xC0000000u) | sign;
  }
  if (e == 0x7ffu) return sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
  return e <= 896u ? sign : (sign | 0x7f800000u);
}

struct DevicePlanTables {
  Column* cols = nullptr;
  double* table = nullptr;
  int32_t* slot_ptr = nullptr;  // [total_steps + n_columns]: CSR offsets per (column, N)
  int32_t* slot_idx = nullptr;  // output column j, bit 31 set for the sin (m < 0) factor
  int32_t* mode_col = nullptr;  // [n_modes]: column index of every mode
  int32_t* mode_N = nullptr;    // [n_modes]: Jacobi degree of every mode
  uint2* split_step = nullptr;  // [table rows]: step descriptors of the split basis
  int4* fused_col = nullptr;    // [columns]: fused contraction layout (see kFusedKind*)
  int32_t* fused_kperm = nullptr;  // [fused_kpad]: slot of every K position, -1 for padding
};

}  // namespace zp

struct zp_plan {
  int device = 0;
  int64_t n_modes = 0;
  int32_t n_max = 0;
  int32_t max_steps = 0;
  std::vector<int32_t> n, m;
  std::vector<zp::Column> cols;      // ordered by n_steps, longest first
  std::vector<double> table;         // rows of kRow doubles
  std::vector<int32_t> slot_ptr, slot_idx, mode_col, mode_N;
  std::vector<uint32_t> split_step;  // 2 words per table row
  std::vector<int32_t> fused_col;    // 4 words per column, then the streams' column lists
  std::vector<int32_t> fused_kperm;
  int64_t fused_kpad = 0;            // K positions of the fused layout (multiple of 32)
  int32_t fused_ncols[zp::kFusedStreams] = {};  // columns per stream
  int32_t fused_units = 0;  // global 8-value units G of the layout (whole 4-unit stages); stream s owns (G - s + S - 1) / S
  int32_t fused_ep = 1;              // row scale exponent of the fused kernel on the unit disc
  zp::DevicePlanTables dev;
  size_t device_bytes = 0;
  void* dev_block = nullptr;  // single allocation backing dev.*
};

namespace zp {

// Error plumbing: set_error stores a message for zp_last_error and returns the status.
zp_status set_error(zp_status s, const std::string& msg);
zp_status cuda_error(cudaError_t e, const char* what);
void clear_error();

// Host-side plan construction (validation, grouping, tables, upload).
zp_status build_plan(const int32_t* n, const int32_t* m, int64_t n_modes, zp_plan** out);
// Host half only: validates and fills the host tables of *p (no device memory touched).
zp_status build_plan_host(const int32_t* n, const int32_t* m, int64_t n_modes, zp_plan* p);
// Byte size of the plan's device tables; offsets[0..8] of cols, table, slot_ptr, slot_idx,
// mode_col, mode_N, split_step, fused_col, fused_kperm inside that block (256-byte aligned
// sections).
size_t plan_device_layout(const zp_plan* p, size_t offsets[kPlanSections]);
// Points p->dev at `base` (laid out as plan_device_layout) and copies the host tables there,
// with cudaMemcpyAsync on `stream` when async, else synchronously.
zp_status plan_upload(zp_plan* p, void* base, cudaStream_t stream, bool async);
// Cached plan for a mode list on the current device (created on first use).  The caller
// keeps *out alive while it uses the plan; the cache may drop its own reference.
zp_status cached_plan(const int32_t* n, const int32_t* m, int64_t n_modes, std::shared_ptr<const zp_plan>* out);
zp_status check_plan_device(const zp_plan* plan);

// Kernel launchers (zp_walk.cu).
// phase_ms: NULL, or [2] receiving the device time of the point preparation and of the walk
// (events around each launch; the stream is synchronised).  rowmax: NULL, or (a walk of Z:
// theta given, max_deriv 0) [modes] words, zeroed by the caller, receiving each output row's
// largest |value| high word << 32.
zp_status launch_walk(const zp_plan* plan, const double* r, const double* theta, int64_t n_points,
                      int max_deriv, double* out, double* out_dtheta, cudaStream_t stream,
                      float* phase_ms = nullptr, unsigned long long* rowmax = nullptr);
zp_status launch_per_mode(const zp_plan* plan, const double* r, int64_t n_points, double* out,
                          cudaStream_t stream);

}  // namespace zp
