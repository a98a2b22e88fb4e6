// Batched series over many instances of uneven size (different mode lists and point counts)
// in one persistent launch per pass, capturable in a CUDA graph.
//
// Forward (one launch): batched_point_kernel<FWD64|FWD32>.  Work items are tiles of TP
// consecutive points of one instance, ordered by cost (modes per point) and handed out
// through an atomic counter; one thread per point walks every |m| column of its instance's
// plan (the float64 Jacobi recursion of Sec. 2 in Algorithm 1's column order, cos/sin(m theta)
// by angle addition between consecutive columns) and accumulates F[p, s] += Z_j C[j, s] for
// up to 16 sets in registers (float64 DFMA, or float32 FFMA on a float32 copy of C).
// Adjoint (two launches): batched_point_kernel<ADJ> accumulates grad_r and grad_theta in
// float64 (H_j = sum_s G[p, s] C[j, s] formed on the fly, dZ/drho from the recursion's own
// derivative lane); batched_column_kernel<PPT> forms grad_C[j, s] = sum_p Z_j(p) G[p, s] with
// one item per (instance, |m| column): each thread sums PPT points locally, each warp
// reduces with a butterfly reduce-scatter of shuffles, warps accumulate into shared memory in
// a fixed order, so the result is deterministic (no floating-point atomics).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "zp_device.cuh"
#include "zp_api_common.h"
#include "zp_fused.h"
#include "zp_series_internal.h"

namespace zp {
namespace {

constexpr int kSC = 16;  // sets per register chunk

struct InstanceDesc {
  const Column* cols;
  const double* table;
  const int32_t* slot_ptr;
  const int32_t* slot_idx;
  int32_t n_cols;
  int32_t max_col_slots;
  int64_t J, P;
  const double* r;
  const double* theta;
  const double* coeffs;   // [J][S] float64
  const float* coeffs32;  // [J][S] float32 copy (FP32 forward), in the batch's buffer
  void* out;              // [P][S]
  const double* grad_out; // [P][S]
  double* grad_coeffs;    // [J][S]
  double* grad_r;
  double* grad_theta;
};

struct PointItem {
  int32_t inst;
  int32_t count;
  int64_t p0;
};

struct ColumnItem {
  int32_t inst;
  int32_t col;
};

enum Mode { FWD64 = 0, FWD32 = 1, ADJ = 2 };

struct BatchArgs {
  const InstanceDesc* inst;
  const PointItem* pitems;
  const ColumnItem* citems;
  int64_t n_pitems, n_citems;
  int* counters;  // [2]: point items, column items
  int64_t S;
  int64_t item_base;  // per-instance launches: first item of the range
  int64_t item_end;   // exclusive end of the range (n_pitems for the persistent launch)
  int persistent;
};

// One point of one instance: forward (F row) or the point part of the adjoint.
template <int MODE>
__device__ void point_work(const InstanceDesc& d, int64_t p, int64_t S) {
  const double rho = d.r[p], th = d.theta[p], u = rho * rho;
  double s1, c1;
  sincos(th, &s1, &c1);
  for (int64_t s0 = 0; s0 < S; s0 += kSC) {
    const int sc = (int)(S - s0 < (int64_t)kSC ? S - s0 : (int64_t)kSC);
    double acc[kSC];
    float accf[kSC];
    double G[kSC];
#pragma unroll
    for (int i = 0; i < kSC; ++i) {
      acc[i] = 0.0;
      accf[i] = 0.0f;
      G[i] = 0.0;
    }
    if constexpr (MODE == ADJ) {
#pragma unroll
      for (int i = 0; i < kSC; ++i)
        if (i < sc) G[i] = d.grad_out[p * S + s0 + i];
    }
    double acc_r = 0.0, acc_t = 0.0;
    double cm = 1.0, sm = 0.0, pm = 1.0, pm1 = 0.0;
    int m_prev = 0;
    for (int c = 0; c < d.n_cols; ++c) {
      const Column col = d.cols[c];
      const int m = col.m;
      if (m == m_prev + 1) {
        const double cn = fma(cm, c1, -sm * s1);
        const double sn = fma(sm, c1, cm * s1);
        cm = cn;
        sm = sn;
        pm1 = pm;
        pm *= rho;
      } else if (m != m_prev || c == 0) {
        if (m != 0) {
          sincos((double)m * th, &sm, &cm);
        } else {
          cm = 1.0;
          sm = 0.0;
        }
        pm1 = m >= 1 ? pow_uint(rho, m - 1) : 0.0;
        pm = m >= 1 ? pm1 * rho : 1.0;
      }
      m_prev = m;
      const double* h = d.table + (size_t)col.table_row * kRow;
      const int32_t* sp = d.slot_ptr + col.slot_base;
      // Taylor lanes 0 (value) and 1 (d/drho, adjoint only) of Q_0 and Q_1.
      double T0 = pm, S0 = fma(h[4], pm * u, -(h[8] * pm));
      double T1 = 0.0, S1 = 0.0;
      if constexpr (MODE == ADJ) {
        T1 = h[1] * pm1;
        S1 = fma(h[5], pm * rho, -(h[9] * pm1));
      }
      const double md = (double)m;
      for (int N = 0; N < col.n_steps; ++N) {
        const double* row = h + (size_t)(kHeaderRows + N) * kRow;
        double q0, q1 = 0.0;
        if (N == 0) {
          q0 = T0;
          q1 = T1;
        } else if (N == 1) {
          q0 = S0;
          q1 = S1;
        } else {
          const double g = fma(row[0], u, -row[1]);
          const double n0 = fma(g, S0, -T0);
          T0 = S0;
          S0 = n0;
          q0 = n0;
          if constexpr (MODE == ADJ) {
            const double n1 = fma(g, S1, fma(row[2] * rho, T0, -T1));
            T1 = S1;
            S1 = n1;
            q1 = n1;
          }
        }
        const int sb = sp[N], se = sp[N + 1];
        if (sb == se) continue;
        const double R0 = row[3] * q0;
        if constexpr (MODE == FWD64) {
          for (int s = sb; s < se; ++s) {
            const uint32_t code = (uint32_t)__ldg(d.slot_idx + s);
            const int64_t j = (int64_t)(code & 0x7fffffffu);
            const double z = R0 * ((code >> 31) ? sm : cm);
            const double* cr = d.coeffs + j * S + s0;
#pragma unroll
            for (int i = 0; i < kSC; ++i)
              if (i < sc) acc[i] = fma(z, __ldg(cr + i), acc[i]);
          }
        } else if constexpr (MODE == FWD32) {
          const float Rf = (float)R0;
          const float cf = (float)cm, sf = (float)sm;
          for (int s = sb; s < se; ++s) {
            const uint32_t code = (uint32_t)__ldg(d.slot_idx + s);
            const int64_t j = (int64_t)(code & 0x7fffffffu);
            const float z = Rf * ((code >> 31) ? sf : cf);
            const float* cr = d.coeffs32 + j * S + s0;
#pragma unroll
            for (int i = 0; i < kSC; ++i)
              if (i < sc) accf[i] = fmaf(z, __ldg(cr + i), accf[i]);
          }
        } else {
          const double R1 = row[4] * q1;
          for (int s = sb; s < se; ++s) {
            const uint32_t code = (uint32_t)__ldg(d.slot_idx + s);
            const int64_t j = (int64_t)(code & 0x7fffffffu);
            const bool is_sin = (code >> 31) != 0;
            const double* cr = d.coeffs + j * S + s0;
            double hv = 0.0;
#pragma unroll
            for (int i = 0; i < kSC; ++i)
              if (i < sc) hv = fma(G[i], __ldg(cr + i), hv);
            const double f = is_sin ? sm : cm;
            const double dt = is_sin ? md * cm : -md * sm;
            acc_r = fma(R1 * f, hv, acc_r);
            acc_t = fma(R0 * dt, hv, acc_t);
          }
        }
      }
    }
    if constexpr (MODE == FWD64) {
      double* o = (double*)d.out + p * S + s0;
#pragma unroll
      for (int i = 0; i < kSC; ++i)
        if (i < sc) o[i] = acc[i];
    } else if constexpr (MODE == FWD32) {
      float* o = (float*)d.out + p * S + s0;
#pragma unroll
      for (int i = 0; i < kSC; ++i)
        if (i < sc) o[i] = accf[i];
    } else {
      // grad_r / grad_theta sum over all sets: chunks accumulate in place.
      if (d.grad_r) d.grad_r[p] = (s0 == 0 ? 0.0 : d.grad_r[p]) + acc_r;
      if (d.grad_theta) d.grad_theta[p] = (s0 == 0 ? 0.0 : d.grad_theta[p]) + acc_t;
    }
  }
}

template <int MODE>
__global__ void batched_point_kernel(BatchArgs a) {
  __shared__ int64_t s_item;
  for (int64_t it = 0;; ++it) {
    int64_t item;
    if (a.persistent) {
      if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(&a.counters[0], 1);
      __syncthreads();
      item = s_item;
      __syncthreads();
    } else {
      item = a.item_base + blockIdx.x + it * gridDim.x;
    }
    if (item >= a.item_end) break;
    const PointItem w = a.pitems[item];
    if ((int)threadIdx.x < w.count) point_work<MODE>(a.inst[w.inst], w.p0 + threadIdx.x, a.S);
  }
}

// Reduce-scatter of 16 doubles across the warp: afterwards lane l holds the warp sum of value
// idx(l) = 8*b4 + 4*b3 + 2*b2 + b1 (b_k = bit k of l); lanes l and l^1 hold the same value.
__device__ __forceinline__ double warp_reduce_scatter16(double (&v)[16], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const double send = b4 ? v[i] : v[i + 8];
    const double keep = b4 ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double send = b3 ? v[i] : v[i + 4];
    const double keep = b3 ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double send = b2 ? v[i] : v[i + 2];
    const double keep = b2 ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const double send = b1 ? v[0] : v[1];
    const double keep = b1 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// grad_C for one (instance, column) item per iteration.  Shared memory: per warp,
// max_col_slots x 16 doubles of running sums.
template <int PPT>
__global__ void batched_column_kernel(BatchArgs a, int max_slots) {
  extern __shared__ double wsum[];  // [warps][max_slots][16]
  __shared__ int64_t s_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int vidx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
  for (;;) {
    if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(&a.counters[1], 1);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();
    if (item >= a.n_citems) break;
    const ColumnItem w = a.citems[item];
    const InstanceDesc d = a.inst[w.inst];
    if (!d.grad_coeffs) continue;  // uniform across the block
    const Column col = d.cols[w.col];
    const int m = col.m;
    const double* h = d.table + (size_t)col.table_row * kRow;
    const int32_t* sp = d.slot_ptr + col.slot_base;
    const int slot0 = sp[0];
    const int nslots = sp[col.n_steps] - slot0;
    const int64_t S = a.S;
    for (int64_t s0 = 0; s0 < S; s0 += kSC) {
      const int sc = (int)(S - s0 < (int64_t)kSC ? S - s0 : (int64_t)kSC);
      for (int i = threadIdx.x; i < nwarps * max_slots * kSC; i += blockDim.x) wsum[i] = 0.0;
      __syncthreads();
      double* mysum = wsum + (size_t)warp * max_slots * kSC;
      for (int64_t pbase = 0; pbase < d.P; pbase += (int64_t)blockDim.x * PPT) {
        // Per thread: PPT points pbase + threadIdx.x + k * blockDim.x.
        double rho[PPT], u[PPT], cm[PPT], sm[PPT], T[PPT], Sx[PPT], G[PPT][kSC];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const int64_t p = pbase + threadIdx.x + (int64_t)k * blockDim.x;
          const bool valid = p < d.P;
          rho[k] = valid ? d.r[p] : 0.0;
          u[k] = rho[k] * rho[k];
          const double th = valid ? d.theta[p] : 0.0;
          if (m != 0) {
            sincos((double)m * th, &sm[k], &cm[k]);
          } else {
            cm[k] = 1.0;
            sm[k] = 0.0;
          }
          if (!valid) {
            cm[k] = 0.0;  // invalid points contribute nothing
            sm[k] = 0.0;
          }
          const double pm = pow_uint(rho[k], m);
          T[k] = pm;
          Sx[k] = fma(h[4], pm * u[k], -(h[8] * pm));
#pragma unroll
          for (int i = 0; i < kSC; ++i) G[k][i] = (valid && i < sc) ? d.grad_out[p * S + s0 + i] : 0.0;
        }
        for (int N = 0; N < col.n_steps; ++N) {
          const double* row = h + (size_t)(kHeaderRows + N) * kRow;
          double q[PPT];
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            if (N == 0) {
              q[k] = T[k];
            } else if (N == 1) {
              q[k] = Sx[k];
            } else {
              const double g = fma(row[0], u[k], -row[1]);
              const double nq = fma(g, Sx[k], -T[k]);
              T[k] = Sx[k];
              Sx[k] = nq;
              q[k] = nq;
            }
          }
          const int sb = sp[N], se = sp[N + 1];
          double rq[PPT];  // R = w_N Q, shared by the step's outputs
#pragma unroll
          for (int k = 0; k < PPT; ++k) rq[k] = row[3] * q[k];
          for (int s = sb; s < se; ++s) {
            const uint32_t code = (uint32_t)__ldg(d.slot_idx + s);
            const bool is_sin = (code >> 31) != 0;
            double v[kSC];
#pragma unroll
            for (int i = 0; i < kSC; ++i) v[i] = 0.0;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
              const double z = rq[k] * (is_sin ? sm[k] : cm[k]);
#pragma unroll
              for (int i = 0; i < kSC; ++i) v[i] = fma(z, G[k][i], v[i]);
            }
            const double tot = warp_reduce_scatter16(v, lane);
            if ((lane & 1) == 0) mysum[(size_t)(s - slot0) * kSC + vidx] += tot;
          }
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nslots * kSC; i += blockDim.x) {
        const int sl = i / kSC, si = i % kSC;
        if (si >= sc) continue;
        double tot = 0.0;
        for (int wv = 0; wv < nwarps; ++wv) tot += wsum[(size_t)wv * max_slots * kSC + i];
        const uint32_t code = (uint32_t)__ldg(d.slot_idx + slot0 + sl);
        const int64_t j = (int64_t)(code & 0x7fffffffu);
        d.grad_coeffs[j * S + s0 + si] = tot;
      }
      __syncthreads();
    }
  }
}

// float32 copies of every instance's coefficients (blockIdx.y = instance).
__global__ void to_float_kernel(const InstanceDesc* __restrict__ inst, int64_t S) {
  const InstanceDesc d = inst[blockIdx.y];
  float* dst = const_cast<float*>(d.coeffs32);
  const int64_t n = d.J * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)d.coeffs[i];
}

}  // namespace
}  // namespace zp

// ----------------------------------------------------------------------------------- host
struct zp_batch {
  int device = 0;
  int64_t n_sets = 0;
  std::vector<zp_instance> inst;          // caller's descriptors (pointers captured)
  std::vector<std::unique_ptr<zp_plan>> plans;
  std::vector<int32_t> inst_plan;         // plan index per instance
  std::vector<zp::InstanceDesc> desc;
  std::vector<size_t> coeff32_off;        // offset (floats) of each instance's float32 coefficients
  int64_t coeff32_total = 0;
  void* dev_block = nullptr;              // plan tables + descriptors + items + counters + float32 C
  zp::InstanceDesc* d_desc = nullptr;
  zp::PointItem* d_pitems = nullptr;
  zp::ColumnItem* d_citems = nullptr;
  int* d_counters = nullptr;
  float* d_coeff32 = nullptr;
  int64_t n_pitems = 0, n_citems = 0, max_pitems = 0;
  int max_col_slots = 1;
  // launch configuration (autotuned): point-tile size, CTAs per SM, column-kernel PPT/threads.
  // Untuned: 8 CTAs per SM (batched_512 float32 forward 93 ms against 125 ms with 4; the float64
  // forward is the same with either).
  int tp = 128, ctas_per_sm = 8, col_ppt = 2, col_threads = 128;
  std::vector<int64_t> inst_item_begin, inst_item_end;  // point items per instance
  // Fused float64-accurate forward on the tensor cores (ZP_PREC_FP64_EMULATED), available when
  // n_sets <= 16 and every instance has at most 5041 modes: instance descriptors, 128-point
  // items ordered by cost, the instance of every 32-mode chunk, coefficient digits and scales.
  bool fused_ok = false;
  void* fused_block = nullptr;
  zp::FusedInst* d_finst = nullptr;
  // The adjoint's point gradients by the same kernel: [n] descriptors of the theta-derivative
  // series (dot with grad_out into grad_theta), then [n] of the rho-derivative (into grad_r).
  zp::FusedInst* d_fadj = nullptr;
  zp::FusedItem* d_fitems = nullptr;
  int32_t* d_fchunk = nullptr;
  int64_t n_fitems = 0, n_fchunks = 0;
  int fused_ndig = zp::kFusedDigits;  // digits per value of the fused launches (the longest instance's)
};

namespace zp {
namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

zp_status build_point_items(zp_batch* b, cudaStream_t stream) {
  std::vector<std::pair<int64_t, int32_t>> order;  // (cost, instance)
  for (size_t i = 0; i < b->inst.size(); ++i) order.push_back({b->inst[i].n_modes, (int32_t)i});
  std::stable_sort(order.begin(), order.end(), [](auto& x, auto& y) { return x.first > y.first; });
  std::vector<PointItem> items;
  b->inst_item_begin.assign(b->inst.size(), 0);
  b->inst_item_end.assign(b->inst.size(), 0);
  for (auto& pr : order) {
    const int32_t i = pr.second;
    b->inst_item_begin[i] = (int64_t)items.size();
    const int64_t P = b->inst[i].n_points;
    if (b->inst[i].n_modes > 0)
      for (int64_t p0 = 0; p0 < P; p0 += b->tp) items.push_back(PointItem{i, (int32_t)std::min<int64_t>(b->tp, P - p0), p0});
    b->inst_item_end[i] = (int64_t)items.size();
  }
  if ((int64_t)items.size() > b->max_pitems) return set_error(ZP_ERR_INVALID_ARG, "tile size below the minimum");
  b->n_pitems = (int64_t)items.size();
  if (!items.empty()) {
    cudaError_t e = cudaMemcpyAsync(b->d_pitems, items.data(), items.size() * sizeof(PointItem),
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_error(e, "copy of work items");
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  }
  return ZP_OK;
}

// Dynamic shared memory of the column kernel for the largest thread count the tuner tries.
zp_status set_column_attributes(const zp_batch* b) {
  const size_t smem = (size_t)(512 / 32) * b->max_col_slots * kSC * sizeof(double);
  const int v = (int)std::min<size_t>(smem, 200 * 1024);
  cudaError_t e = cudaFuncSetAttribute(batched_column_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batched_column_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batched_column_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "cudaFuncSetAttribute(batched_column_kernel)");
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

BatchArgs make_args(const zp_batch* b) {
  BatchArgs a;
  a.inst = b->d_desc;
  a.pitems = b->d_pitems;
  a.citems = b->d_citems;
  a.n_pitems = b->n_pitems;
  a.n_citems = b->n_citems;
  a.counters = b->d_counters;
  a.S = b->n_sets;
  a.item_base = 0;
  a.item_end = b->n_pitems;
  a.persistent = 1;
  return a;
}

template <int MODE>
zp_status launch_points(const zp_batch* b, cudaStream_t st) {
  BatchArgs a = make_args(b);
  cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(counter)");
  const int64_t grid = std::min<int64_t>(std::max<int64_t>(b->n_pitems, 1), (int64_t)sm_count() * b->ctas_per_sm);
  batched_point_kernel<MODE><<<(unsigned)grid, b->tp, 0, st>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "batched_point_kernel launch");
}

zp_status launch_columns(const zp_batch* b, cudaStream_t st) {
  BatchArgs a = make_args(b);
  cudaError_t e = cudaMemsetAsync(b->d_counters + 1, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(counter)");
  const int warps = b->col_threads / 32;
  const size_t smem = (size_t)warps * b->max_col_slots * kSC * sizeof(double);
  if (smem > 200 * 1024) return set_error(ZP_ERR_UNSUPPORTED, "too many duplicated modes in one |m| column");
  const int64_t grid = std::min<int64_t>(std::max<int64_t>(b->n_citems, 1), (int64_t)sm_count() * 4);
  auto go = [&](auto kern) { kern<<<(unsigned)grid, b->col_threads, smem, st>>>(a, b->max_col_slots); };
  switch (b->col_ppt) {
    case 1: go(batched_column_kernel<1>); break;
    case 2: go(batched_column_kernel<2>); break;
    default: go(batched_column_kernel<4>); break;
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "batched_column_kernel launch");
}

// Descriptors, items and buffers of the fused forward (see zp_batch::fused_ok).
zp_status build_fused(zp_batch* b) {
  if (b->n_sets > kFusedMaxSets || b->n_sets == 0) return ZP_OK;
  int64_t kpad_max = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    if (b->plans[b->inst_plan[i]]->fused_kpad > kFusedMaxModes) return ZP_OK;
    if (b->inst[i].n_modes > 0) kpad_max = std::max(kpad_max, b->plans[b->inst_plan[i]]->fused_kpad);
  }
  b->fused_ndig = fused_digits_for(kpad_max);
  const int64_t n = (int64_t)b->inst.size();
  std::vector<FusedInst> fi(n);
  std::vector<int32_t> chunk_inst;
  std::vector<std::pair<int64_t, int32_t>> order;  // (modes, instance): costliest tiles first
  int64_t kc_total = 0;
  for (int64_t i = 0; i < n; ++i) {
    const zp_instance& in = b->inst[i];
    const zp_plan* p = b->plans[b->inst_plan[i]].get();
    FusedInst& d = fi[i];
    d.cols = p->dev.cols;
    d.table = p->dev.table;
    d.steps = p->dev.split_step;
    d.slot_ptr = p->dev.slot_ptr;
    d.slot_idx = p->dev.slot_idx;
    d.mode_col = p->dev.mode_col;
    d.mode_N = p->dev.mode_N;
    d.fcols = p->dev.fused_col;
    d.scols = (const int32_t*)(p->dev.fused_col + p->cols.size());
    for (int st = 0; st < kFusedStreams; ++st) d.ncols_s[st] = p->fused_ncols[st];
    d.units = p->fused_units;
    d.ep_disc = p->fused_ep;
    d.kperm = p->dev.fused_kperm;
    d.Kp = in.n_modes > 0 ? p->fused_kpad : 0;
    d.n_cols = (int32_t)p->cols.size();
    d.KC = (int32_t)((d.Kp + 31) / 32);
    d.kc_base = kc_total;
    d.J = in.n_modes;
    d.P = in.n_points;
    d.S = b->n_sets;
    d.r = in.r;
    d.theta = in.theta;
    d.coeffs = in.coeffs;
    d.out = (double*)in.out;
    kc_total += d.KC;
    for (int32_t c = 0; c < d.KC; ++c) chunk_inst.push_back((int32_t)i);
    if (in.n_modes > 0 && in.n_points > 0) order.push_back({in.n_modes, (int32_t)i});
  }
  std::stable_sort(order.begin(), order.end(), [](auto& x, auto& y) { return x.first > y.first; });
  std::vector<FusedItem> items;
  for (auto& o : order)
    for (int64_t t = 0; t * 128 < b->inst[o.second].n_points; ++t) items.push_back(FusedItem{o.second, (int32_t)t});
  const size_t inst_b = align256(std::max<int64_t>(n, 1) * sizeof(FusedInst));
  const size_t adj_b = align256(std::max<int64_t>(2 * n, 1) * sizeof(FusedInst));
  const size_t item_b = align256(std::max<size_t>(items.size(), 1) * sizeof(FusedItem));
  const size_t chunk_b = align256(std::max<int64_t>(kc_total, 1) * sizeof(int32_t));
  const size_t cexp_b = align256(std::max<int64_t>(n, 1) * kFusedMaxSets * sizeof(int));
  const size_t dig_b = (size_t)std::max<int64_t>(kc_total, 1) * kFusedBChunk;
  cudaError_t e = cudaMalloc(&b->fused_block, inst_b + adj_b + item_b + chunk_b + cexp_b + dig_b);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(fused batch)");
  char* base = (char*)b->fused_block;
  int* cexp = (int*)(base + inst_b + adj_b + item_b + chunk_b);
  uint8_t* dig = (uint8_t*)(base + inst_b + adj_b + item_b + chunk_b + cexp_b);
  for (int64_t i = 0; i < n; ++i) {
    fi[i].cexp = cexp + i * kFusedMaxSets;
    fi[i].bdig = dig + (size_t)fi[i].kc_base * kFusedBChunk;
  }
  // Adjoint descriptors: the same instances, the derivative series' row scales, and the row
  // sums with grad_out written into grad_theta / grad_r instead of a series output.
  std::vector<FusedInst> fa(2 * n);
  for (int64_t i = 0; i < n; ++i) {
    const zp_instance& in = b->inst[i];
    const zp_plan* p = b->plans[b->inst_plan[i]].get();
    for (int k = 0; k < 2; ++k) {
      FusedInst& d = fa[k * n + i];
      d = fi[i];
      d.out = nullptr;
      d.gdot = in.grad_out;
      d.dot_out = k == 0 ? in.grad_theta : in.grad_r;
      d.ep_disc = fused_ep_for(p, k == 0 ? kFusedDTheta : kFusedDRho);
    }
  }
  b->d_finst = (FusedInst*)base;
  b->d_fadj = (FusedInst*)(base + inst_b);
  b->d_fitems = (FusedItem*)(base + inst_b + adj_b);
  b->d_fchunk = (int32_t*)(base + inst_b + adj_b + item_b);
  e = cudaMemcpy(b->d_finst, fi.data(), n * sizeof(FusedInst), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(b->d_fadj, fa.data(), 2 * n * sizeof(FusedInst), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->d_fitems, items.data(), items.size() * sizeof(FusedItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && kc_total > 0)
    e = cudaMemcpy(b->d_fchunk, chunk_inst.data(), kc_total * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "copy of fused batch descriptors");
  b->n_fitems = (int64_t)items.size();
  b->n_fchunks = kc_total;
  b->fused_ok = true;
  return ZP_OK;
}

zp_status batch_forward(zp_batch* b, zp_precision prec, cudaStream_t st) {
  if (prec == ZP_PREC_FP64_EMULATED) {
    if (!b->fused_ok)
      return set_error(ZP_ERR_UNSUPPORTED, "the emulated float64 batched forward takes at most 16 sets and 5041 "
                                           "modes per instance");
    FusedArgs a;
    a.insts = b->d_finst;
    a.items = b->d_fitems;
    a.n_items = b->n_fitems;
    a.ndig = b->fused_ndig;
    if (b->n_fitems == 0) return ZP_OK;
    return fused_launch(a, (int64_t)b->inst.size(), b->d_fchunk, b->n_fchunks, st);
  }
  if (b->n_pitems == 0) return ZP_OK;
  if (prec == ZP_PREC_FP32) {
    if (b->coeff32_total > 0) {
      to_float_kernel<<<dim3(16, (unsigned)b->inst.size()), 256, 0, st>>>(b->d_desc, b->n_sets);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "to_float_kernel launch");
    }
    return launch_points<FWD32>(b, st);
  }
  return launch_points<FWD64>(b, st);
}

}  // namespace
}  // namespace zp

using namespace zp;

static zp_status batch_validate_ptrs(const zp_instance& in, int64_t S, int64_t i) {
  const std::string pre = "instance " + std::to_string(i) + ": ";
  if (in.n_modes < 0 || in.n_points < 0) return set_error(ZP_ERR_INVALID_ARG, pre + "negative size");
  if (in.n_points == 0 || in.n_modes == 0) return ZP_OK;
  zp_status st;
  if ((st = check_device_array(in.r, "r", 8)) != ZP_OK) return set_error(st, pre + zp_last_error());
  if ((st = check_device_array(in.theta, "theta", 8)) != ZP_OK) return set_error(st, pre + zp_last_error());
  if (S > 0 && (st = check_device_array(in.coeffs, "coeffs", 8)) != ZP_OK) return set_error(st, pre + zp_last_error());
  struct Opt {
    const void* p;
    const char* name;
  } opts[] = {{in.out, "out"}, {in.grad_out, "grad_out"}, {in.grad_coeffs, "grad_coeffs"}, {in.grad_r, "grad_r"},
              {in.grad_theta, "grad_theta"}};
  for (const Opt& o : opts)
    if (o.p && (st = check_device_array(o.p, o.name, 4)) != ZP_OK) return set_error(st, pre + zp_last_error());
  return ZP_OK;
}

extern "C" {

zp_status zp_batch_create(const zp_instance* instances, int64_t n_instances, int64_t n_sets, zp_batch** out) {
  clear_error();
  if (!out) return set_error(ZP_ERR_INVALID_ARG, "output pointer is NULL");
  if (n_instances < 0 || n_sets < 0) return set_error(ZP_ERR_INVALID_ARG, "negative size");
  if (n_instances > 0 && !instances) return set_error(ZP_ERR_INVALID_ARG, "instances is NULL");
  if (n_instances >= (int64_t(1) << 31)) return set_error(ZP_ERR_INVALID_ARG, "too many instances");
  std::unique_ptr<zp_batch> b(new zp_batch());
  cudaGetDevice(&b->device);
  b->n_sets = n_sets;
  b->inst.assign(instances, instances + n_instances);
  // One plan per distinct mode list (host tables, packed into one device block below).
  std::map<std::pair<std::vector<int32_t>, std::vector<int32_t>>, int32_t> seen;
  for (int64_t i = 0; i < n_instances; ++i) {
    const zp_instance& in = b->inst[i];
    ZP_TRY(batch_validate_ptrs(in, n_sets, i));
    if (in.n_modes > 0 && (!in.n || !in.m)) return set_error(ZP_ERR_INVALID_ARG, "instance mode list is NULL");
    auto key = std::make_pair(std::vector<int32_t>(in.n, in.n + in.n_modes), std::vector<int32_t>(in.m, in.m + in.n_modes));
    auto it = seen.find(key);
    if (it == seen.end()) {
      std::unique_ptr<zp_plan> p(new zp_plan());
      zp_status st = build_plan_host(in.n, in.m, in.n_modes, p.get());
      if (st != ZP_OK) return set_error(st, "instance " + std::to_string(i) + ": " + zp_last_error());
      it = seen.emplace(std::move(key), (int32_t)b->plans.size()).first;
      b->plans.push_back(std::move(p));
    }
    b->inst_plan.push_back(it->second);
  }
  // Device block: plans | descriptors | point items (smallest tile 32) | column items | counters | float32 C.
  std::vector<size_t> plan_off;
  size_t off = 0;
  for (auto& p : b->plans) {
    size_t o6[kPlanSections];
    plan_off.push_back(off);
    off += align256(plan_device_layout(p.get(), o6));
  }
  const size_t desc_off = off;
  off += align256(std::max<int64_t>(n_instances, 1) * sizeof(InstanceDesc));
  int64_t max_items = 0, n_citems = 0;
  for (auto& in : b->inst) {
    max_items += (in.n_points + 31) / 32;
  }
  for (int64_t i = 0; i < n_instances; ++i)
    if (b->inst[i].n_points > 0 && b->inst[i].n_modes > 0) n_citems += (int64_t)b->plans[b->inst_plan[i]]->cols.size();
  b->max_pitems = max_items;
  const size_t pitem_off = off;
  off += align256(std::max<int64_t>(max_items, 1) * sizeof(PointItem));
  const size_t citem_off = off;
  off += align256(std::max<int64_t>(n_citems, 1) * sizeof(ColumnItem));
  const size_t counter_off = off;
  off += 256;
  const size_t c32_off = off;
  for (auto& in : b->inst) {
    b->coeff32_off.push_back((size_t)b->coeff32_total);
    b->coeff32_total += in.n_modes * n_sets;
  }
  off += align256(std::max<int64_t>(b->coeff32_total, 1) * sizeof(float));
  cudaError_t e = cudaMalloc(&b->dev_block, off);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(batch)");
  char* base = (char*)b->dev_block;
  for (size_t k = 0; k < b->plans.size(); ++k) {
    zp_status st = plan_upload(b->plans[k].get(), base + plan_off[k], nullptr, false);
    if (st != ZP_OK) {
      cudaFree(b->dev_block);
      return st;
    }
  }
  b->d_desc = (InstanceDesc*)(base + desc_off);
  b->d_pitems = (PointItem*)(base + pitem_off);
  b->d_citems = (ColumnItem*)(base + citem_off);
  b->d_counters = (int*)(base + counter_off);
  b->d_coeff32 = (float*)(base + c32_off);
  // Descriptors and column items.
  std::vector<std::pair<int64_t, ColumnItem>> citems;
  for (int64_t i = 0; i < n_instances; ++i) {
    const zp_instance& in = b->inst[i];
    const zp_plan* p = b->plans[b->inst_plan[i]].get();
    InstanceDesc d{};
    d.cols = p->dev.cols;
    d.table = p->dev.table;
    d.slot_ptr = p->dev.slot_ptr;
    d.slot_idx = p->dev.slot_idx;
    d.n_cols = (int32_t)p->cols.size();
    d.J = in.n_modes;
    d.P = in.n_points;
    d.r = in.r;
    d.theta = in.theta;
    d.coeffs = in.coeffs;
    d.coeffs32 = b->d_coeff32 + b->coeff32_off[i];
    d.out = in.out;
    d.grad_out = in.grad_out;
    d.grad_coeffs = in.grad_coeffs;
    d.grad_r = in.grad_r;
    d.grad_theta = in.grad_theta;
    int32_t mx = 1;
    for (size_t c = 0; c < p->cols.size(); ++c) {
      const Column& col = p->cols[c];
      const int32_t ns = p->slot_ptr[col.slot_base + col.n_steps] - p->slot_ptr[col.slot_base];
      mx = std::max(mx, ns);
      if (in.n_points > 0 && in.n_modes > 0)
        citems.push_back({(int64_t)in.n_points * (col.n_steps + 2 * ns), ColumnItem{(int32_t)i, (int32_t)c}});
    }
    d.max_col_slots = mx;
    b->max_col_slots = std::max(b->max_col_slots, (int)mx);
    b->desc.push_back(d);
  }
  std::stable_sort(citems.begin(), citems.end(), [](auto& x, auto& y) { return x.first > y.first; });
  std::vector<ColumnItem> cit;
  for (auto& c : citems) cit.push_back(c.second);
  b->n_citems = (int64_t)cit.size();
  if (!b->desc.empty())
    e = cudaMemcpy(b->d_desc, b->desc.data(), b->desc.size() * sizeof(InstanceDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !cit.empty())
    e = cudaMemcpy(b->d_citems, cit.data(), cit.size() * sizeof(ColumnItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(b->dev_block);
    return cuda_error(e, "copy of batch descriptors");
  }
  zp_status st = build_point_items(b.get(), nullptr);
  if (st == ZP_OK) st = set_column_attributes(b.get());
  if (st == ZP_OK) st = build_fused(b.get());
  if (st != ZP_OK) {
    cudaFree(b->dev_block);
    if (b->fused_block) cudaFree(b->fused_block);
    return st;
  }
  *out = b.release();
  return ZP_OK;
}

zp_status zp_batch_destroy(zp_batch* b) {
  clear_error();
  if (!b) return set_error(ZP_ERR_INVALID_ARG, "batch is NULL");
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->dev_block) cudaFree(b->dev_block);
  if (b->fused_block) cudaFree(b->fused_block);
  cudaSetDevice(cur);
  delete b;
  return ZP_OK;
}

static zp_status zp_batch_forward_impl(zp_batch* b, zp_precision prec, void* stream) {
  clear_error();
  if (!b) return set_error(ZP_ERR_INVALID_ARG, "batch is NULL");
  if (prec != ZP_PREC_FP64 && prec != ZP_PREC_FP32 && prec != ZP_PREC_FP64_EMULATED)
    return set_error(ZP_ERR_INVALID_ARG,
                     "batched forward supports ZP_PREC_FP64_EMULATED, ZP_PREC_FP64 and ZP_PREC_FP32");
  for (size_t i = 0; i < b->inst.size(); ++i)
    if (b->inst[i].n_points > 0 && b->n_sets > 0 && !b->inst[i].out)
      return set_error(ZP_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": out is NULL");
  return batch_forward(b, prec, (cudaStream_t)stream);
}

zp_status zp_batch_forward(zp_batch* b, zp_precision prec, void* stream) {
  zp::NvtxRange zp_range_("zp_batch_forward");
  return zp::entry_finish("zp_batch_forward", stream, zp_batch_forward_impl(b, prec, stream));
}

static zp_status zp_batch_forward_per_instance_impl(zp_batch* b, zp_precision prec, void* stream) {
  clear_error();
  if (!b) return set_error(ZP_ERR_INVALID_ARG, "batch is NULL");
  if (prec != ZP_PREC_FP64) return set_error(ZP_ERR_INVALID_ARG, "per-instance comparison runs float64 only");
  cudaStream_t st = (cudaStream_t)stream;
  BatchArgs a = make_args(b);
  a.persistent = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    const int64_t n = b->inst_item_end[i] - b->inst_item_begin[i];
    if (n <= 0) continue;
    a.item_base = b->inst_item_begin[i];
    a.item_end = b->inst_item_end[i];
    batched_point_kernel<FWD64><<<(unsigned)n, b->tp, 0, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ZP_OK : cuda_error(e, "per-instance launches");
}

zp_status zp_batch_forward_per_instance(zp_batch* b, zp_precision prec, void* stream) {
  zp::NvtxRange zp_range_("zp_batch_forward_per_instance");
  return zp::entry_finish("zp_batch_forward_per_instance", stream, zp_batch_forward_per_instance_impl(b, prec, stream));
}

static zp_status zp_batch_adjoint_impl(zp_batch* b, zp_precision prec, void* stream) {
  clear_error();
  if (!b) return set_error(ZP_ERR_INVALID_ARG, "batch is NULL");
  if (prec != ZP_PREC_FP64 && prec != ZP_PREC_FP64_EMULATED)
    return set_error(ZP_ERR_INVALID_ARG, "batched adjoint supports ZP_PREC_FP64 and ZP_PREC_FP64_EMULATED");
  cudaStream_t st = (cudaStream_t)stream;
  bool need_pt = false, need_c = false;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    const zp_instance& in = b->inst[i];
    if (in.n_points > 0 && in.n_modes > 0 && b->n_sets > 0 && !in.grad_out)
      return set_error(ZP_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": grad_out is NULL");
    need_pt |= in.grad_r || in.grad_theta;
    need_c |= in.grad_coeffs != nullptr;
  }
  // Instances with no modes or no points: zero what exists (empty sums).
  for (size_t i = 0; i < b->inst.size(); ++i) {
    const zp_instance& in = b->inst[i];
    cudaError_t e = cudaSuccess;
    if (in.n_modes == 0 || b->n_sets == 0) {
      if (in.grad_r && in.n_points) e = cudaMemsetAsync(in.grad_r, 0, in.n_points * 8, st);
      if (e == cudaSuccess && in.grad_theta && in.n_points) e = cudaMemsetAsync(in.grad_theta, 0, in.n_points * 8, st);
    }
    if (e == cudaSuccess && in.grad_coeffs && in.n_modes && b->n_sets && in.n_points == 0)
      e = cudaMemsetAsync(in.grad_coeffs, 0, in.n_modes * b->n_sets * 8, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
  }
  if (b->n_sets == 0) return ZP_OK;
  if (need_pt && prec == ZP_PREC_FP64_EMULATED && b->fused_ok) {
    // grad_theta[p] = sum_s G[p][s] (dZ/dtheta C)[p][s] and grad_r likewise with dZ/drho: the
    // fused tensor-core kernel for the two derivative series, each row sum formed in its drain
    // and added onto the zeroed gradients.
    bool need_t = false, need_r = false;
    for (size_t i = 0; i < b->inst.size(); ++i) {
      const zp_instance& in = b->inst[i];
      if (in.n_points == 0 || in.n_modes == 0) continue;
      cudaError_t e = cudaSuccess;
      if (in.grad_theta) e = cudaMemsetAsync(in.grad_theta, 0, in.n_points * 8, st), need_t = true;
      if (e == cudaSuccess && in.grad_r) e = cudaMemsetAsync(in.grad_r, 0, in.n_points * 8, st), need_r = true;
      if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    }
    FusedArgs a;
    a.items = b->d_fitems;
    a.n_items = b->n_fitems;
    a.ndig = b->fused_ndig;
    const int64_t n = (int64_t)b->inst.size();
    bool digits = true;  // the coefficient digits once, for the first pass
    if (need_t) {
      a.insts = b->d_fadj;
      ZP_TRY(fused_launch(a, n, b->d_fchunk, b->n_fchunks, st, kFusedDTheta, digits));
      digits = false;
    }
    if (need_r) {
      a.insts = b->d_fadj + n;
      ZP_TRY(fused_launch(a, n, b->d_fchunk, b->n_fchunks, st, kFusedDRho, digits));
    }
  } else if (need_pt && b->n_pitems) {
    ZP_TRY(launch_points<ADJ>(b, st));
  }
  if (need_c && prec == ZP_PREC_FP64_EMULATED) {
    // grad_C = Z G per instance by the float64-accurate tensor-core GEMM, Z walked into
    // scratch (grad_r and grad_theta above: the point kernel forms H = C G^T on the fly).
    for (size_t i = 0; i < b->inst.size(); ++i) {
      const zp_instance& in = b->inst[i];
      if (in.n_points == 0 || in.n_modes == 0 || !in.grad_coeffs) continue;
      ZP_TRY(series_adjoint_fp64(b->plans[b->inst_plan[i]].get(), in.r, in.theta, in.n_points, in.coeffs, b->n_sets,
                                 in.grad_out, in.grad_coeffs, nullptr, nullptr, st, HessOut(), true));
    }
    return ZP_OK;
  }
  if (need_c && b->n_citems) ZP_TRY(launch_columns(b, st));
  return ZP_OK;
}

zp_status zp_batch_adjoint(zp_batch* b, void* stream) {
  zp::NvtxRange zp_range_("zp_batch_adjoint");
  return zp::entry_finish("zp_batch_adjoint", stream, zp_batch_adjoint_impl(b, ZP_PREC_FP64, stream));
}

zp_status zp_batch_adjoint_prec(zp_batch* b, zp_precision prec, void* stream) {
  zp::NvtxRange zp_range_("zp_batch_adjoint_prec");
  return zp::entry_finish("zp_batch_adjoint_prec", stream, zp_batch_adjoint_impl(b, prec, stream));
}

zp_status zp_batch_set_config(zp_batch* b, int32_t tile_points, int32_t ctas_per_sm, int32_t col_ppt,
                              int32_t col_threads) {
  clear_error();
  if (!b) return set_error(ZP_ERR_INVALID_ARG, "batch is NULL");
  if (tile_points < 32 || tile_points > 1024 || tile_points % 32)
    return set_error(ZP_ERR_INVALID_ARG, "tile_points must be a multiple of 32 in 32..1024");
  if (ctas_per_sm < 1 || ctas_per_sm > 32) return set_error(ZP_ERR_INVALID_ARG, "ctas_per_sm must be 1..32");
  if (col_ppt != 1 && col_ppt != 2 && col_ppt != 4) return set_error(ZP_ERR_INVALID_ARG, "col_ppt must be 1, 2 or 4");
  if (col_threads < 32 || col_threads > 512 || col_threads % 32)
    return set_error(ZP_ERR_INVALID_ARG, "col_threads must be a multiple of 32 in 32..512");
  const int old_tp = b->tp;
  b->tp = tile_points;
  b->ctas_per_sm = ctas_per_sm;
  b->col_ppt = col_ppt;
  b->col_threads = col_threads;
  if (old_tp != tile_points) return build_point_items(b, nullptr);
  return ZP_OK;
}

zp_status zp_batch_get_config(const zp_batch* b, int32_t* cfg) {
  clear_error();
  if (!b || !cfg) return set_error(ZP_ERR_INVALID_ARG, "NULL argument");
  cfg[0] = b->tp;
  cfg[1] = b->ctas_per_sm;
  cfg[2] = b->col_ppt;
  cfg[3] = b->col_threads;
  return ZP_OK;
}

// Autotuner: times every candidate launch configuration on the batch itself (one warm-up
// run, then the mean of `reps` runs, CUDA events on `stream`) and keeps the fastest.
// which: 0 = forward (precision prec), 1 = adjoint.  Writes the chosen configuration to cfg[4]
// and the best time in ms to *best_ms.  Synchronises `stream`.
}  // extern "C"

namespace zp {
namespace {
// Tuning results kept for the process and, when the environment variable ZP_TUNE_CACHE names a
// file, across processes: one line per key, "key tile ctas ppt threads best_ms".  The key holds
// what decides the best launch: the GPU (compute capability, SM count) and the batch's shape
// (instances, points, modes, largest n, sets), the pass and the precision.
struct TuneCache {
  std::mutex mu;
  bool loaded = false;
  std::map<std::string, std::array<float, 5>> entries;
};
TuneCache& tune_cache() {
  static TuneCache c;
  return c;
}
const char* tune_cache_path() { return std::getenv("ZP_TUNE_CACHE"); }

std::string tune_key(const zp_batch* b, int32_t which, zp_precision prec) {
  int dev = 0, major = 0, minor = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t points = 0, modes = 0;
  int32_t n_max = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    points += b->inst[i].n_points;
    modes += b->inst[i].n_modes;
    n_max = std::max(n_max, b->plans[b->inst_plan[i]]->n_max);
  }
  std::ostringstream k;
  k << "sm" << major << minor << "x" << sms << "/inst" << b->inst.size() << "/pts" << points << "/modes" << modes
    << "/nmax" << n_max << "/sets" << b->n_sets << "/pass" << which << "/prec" << (int)prec;
  return k.str();
}

void tune_cache_load_locked(TuneCache& c) {
  if (c.loaded) return;
  c.loaded = true;
  const char* path = tune_cache_path();
  if (!path) return;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ls(line);
    std::string key;
    std::array<float, 5> v{};
    if (ls >> key >> v[0] >> v[1] >> v[2] >> v[3] >> v[4]) c.entries[key] = v;
  }
}

bool tune_cache_get(const std::string& key, std::array<float, 5>* v) {
  TuneCache& c = tune_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  tune_cache_load_locked(c);
  auto it = c.entries.find(key);
  if (it == c.entries.end()) return false;
  *v = it->second;
  return true;
}

void tune_cache_put(const std::string& key, const std::array<float, 5>& v) {
  TuneCache& c = tune_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  tune_cache_load_locked(c);
  c.entries[key] = v;
  const char* path = tune_cache_path();
  if (!path) return;
  std::ofstream out(path, std::ios::app);
  if (out) out << key << " " << v[0] << " " << v[1] << " " << v[2] << " " << v[3] << " " << v[4] << "\n";
}
}  // namespace
}  // namespace zp

extern "C" {

zp_status zp_batch_tune(zp_batch* b, int32_t which, zp_precision prec, int32_t reps, void* stream, int32_t* cfg,
                        float* best_ms) {
  clear_error();
  if (!b) return set_error(ZP_ERR_INVALID_ARG, "batch is NULL");
  // A configuration tuned before for this GPU and batch shape (this process or the cache file).
  const std::string key = tune_key(b, which, prec);
  std::array<float, 5> hit{};
  if (tune_cache_get(key, &hit)) {
    ZP_TRY(zp_batch_set_config(b, (int32_t)hit[0], (int32_t)hit[1], (int32_t)hit[2], (int32_t)hit[3]));
    if (cfg)
      for (int k = 0; k < 4; ++k) cfg[k] = (int32_t)hit[k];
    if (best_ms) *best_ms = hit[4];
    return ZP_OK;
  }
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int32_t best_cfg[4] = {b->tp, b->ctas_per_sm, b->col_ppt, b->col_threads};
  const int tps[] = {64, 128, 256};
  const int ctas[] = {2, 4, 8};
  std::vector<std::array<int, 4>> cands;
  if (which == 0 && prec == ZP_PREC_FP64_EMULATED) {
    // The fused forward takes none of these parameters: one timing of the current configuration.
    cands.push_back({b->tp, b->ctas_per_sm, b->col_ppt, b->col_threads});
  } else if (which == 0) {
    for (int tp : tps)
      for (int c : ctas) cands.push_back({tp, c, b->col_ppt, b->col_threads});
  } else {
    for (int tp : {128, 256})
      for (int pp : {2, 4})
        for (int ct : {64, 128}) cands.push_back({tp, b->ctas_per_sm, pp, ct});
  }
  zp_status result = ZP_OK;
  for (auto& cnd : cands) {
    if ((result = zp_batch_set_config(b, cnd[0], cnd[1], cnd[2], cnd[3])) != ZP_OK) break;
    auto run = [&]() { return which == 0 ? zp_batch_forward(b, prec, stream) : zp_batch_adjoint(b, stream); };
    if ((result = run()) != ZP_OK) {
      // A configuration the GPU cannot launch (registers, shared memory) is skipped.
      if (result == ZP_ERR_UNSUPPORTED) {
        result = ZP_OK;
        continue;
      }
      break;
    }
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && result == ZP_OK; ++k) result = run();
    cudaEventRecord(e1, st);
    if (result != ZP_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      result = cuda_error(e, "tuning run");
      break;
    }
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    t /= reps;
    if (t < best) {
      best = t;
      for (int k = 0; k < 4; ++k) best_cfg[k] = cnd[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != ZP_OK) return result;
  ZP_TRY(zp_batch_set_config(b, best_cfg[0], best_cfg[1], best_cfg[2], best_cfg[3]));
  if (cfg)
    for (int k = 0; k < 4; ++k) cfg[k] = best_cfg[k];
  if (best_ms) *best_ms = best;
  tune_cache_put(key, {(float)best_cfg[0], (float)best_cfg[1], (float)best_cfg[2], (float)best_cfg[3], best});
  return ZP_OK;
}

}  // extern "C"
