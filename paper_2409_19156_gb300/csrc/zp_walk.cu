// The per-(point, |m|-column) recursion walk: radial polynomials, rho-derivatives, Z.
//
// Work decomposition (Algorithm 1 of Sec. 3, mapped to the GPU): one thread owns
// one or two consecutive points of one |m| column and walks the Jacobi degree N = 0 .. N_max in
// registers, storing every requested (n, m) of that column as it passes (the store list
// comes from the plan; the duplicated-modes variant of Sec. 3 is several entries per N).
// The recursion is the beta = 0 Jacobi recursion of Sec. 2 in the rescaled form built by
// the plan (see zp_plan.cpp):
//   Q_N = g_N Q_{N-1} - Q_{N-2},   g_N(rho) = A_N rho^2 - B_N,   R_N = w_N Q_N.
// Derivatives carry Taylor lanes S_k = Q^(k) / k!; by Leibniz,
//   S_k,N = g S_k,N-1 + g' S_{k-1},N-1 + (g''/2) S_{k-2},N-1 - S_k,N-2,
// with g' = 2 A_N rho, g''/2 = A_N and g''' = 0, and d^k R / drho^k = (k! w_N) S_k.
// Per step and point that is 3 (k = 0), 7 (k <= 1), 11 (k <= 2) or 15 (k <= 3) float64
// operations, which on GB300 (two float64 lanes per SM per clock) makes this kernel
// float64-issue bound; the stores (point-fastest rows, 16-byte vectors) are coalesced.
//
// Seeds (Sec. 2 explicit Jacobi sum for P_0, P_1 through the Jacobi relation):
//   R_{m}^{m} = rho^m,   R_{m+2}^{m} = (m+2) rho^(m+2) - (m+1) rho^m.
// For large launches a point-preparation kernel first tabulates rho^j and cos / sin(j theta)
// per point (j up to the largest |m| + 2), so each (point, column) seed costs a few loads
// instead of a power by squaring and a sincos.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "zp_device.cuh"
#include "zp_api_common.h"
#include "zp_internal.h"
#include "zp_series_internal.h"

namespace zp {
namespace {

constexpr int kThreads = 128;      // threads per block of a full-size launch, 2 points each
constexpr int kThreadsSmall = 32;  // short launches: 1 point per thread, more and shorter warps
constexpr int kPPT = 2;

struct WalkArgs {
  const Column* cols;
  const double* table;
  const int32_t* slot_ptr;
  const int32_t* slot_idx;
  const double* r;
  const double* theta;
  int64_t P;
  int64_t J;
  double* out;
  double* out_dtheta;
  // Optional point tables [j][P] (NULL: computed per thread): pw = rho^j (j <= pw_max),
  // cs / sn = cos / sin(j theta) (j <= the largest |m|).
  const double* pw = nullptr;
  const double* cs = nullptr;
  const double* sn = nullptr;
  int pw_max = 0;
  // Optional (NULL: none; walks of Z at k = 0 only): per output row j, the largest high word
  // of |value| over all points, atomically maxed into rowmax[j] << 32 (zeroed by the caller):
  // what the float64-accurate GEMM needs for its power-of-two row scales.
  unsigned long long* rowmax = nullptr;
};

// Point preparation: rho^j for j = 0..pw_max and (theta given) cos / sin(j theta) for
// j = 0..trig_max, point-fastest rows.  Every 16th entry is computed directly (a power by
// squaring, a sincos of j theta) and the entries between by one multiplication (rho^(j+1) =
// rho^j rho) or one angle addition, so rounding errors grow over at most 15 steps.
__global__ void __launch_bounds__(128) point_prep_kernel(const double* __restrict__ r, const double* __restrict__ theta,
                                                         int64_t P, int pw_max, int trig_max, double* __restrict__ pw,
                                                         double* __restrict__ cs, double* __restrict__ sn);

__global__ void __launch_bounds__(128) point_prep_kernel(const double* __restrict__ r, const double* __restrict__ theta,
                                                         int64_t P, int pw_max, int trig_max, double* __restrict__ pw,
                                                         double* __restrict__ cs, double* __restrict__ sn) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double rho = r[p];
  double v = 1.0;
  for (int j = 0; j <= pw_max; ++j) {
    v = (j % 16 == 0) ? pow_uint(rho, j) : v * rho;
    __stcg(pw + (int64_t)j * P + p, v);
  }
  if (theta == nullptr) return;
  const double th = theta[p];
  double s1, c1;
  sincos(th, &s1, &c1);
  double c = 1.0, s = 0.0;
  for (int j = 0; j <= trig_max; ++j) {
    if (j % 16 == 0) {
      sincos((double)j * th, &s, &c);
    } else {
      const double cn = fma(c, c1, -s * s1);
      s = fma(s, c1, c * s1);
      c = cn;
    }
    __stcg(cs + (int64_t)j * P + p, c);
    __stcg(sn + (int64_t)j * P + p, s);
  }
}

template <int PPT>
__device__ __forceinline__ void store_pts(double* dst, int64_t p, double v0, double v1, bool two, bool vec) {
  if constexpr (PPT == 1) {
    __stcs(dst + p, v0);
    return;
  }
  if (vec) {
    __stcs(reinterpret_cast<double2*>(dst + p), make_double2(v0, v1));
  } else {
    __stcs(dst + p, v0);
    if (two) __stcs(dst + p + 1, v1);
  }
}

// KMAX: highest rho-derivative; ANG: multiply by cos/sin(|m| theta) (Z instead of R);
// VEC: 16-byte stores (P even and outputs 16-byte aligned); DUP (with ANG): the plan has steps
// with more than two outputs (duplicated modes), whose angular products are formed once.
// TPB: threads per block: 128 with two points per thread, or 32 with one point per thread for
// short launches (a short launch is bound by its longest warp's dependent float64 chain, so
// more, shorter warps spread over more SMs finish sooner).
template <int KMAX, bool ANG, bool VEC, bool DUP = false, int TPB = kThreads>
__global__ void __launch_bounds__(TPB) walk_kernel(WalkArgs a) {
  constexpr int PPT = TPB == kThreads ? kPPT : 1;
  extern __shared__ double smem[];
  const Column col = a.cols[blockIdx.y];
  const int n_rows = kHeaderRows + col.n_steps;
  double* tab = smem;
  int32_t* sptr = reinterpret_cast<int32_t*>(smem + (size_t)n_rows * kRow);
  {
    const double* src = a.table + (size_t)col.table_row * kRow;
    for (int i = threadIdx.x; i < n_rows * kRow; i += TPB) tab[i] = src[i];
    const int32_t* s2 = a.slot_ptr + col.slot_base;
    for (int i = threadIdx.x; i <= col.n_steps; i += TPB) sptr[i] = s2[i];
  }
  __syncthreads();

  const int64_t p0 = ((int64_t)blockIdx.x * TPB + (int64_t)threadIdx.x) * PPT;
  if (p0 >= a.P) return;
  const bool two = PPT == 2 && p0 + 1 < a.P;
  const int m = col.m;

  double rho[PPT], u[PPT];
  rho[0] = a.r[p0];
  if constexpr (PPT == 2) rho[PPT - 1] = two ? a.r[p0 + 1] : 0.0;
#pragma unroll
  for (int i = 0; i < PPT; ++i) u[i] = rho[i] * rho[i];

  double cs[PPT], sn[PPT];
  if constexpr (ANG) {
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      cs[i] = 1.0;
      sn[i] = 0.0;
    }
    if (a.cs != nullptr) {
      cs[0] = a.cs[(int64_t)m * a.P + p0];
      sn[0] = a.sn[(int64_t)m * a.P + p0];
      if constexpr (PPT == 2) {
        if (two) {
          cs[PPT - 1] = a.cs[(int64_t)m * a.P + p0 + 1];
          sn[PPT - 1] = a.sn[(int64_t)m * a.P + p0 + 1];
        }
      }
    } else if (m != 0) {
      sincos((double)m * a.theta[p0], &sn[0], &cs[0]);
      if constexpr (PPT == 2) {
        const double th1 = two ? a.theta[p0 + 1] : 0.0;
        sincos((double)m * th1, &sn[PPT - 1], &cs[PPT - 1]);
      }
    }
  }

  // Seeds.  pw[i] = rho^(m - KMAX + i) for i = 0 .. KMAX+2 (0 for negative exponents, whose
  // coefficients vanish).
  double S[PPT][KMAX + 1], T[PPT][KMAX + 1];
  {
    const double* h = tab;
    const int e0 = m - KMAX;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      double pw[KMAX + 3];
      if (a.pw != nullptr) {
        const int64_t pi = (i == 0 || two) ? p0 + i : p0;
#pragma unroll
        for (int t = 0; t < KMAX + 3; ++t) pw[t] = e0 + t >= 0 ? a.pw[(int64_t)(e0 + t) * a.P + pi] : 0.0;
      } else {
        double cur = e0 >= 0 ? pow_uint(rho[i], e0) : 0.0;
#pragma unroll
        for (int t = 0; t < KMAX + 3; ++t) {
          if (t > 0) cur = (e0 + t == 0) ? 1.0 : cur * rho[i];
          pw[t] = cur;
        }
      }
#pragma unroll
      for (int k = 0; k <= KMAX; ++k) {
        T[i][k] = h[k] * pw[KMAX - k];                                      // N = 0: rho^m
        S[i][k] = fma(h[4 + k], pw[KMAX - k + 2], -(h[8 + k] * pw[KMAX - k]));  // N = 1
      }
    }
  }

  // Row maximum of output row j (walks of Z at k = 0): the warp's live lanes reduce the high
  // words of |v| and one of them maxes the result into rowmax[j].
  auto note_max = [&](int64_t j, double v0, double v1) {
    uint32_t h = (uint32_t)__double2hiint(v0) & 0x7fffffffu;
    if (PPT == 2 && two) h = max(h, (uint32_t)__double2hiint(v1) & 0x7fffffffu);
    const unsigned mask = __activemask();
    const uint32_t mx = __reduce_max_sync(mask, h);
    if ((int)(threadIdx.x & 31u) == __ffs((int)mask) - 1) atomicMax(a.rowmax + j, (unsigned long long)mx << 32);
  };
  auto store_step = [&](int N, const double (&V)[PPT][KMAX + 1]) {
    const int s_begin = sptr[N], s_end = sptr[N + 1];
    if (s_begin == s_end) return;
    const double* row = tab + (size_t)(kHeaderRows + N) * kRow;
    // row[7] holds 0.0: multiplies are issued as FMAs with a zero addend the compiler cannot
    // fold away, because GB300 issues DFMA faster than DMUL (1.88 vs 1.59 lanes/SM/clk).
    const double zero = row[7];
    double R[PPT][KMAX + 1];
#pragma unroll
    for (int k = 0; k <= KMAX; ++k) {
      const double W = row[3 + k];
#pragma unroll
      for (int i = 0; i < PPT; ++i) R[i][k] = fma(W, V[i][k], zero);
    }
    if constexpr (ANG && DUP) {
      if (s_end - s_begin > 2) {
        // Duplicated modes (several outputs per (column, N)): each angular product once per
        // (step, k), stored to every output of the step.
#pragma unroll
        for (int k = 0; k <= KMAX; ++k) {
          double rc[PPT], rs[PPT];
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            rc[i] = fma(R[i][k], cs[i], zero);
            rs[i] = fma(R[i][k], sn[i], zero);
          }
          for (int s = s_begin; s < s_end; ++s) {
            const uint32_t code = (uint32_t)__ldg(a.slot_idx + s);
            const int64_t j = (int64_t)(code & 0x7fffffffu);
            const bool is_sin = (code >> 31) != 0;
            store_pts<PPT>(a.out + ((int64_t)k * a.J + j) * a.P, p0, is_sin ? rs[0] : rc[0], is_sin ? rs[PPT - 1] : rc[PPT - 1], two,
                       VEC);
            if constexpr (KMAX == 0)
              if (a.rowmax) note_max(j, is_sin ? rs[0] : rc[0], is_sin ? rs[PPT - 1] : rc[PPT - 1]);
          }
        }
        if (a.out_dtheta) {
          // d/dtheta: m R cos(m theta) for a sin output, -m R sin(m theta) for a cos output.
          const double md = (double)m;
          double dsn[PPT], dcs[PPT];
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            dsn[i] = fma(R[i][0], md * cs[i], zero);
            dcs[i] = fma(R[i][0], -md * sn[i], zero);
          }
          for (int s = s_begin; s < s_end; ++s) {
            const uint32_t code = (uint32_t)__ldg(a.slot_idx + s);
            const int64_t j = (int64_t)(code & 0x7fffffffu);
            const bool is_sin = (code >> 31) != 0;
            store_pts<PPT>(a.out_dtheta + j * a.P, p0, is_sin ? dsn[0] : dcs[0], is_sin ? dsn[PPT - 1] : dcs[PPT - 1], two, VEC);
          }
        }
        return;
      }
    }
    for (int s = s_begin; s < s_end; ++s) {
      const uint32_t code = (uint32_t)__ldg(a.slot_idx + s);
      const int64_t j = (int64_t)(code & 0x7fffffffu);
      if constexpr (ANG) {
        const bool is_sin = (code >> 31) != 0;
        double f[PPT];
#pragma unroll
        for (int i = 0; i < PPT; ++i) f[i] = is_sin ? sn[i] : cs[i];
#pragma unroll
        for (int k = 0; k <= KMAX; ++k) {
          const double v0 = fma(R[0][k], f[0], zero), v1 = fma(R[PPT - 1][k], f[PPT - 1], zero);
          store_pts<PPT>(a.out + ((int64_t)k * a.J + j) * a.P, p0, v0, v1, two, VEC);
          if constexpr (KMAX == 0)
            if (a.rowmax) note_max(j, v0, v1);
        }
        if (a.out_dtheta) {
          const double md = (double)m;
          double dt[PPT];
#pragma unroll
          for (int i = 0; i < PPT; ++i) dt[i] = is_sin ? md * cs[i] : -md * sn[i];
          store_pts<PPT>(a.out_dtheta + j * a.P, p0, fma(R[0][0], dt[0], zero), fma(R[PPT - 1][0], dt[PPT - 1], zero), two, VEC);
        }
      } else {
#pragma unroll
        for (int k = 0; k <= KMAX; ++k)
          store_pts<PPT>(a.out + ((int64_t)k * a.J + j) * a.P, p0, R[0][k], R[PPT - 1][k], two, VEC);
      }
    }
  };

  store_step(0, T);
  if (col.n_steps < 2) return;
  store_step(1, S);
  // Derivative walks of the 128-thread form take eight steps per iteration: the independent
  // float64 chains of the unrolled steps overlap their latencies (radial n <= 100, k <= 3,
  // 100000 points: 6.58 ms with one step, 6.48 with two, 6.34 with four, 6.29 with eight; no
  // spills).  The value-only walk keeps one step (unrolled by two or four it measured 8 %
  // slower), and so do the short launches' 32-thread blocks (latency-bound; unrolling them only
  // adds compile time).
#pragma unroll((KMAX >= 1 && TPB == kThreads) ? 8 : 1)
  for (int N = 2; N < col.n_steps; ++N) {
    const double* row = tab + (size_t)(kHeaderRows + N) * kRow;
    const double A = row[0], B = row[1], A2 = row[2], zero = row[7];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const double g = fma(A, u[i], -B);
      double nw[KMAX + 1];
      nw[0] = fma(g, S[i][0], -T[i][0]);
      if constexpr (KMAX >= 1) {
        const double hg = fma(A2, rho[i], zero);
        nw[1] = fma(g, S[i][1], fma(hg, S[i][0], -T[i][1]));
        if constexpr (KMAX >= 2) nw[2] = fma(g, S[i][2], fma(hg, S[i][1], fma(A, S[i][0], -T[i][2])));
        if constexpr (KMAX >= 3) nw[3] = fma(g, S[i][3], fma(hg, S[i][2], fma(A, S[i][1], -T[i][3])));
      }
#pragma unroll
      for (int k = 0; k <= KMAX; ++k) {
        T[i][k] = S[i][k];
        S[i][k] = nw[k];
      }
    }
    store_step(N, S);
  }
}

// Algorithm 2 of Sec. 3: one thread per (point, mode), each running its own recursion to
// its own degree and storing only the last value (k = 0).  Comparison kernel.
__global__ void __launch_bounds__(kThreads) per_mode_kernel(const Column* cols, const double* table,
                                                            const int32_t* mode_col, const int32_t* mode_N,
                                                            const double* r, int64_t P, int64_t J, double* out) {
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= P) return;
  const double rho = r[p], u = rho * rho;
  for (int64_t j = blockIdx.y; j < J; j += gridDim.y) {
    const Column col = cols[mode_col[j]];
    const int N = mode_N[j];
    const double* h = table + (size_t)col.table_row * kRow;
    const double rm = pow_uint(rho, col.m);
    double q0 = rm;                                  // Q_0
    double q1 = fma(h[4], rm * u, -(h[8] * rm));      // Q_1 = (m+2) rho^(m+2) - (m+1) rho^m
    double q = N == 0 ? q0 : q1;
    for (int s = 2; s <= N; ++s) {
      const double* row = h + (size_t)(kHeaderRows + s) * kRow;
      q = fma(fma(row[0], u, -row[1]), q1, -q0);
      q0 = q1;
      q1 = q;
    }
    __stcs(out + j * P + p, q * h[(size_t)(kHeaderRows + N) * kRow + 3]);
  }
}

template <int KMAX, bool ANG, int TPB>
cudaError_t launch_walk_tpb(const WalkArgs& a, dim3 grid, size_t smem, bool vec, bool dup, cudaStream_t st) {
  if (ANG && dup) {
    if (vec)
      walk_kernel<KMAX, ANG, true, true, TPB><<<grid, TPB, smem, st>>>(a);
    else
      walk_kernel<KMAX, ANG, false, true, TPB><<<grid, TPB, smem, st>>>(a);
  } else if (vec) {
    walk_kernel<KMAX, ANG, true, false, TPB><<<grid, TPB, smem, st>>>(a);
  } else {
    walk_kernel<KMAX, ANG, false, false, TPB><<<grid, TPB, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <int KMAX, bool ANG>
cudaError_t launch_walk_t(const WalkArgs& a, dim3 grid, bool small, size_t smem, bool vec, bool dup,
                          cudaStream_t st) {
  return small ? launch_walk_tpb<KMAX, ANG, kThreadsSmall>(a, grid, smem, vec, dup, st)
               : launch_walk_tpb<KMAX, ANG, kThreads>(a, grid, smem, vec, dup, st);
}

}  // namespace

namespace {
// Events around the launches of one call, for zp_radial_plan_timed.
struct WalkTimer {
  float* ms;
  cudaStream_t stream;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool prep = false;
  WalkTimer(float* m, cudaStream_t s) : ms(m), stream(s) {
    if (!ms) return;
    for (auto& e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], stream);
  }
  void mark(int i) {
    if (ms) cudaEventRecord(ev[i], stream);
  }
  zp_status finish() {
    if (!ms) return ZP_OK;
    cudaError_t e = cudaEventSynchronize(ev[2]);
    float t0 = 0.0f, t1 = 0.0f;
    if (e == cudaSuccess && prep) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, prep ? ev[1] : ev[0], ev[2]);
    ms[0] = t0;
    ms[1] = t1;
    return e == cudaSuccess ? ZP_OK : cuda_error(e, "walk timing");
  }
  ~WalkTimer() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};
}  // namespace

zp_status launch_walk(const zp_plan* plan, const double* r, const double* theta, int64_t n_points, int max_deriv,
                      double* out, double* out_dtheta, cudaStream_t stream, float* phase_ms,
                      unsigned long long* rowmax) {
  if (phase_ms) phase_ms[0] = phase_ms[1] = 0.0f;
  if (rowmax && (max_deriv != 0 || theta == nullptr))
    return set_error(ZP_ERR_INVALID_ARG, "row maxima are formed for walks of Z at k = 0 only");
  if (n_points == 0 || plan->n_modes == 0) return ZP_OK;
  WalkTimer timer(phase_ms, stream);
  WalkArgs a;
  a.cols = plan->dev.cols;
  a.table = plan->dev.table;
  a.slot_ptr = plan->dev.slot_ptr;
  a.slot_idx = plan->dev.slot_idx;
  a.r = r;
  a.theta = theta;
  a.P = n_points;
  a.J = plan->n_modes;
  a.out = out;
  a.out_dtheta = out_dtheta;
  a.rowmax = rowmax;
  // Short launches (fewer than eight 128-thread blocks per SM) take 32-thread blocks of one
  // point per thread: more, shorter warps over more SMs.
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n_cols = (int64_t)plan->cols.size();
  const bool small = ((n_points + kThreads * kPPT - 1) / (kThreads * kPPT)) * n_cols < 8 * (int64_t)sms;
  const int64_t per_block = small ? kThreadsSmall : kThreads * kPPT;
  const int64_t blocks_x = (n_points + per_block - 1) / per_block;
  if (blocks_x > 0x7fffffffLL) return set_error(ZP_ERR_INVALID_ARG, "n_points too large for one launch");
  dim3 grid((unsigned)blocks_x, (unsigned)n_cols);
  const size_t smem = (size_t)(kHeaderRows + plan->max_steps) * kRow * sizeof(double) +
                      (size_t)(plan->max_steps + 1) * sizeof(int32_t);
  const bool vec = (n_points % 2 == 0) && ((uintptr_t)out % 16 == 0) &&
                   (out_dtheta == nullptr || (uintptr_t)out_dtheta % 16 == 0);
  const bool ang = theta != nullptr;
  cudaError_t e;
  // Point tables when they pay: enough points and columns to amortise one more launch, and
  // orders low enough that the tables stay small (at most 2 + 2 x 131 rows of P doubles).
  int m_max = 0;
  for (const Column& c : plan->cols) m_max = std::max(m_max, (int)c.m);
  ScratchBuffer tables;
  if (n_points >= 8192 && plan->cols.size() >= 4 && m_max <= 128) {
    const int pw_max = m_max + 2;
    const size_t rows = (size_t)(pw_max + 1) + (ang ? 2 * (size_t)(m_max + 1) : 0);
    // The tables are an optimisation: without the memory for them the walk computes its seeds.
    if (tables.alloc(rows * (size_t)n_points * sizeof(double), stream) != ZP_OK) {
      cudaGetLastError();
      clear_error();
    }
  }
  if (tables.ptr) {
    const int pw_max = m_max + 2;
    double* pw = (double*)tables.ptr;
    double* cs = ang ? pw + (size_t)(pw_max + 1) * n_points : nullptr;
    double* sn = ang ? cs + (size_t)(m_max + 1) * n_points : nullptr;
    point_prep_kernel<<<(unsigned)((n_points + 127) / 128), 128, 0, stream>>>(r, theta, n_points, pw_max, m_max, pw,
                                                                             cs, sn);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "point_prep_kernel launch");
    timer.prep = true;
    timer.mark(1);
    a.pw = pw;
    a.pw_max = pw_max;
    a.cs = cs;
    a.sn = sn;
  }
  // Duplicated modes: some (column, N) step stores to more than two outputs.
  bool dup = false;
  for (size_t i = 0; i + 1 < plan->slot_ptr.size() && !dup; ++i) dup = plan->slot_ptr[i + 1] - plan->slot_ptr[i] > 2;
  switch (max_deriv) {
    case 0: e = ang ? launch_walk_t<0, true>(a, grid, small, smem, vec, dup, stream) : launch_walk_t<0, false>(a, grid, small, smem, vec, dup, stream); break;
    case 1: e = ang ? launch_walk_t<1, true>(a, grid, small, smem, vec, dup, stream) : launch_walk_t<1, false>(a, grid, small, smem, vec, dup, stream); break;
    case 2: e = ang ? launch_walk_t<2, true>(a, grid, small, smem, vec, dup, stream) : launch_walk_t<2, false>(a, grid, small, smem, vec, dup, stream); break;
    case 3: e = ang ? launch_walk_t<3, true>(a, grid, small, smem, vec, dup, stream) : launch_walk_t<3, false>(a, grid, small, smem, vec, dup, stream); break;
    default: return set_error(ZP_ERR_DERIV_ORDER, "max_deriv outside 0..3");
  }
  if (e != cudaSuccess) return cuda_error(e, "walk_kernel launch");
  timer.mark(2);
  return timer.finish();
}

zp_status launch_per_mode(const zp_plan* plan, const double* r, int64_t n_points, double* out, cudaStream_t stream) {
  if (n_points == 0 || plan->n_modes == 0) return ZP_OK;
  const int64_t blocks_x = (n_points + kThreads - 1) / kThreads;
  if (blocks_x > 0x7fffffffLL) return set_error(ZP_ERR_INVALID_ARG, "n_points too large for one launch");
  dim3 grid((unsigned)blocks_x, (unsigned)(plan->n_modes < 65535 ? plan->n_modes : 65535));
  per_mode_kernel<<<grid, kThreads, 0, stream>>>(plan->dev.cols, plan->dev.table, plan->dev.mode_col, plan->dev.mode_N,
                                                 r, n_points, plan->n_modes, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "per_mode_kernel launch");
  return ZP_OK;
}

}  // namespace zp
