// Least-squares fit of Zernike series coefficients (the "fit" counterpart of zp_series_eval).
//
//   minimise  sum_p w_p || sum_j Z_j(p) C[j, :] - Y[p, :] ||^2  +  ridge ||C||^2
//   =>  (Z W Z^T + ridge I) C = Z W Y          (normal equations, Z = basis [J][P])
//
// Steps: the basis by the walk kernel (float64, into scratch), the rows scaled by sqrt(w) when
// weights are given, the Gram matrix and the right-hand side by cuBLAS DGEMM (or by the
// float64-accurate tensor-core GEMM of zp_mma.cu for ZP_PREC_FP64_EMULATED), the
// ridge added on the diagonal, a right-looking blocked Cholesky factorisation in the library's
// own kernels, and the two triangular solves (up to 640 modes one kernel that stages L in shared
// memory and stores straight into the caller's row-major [J][S] output; beyond, blocked solves
// of 32 rows at a time and a transpose kernel).  The call synchronises its stream at the end to
// read the factorisation status.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "zp_api_common.h"
#include "zp_series_internal.h"

namespace zp {
namespace {

// sw[p] = sqrt(w[p]) once per point; then Z[j][p] *= sw[p] and Ys[p][s] = sw[p] Y[p][s] by
// multiplies (a float64 sqrt per element cost 0.25 ms per 16M elements on this part).
__global__ void sqrt_weights_kernel(const double* w, double* sw, int64_t P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    sw[i] = sqrt(w[i]);
}
// Rows of Z over blockIdx.y (grid-stride), points over x.
__global__ void scale_rows_kernel(double* Z, int64_t J, int64_t P, const double* sw) {
  for (int64_t j = blockIdx.y; j < J; j += gridDim.y) {
    double* row = Z + j * P;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
      row[p] *= sw[p];
  }
}
// Points over blockIdx.x (grid-stride), sets over threads.
__global__ void scale_samples_kernel(const double* Y, double* Ys, int64_t P, int64_t S, const double* sw) {
  for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
    const double f = sw[p];
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) Ys[p * S + s] = Y[p * S + s] * f;
  }
}
__global__ void add_ridge_kernel(double* G, int64_t J, double ridge) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J; i += (int64_t)gridDim.x * blockDim.x)
    G[i * J + i] += ridge;
}

// Smallest and largest squared pivot of the Cholesky factor (single block).
__global__ void pivot_range_kernel(const double* L, int64_t J, double* out) {
  __shared__ double smin[256], smax[256];
  double lo = 1.0 / 0.0, hi = 0.0;
  for (int64_t i = threadIdx.x; i < J; i += blockDim.x) {
    const double d = L[i * J + i];
    const double d2 = d * d;
    lo = d2 < lo ? d2 : lo;
    hi = d2 > hi ? d2 : hi;
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      smin[threadIdx.x] = smin[threadIdx.x + s] < smin[threadIdx.x] ? smin[threadIdx.x + s] : smin[threadIdx.x];
      smax[threadIdx.x] = smax[threadIdx.x + s] > smax[threadIdx.x] ? smax[threadIdx.x + s] : smax[threadIdx.x];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smin[0];
    out[1] = smax[0];
  }
}

// ---- Cholesky factorisation and solve for small normal matrices (J <= kCholMaxJ) ----------
// cuSOLVER's potrf / potrs take 1.3 + 0.9 ms for J = 325 (latency-bound panel kernels); these
// kernels do the same in a few tens of launches without grid-wide waits.  A is column-major
// J x J, lower triangle; every element is written by one thread in a fixed order (the results
// are deterministic).
constexpr int kNb = 32;          // panel width
constexpr int kCholMaxJ = 640;   // shared-memory staging limit of the solve kernel
constexpr int kSolveCols = 2;    // right-hand sides per CTA of the solve kernel

// Pivot d = sqrt(v) and its reciprocal.  In the float32 range: the reciprocal square root by
// Newton-Raphson iteration (r <- r (3 - v r^2) / 2, quadratic convergence) from the float32
// estimate rsqrtf, two steps to float64 precision, d = v r; one thread's dependent float64 chain
// is much shorter this way than a float64 sqrt and a division.  Elsewhere (and for v <= 0 or NaN,
// which the caller reports): sqrt and a division.
__device__ __forceinline__ void pivot_sqrt(double v, double* d, double* rd) {
  if (v > 1e-30 && v < 1e30) {
    double r = (double)rsqrtf((float)v);
    r = r * fma(-0.5 * v, r * r, 1.5);
    r = r * fma(-0.5 * v, r * r, 1.5);
    *rd = r;
    *d = v * r;
  } else {
    *d = sqrt(v);
    *rd = 1.0 / *d;
  }
}

// Panel k0 (columns k0 .. k0 + nb - 1, the updates of earlier panels already applied): every
// CTA factors the nb x nb diagonal block in shared memory (identical arithmetic, so the copies
// agree bitwise); CTA 0 writes the factor back, CTA b >= 1 solves rows k0 + 32 b ... of the
// panel against it (L_rows = A_rows L_kk^-T).  info[0]: 1 + the first column whose pivot is not
// positive (left 0 when there is none).
__global__ void __launch_bounds__(256) chol_panel_kernel(double* A, int J, int k0, int* info) {
  __shared__ double D[kNb][kNb + 1];
  __shared__ double R[kNb][kNb + 1];
  __shared__ double rd[kNb];
  const int nb = min(kNb, J - k0);
  const int tid = threadIdx.x;
  const int tx = tid % kNb, ty = tid / kNb;  // 256 threads: 8 rows of 32
#pragma unroll
  for (int c = ty; c < kNb; c += 8)
    D[tx][c] = (tx < nb && c < nb && tx >= c) ? A[(size_t)(k0 + tx) + (size_t)(k0 + c) * J] : 0.0;
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (tid == 0) {
      const double v = D[c][c];
      if (!(v > 0.0) && blockIdx.x == 0) atomicCAS(info, 0, k0 + c + 1);
      double d, r;
      pivot_sqrt(v, &d, &r);
      D[c][c] = d;
      rd[c] = r;
    }
    __syncthreads();
    if (tid > c && tid < nb) D[tid][c] *= rd[c];
    __syncthreads();
    // Trailing block: (r, q) = (tx, q) with c < q <= r < nb.
#pragma unroll
    for (int q = ty; q < kNb; q += 8)
      if (q > c && q <= tx && tx < nb) D[tx][q] = fma(-D[tx][c], D[q][c], D[tx][q]);
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    for (int e = tid; e < nb * nb; e += blockDim.x) {
      const int r = e % nb, c = e / nb;
      if (r >= c) A[(size_t)(k0 + r) + (size_t)(k0 + c) * J] = D[r][c];
    }
    return;
  }
  const int i0 = k0 + nb + ((int)blockIdx.x - 1) * kNb;
  const int rows = min(kNb, J - i0);
  if (rows <= 0) return;
  for (int e = tid; e < rows * nb; e += blockDim.x) {
    const int r = e % rows, c = e / rows;
    R[r][c] = A[(size_t)(i0 + r) + (size_t)(k0 + c) * J];
  }
  __syncthreads();
  // Rows below the diagonal block exist only for full-width panels (nb = 32): the row is solved
  // in registers, fully unrolled (a shared-memory row would serialise on store-load ordering).
  if (tid < rows) {
    double x[kNb];
#pragma unroll
    for (int c = 0; c < kNb; ++c) x[c] = R[tid][c];
#pragma unroll
    for (int c = 0; c < kNb; ++c) {
      x[c] *= rd[c];
#pragma unroll
      for (int q = c + 1; q < kNb; ++q) x[q] = fma(-x[c], D[q][c], x[q]);
    }
#pragma unroll
    for (int c = 0; c < kNb; ++c) R[tid][c] = x[c];
  }
  __syncthreads();
  for (int e = tid; e < rows * nb; e += blockDim.x) {
    const int r = e % rows, c = e / rows;
    A[(size_t)(i0 + r) + (size_t)(k0 + c) * J] = R[r][c];
  }
}

// Trailing update after panel k0: A[i][j] -= sum_u L[i][k0+u] L[j][k0+u] for k0 + 32 <= j <= i,
// one 32 x 32 tile (tile row ti >= tile column tj) per CTA, 4 outputs per thread.
__global__ void __launch_bounds__(256) chol_update_kernel(double* A, int J, int k0) {
  __shared__ double Li[kNb][kNb + 1], Lj[kNb][kNb + 1];
  const int k1 = k0 + kNb;
  const int t = (int)blockIdx.x;
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int i0 = k1 + ti * kNb, j0 = k1 + tj * kNb;
  const int ri = min(kNb, J - i0), rj = min(kNb, J - j0);
  const int tid = threadIdx.x;
  for (int e = tid; e < kNb * kNb; e += blockDim.x) {
    const int r = e % kNb, c = e / kNb;
    Li[r][c] = r < ri ? A[(size_t)(i0 + r) + (size_t)(k0 + c) * J] : 0.0;
    Lj[r][c] = r < rj ? A[(size_t)(j0 + r) + (size_t)(k0 + c) * J] : 0.0;
  }
  __syncthreads();
  const int r = tid % kNb;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = tid / kNb + 8 * q;
    const int i = i0 + r, j = j0 + c;
    if (r < ri && c < rj && i >= j) {
      double acc = 0.0;
#pragma unroll 8
      for (int u = 0; u < kNb; ++u) acc = fma(Li[r][u], Lj[c][u], acc);
      A[(size_t)i + (size_t)j * J] -= acc;
    }
  }
}

// Solves L L^T X = B for kSolveCols columns of B per CTA (B column-major J x S) and stores X
// row-major [J][S] (the caller's coefficient layout): the forward substitution L y = b walks
// the columns of L, the backward one L^T x = y its rows; L is staged in shared memory 32
// columns (rows) at a time.  Shared memory: (32 + 2 kSolveCols + 1) J doubles.
__global__ void __launch_bounds__(256) chol_solve_kernel(const double* __restrict__ L, int J,
                                                         const double* __restrict__ B, int S, double* __restrict__ X) {
  extern __shared__ double sm[];
  double* Lb = sm;                       // [32][J]
  double* y = Lb + (size_t)kNb * J;      // [kSolveCols][J] working right-hand sides
  double* z = y + (size_t)kSolveCols * J;  // [kSolveCols][J] forward solution
  double* rdg = z + (size_t)kSolveCols * J;  // [J] reciprocals of the pivots
  const int tid = threadIdx.x;
  const int s0 = (int)blockIdx.x * kSolveCols;
  const int ns = min(kSolveCols, S - s0);
  for (int e = tid; e < J; e += blockDim.x) rdg[e] = 1.0 / L[(size_t)e + (size_t)e * J];
  for (int e = tid; e < kSolveCols * J; e += blockDim.x) {
    const int k = e / J, t = e % J;
    y[e] = k < ns ? B[(size_t)t + (size_t)(s0 + k) * J] : 0.0;
  }
  __syncthreads();
  for (int c0 = 0; c0 < J; c0 += kNb) {
    const int nc = min(kNb, J - c0);
    // Eight loads in flight per thread (the staged block comes from L2).
    for (int base = tid; base < nc * J; base += 8 * (int)blockDim.x) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = base + q * (int)blockDim.x, u = e / J, t = e % J;
        v[q] = (e < nc * J && t > c0 + u) ? L[(size_t)t + (size_t)(c0 + u) * J] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = base + q * (int)blockDim.x;
        if (e < nc * J) Lb[(size_t)(e / J) * J + e % J] = v[q];
      }
    }
    __syncthreads();
    for (int u = 0; u < nc; ++u) {
      const int c = c0 + u;
      double yc[kSolveCols];
#pragma unroll
      for (int k = 0; k < kSolveCols; ++k) yc[k] = y[(size_t)k * J + c] * rdg[c];
      if (tid == 0) {
#pragma unroll
        for (int k = 0; k < kSolveCols; ++k) z[(size_t)k * J + c] = yc[k];
      }
      for (int t = c + 1 + tid; t < J; t += blockDim.x) {
        const double l = Lb[(size_t)u * J + t];
#pragma unroll
        for (int k = 0; k < kSolveCols; ++k) y[(size_t)k * J + t] = fma(-l, yc[k], y[(size_t)k * J + t]);
      }
      __syncthreads();
    }
  }
  for (int i0 = (J - 1) / kNb * kNb; i0 >= 0; i0 -= kNb) {
    const int nr = min(kNb, J - i0);
    for (int base = tid; base < nr * (i0 + nr); base += 8 * (int)blockDim.x) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = base + q * (int)blockDim.x, u = e % nr, t = e / nr;
        v[q] = (e < nr * (i0 + nr) && t < i0 + u) ? L[(size_t)(i0 + u) + (size_t)t * J] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = base + q * (int)blockDim.x;
        if (e < nr * (i0 + nr)) Lb[(size_t)(e % nr) * J + e / nr] = v[q];
      }
    }
    __syncthreads();
    for (int u = nr - 1; u >= 0; --u) {
      const int i = i0 + u;
      double xi[kSolveCols];
#pragma unroll
      for (int k = 0; k < kSolveCols; ++k) xi[k] = z[(size_t)k * J + i] * rdg[i];
      if (tid == 0) {
        for (int k = 0; k < ns; ++k) X[(size_t)i * S + (size_t)(s0 + k)] = xi[k];
      }
      for (int t = tid; t < i; t += blockDim.x) {
        const double l = Lb[(size_t)u * J + t];
#pragma unroll
        for (int k = 0; k < kSolveCols; ++k) z[(size_t)k * J + t] = fma(-l, xi[k], z[(size_t)k * J + t]);
      }
      __syncthreads();
    }
  }
}

// Blocked triangular solves for normal matrices beyond the solve kernel's shared-memory limit,
// 32 rows (one diagonal block) at a time: a diagonal-block kernel solves the block's rows for 32
// right-hand sides per CTA, an update kernel subtracts the solved block from the rows still to
// be solved (tiles of 32 rows x 32 right-hand sides).  B is column-major J x S, solved in place;
// every element is written by one thread in a fixed order (deterministic).
// FWD: L y = b (rows k0 .. k0+31 after the rows above are folded in); else L^T x = y (rows
// k0 .. k0+31 after the rows below are folded in).
template <bool FWD>
__global__ void __launch_bounds__(256) trsm_diag_kernel(const double* __restrict__ L, int J, double* B, int S, int k0) {
  __shared__ double D[kNb][kNb + 1];
  __shared__ double X[kNb][kNb + 1];  // [row][rhs]
  const int nb = min(kNb, J - k0);
  const int s0 = (int)blockIdx.x * kNb;
  const int ns = min(kNb, S - s0);
  for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
    const int r = e % kNb, c = e / kNb;
    D[r][c] = (r < nb && c < nb) ? L[(size_t)(k0 + r) + (size_t)(k0 + c) * J] : 0.0;
    X[r][c] = (r < nb && c < ns) ? B[(size_t)(k0 + r) + (size_t)(s0 + c) * J] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < kNb && (int)threadIdx.x < ns) {
    const int c = threadIdx.x;
    if constexpr (FWD) {
      for (int r = 0; r < nb; ++r) {
        double v = X[r][c];
        for (int q = 0; q < r; ++q) v = fma(-D[r][q], X[q][c], v);
        X[r][c] = v / D[r][r];
      }
    } else {
      for (int r = nb - 1; r >= 0; --r) {
        double v = X[r][c];
        for (int q = r + 1; q < nb; ++q) v = fma(-D[q][r], X[q][c], v);
        X[r][c] = v / D[r][r];
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb * ns; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    B[(size_t)(k0 + r) + (size_t)(s0 + c) * J] = X[r][c];
  }
}

// FWD: rows i >= k0 + 32 of B minus L[i][k0..k0+31] times the solved block; else rows i < k0
// minus L[k0..k0+31][i] (= L^T[i][k0..]) times it.  One 32 x 32 tile of (row, rhs) per CTA.
template <bool FWD>
__global__ void __launch_bounds__(256) trsm_update_kernel(const double* __restrict__ L, int J, double* B, int S, int k0) {
  __shared__ double Lt[kNb][kNb + 1];  // [row of the tile][q]
  __shared__ double Xs[kNb][kNb + 1];  // [q][rhs]
  const int nb = min(kNb, J - k0);
  const int i0 = FWD ? k0 + kNb + (int)blockIdx.y * kNb : (int)blockIdx.y * kNb;
  const int i1 = FWD ? J : k0;
  const int s0 = (int)blockIdx.x * kNb;
  const int nr = min(kNb, i1 - i0), ns = min(kNb, S - s0);
  if (nr <= 0) return;
  for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
    const int r = e % kNb, q = e / kNb;
    Lt[r][q] = (r < nr && q < nb) ? (FWD ? L[(size_t)(i0 + r) + (size_t)(k0 + q) * J] : L[(size_t)(k0 + q) + (size_t)(i0 + r) * J])
                                  : 0.0;
    Xs[r][q] = (r < nb && q < ns) ? B[(size_t)(k0 + r) + (size_t)(s0 + q) * J] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x % kNb;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = threadIdx.x / kNb + 8 * k;
    if (r < nr && c < ns) {
      double acc = 0.0;
#pragma unroll 8
      for (int q = 0; q < kNb; ++q) acc = fma(Lt[r][q], Xs[q][c], acc);
      B[(size_t)(i0 + r) + (size_t)(s0 + c) * J] -= acc;
    }
  }
}

// Right-looking blocked Cholesky factorisation of the J x J normal matrix in place (lower
// triangle, column-major); info[0] as in chol_panel_kernel (zeroed here).
zp_status cholesky_factor(double* A, int J, int* info, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
  for (int k0 = 0; k0 < J; k0 += kNb) {
    const int nb = std::min(kNb, J - k0);
    const int below = J - k0 - nb;
    chol_panel_kernel<<<1 + (below + kNb - 1) / kNb, 256, 0, stream>>>(A, J, k0, info);
    if (below > 0) {
      const int64_t nt = (below + kNb - 1) / kNb;
      chol_update_kernel<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, stream>>>(A, J, k0);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "Cholesky panel launch");
  }
  return ZP_OK;
}

// Solves L L^T X = B for the factor in A: B column-major J x S (overwritten), the solution
// stored row-major [J][S] in X by the transpose kernel.
zp_status blocked_cholesky_solve(const double* A, int J, double* B, int S, double* X, cudaStream_t stream);

// Factors the J x J normal matrix (J <= kCholMaxJ) in place and solves for the J x S
// right-hand sides B (column-major), storing the solution row-major [J][S] in X; info[0] as in
// chol_panel_kernel (zeroed here).
zp_status small_cholesky_solve(double* A, int J, const double* B, int S, double* X, int* info, cudaStream_t stream) {
  ZP_TRY(cholesky_factor(A, J, info, stream));
  cudaError_t e;
  const size_t smem = (size_t)(kNb + 2 * kSolveCols + 1) * J * sizeof(double);
  static DeviceMemo<int> attr;  // the largest solve's shared memory, allowed once per device
  int dummy = 0;
  ZP_TRY(attr.get(&dummy, [](int* x) -> zp_status {
    *x = (kNb + 2 * kSolveCols + 1) * kCholMaxJ * (int)sizeof(double);
    const cudaError_t err = cudaFuncSetAttribute(chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, *x);
    return err == cudaSuccess ? ZP_OK : cuda_error(err, "cudaFuncSetAttribute(chol_solve_kernel)");
  }));
  chol_solve_kernel<<<(S + kSolveCols - 1) / kSolveCols, 256, smem, stream>>>(A, J, B, S, X);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "chol_solve_kernel launch");
  return ZP_OK;
}

// out row-major [J][S] from in column-major J x S (32 x 32 tiles through shared memory).
__global__ void __launch_bounds__(256) transpose_kernel(const double* __restrict__ in, int64_t J, int64_t S,
                                                        double* __restrict__ out) {
  __shared__ double t[32][33];
  const int64_t s0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    const int jj = e % 32, ss = e / 32;
    if (j0 + jj < J && s0 + ss < S) t[ss][jj] = in[(j0 + jj) + (s0 + ss) * J];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    const int ss = e % 32, jj = e / 32;
    if (j0 + jj < J && s0 + ss < S) out[(j0 + jj) * S + (s0 + ss)] = t[ss][jj];
  }
}

zp_status blocked_cholesky_solve(const double* A, int J, double* B, int S, double* X, cudaStream_t stream) {
  const unsigned cols = (unsigned)((S + kNb - 1) / kNb);
  cudaError_t e;
  for (int k0 = 0; k0 < J; k0 += kNb) {
    trsm_diag_kernel<true><<<cols, 256, 0, stream>>>(A, J, B, S, k0);
    const int below = J - k0 - kNb;
    if (below > 0) trsm_update_kernel<true><<<dim3(cols, (unsigned)((below + kNb - 1) / kNb)), 256, 0, stream>>>(A, J, B, S, k0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "forward substitution launch");
  }
  for (int k0 = (J - 1) / kNb * kNb; k0 >= 0; k0 -= kNb) {
    trsm_diag_kernel<false><<<cols, 256, 0, stream>>>(A, J, B, S, k0);
    if (k0 > 0) trsm_update_kernel<false><<<dim3(cols, (unsigned)((k0 + kNb - 1) / kNb)), 256, 0, stream>>>(A, J, B, S, k0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "backward substitution launch");
  }
  transpose_kernel<<<dim3((unsigned)((S + 31) / 32), (unsigned)((J + 31) / 32)), 256, 0, stream>>>(B, J, S, X);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "transpose_kernel launch");
  return ZP_OK;
}

struct BlasHandles {
  std::mutex mu;
  std::vector<cublasHandle_t> blas;
};
BlasHandles& blas_handles() {
  static BlasHandles h;
  return h;
}

}  // namespace

zp_status series_fit_fp64(const zp_plan* plan, const double* r, const double* theta, const double* w, int64_t P,
                          const double* Y, int64_t S, double ridge, double* coeffs, cudaStream_t stream,
                          bool emulated) {
  const int64_t J = plan->n_modes;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  // cuBLAS only for the DGEMM baseline (ZP_PREC_FP64).
  BlasHandles& hs = blas_handles();
  std::unique_lock<std::mutex> lock(hs.mu, std::defer_lock);
  cublasHandle_t blas = nullptr;
  if (!emulated) {
    lock.lock();
    if ((int)hs.blas.size() <= dev) hs.blas.resize(dev + 1, nullptr);
    if (!hs.blas[dev] && cublasCreate(&hs.blas[dev]) != CUBLAS_STATUS_SUCCESS)
      return set_error(ZP_ERR_CUDA, "cublasCreate failed");
    blas = hs.blas[dev];
    if (cublasSetStream(blas, stream) != CUBLAS_STATUS_SUCCESS)
      return set_error(ZP_ERR_CUDA, "setting the stream of the cuBLAS handle failed");
  }

  ScratchBuffer zbuf, ybuf, gram, rhs, info;
  ZP_TRY(zbuf.alloc((size_t)J * P * sizeof(double), stream));
  ZP_TRY(gram.alloc((size_t)J * J * sizeof(double), stream));
  ZP_TRY(rhs.alloc((size_t)J * S * sizeof(double), stream));
  ZP_TRY(info.alloc(4 * sizeof(double), stream));  // [0]: potrf status (int), [2..3]: pivot range
  double* Z = (double*)zbuf.ptr;
  ZP_TRY(launch_walk(plan, r, theta, P, 0, Z, nullptr, stream));
  const double* Yuse = Y;
  ScratchBuffer swbuf;
  if (w) {
    ZP_TRY(ybuf.alloc((size_t)P * S * sizeof(double), stream));
    ZP_TRY(swbuf.alloc((size_t)P * sizeof(double), stream));
    double* sw = (double*)swbuf.ptr;
    sqrt_weights_kernel<<<(unsigned)std::min<int64_t>((P + 255) / 256, 4096), 256, 0, stream>>>(w, sw, P);
    const dim3 rgrid((unsigned)std::min<int64_t>((P + 255) / 256, 64), (unsigned)std::min<int64_t>(J, 4096));
    scale_rows_kernel<<<rgrid, 256, 0, stream>>>(Z, J, P, sw);
    scale_samples_kernel<<<(unsigned)std::min<int64_t>(P, 16384), 256, 0, stream>>>(Y, (double*)ybuf.ptr, P, S, sw);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "weight scaling launch");
    Yuse = (const double*)ybuf.ptr;
  }
  const double one = 1.0, zero = 0.0;
  if (emulated) {
    // Gram[i][j] = sum_p Z[i][p] Z[j][p] (exactly symmetric: both operands carry the same
    // scales and slices); RHS column-major J x S = row-major [S][J]: rhs[s][j] = sum_p Y[p][s] Z[j][p].
    ZP_TRY(emulated_gemm_fp64(J, J, P, Z, P, 1, Z, P, 1, (double*)gram.ptr, J, stream));
    ZP_TRY(emulated_gemm_fp64(S, J, P, Yuse, 1, S, Z, P, 1, (double*)rhs.ptr, J, stream));
  } else {
    // Z row-major [J][P] is column-major P x J (Zc).  Gram = Zc^T Zc: a full DGEMM (cuBLAS's
    // DSYRK measured three times slower for these shapes), of which potrf reads the lower half.
    if (cublasDgemm_64(blas, CUBLAS_OP_T, CUBLAS_OP_N, J, J, P, &one, Z, P, Z, P, &zero, (double*)gram.ptr, J) !=
        CUBLAS_STATUS_SUCCESS)
      return set_error(ZP_ERR_CUDA, "cublasDgemm (Gram) failed");
    // RHS (column-major J x S) = Zc^T (J x P) * Yc^T (P x S), Y row-major [P][S] = column-major S x P.
    if (cublasDgemm_64(blas, CUBLAS_OP_T, CUBLAS_OP_T, J, S, P, &one, Z, P, Yuse, S, &zero, (double*)rhs.ptr, J) !=
        CUBLAS_STATUS_SUCCESS)
      return set_error(ZP_ERR_CUDA, "cublasDgemm failed");
  }
  if (ridge > 0.0) {
    add_ridge_kernel<<<(unsigned)((J + 255) / 256), 256, 0, stream>>>((double*)gram.ptr, J, ridge);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "add_ridge_kernel launch");
  }
  if (J <= kCholMaxJ) {
    ZP_TRY(small_cholesky_solve((double*)gram.ptr, (int)J, (const double*)rhs.ptr, (int)S, coeffs, (int*)info.ptr,
                                stream));
  } else {
    ZP_TRY(cholesky_factor((double*)gram.ptr, (int)J, (int*)info.ptr, stream));
    ZP_TRY(blocked_cholesky_solve((const double*)gram.ptr, (int)J, (double*)rhs.ptr, (int)S, coeffs, stream));
  }
  pivot_range_kernel<<<1, 256, 0, stream>>>((const double*)gram.ptr, J, (double*)info.ptr + 2);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "pivot_range_kernel launch");
  double h_info[4] = {0, 0, 0, 0};
  if ((e = cudaMemcpyAsync(h_info, info.ptr, sizeof(h_info), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return cuda_error(e, "reading the factorisation status");
  int status = 0;
  memcpy(&status, h_info, sizeof(int));
  // A rank-deficient normal matrix can factor with tiny positive pivots in floating point;
  // a squared-pivot ratio below 1e-14 (condition number above ~1e14) is reported as singular.
  if (status != 0 || !(h_info[2] > 1e-14 * h_info[3]))
    return set_error(ZP_ERR_INVALID_ARG, "normal matrix not positive definite (potrf status " + std::to_string(status) +
                                             ", squared pivot ratio " + std::to_string(h_info[2] / h_info[3]) +
                                             "): fewer independent points than modes, or duplicated modes; add a "
                                             "ridge");
  return ZP_OK;
}

}  // namespace zp

using namespace zp;

extern "C" {

static zp_status zp_series_fit_plan_impl(const zp_plan* plan, const double* r, const double* theta, const double* weights,
                             int64_t n_points, const double* samples, int64_t n_sets, double ridge, double* coeffs,
                             void* stream) {
  return zp_series_fit_plan_prec(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs,
                                 ZP_PREC_FP64_EMULATED, stream);
}

zp_status zp_series_fit_plan(const zp_plan* plan, const double* r, const double* theta, const double* weights,
                             int64_t n_points, const double* samples, int64_t n_sets, double ridge, double* coeffs,
                             void* stream) {
  zp::NvtxRange zp_range_("zp_series_fit_plan");
  return zp::entry_finish("zp_series_fit_plan", stream, zp_series_fit_plan_impl(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, stream));
}

static zp_status zp_series_fit_plan_prec_impl(const zp_plan* plan, const double* r, const double* theta, const double* weights,
                                  int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                                  double* coeffs, zp_precision prec, void* stream) {
  clear_error();
  if (prec != ZP_PREC_FP64 && prec != ZP_PREC_FP64_EMULATED)
    return set_error(ZP_ERR_INVALID_ARG, "the fit takes ZP_PREC_FP64 or ZP_PREC_FP64_EMULATED");
  ZP_TRY(check_plan_device(plan));
  if (n_points < 0 || n_sets < 0) return set_error(ZP_ERR_INVALID_ARG, "negative size");
  if (!(ridge >= 0.0)) return set_error(ZP_ERR_INVALID_ARG, "ridge must be >= 0");
  if (plan->n_modes > 46340) return set_error(ZP_ERR_UNSUPPORTED, "fit supports at most 46340 modes");
  if (plan->n_modes == 0 || n_sets == 0) return ZP_OK;
  if (n_points == 0) return set_error(ZP_ERR_INVALID_ARG, "no points to fit");
  ZP_TRY(check_device_array(r, "r", 8));
  ZP_TRY(check_device_array(theta, "theta", 8));
  ZP_TRY(check_device_array(samples, "samples", 8));
  ZP_TRY(check_device_array(coeffs, "coeffs", 8));
  if (weights) ZP_TRY(check_device_array(weights, "weights", 8));
  if (n_sets > 0x7fffffff || plan->n_modes * n_sets > 0x7fffffffLL)
    return set_error(ZP_ERR_UNSUPPORTED, "fit output too large");
  return series_fit_fp64(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, (cudaStream_t)stream,
                         prec == ZP_PREC_FP64_EMULATED);
}

zp_status zp_series_fit_plan_prec(const zp_plan* plan, const double* r, const double* theta, const double* weights,
                                  int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                                  double* coeffs, zp_precision prec, void* stream) {
  zp::NvtxRange zp_range_("zp_series_fit_plan_prec");
  return zp::entry_finish("zp_series_fit_plan_prec", stream, zp_series_fit_plan_prec_impl(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, prec, stream));
}

static zp_status zp_series_fit_impl(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                        const double* weights, int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                        double* coeffs, void* stream) {
  clear_error();
  std::shared_ptr<const zp_plan> held;
  ZP_TRY(cached_plan(n, m, n_modes, &held));
  const zp_plan* plan = held.get();
  return zp_series_fit_plan(plan, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, stream);
}

zp_status zp_series_fit(const int32_t* n, const int32_t* m, int64_t n_modes, const double* r, const double* theta,
                        const double* weights, int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                        double* coeffs, void* stream) {
  zp::NvtxRange zp_range_("zp_series_fit");
  return zp::entry_finish("zp_series_fit", stream, zp_series_fit_impl(n, m, n_modes, r, theta, weights, n_points, samples, n_sets, ridge, coeffs, stream));
}

}  // extern "C"
