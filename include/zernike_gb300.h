/*
 * zernike_gb300.h -- C ABI of the GB300 (sm_103a) Zernike basis / series library.
 *
 * The library evaluates the radial Zernike polynomials R_n^m(rho), their rho-derivatives
 * of order 0..3, the Zernike functions Z_n^m(rho, theta) = R_n^{|m|}(rho) cos(m theta)
 * (m >= 0) or R_n^{|m|}(rho) sin(|m| theta) (m < 0), and series of them, through the
 * Jacobi form R_n^m(rho) = (-1)^((n-m)/2) rho^m P_{(n-m)/2}^{(m,0)}(1 - 2 rho^2) and the
 * three-term Jacobi recursion in n for each m (Sec. 2: the Jacobi relation, the beta = 0
 * recursion; Sec. 3: Algorithm 1's per-m column walk).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Mode lists n[], m[] are HOST int32 arrays of length n_modes.  A mode is valid when
 *    n >= 0, |m| <= n and n - |m| is even (Sec. 2).  Duplicated modes are allowed (the
 *    duplicated-modes variant of Sec. 3); each occurrence gets its own output column.
 *    Output columns follow the caller's mode order.  Radial entry points use |m|.
 *  - Point arrays r[] (and theta[]) are DEVICE float64 arrays of length n_points.  r is
 *    evaluated as the polynomial it is: values outside [0, 1] are not clamped.
 *  - Outputs are DEVICE arrays owned and allocated by the caller; the library never keeps a
 *    pointer to them after the call returns.
 *  - DEVICE means reachable by the current device at that address: its own memory, managed
 *    memory, or pinned host memory mapped at the same address (cudaHostAlloc, cudaHostRegister
 *    under unified addressing), which the kernels then read or write across the host link.  Layouts are row-major with the point index
 *    fastest unless stated.
 *  - Arguments are validated on the host before anything is launched.  On any error the
 *    call returns a non-zero zp_status, launches nothing and leaves outputs untouched;
 *    zp_last_error() then holds a one-line description (per host thread).
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream) on the CURRENT device.  n_points == 0 or n_modes == 0 returns
 *    ZP_OK without launching.
 *  - The mode-list entry points build (and cache, keyed by the exact mode list and device)
 *    a plan on first use; that first call copies small tables to the device synchronously.
 *    Inside CUDA-graph capture use the *_plan variants with a plan created beforehand.
 *  - Every compute entry point opens an NVTX range named after itself (visible in Nsight
 *    timelines).  The environment variable ZP_DEBUG (read once per process) adds checks: 1
 *    synchronises the caller's stream at the end of each compute call (outside stream capture)
 *    and turns an asynchronous CUDA error or a bounded device wait that gave up into that call's
 *    status; 2 also prints one line per call to stderr.  The default (unset, 0) adds nothing.
 */
#ifndef ZERNIKE_GB300_H
#define ZERNIKE_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ZP_API __attribute__((visibility("default")))
#else
#define ZP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ZP_OK = 0,
  ZP_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad enum, misaligned pointer */
  ZP_ERR_INVALID_MODE = 2,  /* a mode breaks n >= 0, |m| <= n, n - |m| even, or n > ZP_MAX_N */
  ZP_ERR_DERIV_ORDER = 3,   /* derivative order outside 0..3 */
  ZP_ERR_CUDA = 4,          /* a CUDA runtime or cuBLAS call failed */
  ZP_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  ZP_ERR_UNSUPPORTED = 6,   /* valid request the library cannot serve (e.g. wrong GPU) */
  ZP_ERR_NO_MEMORY = 7      /* a device allocation failed */
} zp_status;

typedef enum {
  ZP_PREC_FP64 = 0,   /* the plain float64 basis-then-GEMM form, kept as the baseline: the basis
                         is written to scratch and contracted by cuBLAS DGEMM; outputs float64.
                         The library's default float64 path is ZP_PREC_FP64_EMULATED */
  ZP_PREC_BF16X3 = 1, /* float64 basis, contraction on tensor cores as hi*hi + hi*lo + lo*hi
                         with bfloat16 halves and float32 accumulation; outputs float32 */
  ZP_PREC_TF32 = 2,   /* float64 basis rounded to TF32, tensor-core contraction with float32
                         accumulation; outputs float32 */
  ZP_PREC_FP32 = 3,   /* float64 basis rounded to float32, float32 contraction on the CUDA
                         cores; outputs float32 (batched forward only) */
  ZP_PREC_FP64_EMULATED = 4 /* float64-accurate contraction on the tensor cores: rows of Z and
                         columns of C scaled by powers of two and cut into small-integer bf16
                         slices (54 bits, error-free), exact sums per slice diagonal, exact
                         integer recombination rounded once to float64; outputs float64
                         (zp_series_eval only, <= 16320 modes).  The error is bounded by the
                         scales, about n_modes * 2^-54 * max_j |Z[j][p]| * max_j |C[j][s]| for
                         F[p][s], rather than by sum_j |Z C| as for float64 arithmetic: a
                         coefficient set whose entries span many orders of magnitude keeps
                         fewer bits on its small entries than the FP64 path.  An infinity or
                         NaN in a coefficient set (or in a point's basis row) makes that set's
                         (point's) outputs NaN.  Scratch (stream-ordered): the slices of C and
                         of a slab of points and the slab's int32 diagonal sums, about 4.5 GB at
                         most */
} zp_precision;

/* Largest radial order accepted (recursion tables live in shared memory). */
#define ZP_MAX_N 1000

typedef struct zp_plan zp_plan;

/* One-line text for a status code (static storage). */
ZP_API const char* zp_status_string(zp_status status);

/* Description of the last error raised on the calling host thread ("" if none). */
ZP_API const char* zp_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
ZP_API int32_t zp_version(void);

/*
 * Plans.  A plan holds everything derived from a mode list: validation, the grouping of
 * modes into |m| columns ordered by recursion length (Algorithm 1's outer loop over
 * alpha = m), the Jacobi-degree N = (n - |m|)/2 of every output column, and the recursion
 * coefficient tables of the beta = 0 Jacobi recursion (Sec. 2), uploaded to the current
 * device.  zp_plan_create copies tables synchronously (call it outside stream capture).
 * A plan may be used from any stream of the device it was created on; it is read-only
 * after creation and may be shared by concurrent calls.  zp_plan_destroy frees it
 * (synchronising the device first).  *out is written only on success.
 */
ZP_API zp_status zp_plan_create(const int32_t* n, const int32_t* m, int64_t n_modes, zp_plan** out);
ZP_API zp_status zp_plan_destroy(zp_plan* plan);
/* n_modes, largest n, number of distinct |m| columns of a plan (any pointer may be NULL). */
ZP_API zp_status zp_plan_info(const zp_plan* plan, int64_t* n_modes, int32_t* n_max, int32_t* n_columns);

/*
 * Radial polynomials and rho-derivatives (Sec. 2 Jacobi relation and recursion; derivative
 * orders as in the accuracy study of Sec. 4, Fig. 1).
 *   out: DEVICE float64 [max_deriv+1][n_modes][n_points];
 *        out[(k*n_modes + j)*n_points + p] = d^k/drho^k R_{n_j}^{|m_j|}(r_p).
 *   max_deriv in 0..3.
 */
ZP_API zp_status zp_radial(const int32_t* n, const int32_t* m, int64_t n_modes,
                    const double* r, int64_t n_points, int32_t max_deriv,
                    double* out, void* stream);
ZP_API zp_status zp_radial_plan(const zp_plan* plan, const double* r, int64_t n_points,
                         int32_t max_deriv, double* out, void* stream);
/*
 * zp_radial_plan with per-kernel timing: CUDA events are recorded on `stream` around each
 * launch and phase_ms[0] receives the device time of the point-preparation kernel (powers of
 * rho; 0 when the launch is too small to use it), phase_ms[1] that of the recursion walk.
 * Same outputs as zp_radial_plan.  The call synchronises `stream` before returning
 * (instrumentation; not for graph capture).
 */
ZP_API zp_status zp_radial_plan_timed(const zp_plan* plan, const double* r, int64_t n_points,
                                      int32_t max_deriv, double* out, void* stream, float* phase_ms);

/*
 * Zernike functions (Sec. 2 definition of Z) and their derivatives.
 *   out:        DEVICE float64 [max_deriv+1][n_modes][n_points],
 *               out[(k*n_modes + j)*n_points + p] = d^k/drho^k Z_{n_j}^{m_j}(r_p, theta_p).
 *   out_dtheta: DEVICE float64 [n_modes][n_points] = d/dtheta Z_{n_j}^{m_j}, or NULL.
 */
ZP_API zp_status zp_basis(const int32_t* n, const int32_t* m, int64_t n_modes,
                   const double* r, const double* theta, int64_t n_points, int32_t max_deriv,
                   double* out, double* out_dtheta, void* stream);
ZP_API zp_status zp_basis_plan(const zp_plan* plan, const double* r, const double* theta,
                        int64_t n_points, int32_t max_deriv, double* out, double* out_dtheta,
                        void* stream);

/*
 * Algorithm 2 of Sec. 3 (the paper's per-mode GPU variant): every (point, mode) runs its
 * own recursion from P_0, P_1 up to its own degree and stores only the last value.  Kept
 * as the comparison kernel for the per-column walk; same output layout as zp_radial with
 * max_deriv = 0.
 */
ZP_API zp_status zp_radial_per_mode(const zp_plan* plan, const double* r, int64_t n_points,
                             double* out, void* stream);

/*
 * Series of Zernike functions (the spectral expansion motivated in Sec. 3's footnote):
 *   F[p, s] = sum_j Z_j(r_p, theta_p) * coeffs[j, s].
 *   coeffs: DEVICE float64 [n_modes][n_sets] row-major.
 *   out:    DEVICE [n_points][n_sets] row-major; float64 for ZP_PREC_FP64, float32 for
 *           ZP_PREC_BF16X3 / ZP_PREC_TF32.
 * ZP_PREC_FP64_EMULATED is the float64-accurate form to use; ZP_PREC_FP64 is the plain
 * baseline: it writes the basis to scratch device memory (allocated stream-ordered on `stream`
 * from the library's scratch pool, see zp_release_scratch, and released to it before return)
 * and contracts with cuBLAS DGEMM.  The split forms run the float64 recursion into
 * tensor-core operand tiles in scratch (slabs of whole waves of point tiles) and contract them
 * with tcgen05 MMAs and float32 accumulation.  ZP_PREC_FP64_EMULATED with n_sets <= 16 and at
 * most 5041 padded modes builds the basis inside the tensor-core kernel (no basis in memory):
 * each value Q_N cos/sin(m theta) is scaled by one power of two per point (on the unit disc
 * the plan's bound on |Z| over its smallest recursion weight; off the disc the point's own
 * largest value) and cut into 11 digits of 5 bits, or 9 of 6 bits when the padded modes are
 * at most 1489 (54 or 55 fraction bits: the error bound above with that power of two in place
 * of max_j |Z[j][p]|).
 */
ZP_API zp_status zp_series_eval(const int32_t* n, const int32_t* m, int64_t n_modes,
                         const double* r, const double* theta, int64_t n_points,
                         const double* coeffs, int64_t n_sets, zp_precision prec,
                         void* out, void* stream);
ZP_API zp_status zp_series_eval_plan(const zp_plan* plan, const double* r, const double* theta,
                              int64_t n_points, const double* coeffs, int64_t n_sets,
                              zp_precision prec, void* out, void* stream);

/*
 * zp_series_eval_plan for ZP_PREC_BF16X3 / ZP_PREC_TF32 with per-phase timing: CUDA events
 * are recorded on `stream` around each launch and phase_ms[0..2] receives the summed device
 * time of the coefficient split, the basis split and the tensor-core GEMM launches.  The
 * call synchronises `stream` before returning (instrumentation; not for graph capture).
 */
ZP_API zp_status zp_series_eval_timed(const zp_plan* plan, const double* r, const double* theta,
                                      int64_t n_points, const double* coeffs, int64_t n_sets,
                                      zp_precision prec, void* out, void* stream, float* phase_ms);

/*
 * Adjoint of the series (the reverse-mode derivative that Sec. 3 provides by a custom
 * rule), float64 results.  With G = grad_out (DEVICE float64 [n_points][n_sets]):
 *   grad_coeffs[j, s] = sum_p Z_j(p) G[p, s]                         ([n_modes][n_sets])
 *   grad_r[p]         = sum_j dZ_j/drho(p)   sum_s coeffs[j, s] G[p, s]      ([n_points])
 *   grad_theta[p]     = sum_j dZ_j/dtheta(p) sum_s coeffs[j, s] G[p, s]      ([n_points])
 * Any of the three outputs may be NULL (not computed).  The basis is recomputed, never
 * read from a previous forward call.  Reductions are deterministic (no float atomics).
 * The contractions grad_coeffs = Z G and H = C G^T run on the float64-accurate tensor-core
 * GEMM of ZP_PREC_FP64_EMULATED (zp_series_adjoint_plan_prec selects the DGEMM baseline).
 */
ZP_API zp_status zp_series_adjoint(const int32_t* n, const int32_t* m, int64_t n_modes,
                            const double* r, const double* theta, int64_t n_points,
                            const double* coeffs, int64_t n_sets, const double* grad_out,
                            double* grad_coeffs, double* grad_r, double* grad_theta,
                            void* stream);
ZP_API zp_status zp_series_adjoint_plan(const zp_plan* plan, const double* r, const double* theta,
                                 int64_t n_points, const double* coeffs, int64_t n_sets,
                                 const double* grad_out, double* grad_coeffs, double* grad_r,
                                 double* grad_theta, void* stream);
/*
 * zp_series_adjoint_plan with a choice of contraction arithmetic: ZP_PREC_FP64 (the cuBLAS
 * DGEMM baseline) or ZP_PREC_FP64_EMULATED (the default: grad_coeffs = Z G and H = C G^T by the
 * float64-accurate tensor-core GEMM of ZP_PREC_FP64_EMULATED, with the scale-relative error
 * bound stated there: about K 2^-54 times the largest operand magnitudes of the row and
 * column, K = n_points for grad_coeffs and n_sets for H).  grad_r and grad_theta are then
 * reduced in float64 as for ZP_PREC_FP64 -- except for n_sets <= 16 (and at most 5041 padded
 * modes), where they are the row sums grad_out[p] . (dZ/dtheta C)[p] and grad_out[p] . (dZ/drho
 * C)[p] of the fused kernel's derivative series (no modes x points matrix H; deterministic).
 * Other precisions: ZP_ERR_INVALID_ARG.
 */
ZP_API zp_status zp_series_adjoint_plan_prec(const zp_plan* plan, const double* r, const double* theta,
                                             int64_t n_points, const double* coeffs, int64_t n_sets,
                                             const double* grad_out, double* grad_coeffs, double* grad_r,
                                             double* grad_theta, zp_precision prec, void* stream);

/*
 * Second derivatives for Jacobian/Hessian work (Sec. 3 mentions Jacobian and Hessian
 * calculations through automatic differentiation).  For the scalar L = sum_{p,s} F[p,s] G[p,s]
 * the Hessian in the point coordinates is block diagonal (r_p, theta_p enter row p only);
 * this returns each point's block and gradient, float64:
 *   grad_r[p]  = dL/dr_p,        grad_theta[p] = dL/dtheta_p,
 *   hess_rr[p] = d2L/dr_p^2,     hess_rt[p] = d2L/dr_p dtheta_p,     hess_tt[p] = d2L/dtheta_p^2.
 * Any output may be NULL.  grad_out = G, DEVICE float64 [n_points][n_sets].  Same basis
 * recomputation and reduction as zp_series_adjoint (one extra Taylor lane; H = C G^T on the
 * float64-accurate tensor-core GEMM).
 */
ZP_API zp_status zp_series_point_hessian(const int32_t* n, const int32_t* m, int64_t n_modes,
                                         const double* r, const double* theta, int64_t n_points,
                                         const double* coeffs, int64_t n_sets, const double* grad_out,
                                         double* grad_r, double* grad_theta, double* hess_rr,
                                         double* hess_rt, double* hess_tt, void* stream);
ZP_API zp_status zp_series_point_hessian_plan(const zp_plan* plan, const double* r,
                                              const double* theta, int64_t n_points,
                                              const double* coeffs, int64_t n_sets,
                                              const double* grad_out, double* grad_r,
                                              double* grad_theta, double* hess_rr, double* hess_rt,
                                              double* hess_tt, void* stream);

/*
 * Hessian-vector product of L = sum_{p,s} F[p,s] G[p,s] in the point coordinates for a
 * tangent (v_r, v_theta) (DEVICE float64 [n_points] each): with the per-point blocks of
 * zp_series_point_hessian,
 *   hv_r[p]     = hess_rr[p] v_r[p] + hess_rt[p] v_theta[p],
 *   hv_theta[p] = hess_rt[p] v_r[p] + hess_tt[p] v_theta[p]
 * (the Hessian is block diagonal, so the product is per point), formed inside the same kernel
 * without storing the blocks.  Either output may be NULL.
 */
ZP_API zp_status zp_series_point_hvp_plan(const zp_plan* plan, const double* r, const double* theta,
                                          int64_t n_points, const double* coeffs, int64_t n_sets,
                                          const double* grad_out, const double* v_r, const double* v_theta,
                                          double* hv_r, double* hv_theta, void* stream);

/*
 * Least-squares fit of series coefficients (the "fit" counterpart of zp_series_eval):
 *   minimise sum_p w_p || sum_j Z_j(r_p, theta_p) C[j, :] - Y[p, :] ||^2 + ridge ||C||^2
 * through the normal equations (Z W Z^T + ridge I) C = Z W Y, float64 results (basis by the
 * recursion walk, Gram matrix and right-hand side by the float64-accurate tensor-core GEMM of
 * ZP_PREC_FP64_EMULATED, Cholesky factorisation and the two triangular solves by the library's
 * own blocked kernels).
 *   weights: DEVICE float64 [n_points] (w_p >= 0) or NULL (all 1).
 *   samples: DEVICE float64 [n_points][n_sets] (Y, row-major).
 *   coeffs:  DEVICE float64 [n_modes][n_sets] (output, row-major).
 *   ridge >= 0 (Tikhonov term; 0 for plain least squares).
 * Scratch is allocated stream-ordered on `stream`.  The call synchronises `stream` to read the
 * factorisation status: a singular or numerically singular normal matrix (squared Cholesky
 * pivot ratio below 1e-14: fewer independent points than modes, or a duplicated mode without
 * ridge) returns ZP_ERR_INVALID_ARG after writing coeffs.  At most 46340 modes.
 */
ZP_API zp_status zp_series_fit(const int32_t* n, const int32_t* m, int64_t n_modes,
                               const double* r, const double* theta, const double* weights,
                               int64_t n_points, const double* samples, int64_t n_sets, double ridge,
                               double* coeffs, void* stream);
ZP_API zp_status zp_series_fit_plan(const zp_plan* plan, const double* r, const double* theta,
                                    const double* weights, int64_t n_points, const double* samples,
                                    int64_t n_sets, double ridge, double* coeffs, void* stream);
/*
 * zp_series_fit_plan with a choice of arithmetic for the Gram matrix Z W Z^T and the
 * right-hand side Z W Y: ZP_PREC_FP64 (the cuBLAS DGEMM baseline) or ZP_PREC_FP64_EMULATED (the
 * default: the float64-accurate tensor-core GEMM, error about n_points 2^-54 times the largest magnitudes
 * of the rows involved).  The Cholesky factorisation and solve are float64 either way.  Other precisions: ZP_ERR_INVALID_ARG.
 */
ZP_API zp_status zp_series_fit_plan_prec(const zp_plan* plan, const double* r, const double* theta,
                                         const double* weights, int64_t n_points, const double* samples,
                                         int64_t n_sets, double ridge, double* coeffs, zp_precision prec,
                                         void* stream);

/*
 * Batched series over many instances of uneven size (different mode lists, point counts)
 * in one persistent launch per pass; the launches are stream-ordered and contain no host
 * synchronisation, so zp_batch_forward / zp_batch_adjoint can be captured in a CUDA graph.
 * The paper evaluates one mode set at a time (Sec. 3, Algorithm 1); this is the throughput
 * form of the same per-column recursion for many independent problems.
 *
 * zp_instance: HOST mode list n[], m[] (n_modes entries); DEVICE arrays r, theta
 * [n_points], coeffs [n_modes][n_sets] (float64); out [n_points][n_sets] (float64 for
 * ZP_PREC_FP64, float32 for ZP_PREC_FP32); for the adjoint grad_out [n_points][n_sets]
 * (float64) and optional outputs grad_coeffs [n_modes][n_sets], grad_r, grad_theta
 * [n_points] (float64, NULL = not computed).  All sets share one n_sets.
 * zp_batch_create validates every instance, builds one plan per distinct mode list, copies
 * tables and descriptors to the device (synchronously) and keeps the device pointers: the
 * arrays must stay allocated, and may change contents, between calls.  The passes of one batch
 * share its scratch (work counters, coefficient digits): issue them on one stream, or order
 * streams with events, never concurrently.
 */
typedef struct {
  const int32_t* n;
  const int32_t* m;
  int64_t n_modes;
  const double* r;
  const double* theta;
  int64_t n_points;
  const double* coeffs;
  void* out;
  const double* grad_out;
  double* grad_coeffs;
  double* grad_r;
  double* grad_theta;
} zp_instance;

typedef struct zp_batch zp_batch;

ZP_API zp_status zp_batch_create(const zp_instance* instances, int64_t n_instances, int64_t n_sets,
                                 zp_batch** out);
ZP_API zp_status zp_batch_destroy(zp_batch* batch);
/* F for every instance: one launch (plus a float32 copy of C for ZP_PREC_FP32). */
ZP_API zp_status zp_batch_forward(zp_batch* batch, zp_precision prec, void* stream);
/* The same float64 forward as one launch per instance (comparison path). */
ZP_API zp_status zp_batch_forward_per_instance(zp_batch* batch, zp_precision prec, void* stream);
/* grad_r, grad_theta (one launch) and grad_coeffs (one launch), float64 on the CUDA cores,
 * deterministic (the same as zp_batch_adjoint_prec with ZP_PREC_FP64). */
ZP_API zp_status zp_batch_adjoint(zp_batch* batch, void* stream);
/* The adjoint with a chosen contraction: ZP_PREC_FP64 as zp_batch_adjoint; or
 * ZP_PREC_FP64_EMULATED (float64-accurate on the tensor cores, deterministic, no host
 * synchronisation): grad_theta[p] = sum_s grad_out[p][s] (dZ/dtheta C)[p][s] and grad_r likewise
 * with dZ/drho, each derivative series by the fused kernel of ZP_PREC_FP64_EMULATED's batched
 * forward (one launch each; its row sums added onto the zeroed gradients) when n_sets <= 16 and
 * every instance has at most 5041 modes, else by the float64 point kernel; and per instance
 * grad_coeffs = Z G by the float64-accurate GEMM of zp_series_adjoint_plan (Z walked into
 * library scratch).  Other precisions: ZP_ERR_INVALID_ARG. */
ZP_API zp_status zp_batch_adjoint_prec(zp_batch* batch, zp_precision prec, void* stream);
/* Launch configuration: point-tile size (threads per CTA of the point kernel, multiple of 32),
 * persistent CTAs per SM, points per thread (1, 2, 4) and threads per CTA of the grad_coeffs
 * kernel (a new batch: 128, 8, 2, 128).  cfg[4] receives the current values. */
ZP_API zp_status zp_batch_set_config(zp_batch* batch, int32_t tile_points, int32_t ctas_per_sm,
                                     int32_t col_ppt, int32_t col_threads);
ZP_API zp_status zp_batch_get_config(const zp_batch* batch, int32_t* cfg);
/* Autotuner: times each candidate configuration on this batch (which = 0: forward with
 * `prec`, 1: adjoint), one warm-up then `reps` timed runs with CUDA events on `stream`, and
 * keeps the fastest; cfg[4] (may be NULL) and *best_ms receive the result.  Synchronises
 * `stream`; outputs hold the result of the last candidate run.  Results are kept per GPU
 * (compute capability, SM count) and batch shape (instances, points, modes, largest n, sets,
 * pass, precision): a later tune of the same key applies the kept configuration without
 * launching anything.  When the environment variable ZP_TUNE_CACHE names a file, results are
 * appended there (one line per key) and read back by later processes. */
ZP_API zp_status zp_batch_tune(zp_batch* batch, int32_t which, zp_precision prec, int32_t reps,
                               void* stream, int32_t* cfg, float* best_ms);

/*
 * Allocation-free series evaluation.  (The paper has no counterpart: this is a library
 * service for callers that cannot allocate device memory while they run, such as code in a
 * host callback or an allocator hook, applications that reserve all device memory at
 * start-up, or latency-critical loops where a cudaMalloc would stall other work.)
 *
 * Same arguments and result as zp_series_eval with ZP_PREC_BF16X3 or ZP_PREC_TF32 (out is
 * float32 [n_points][n_sets], 16-byte aligned), but no device memory is allocated: the plan
 * tables, the split coefficient tiles and the split basis live in one file-scope device array
 * of ZP_STATIC_SCRATCH_BYTES, present on every GPU that loads the library until the process
 * exits.  The array is shared by every call and keeps the last call's contents; each call
 * rewrites everything it reads, so nothing needs clearing.  Calls that overlap on the GPU
 * (different streams, or different host threads) race on the array: serialise them, for
 * example by issuing them on one stream.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current).  Under CUDA's default lazy
 * module loading the array's memory is committed when the library's module is first loaded
 * on a device, which may be that first call: a caller that will later be unable to allocate
 * should make one small call first (or run with CUDA_MODULE_LOADING=EAGER).  The tables
 * travel by cudaMemcpyAsync from pageable host memory on `stream`, so the call cannot be
 * captured in a CUDA graph: on a capturing stream it returns ZP_ERR_INVALID_ARG.
 * Limits: the plan tables, the coefficient tiles (ceil(n_sets/256) * ceil(n_modes/32) * 32 KiB)
 * and one 128-point basis tile (ceil(n_modes/32) * 16 KiB), for either precision, must fit in
 * ZP_STATIC_SCRATCH_BYTES (n_modes * n_sets is bounded before any size is multiplied); larger
 * problems are rejected with ZP_ERR_INVALID_ARG before anything is launched.  Points beyond one tile are
 * processed in slabs, so n_points has no limit of its own.
 */
#define ZP_STATIC_SCRATCH_BYTES (64u << 20)
ZP_API zp_status zp_series_eval_static(const int32_t* n, const int32_t* m, int64_t n_modes,
                                       const double* r, const double* theta, int64_t n_points,
                                       const double* coeffs, int64_t n_sets, zp_precision prec,
                                       float* out, void* stream);

/*
 * Float64 issue-rate probe (measurement service; the paper has no counterpart: it states its
 * hardware's float64 rate, GB300's has to be measured).  Runs one wave of CTAs on the current
 * device in which every thread issues `iters` rounds of 16 independent dependent chains of one
 * float64 operation, op = 0 (fused multiply-add), 1 (multiply) or 2 (add), after a short
 * warm-up launch, and synchronises `stream`.  result[6] (HOST) receives: [0] operations
 * issued, [1] milliseconds (CUDA events around the launch), [2] operations per second, [3]
 * lanes per SM per clock (from the SM cycle counter, independent of the clock the GPU ran
 * at), [4] the SM clock implied by cycles over time (MHz), [5] the SM count.  iters: a
 * multiple of 4 in 4..2^24.  Allocates a few KB of stream-ordered scratch.
 */
ZP_API zp_status zp_probe_fp64(int32_t op, int32_t iters, void* stream, double* result);

/*
 * Reads (and optionally clears) the library's device-side wait-status word on the current
 * device, synchronously.  Returns ZP_ERR_TIMEOUT if a bounded wait inside a tensor-core
 * kernel gave up since the last reset (the kernel then skipped its remaining work and its
 * outputs are incomplete), ZP_OK otherwise.
 */
ZP_API zp_status zp_device_wait_status(int32_t reset);

/*
 * Returns the library's retained scratch memory on the current device to the system.  The
 * series, adjoint and fit calls draw their scratch from a library-owned stream-ordered memory
 * pool per device that keeps up to 16 GiB of freed scratch reserved across synchronisations
 * (so that calls which synchronise do not map their scratch again each time).  Memory still
 * in use by pending work is kept: synchronise the streams that used the library first.
 * ZP_OK when the device has no pool yet.
 */
ZP_API zp_status zp_release_scratch(void);

/*
 * Failure-detection self-test: launches (asynchronously, on `stream`) one thread that waits on
 * a device barrier nothing arrives on, with the same bounded wait the tensor-core kernels use,
 * giving up after limit_ms (1..2000).  A following zp_device_wait_status then reports
 * ZP_ERR_TIMEOUT, and the context stays usable.
 */
ZP_API zp_status zp_device_wait_selftest(int32_t limit_ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ZERNIKE_GB300_H */
