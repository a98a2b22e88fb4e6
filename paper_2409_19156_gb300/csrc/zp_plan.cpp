// Plan construction: validation, grouping of modes into |m| columns, recursion tables.
//
// The per-column walk is Algorithm 1 of Sec. 3 (outer loop over alpha = |m|, inner loop
// over the Jacobi degree N, store every requested (n, m) on the way).  The coefficients
// come from the beta = 0 Jacobi recursion of Sec. 2,
//   P_N = [(2N+a-1)((2N+a)(2N+a-2) x + a^2) / D] P_{N-1} - [2(N+a-1)(N-1)(2N+a) / D] P_{N-2},
//   D = 2N(N+a)(2N+a-2),  a = |m|,
// rewritten for R_N = (-1)^N rho^m P_N(1 - 2 rho^2) (the Jacobi relation):
//   R_N = (2 a_N rho^2 - a_N - b_N) R_{N-1} - c_N R_{N-2}
// with a_N, b_N, c_N the three printed ratios.  The library carries Q_N = R_N / w_N with
// w_0 = w_1 = 1 and w_N = c_N w_{N-2}, which turns the recursion into
//   Q_N = (A_N rho^2 - B_N) Q_{N-1} - Q_{N-2},  A_N = 2 a_N w_{N-1}/w_N, B_N = (a_N+b_N) w_{N-1}/w_N
// and saves one multiply per derivative lane per step; stores multiply by W_k = k! w_N.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>

#include "zp_internal.h"

namespace zp {

namespace {
thread_local std::string g_last_error;
}

zp_status set_error(zp_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

zp_status cuda_error(cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return set_error(ZP_ERR_NO_MEMORY, msg);
  // A launch configuration the GPU cannot hold (registers, shared memory): not a device fault.
  if (e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidConfiguration) return set_error(ZP_ERR_UNSUPPORTED, msg);
  return set_error(ZP_ERR_CUDA, msg);
}

void clear_error() { g_last_error.clear(); }

static long double binom_ld(int n, int k) {
  if (k < 0 || k > n) return 0.0L;
  long double v = 1.0L;
  for (int i = 1; i <= k; ++i) v = v * (long double)(n - k + i) / (long double)i;
  return v;
}

static void fill_column_table(int m, int n_steps, double* rows) {
  // Header rows: seed constants (Taylor coefficients of rho^m and of R_{m+2}^m).
  double* h = rows;
  for (int k = 0; k < 4; ++k) {
    h[k] = (double)binom_ld(m, k);
    h[4 + k] = (double)((long double)(m + 2) * binom_ld(m + 2, k));
    h[8 + k] = (double)((long double)(m + 1) * binom_ld(m, k));
  }
  for (int k = 12; k < 16; ++k) h[k] = 0.0;
  double* t = rows + kHeaderRows * kRow;
  std::vector<long double> w(std::max(n_steps, 2), 1.0L);
  for (int N = 0; N < n_steps; ++N) {
    double* row = t + (size_t)N * kRow;
    long double A = 0.0L, B = 0.0L;
    if (N >= 2) {
      const long double a = m;
      const long double D = 2.0L * N * (N + a) * (2.0L * N + a - 2.0L);
      const long double aN = (2.0L * N + a - 1.0L) * (2.0L * N + a) * (2.0L * N + a - 2.0L) / D;
      const long double bN = (2.0L * N + a - 1.0L) * a * a / D;
      const long double cN = 2.0L * (N + a - 1.0L) * (N - 1.0L) * (2.0L * N + a) / D;
      w[N] = cN * w[N - 2];
      A = 2.0L * aN * w[N - 1] / w[N];
      B = (aN + bN) * w[N - 1] / w[N];
    }
    row[0] = (double)A;
    row[1] = (double)B;
    row[2] = (double)(2.0L * A);
    row[3] = (double)w[N];
    row[4] = (double)w[N];
    row[5] = (double)(2.0L * w[N]);
    row[6] = (double)(6.0L * w[N]);
    row[7] = 0.0;
  }
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

zp_status build_plan_host(const int32_t* n, const int32_t* m, int64_t n_modes, zp_plan* p) {
  if (n_modes < 0) return set_error(ZP_ERR_INVALID_ARG, "n_modes < 0");
  if (n_modes > 0 && (!n || !m)) return set_error(ZP_ERR_INVALID_ARG, "mode arrays are NULL");
  if (n_modes >= (int64_t(1) << 31)) return set_error(ZP_ERR_INVALID_ARG, "n_modes >= 2^31");
  int32_t n_max = 0;
  for (int64_t j = 0; j < n_modes; ++j) {
    const int32_t nj = n[j], mj = m[j];
    const int64_t am = mj < 0 ? -(int64_t)mj : (int64_t)mj;
    if (nj < 0 || am > nj || (((int64_t)nj - am) & 1)) {
      return set_error(ZP_ERR_INVALID_MODE, "invalid mode at index " + std::to_string(j) + ": (n=" +
                                                std::to_string(nj) + ", m=" + std::to_string(mj) +
                                                ") needs n >= 0, |m| <= n, n - |m| even");
    }
    if (nj > ZP_MAX_N) {
      return set_error(ZP_ERR_INVALID_MODE, "mode n=" + std::to_string(nj) + " above ZP_MAX_N");
    }
    n_max = std::max(n_max, nj);
  }
  // The host tables need no device; without one (device -1) the later upload fails instead.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = -1;
  }

  p->device = dev;
  p->n_modes = n_modes;
  p->n_max = n_max;
  p->n.assign(n, n + n_modes);
  p->m.assign(m, m + n_modes);

  // Steps per |m| column = 1 + largest requested Jacobi degree of that column.
  std::vector<int32_t> steps_of_m(n_max + 1, 0);
  for (int64_t j = 0; j < n_modes; ++j) {
    const int32_t am = std::abs(m[j]);
    steps_of_m[am] = std::max(steps_of_m[am], (n[j] - am) / 2 + 1);
  }
  for (int32_t am = 0; am <= n_max; ++am) {
    if (steps_of_m[am] > 0) p->cols.push_back(zp::Column{am, steps_of_m[am], 0, 0});
  }
  // Longest recursion first: better tail behaviour when blocks are scheduled in order.
  std::stable_sort(p->cols.begin(), p->cols.end(),
                   [](const Column& a, const Column& b) { return a.n_steps > b.n_steps; });
  std::vector<int32_t> col_of_m(n_max + 1, -1);
  int32_t row = 0, slot = 0;
  for (size_t c = 0; c < p->cols.size(); ++c) {
    Column& col = p->cols[c];
    col.table_row = row;
    col.slot_base = slot;
    row += kHeaderRows + col.n_steps;
    slot += col.n_steps + 1;
    col_of_m[col.m] = (int32_t)c;
    p->max_steps = std::max(p->max_steps, col.n_steps);
  }
  p->table.assign((size_t)row * kRow, 0.0);
  for (const Column& col : p->cols) fill_column_table(col.m, col.n_steps, p->table.data() + (size_t)col.table_row * kRow);

  // CSR of output columns per (column, N), in the caller's mode order.
  std::vector<int32_t> count((size_t)slot, 0);
  p->mode_col.resize(n_modes);
  p->mode_N.resize(n_modes);
  for (int64_t j = 0; j < n_modes; ++j) {
    const int32_t am = std::abs(m[j]);
    const int32_t c = col_of_m[am];
    const int32_t N = (n[j] - am) / 2;
    p->mode_col[j] = c;
    p->mode_N[j] = N;
    count[(size_t)p->cols[c].slot_base + N]++;
  }
  p->slot_ptr.assign((size_t)slot, 0);
  {
    int32_t acc = 0;
    for (size_t c = 0; c < p->cols.size(); ++c) {
      const Column& col = p->cols[c];
      for (int32_t N = 0; N <= col.n_steps; ++N) {
        const size_t s = (size_t)col.slot_base + N;
        p->slot_ptr[s] = acc;
        if (N < col.n_steps) acc += count[s];
      }
    }
    p->slot_idx.assign((size_t)acc, 0);
  }
  std::vector<int32_t> fill((size_t)slot, 0);
  for (int64_t j = 0; j < n_modes; ++j) {
    const size_t s = (size_t)p->cols[p->mode_col[j]].slot_base + p->mode_N[j];
    const int32_t pos = p->slot_ptr[s] + fill[s]++;
    p->slot_idx[pos] = (int32_t)((uint32_t)j | (m[j] < 0 ? 0x80000000u : 0u));
  }
  // Step descriptors of the split basis: slot count and sin flags, and the float32 weight.
  p->split_step.assign(2 * (size_t)row, 0u);
  for (const Column& col : p->cols) {
    for (int32_t N = 0; N < col.n_steps; ++N) {
      const size_t s = (size_t)col.slot_base + N;
      const int32_t b = p->slot_ptr[s], cnt = p->slot_ptr[s + 1] - b;
      uint32_t code = kStepIrregular;
      if (cnt <= kStepMaxFlags) {
        code = (uint32_t)cnt;
        for (int32_t i = 0; i < cnt; ++i) code |= ((uint32_t)p->slot_idx[(size_t)b + i] >> 31) << (8 + i);
      }
      const size_t r = (size_t)col.table_row + kHeaderRows + N;
      uint64_t wbits;
      std::memcpy(&wbits, &p->table[r * kRow + 3], sizeof(wbits));
      p->split_step[2 * r] = code;
      p->split_step[2 * r + 1] = trunc_float_bits((uint32_t)(wbits >> 32), (uint32_t)wbits);
    }
  }
  // Fused contraction layout.  The columns are dealt to kFusedStreams streams (producer
  // threads per point) in walk order, round robin (a stream's consecutive columns then lie
  // kFusedStreams apart in |m| for a full mode set, one angle step each) unless that stream is
  // more than two 8-value units ahead of the least loaded one, which then takes the column;
  // each column's outputs fill whole units (slot order, zero padded), and the K order
  // interleaves the streams unit by unit: unit j of stream s is global unit kFusedStreams j + s.
  constexpr int NS = kFusedStreams;
  const size_t nc = p->cols.size();
  p->fused_col.assign(5 * nc, 0);
  int32_t units[NS] = {};
  std::vector<int32_t> scol[NS];
  std::vector<int32_t> col_first(nc, 0), col_stream(nc, 0);
  for (size_t c = 0; c < nc; ++c) {
    const Column& col = p->cols[c];
    const int32_t first = p->slot_ptr[col.slot_base], last = p->slot_ptr[(size_t)col.slot_base + col.n_steps];
    int kind = -1;
    uint32_t fa = 0, fb = 0;
    for (int32_t N = 0; N < col.n_steps; ++N) {
      const size_t s = (size_t)col.slot_base + N;
      const int32_t b = p->slot_ptr[s], cnt = p->slot_ptr[s + 1] - b;
      const uint32_t a0 = cnt > 0 ? (uint32_t)p->slot_idx[b] >> 31 : 0u;
      const uint32_t a1 = cnt > 1 ? (uint32_t)p->slot_idx[(size_t)b + 1] >> 31 : 0u;
      const int k = (cnt == 1) ? kFusedKindOne : (cnt == 2 ? kFusedKindTwo : kFusedKindGeneric);
      if (N == 0) {
        kind = k;
        fa = a0;
        fb = a1;
      } else if (k != kind || a0 != fa || (k == kFusedKindTwo && a1 != fb)) {
        kind = kFusedKindGeneric;
      }
    }
    if (kind < 0) kind = kFusedKindGeneric;
    const int32_t nvals = last - first;
    int least = 0;
    for (int s2 = 1; s2 < NS; ++s2)
      if (units[s2] < units[least]) least = s2;
    const int st = units[c % NS] > units[least] + 2 ? least : (int)(c % NS);
    col_stream[c] = st;
    col_first[c] = units[st];
    p->fused_col[4 * c] = kind | (int32_t)(fa << 8) | (int32_t)(fb << 9);
    p->fused_col[4 * c + 1] = st;
    p->fused_col[4 * c + 2] = units[st];
    p->fused_col[4 * c + 3] = nvals;
    units[st] += (nvals + 7) / 8;
    scol[st].push_back((int32_t)c);
  }
  size_t at = 4 * nc;
  for (int st = 0; st < NS; ++st) {
    for (size_t i = 0; i < scol[st].size(); ++i) p->fused_col[at + i] = scol[st][i];
    at += scol[st].size();
    p->fused_ncols[st] = (int32_t)scol[st].size();
  }
  // Global units G: the fewest, in whole 4-unit (32-position) stages, that give every stream
  // its units (stream s owns the global units g < G with g = s mod NS: (G - s + NS - 1) / NS of
  // them, so streams end at most one unit apart).
  int32_t G = 0;
  for (int st = 0; st < NS; ++st)
    if (units[st] > 0) G = std::max(G, NS * (units[st] - 1) + st + 1);
  G = (G + 3) / 4 * 4;
  p->fused_units = G;
  p->fused_kperm.assign((size_t)G * 8, -1);
  for (size_t c = 0; c < nc; ++c) {
    const Column& col = p->cols[c];
    const int32_t first = p->slot_ptr[col.slot_base];
    for (int32_t i = 0; i < p->fused_col[4 * c + 3]; ++i) {
      const int32_t unit = NS * (col_first[c] + i / 8) + col_stream[c];
      p->fused_kperm[(size_t)unit * 8 + i % 8] = first + i;
    }
  }
  p->fused_kpad = (int64_t)p->fused_kperm.size();
  // The fused kernel digitises Q_N cos/sin(m theta) and carries the weight w_N on the
  // coefficient side; on the unit disc |R| <= 1, so |Q| <= 1 / w_N: the row scale 2^e covers
  // the largest 1 / w_N of the plan's outputs (with a margin for the recursion's rounding).
  double inv_w = 1.0;
  for (const Column& col : p->cols)
    for (int32_t N = 0; N < col.n_steps; ++N) {
      const size_t s = (size_t)col.slot_base + N;
      if (p->slot_ptr[s + 1] == p->slot_ptr[s]) continue;
      const double w = p->table[((size_t)col.table_row + kHeaderRows + N) * kRow + 3];
      inv_w = std::max(inv_w, 1.0 / w);
    }
  int e = 0;
  while (std::ldexp(1.0, e) <= inv_w * (1.0 + 1e-9)) ++e;
  p->fused_ep = e;
  return ZP_OK;
}

size_t plan_device_layout(const zp_plan* p, size_t offsets[kPlanSections]) {
  const size_t b_cols = align_up(p->cols.size() * sizeof(Column), 256);
  const size_t b_table = align_up(p->table.size() * sizeof(double), 256);
  const size_t b_sptr = align_up(p->slot_ptr.size() * sizeof(int32_t), 256);
  const size_t b_sidx = align_up(std::max<size_t>(p->slot_idx.size(), 1) * sizeof(int32_t), 256);
  const size_t b_mode = align_up(std::max<int64_t>(p->n_modes, 1) * sizeof(int32_t), 256);
  const size_t b_step = align_up(std::max<size_t>(p->split_step.size(), 2) * sizeof(uint32_t), 256);
  const size_t b_fcol = align_up(std::max<size_t>(p->fused_col.size(), 4) * sizeof(int32_t), 256);
  const size_t b_fperm = align_up(std::max<size_t>(p->fused_kperm.size(), 1) * sizeof(int32_t), 256);
  offsets[0] = 0;
  offsets[1] = b_cols;
  offsets[2] = b_cols + b_table;
  offsets[3] = b_cols + b_table + b_sptr;
  offsets[4] = b_cols + b_table + b_sptr + b_sidx;
  offsets[5] = b_cols + b_table + b_sptr + b_sidx + b_mode;
  offsets[6] = b_cols + b_table + b_sptr + b_sidx + 2 * b_mode;
  offsets[7] = offsets[6] + b_step;
  offsets[8] = offsets[7] + b_fcol;
  return offsets[8] + b_fperm;
}

zp_status plan_upload(zp_plan* p, void* base_ptr, cudaStream_t stream, bool async) {
  size_t off[kPlanSections];
  plan_device_layout(p, off);
  char* base = (char*)base_ptr;
  p->dev.cols = (Column*)(base + off[0]);
  p->dev.table = (double*)(base + off[1]);
  p->dev.slot_ptr = (int32_t*)(base + off[2]);
  p->dev.slot_idx = (int32_t*)(base + off[3]);
  p->dev.mode_col = (int32_t*)(base + off[4]);
  p->dev.mode_N = (int32_t*)(base + off[5]);
  p->dev.split_step = (uint2*)(base + off[6]);
  p->dev.fused_col = (int4*)(base + off[7]);
  p->dev.fused_kperm = (int32_t*)(base + off[8]);
  struct Part {
    void* dst;
    const void* src;
    size_t bytes;
  } parts[] = {
      {p->dev.cols, p->cols.data(), p->cols.size() * sizeof(Column)},
      {p->dev.table, p->table.data(), p->table.size() * sizeof(double)},
      {p->dev.slot_ptr, p->slot_ptr.data(), p->slot_ptr.size() * sizeof(int32_t)},
      {p->dev.slot_idx, p->slot_idx.data(), p->slot_idx.size() * sizeof(int32_t)},
      {p->dev.mode_col, p->mode_col.data(), p->mode_col.size() * sizeof(int32_t)},
      {p->dev.mode_N, p->mode_N.data(), p->mode_N.size() * sizeof(int32_t)},
      {p->dev.split_step, p->split_step.data(), p->split_step.size() * sizeof(uint32_t)},
      {p->dev.fused_col, p->fused_col.data(), p->fused_col.size() * sizeof(int32_t)},
      {p->dev.fused_kperm, p->fused_kperm.data(), p->fused_kperm.size() * sizeof(int32_t)},
  };
  for (const Part& part : parts) {
    if (part.bytes == 0) continue;
    cudaError_t e = async ? cudaMemcpyAsync(part.dst, part.src, part.bytes, cudaMemcpyHostToDevice, stream)
                          : cudaMemcpy(part.dst, part.src, part.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "copy of plan tables");
  }
  return ZP_OK;
}

zp_status build_plan(const int32_t* n, const int32_t* m, int64_t n_modes, zp_plan** out) {
  if (!out) return set_error(ZP_ERR_INVALID_ARG, "plan output pointer is NULL");
  std::unique_ptr<zp_plan> p(new zp_plan());
  zp_status st = build_plan_host(n, m, n_modes, p.get());
  if (st != ZP_OK) return st;
  size_t off[kPlanSections];
  const size_t total = plan_device_layout(p.get(), off);
  cudaError_t e = cudaMalloc(&p->dev_block, total);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(plan tables)");
  p->device_bytes = total;
  st = plan_upload(p.get(), p->dev_block, nullptr, false);
  if (st != ZP_OK) {
    cudaFree(p->dev_block);
    return st;
  }
  *out = p.release();
  return ZP_OK;
}

static void free_plan(zp_plan* p) {
  if (!p) return;
  if (p->dev_block) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->dev_block);
    cudaSetDevice(cur);
  }
  delete p;
}

zp_status check_plan_device(const zp_plan* plan) {
  if (!plan) return set_error(ZP_ERR_INVALID_ARG, "plan is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev != plan->device) {
    return set_error(ZP_ERR_INVALID_ARG, "plan was created on device " + std::to_string(plan->device) +
                                             " but the current device is " + std::to_string(dev));
  }
  return ZP_OK;
}

namespace {
struct PlanKey {
  int device;
  std::vector<int32_t> n, m;
  bool operator==(const PlanKey& o) const { return device == o.device && n == o.n && m == o.m; }
};
struct PlanKeyHash {
  size_t operator()(const PlanKey& k) const {
    uint64_t h = 1469598103934665603ull ^ (uint64_t)k.device;
    for (size_t i = 0; i < k.n.size(); ++i) {
      h = (h ^ (uint32_t)k.n[i]) * 1099511628211ull;
      h = (h ^ (uint32_t)k.m[i]) * 1099511628211ull;
    }
    return (size_t)h;
  }
};
std::mutex g_cache_mu;
std::unordered_map<PlanKey, std::shared_ptr<const zp_plan>, PlanKeyHash> g_cache;
constexpr size_t kCacheMax = 64;
}  // namespace

zp_status cached_plan(const int32_t* n, const int32_t* m, int64_t n_modes, std::shared_ptr<const zp_plan>* out) {
  if (n_modes < 0) return set_error(ZP_ERR_INVALID_ARG, "n_modes < 0");
  if (n_modes > 0 && (!n || !m)) return set_error(ZP_ERR_INVALID_ARG, "mode arrays are NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  PlanKey key{dev, std::vector<int32_t>(n, n + n_modes), std::vector<int32_t>(m, m + n_modes)};
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *out = it->second;
    return ZP_OK;
  }
  zp_plan* p = nullptr;
  zp_status s = build_plan(n, m, n_modes, &p);
  if (s != ZP_OK) return s;
  // Callers hold a reference for the duration of their call; an evicted plan is freed when
  // the last reference drops (freeing synchronises the device first, so work already
  // enqueued with it completes).
  std::shared_ptr<const zp_plan> sp(p, [](const zp_plan* q) { free_plan(const_cast<zp_plan*>(q)); });
  if (g_cache.size() >= kCacheMax) g_cache.clear();
  g_cache.emplace(std::move(key), sp);
  *out = sp;
  return ZP_OK;
}

}  // namespace zp

extern "C" {

const char* zp_status_string(zp_status s) {
  switch (s) {
    case ZP_OK: return "ok";
    case ZP_ERR_INVALID_ARG: return "invalid argument";
    case ZP_ERR_INVALID_MODE: return "invalid Zernike mode";
    case ZP_ERR_DERIV_ORDER: return "derivative order outside 0..3";
    case ZP_ERR_CUDA: return "CUDA error";
    case ZP_ERR_TIMEOUT: return "device wait timed out";
    case ZP_ERR_UNSUPPORTED: return "unsupported";
    case ZP_ERR_NO_MEMORY: return "out of device memory";
  }
  return "unknown status";
}

const char* zp_last_error(void) { return zp::g_last_error.c_str(); }

int32_t zp_version(void) { return 100; }

zp_status zp_plan_create(const int32_t* n, const int32_t* m, int64_t n_modes, zp_plan** out) {
  zp::clear_error();
  return zp::build_plan(n, m, n_modes, out);
}

zp_status zp_plan_destroy(zp_plan* plan) {
  zp::clear_error();
  if (!plan) return zp::set_error(ZP_ERR_INVALID_ARG, "plan is NULL");
  zp::free_plan(plan);
  return ZP_OK;
}

zp_status zp_plan_info(const zp_plan* plan, int64_t* n_modes, int32_t* n_max, int32_t* n_columns) {
  zp::clear_error();
  if (!plan) return zp::set_error(ZP_ERR_INVALID_ARG, "plan is NULL");
  if (n_modes) *n_modes = plan->n_modes;
  if (n_max) *n_max = plan->n_max;
  if (n_columns) *n_columns = (int32_t)plan->cols.size();
  return ZP_OK;
}

}  // extern "C"
