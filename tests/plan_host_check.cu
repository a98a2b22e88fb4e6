// Host driver for tests/test_plan_host.py: builds the host half of a plan (no GPU needed)
// for the mode list on stdin ("n_modes" then n_modes pairs "n m") and prints its tables.
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <vector>

#include "zp_internal.h"

int main() {
  long long count = 0;
  if (std::scanf("%lld", &count) != 1 || count < 0) return 2;
  std::vector<int32_t> n((size_t)count), m((size_t)count);
  for (long long j = 0; j < count; ++j)
    if (std::scanf("%d %d", &n[(size_t)j], &m[(size_t)j]) != 2) return 2;
  zp_plan plan;
  const zp_status st = zp::build_plan_host(n.data(), m.data(), count, &plan);
  std::printf("status %d\n", (int)st);
  if (st != ZP_OK) return 0;
  std::printf("cols %zu\n", plan.cols.size());
  for (const zp::Column& c : plan.cols) std::printf("%d %d %d %d\n", c.m, c.n_steps, c.table_row, c.slot_base);
  std::printf("table %zu\n", plan.table.size());
  for (double v : plan.table) {
    uint64_t b;
    std::memcpy(&b, &v, sizeof(b));
    std::printf("%016" PRIx64 "\n", b);
  }
  std::printf("slot_ptr %zu\n", plan.slot_ptr.size());
  for (int32_t v : plan.slot_ptr) std::printf("%d\n", v);
  std::printf("slot_idx %zu\n", plan.slot_idx.size());
  for (int32_t v : plan.slot_idx) std::printf("%u\n", (unsigned)v);
  std::printf("split_step %zu\n", plan.split_step.size());
  for (uint32_t v : plan.split_step) std::printf("%u\n", v);
  std::printf("fused %d %d %lld %d\n", zp::kFusedStreams, plan.fused_units, (long long)plan.fused_kpad, plan.fused_ep);
  for (int s = 0; s < zp::kFusedStreams; ++s) std::printf("%d\n", plan.fused_ncols[s]);
  std::printf("fused_col %zu\n", plan.fused_col.size());
  for (int32_t v : plan.fused_col) std::printf("%d\n", v);
  std::printf("fused_kperm %zu\n", plan.fused_kperm.size());
  for (int32_t v : plan.fused_kperm) std::printf("%d\n", v);
  return 0;
}
