// Split-precision tensor-core series evaluation (placeholder until the tcgen05 path lands).
#include "zp_series_internal.h"

namespace zp {

zp_status series_eval_split(const zp_plan*, const double*, const double*, int64_t, const double*, int64_t,
                            zp_precision, float*, cudaStream_t) {
  return set_error(ZP_ERR_UNSUPPORTED, "split-precision series not built yet");
}

}  // namespace zp
