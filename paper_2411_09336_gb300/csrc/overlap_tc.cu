// Split-precision tensor-core transfer sweep (placeholder until the tcgen05
// kernel lands): reports that the path is unavailable.
#include "qk_internal.h"

namespace qk {
void free_tc_cache(qk_mps_batch* b) { b->tc_cache = nullptr; }
qk_status gram_split(const qk_mps_batch*, const qk_mps_batch*, double*, int64_t, double,
                     cudaStream_t, int64_t*) {
  return fail(QK_ERR_INVALID_ARG, "qk_gram: split-precision path not available in this build");
}
qk_status pairs_split(const qk_mps_batch*, const qk_mps_batch*, const int32_t*, int64_t, double*,
                      cudaStream_t) {
  return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs: split-precision path not available in this build");
}
}  // namespace qk
