// Learned surrogate entry points (placeholder until the MLP kernels land).
#include "qk_internal.h"

using namespace qk;
#define QK_SURR_NA return fail(QK_ERR_INVALID_ARG, "surrogate not available in this build")
extern "C" {
qk_status qk_surrogate_create(int32_t, int32_t, uint64_t, qk_surrogate**) { QK_SURR_NA; }
qk_status qk_surrogate_free(qk_surrogate*) { return QK_OK; }
int64_t qk_surrogate_param_count(const qk_surrogate*) { return 0; }
qk_status qk_surrogate_get_params(const qk_surrogate*, float*) { QK_SURR_NA; }
qk_status qk_surrogate_set_params(qk_surrogate*, const float*) { QK_SURR_NA; }
qk_status qk_surrogate_set_target_scale(qk_surrogate*, double, double) { QK_SURR_NA; }
qk_status qk_surrogate_loss_grad(qk_surrogate*, const double*, int64_t, const double*, int64_t, int32_t,
                                 const int32_t*, const double*, int64_t, float*, double*, void*) { QK_SURR_NA; }
qk_status qk_surrogate_train(qk_surrogate*, const double*, int64_t, const double*, int64_t, int32_t,
                             const int32_t*, const double*, int64_t, int32_t, int32_t, float, uint64_t,
                             void*, double*) { QK_SURR_NA; }
qk_status qk_surrogate_predict(const qk_surrogate*, const double*, int64_t, const double*, int64_t, int32_t,
                               const int32_t*, int64_t, double*, void*) { QK_SURR_NA; }
qk_status qk_surrogate_calibrate(qk_surrogate*, const double*, int64_t, const double*, int64_t, int32_t,
                                 const int32_t*, const double*, int64_t, double, int32_t, void*) { QK_SURR_NA; }
qk_status qk_surrogate_bins(const qk_surrogate*, int32_t*, double*, double*) { QK_SURR_NA; }
qk_status qk_gram_surrogate(const qk_surrogate*, const qk_mps_batch*, const qk_mps_batch*, const double*,
                            const double*, double, double*, int64_t, uint8_t*, qk_prec, void*, int64_t*) { QK_SURR_NA; }
}
