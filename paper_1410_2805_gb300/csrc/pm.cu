// Long-range spectral particle-mesh force (Sec. 2.3).
#include "hacc_internal.cuh"

namespace hacc {

hacc_status pm_accel(hacc_ctx *ctx, const hacc_box *box, const hacc_pm *pm, int64_t n, const float4 *pos,
                     float4 *acc, float4 *vel_kick, float kick, cudaStream_t s) {
    (void)box; (void)pm; (void)n; (void)pos; (void)acc; (void)vel_kick; (void)kick; (void)s;
    return set_error(ctx, HACC_EINVAL, "the PM stage is not built yet");
}

void pm_destroy(hacc_ctx *ctx) { (void)ctx; }

}  // namespace hacc
