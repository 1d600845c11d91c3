// Batched grouped product: placeholder until the persistent kernel lands.
#include "gfp_internal.h"

extern "C" {

GFP_API gfp_status gfp_batched_workspace_size(int64_t count, const gfp_problem *probs,
                                              size_t *bytes) {
    if (count < 0 || (count > 0 && !probs) || !bytes) return GFP_EINVAL;
    *bytes = 0;
    return GFP_EUNSUPPORTED;
}

GFP_API gfp_status gfp_batched_prepare(int64_t, const gfp_problem *, gfp_algo, gfp_status *,
                                       void *, size_t, void *) {
    return GFP_EUNSUPPORTED;
}

GFP_API gfp_status gfp_batched_launch(void *, size_t, void *) { return GFP_EUNSUPPORTED; }

GFP_API gfp_status gfp_gemm_batched(int64_t, const gfp_problem *, gfp_algo, gfp_status *, void *,
                                    size_t, void *) {
    return GFP_EUNSUPPORTED;
}

}  // extern "C"
