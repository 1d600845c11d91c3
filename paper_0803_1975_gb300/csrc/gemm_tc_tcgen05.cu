// Exact C = A B mod p on the tcgen05 tensor cores (kind::f16): placeholder
// until the kernel lands; reports GFP_EUNSUPPORTED.
#include "gfp_internal.h"

namespace gfp {

int64_t tc_kblock_f32(uint32_t p) {
    const int64_t h = p == 2 ? 1 : (p - 1) / 2;
    int64_t kb = ((int64_t(1) << 24) - 1 - p) / (h * h);
    return kb / 64 * 64;
}

size_t tc_f16_workspace(int64_t, int64_t, int64_t) { return 0; }

gfp_status launch_tc_f16(uint32_t, int64_t, int64_t, int64_t, const uint8_t *, int64_t,
                         const uint8_t *, int64_t, uint8_t *, int64_t, void *, size_t,
                         cudaStream_t) {
    return GFP_EUNSUPPORTED;
}

}  // namespace gfp
