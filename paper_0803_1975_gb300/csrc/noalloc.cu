// gfp_gemm_noalloc: the exact int8 tensor-core product (the GFP_ALGO_TC_MMA_S8
// form of gfp_gemm) for callers that cannot allocate device memory -- code
// running under a fixed device-memory budget set at start-up, code inside a
// framework whose allocator owns every device allocation, and latency-bound
// paths where an allocation could synchronize the device.  Such callers
// cannot provide the workspace gfp_gemm asks for, so this entry point uses a
// scratch buffer compiled into the library instead.
//
// The scratch is a file-scope __device__ array of GFP_NOALLOC_SCRATCH_BYTES;
// every GPU that loads the library keeps it for the life of the process.  In
// host code the array's name does not denote a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it with the device's current context; later
// calls in the same context reuse it.  A call that finds another context
// current (the primary context was destroyed by cudaDeviceReset and created
// again, which loads the module, and so the array, anew) looks it up again.
// All calls share the array, so calls whose kernels overlap on the GPU race
// on it.  The two preprocessing kernels rewrite every byte of the scratch a
// call uses (padding included), so nothing has to be cleared between calls.
#include <mutex>

#include <cuda.h>

#include "gfp_internal.h"

namespace gfp {
namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[GFP_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};
CUcontext g_noalloc_ctx[64] = {nullptr};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

CtxGetCurrentFn ctx_get_current_fn() {
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

// Device address of the scratch in the current context of the current device
// (looked up once per context).
gfp_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return GFP_EUNSUPPORTED;
    CtxGetCurrentFn get = ctx_get_current_fn();
    if (!get) return GFP_EUNSUPPORTED;
    CUcontext ctx = nullptr;
    if (get(&ctx) != CUDA_SUCCESS) return GFP_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!ctx || !g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
        // the lookup also makes the device's primary context current if none is
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        if (get(&ctx) != CUDA_SUCCESS || !ctx) return GFP_EUNSUPPORTED;
        g_noalloc_ptr[dev] = ptr;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_ptr[dev];
    return GFP_OK;
}

}  // namespace
}  // namespace gfp

using namespace gfp;

extern "C" {

GFP_API gfp_status gfp_gemm_noalloc(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                                    int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C,
                                    int64_t ldc, void *stream) {
    if (m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    if (m == 0 || n == 0) return GFP_OK;
    if (!C || ldc < n) return GFP_EINVAL;
    if (k > 0 && (!A || !B || lda < k || ldb < n)) return GFP_EINVAL;
    if (tc_mma_workspace(m, k, n) > (size_t)GFP_NOALLOC_SCRATCH_BYTES) return GFP_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 0) {
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc, 0, (size_t)n, (size_t)m, s);
        return e == cudaSuccess ? GFP_OK : cuda_fail(e);
    }
    void *scratch = nullptr;
    gfp_status st = noalloc_scratch(&scratch);
    if (st != GFP_OK) return st;
    return launch_tc_mma(p, m, k, n, A, lda, B, ldb, C, ldc, scratch,
                         (size_t)GFP_NOALLOC_SCRATCH_BYTES, s);
}

}  // extern "C"
