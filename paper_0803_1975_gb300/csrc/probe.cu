// Instruction-rate probes: the throughput of the instructions the CUDA-core
// forms are built from, measured on the GPU at hand, so that their kernels
// can be reported against measured ceilings (no counterpart in the paper).
// The dense rates of the tcgen05 kinds come from tc_mma_rates
// (gemm_tc_tcgen05.cu).
//
// Each probe runs independent dependency chains of one instruction per
// thread (8; 16 for the double-precision FMA, whose latency is longer; 4
// chains of int8 warp MMAs per warp), `iters` steps each, on 4 CTAs of 256
// threads per SM (32 warps per SM hide the instruction latencies), timed
// with CUDA events (best of 3 after one untimed run).  Every chain feeds the
// next step of itself, so no step can be hoisted or folded; the chains'
// values reach a conditional store that never happens but that the compiler
// cannot rule out.
#include <cstdint>

#include "gfp_internal.h"

namespace gfp {
namespace {

constexpr int kChains = 8;
constexpr int kFpChains = 16;

template <int OP>
__global__ void __launch_bounds__(256) pipe_probe_kernel(uint64_t *sink, uint32_t seed, uint64_t x64, uint64_t y64,
                                                         int iters) {
    const uint32_t x = seed | 1u, y = seed * 2654435761u;
    uint32_t a[kChains];
    uint64_t w[kChains];
    double f[kFpChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = threadIdx.x * 97u + c;
        w[c] = ((uint64_t)blockIdx.x << 32) | (threadIdx.x + c);
    }
#pragma unroll
    for (int c = 0; c < kFpChains; ++c) f[c] = 1.0 + 1e-9 * (threadIdx.x + c);
    const double fx = 0.999999, fy = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (OP == 0)        // 32-bit multiply-add (IMAD)
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(x), "r"(y));
            else if constexpr (OP == 1)   // 32 x 32 -> 64-bit multiply-add (IMAD.WIDE)
                asm volatile("{\n.reg .u32 lo;\ncvt.u32.u64 lo, %0;\nmad.wide.u32 %0, lo, %1, %0;\n}" : "+l"(w[c]) : "r"(x));
            else if constexpr (OP == 2)   // 64-bit multiply-add, low half (the dot form's word step);
                                          // both factors full 64-bit values the compiler cannot see
                asm volatile("mad.lo.u64 %0, %0, %1, %2;" : "+l"(w[c]) : "l"(x64), "l"(y64));
            else if constexpr (OP == 3)   // four byte products and their sum (dp4a)
                asm volatile("dp4a.u32.u32 %0, %0, %1, %0;" : "+r"(a[c]) : "r"(x));
        }
        if constexpr (OP == 4) {          // double-precision fused multiply-add
#pragma unroll
            for (int c = 0; c < kFpChains; ++c)
                asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(f[c]) : "d"(fx), "d"(fy));
        }
        if constexpr (OP == 5) {
            // int8 warp MMA, 16 x 8 x 32 per instruction with int32 accumulation:
            // chains through the accumulators (4 registers each, two per chain)
#pragma unroll
            for (int c = 0; c < kChains; c += 2) {
                uint32_t d0 = a[c], d1 = a[c + 1], d2 = (uint32_t)w[c], d3 = (uint32_t)w[c + 1];
                asm volatile(
                    "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                    "{%8, %9}, {%0, %1, %2, %3};"
                    : "+r"(d0), "+r"(d1), "+r"(d2), "+r"(d3)
                    : "r"(x), "r"(y), "r"(x ^ y), "r"(x + y), "r"(x), "r"(y));
                a[c] = d0;
                a[c + 1] = d1;
                w[c] = d2;
                w[c + 1] = d3;
            }
        }
    }
    uint64_t v = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) v += a[c] + w[c];
#pragma unroll
    for (int c = 0; c < kFpChains; ++c) v += (uint64_t)__double_as_longlong(f[c]);
    if (v == 0x9E3779B97F4A7C15ull) sink[0] = v;
}

template <int OP>
gfp_status time_probe(uint64_t *sink, int grid, int iters, cudaStream_t s, double *per_s) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError());
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError());
    }
    float best = 0;
    gfp_status st = GFP_OK;
    for (int rep = 0; rep < 4 && st == GFP_OK; ++rep) {
        cudaEventRecord(e0, s);
        const uint64_t x64 = 0x9E3779B97F4A7C15ull ^ ((uint64_t)rep << 40), y64 = 0xD1B54A32D192ED03ull + rep;
        pipe_probe_kernel<OP><<<grid, 256, 0, s>>>(sink, 0x12345u + rep, x64, y64, iters);
        cudaEventRecord(e1, s);
        st = check_launch();
        if (st != GFP_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = cuda_fail(e);
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0 || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // OP 5 counts operations of the MMA: each warp issues kChains / 2 MMAs
    // of 2 x 16 x 8 x 32 per step
    const double per_step = OP == 5   ? (double)grid * 8.0 * (kChains / 2) * 2.0 * 16 * 8 * 32
                            : OP == 4 ? (double)grid * 256.0 * kFpChains
                                      : (double)grid * 256.0 * kChains;
    if (st == GFP_OK) *per_s = per_step * iters / (best * 1e-3);
    return st;
}

}  // namespace
}  // namespace gfp

using namespace gfp;

extern "C" {

GFP_API gfp_status gfp_pipe_rates(double *rates, int n_rates, void *workspace, size_t ws_bytes, void *stream) {
    if (!rates || n_rates < 1) return GFP_EINVAL;
    if (!workspace || ws_bytes < 256 || ((uintptr_t)workspace & 255)) return GFP_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *sink = static_cast<uint64_t *>(workspace);
    const int grid = 4 * num_sms();
    const int iters = 4096;
    gfp_status st = GFP_OK;
    double r[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (st == GFP_OK && n_rates > 0) st = time_probe<0>(sink, grid, iters, s, &r[0]);
    if (st == GFP_OK && n_rates > 1) st = time_probe<1>(sink, grid, iters, s, &r[1]);
    if (st == GFP_OK && n_rates > 2) st = time_probe<2>(sink, grid, iters, s, &r[2]);
    if (st == GFP_OK && n_rates > 3) st = time_probe<3>(sink, grid, iters, s, &r[3]);
    if (st == GFP_OK && n_rates > 4) st = time_probe<4>(sink, grid, iters / 16, s, &r[4]);
    if (st == GFP_OK && n_rates > 5) st = time_probe<5>(sink, grid, iters / 4, s, &r[5]);
    if (st == GFP_OK && n_rates > 6)
        st = tc_mma_rates(&r[6], reinterpret_cast<int *>(static_cast<uint8_t *>(workspace) + 128), s);
    if (st != GFP_OK) return st;
    for (int i = 0; i < n_rates && i < 13; ++i) rates[i] = r[i];
    return GFP_OK;
}

}  // extern "C"
