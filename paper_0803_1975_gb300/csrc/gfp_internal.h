// Internal declarations shared by the translation units of libgfp.
#pragma once

#include <cstddef>
#include <cstdint>

#include <atomic>

#include <cuda.h>
#include <cuda_runtime.h>

#include "gfp.h"

namespace gfp {

// ---- status helpers -------------------------------------------------------
gfp_status cuda_fail(cudaError_t e);   // records e for gfp_last_cuda_error()
inline gfp_status check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}
int num_sms();                         // SM count of the current device (cached per device)

// Raise a kernel's dynamic shared-memory limit on the current device, once
// per device (the attribute belongs to the device's context); `done` is the
// kernel's own mask of devices already set.
inline cudaError_t smem_attr_once(const void *kernel, int bytes, std::atomic<uint64_t> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// ---- parameters (params.cpp) ------------------------------------------------
bool is_prime_small(uint32_t p);       // p prime and 2 <= p <= 251
int log2_exact(uint64_t Q);            // t with Q = 2^t, or -1
// Largest packed word (p-1)(1+Q+...+Q^d) compared with 2^bits: true when < 2^bits.
bool amax_below(uint32_t p, int t, int d, int bits);
bool amax_below_v(uint32_t v, int t, int d, int bits);   // v (1+Q+...+Q^d) < 2^bits
gfp_status check_dqt(uint32_t p, int64_t k, int d, uint64_t Q, gfp_form form, gfp_word word,
                     int64_t kb);
// The same with entries of A at most va and of B at most vb (both <= p - 1).
gfp_status check_dqt_vb(uint32_t p, int64_t k, int d, uint64_t Q, gfp_form form, gfp_word word,
                        int64_t kb, uint32_t va, uint32_t vb);
gfp_status check_pack(uint32_t p, int d, uint64_t Q, gfp_word word);
gfp_status check_pack_vb(uint32_t p, uint32_t v, int d, uint64_t Q, gfp_word word);
gfp_status launch_amax(int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx, uint32_t *out,
                       cudaStream_t s);
// C = A B over Z/2^64 for word matrices (A m x kc, B kc x n, C m x n, leading
// dimensions in words): the raw sums of the dot form, no digit extracted.
gfp_status launch_word_product_u64(const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb,
                                   uint64_t *C, int64_t ldc, int64_t m, int64_t kc, int64_t n,
                                   cudaStream_t s);
// Strassen-Winograd over Z/2^64 on the dot form's words (winograd.cu).
size_t winograd_workspace_bytes(int64_t m, int64_t kc, int64_t n, int levels);
gfp_status launch_winograd_u64(uint32_t p, int64_t m, int64_t kc, int64_t n, int d, int t, const uint64_t *CA,
                               int64_t lda, const uint64_t *CB, int64_t ldb, uint8_t *C, int64_t ldc, int levels,
                               void *ws, size_t ws_bytes, cudaStream_t s);
size_t word_bytes(gfp_word w);

// Lemire, Kaser, Kurz, "Faster remainder by direct computation" (2019):
// for 32-bit a and divisor p, a mod p = hi64((M * a mod 2^64) * p) with
// M = floor((2^64 - 1) / p) + 1.
inline uint64_t fastmod_magic(uint32_t p) { return UINT64_MAX / p + 1; }

// ---- kernel launchers ---------------------------------------------------------
gfp_status launch_pack(uint32_t p, int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx,
                       int d, int t, gfp_layout lay, gfp_word word, void *W, int64_t ldw,
                       cudaStream_t s);
gfp_status launch_unpack(int64_t rows, int64_t cols, const void *W, int64_t ldw, int d, int t,
                         gfp_layout lay, gfp_word word, uint8_t *X, int64_t ldx, cudaStream_t s);

// dp4a needs the workspace dp4a_workspace_bytes(k, n) for B transposed
gfp_status launch_plain(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                        int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                        bool dp4a, void *ws, size_t ws_bytes, cudaStream_t s);
size_t dp4a_workspace_bytes(int64_t k, int64_t n);
gfp_status launch_transpose_bytes(const uint8_t *B, int64_t ldb, int64_t k, int64_t n, uint8_t *out, int64_t kp,
                                  int64_t np, cudaStream_t s);
gfp_status launch_dot(uint32_t p, int64_t m, int64_t kc, int64_t n, int d, int t, gfp_word word,
                      const void *CA, int64_t lda, const void *CB, int64_t ldb, uint8_t *C,
                      int64_t ldc, int64_t kbw, cudaStream_t s);
gfp_status launch_mixed(uint32_t p, int64_t m, int64_t k, int64_t nc, int d, int t, gfp_word word,
                        const uint8_t *A, int64_t lda, const void *CB, int64_t ldb, void *CC,
                        int64_t ldc, cudaStream_t s);

gfp_status launch_left(uint32_t p, int64_t mc, int64_t k, int64_t n, int d, int t, gfp_word word,
                       const void *CA, int64_t lda, const uint8_t *B, int64_t ldb, void *CC,
                       int64_t ldc, cudaStream_t s);
gfp_status launch_full(uint32_t p, int64_t mc, int64_t k, int64_t nc, int dq, int dth, int t,
                       gfp_word word, const void *CA, int64_t lda, const void *CB, int64_t ldb,
                       void *CC, int64_t ldc, cudaStream_t s);
gfp_status launch_block(bool pack, int64_t rows, int64_t cols, const uint8_t *X, uint8_t *Xout,
                        int64_t ldx, int dq, int dth, int t, gfp_word word, const void *Win, void *Wout,
                        int64_t ldw, cudaStream_t s);
gfp_status check_full(uint32_t p, int64_t k, int dq, int dth, uint64_t Q, gfp_word word);

gfp_status launch_dot_compc(uint32_t p, int64_t m, int64_t kc, int64_t n, int d, int t, gfp_word word,
                            const void *CA, int64_t lda, const void *CB, int64_t ldb, int64_t kbw, int d_out,
                            int t_out, void *CC, int64_t ldcc, cudaStream_t s);

// tensor-core forms (gemm_tc_mma.cu, gemm_tc_tcgen05.cu)
size_t tc_mma_workspace(int64_t m, int64_t k, int64_t n);
gfp_status launch_tc_mma(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                         int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                         void *ws, size_t ws_bytes, cudaStream_t s);
size_t tc_f16_workspace(int64_t m, int64_t k, int64_t n);
gfp_status launch_tc_f16(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                         int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                         void *ws, size_t ws_bytes, cudaStream_t s);
size_t tc_f8_workspace(int64_t m, int64_t k, int64_t n);
size_t tc_e2m1_workspace(int64_t m, int64_t k, int64_t n);
gfp_status launch_tc_e2m1(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A, int64_t lda,
                          const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc, void *ws, size_t ws_bytes,
                          cudaStream_t s);
int64_t tc_kblock_e2m1(uint32_t p);
gfp_status tc_mma_rates(double *out, int *status_dev, cudaStream_t s);   // fp16, e4m3, e2m1 (mxf4, mxf4nvf4) flops/s     // largest kb (multiple of 256) with kb ((p-1)/2)^2 + p < 2^24
gfp_status launch_tc_f8(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                        int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                        void *ws, size_t ws_bytes, cudaStream_t s);
// grouped tcgen05 launch (batched.cu builds the schedule; tc_group.h)
bool tc_make_map_u8(CUtensorMap *map, const void *base, int64_t rows, int64_t kp, int box_rows);
gfp_status launch_tc_grouped(const void *grp, int grid, int *status, cudaStream_t s);
int tc_grouped_ctas_per_sm();
gfp_status tc_selftest_wait_limit(void *ws, size_t ws_bytes, uint64_t limit_ns, int *status_host, cudaStream_t s);
int64_t tc_kblock_s32(uint32_t p);      // largest kb with kb ((p-1)/2)^2 + p < 2^30
int64_t tc_kblock_f32(uint32_t p);      // largest kb (multiple of 128) with kb ((p-1)/2)^2 + p < 2^24

}  // namespace gfp
