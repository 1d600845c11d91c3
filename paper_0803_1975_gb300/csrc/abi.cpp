// C-ABI entry points: host-side validation, then dispatch to the kernels.
// Nothing is launched unless every argument has been checked.
#include <cstring>

#include "gfp_internal.h"

namespace gfp {

static thread_local int g_last_cuda_error = 0;

gfp_status cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return GFP_ECUDA;
}

int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cache[dev] = v;
    }
    return cache[dev];
}

static bool valid_layout(gfp_layout l) {
    return l == GFP_LAYOUT_ROWS_REV || l == GFP_LAYOUT_COLS || l == GFP_LAYOUT_ROWS;
}

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Words per row and word rows of a packed matrix of a rows x cols residue matrix.
static void packed_shape(gfp_layout lay, int64_t rows, int64_t cols, int d, int64_t *wrows,
                         int64_t *wcols) {
    if (lay == GFP_LAYOUT_COLS) {
        *wrows = cdiv(rows, d + 1);
        *wcols = cols;
    } else {
        *wrows = rows;
        *wcols = cdiv(cols, d + 1);
    }
}

}  // namespace gfp

using namespace gfp;

extern "C" {

GFP_API int gfp_last_cuda_error(void) { return g_last_cuda_error; }

GFP_API gfp_status gfp_pack(uint32_t p, int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx,
                            int d, uint64_t Q, gfp_layout lay, gfp_word word, void *W, int64_t ldw,
                            void *stream) {
    return gfp_pack_vb(p, p - 1, rows, cols, X, ldx, d, Q, lay, word, W, ldw, stream);
}

GFP_API gfp_status gfp_pack_vb(uint32_t p, uint32_t amax, int64_t rows, int64_t cols, const uint8_t *X,
                               int64_t ldx, int d, uint64_t Q, gfp_layout lay, gfp_word word, void *W,
                               int64_t ldw, void *stream) {
    if (rows < 0 || cols < 0 || !valid_layout(lay) || word_bytes(word) == 0) return GFP_EINVAL;
    gfp_status st = check_pack_vb(p, amax, d, Q, word);
    if (st != GFP_OK) return st;
    if (rows == 0 || cols == 0) return GFP_OK;
    int64_t wr, wc;
    packed_shape(lay, rows, cols, d, &wr, &wc);
    if (!X || !W || ldx < cols || ldw < wc) return GFP_EINVAL;
    return launch_pack(p, rows, cols, X, ldx, d, log2_exact(Q), lay, word, W, ldw,
                       (cudaStream_t)stream);
}

GFP_API gfp_status gfp_unpack(uint32_t p, int64_t rows, int64_t cols, const void *W, int64_t ldw,
                              int d, uint64_t Q, gfp_layout lay, gfp_word word, uint8_t *X,
                              int64_t ldx, void *stream) {
    if (rows < 0 || cols < 0 || !valid_layout(lay) || word_bytes(word) == 0) return GFP_EINVAL;
    gfp_status st = check_pack(p, d, Q, word);
    if (st != GFP_OK) return st;
    if (rows == 0 || cols == 0) return GFP_OK;
    int64_t wr, wc;
    packed_shape(lay, rows, cols, d, &wr, &wc);
    if (!X || !W || ldx < cols || ldw < wc) return GFP_EINVAL;
    return launch_unpack(rows, cols, W, ldw, d, log2_exact(Q), lay, word, X, ldx,
                         (cudaStream_t)stream);
}

static gfp_status resolve_algo(uint32_t p, int64_t m, int64_t k, int64_t n, gfp_algo algo,
                               gfp_algo *out) {
    switch (algo) {
        case GFP_ALGO_PLAIN:
        case GFP_ALGO_DP4A:
        case GFP_ALGO_TC_MMA_S8:
        case GFP_ALGO_TC_F16: *out = algo; return GFP_OK;
        case GFP_ALGO_TC_F8:
            if (p > 31) return GFP_EUNSUPPORTED;
            *out = algo;
            return GFP_OK;
        case GFP_ALGO_TC_E2M1:
            if (p > 7) return GFP_EUNSUPPORTED;
            *out = algo;
            return GFP_OK;
        case GFP_ALGO_AUTO: {
            // Measured on GB300: tcgen05 with fp8 operands (p <= 31) or fp16
            // operands is the fastest exact form at every size worth a launch,
            // except large products with p <= 7, where the e2m1 operands win
            // once k is long enough to pay for converting A as well (8192^3:
            // 0.309 vs 0.362 ms; 4096^3 even; 16384 x 2048 x 16384: 0.446 vs
            // 0.379 ms).
            if (p <= 7 && k >= 6144 && m >= 4096 && n >= 4096) *out = GFP_ALGO_TC_E2M1;
            else *out = p <= 31 ? GFP_ALGO_TC_F8 : GFP_ALGO_TC_F16;
            return GFP_OK;
        }
    }
    return GFP_EINVAL;
}

GFP_API gfp_status gfp_gemm_workspace_size(uint32_t p, int64_t m, int64_t k, int64_t n,
                                           gfp_algo algo, size_t *bytes) {
    if (!bytes || m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    gfp_algo a;
    gfp_status st = resolve_algo(p, m, k, n, algo, &a);
    if (st != GFP_OK) return st;
    *bytes = 0;
    if (a == GFP_ALGO_DP4A) *bytes = dp4a_workspace_bytes(k, n);
    if (a == GFP_ALGO_TC_MMA_S8) *bytes = tc_mma_workspace(m, k, n);
    if (a == GFP_ALGO_TC_F16) *bytes = tc_f16_workspace(m, k, n);
    if (a == GFP_ALGO_TC_F8) *bytes = tc_f8_workspace(m, k, n);
    if (a == GFP_ALGO_TC_E2M1) *bytes = tc_e2m1_workspace(m, k, n);
    return GFP_OK;
}

GFP_API gfp_status gfp_gemm(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                            int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                            gfp_algo algo, void *workspace, size_t ws_bytes, void *stream) {
    if (m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    gfp_algo a;
    gfp_status st = resolve_algo(p, m, k, n, algo, &a);
    if (st != GFP_OK) return st;
    if (m == 0 || n == 0) return GFP_OK;
    if (!C || ldc < n) return GFP_EINVAL;
    if (k > 0 && (!A || !B || lda < k || ldb < n)) return GFP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 0) {
        // empty sum: C = 0
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc, 0, (size_t)n, (size_t)m, s);
        return e == cudaSuccess ? GFP_OK : cuda_fail(e);
    }
    if (a == GFP_ALGO_PLAIN || a == GFP_ALGO_DP4A) {
        const unsigned __int128 tot = (unsigned __int128)k * (p - 1) * (p - 1);
        if (tot >= ((unsigned __int128)1 << 32)) return GFP_EBOUND;
        if (a == GFP_ALGO_DP4A &&
            (!workspace || ws_bytes < dp4a_workspace_bytes(k, n) || ((uintptr_t)workspace & 255)))
            return GFP_EWORKSPACE;
        return launch_plain(p, m, k, n, A, lda, B, ldb, C, ldc, a == GFP_ALGO_DP4A, workspace, ws_bytes, s);
    }
    const size_t need = a == GFP_ALGO_TC_MMA_S8 ? tc_mma_workspace(m, k, n)
                        : a == GFP_ALGO_TC_F8   ? tc_f8_workspace(m, k, n)
                        : a == GFP_ALGO_TC_E2M1 ? tc_e2m1_workspace(m, k, n)
                                                : tc_f16_workspace(m, k, n);
    if (need > 0 && (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)))
        return GFP_EWORKSPACE;
    if (a == GFP_ALGO_TC_MMA_S8)
        return launch_tc_mma(p, m, k, n, A, lda, B, ldb, C, ldc, workspace, ws_bytes, s);
    if (a == GFP_ALGO_TC_F8)
        return launch_tc_f8(p, m, k, n, A, lda, B, ldb, C, ldc, workspace, ws_bytes, s);
    if (a == GFP_ALGO_TC_E2M1)
        return launch_tc_e2m1(p, m, k, n, A, lda, B, ldb, C, ldc, workspace, ws_bytes, s);
    return launch_tc_f16(p, m, k, n, A, lda, B, ldb, C, ldc, workspace, ws_bytes, s);
}

GFP_API gfp_status gfp_gemm_compressed(uint32_t p, int64_t m, int64_t k, int64_t n, int d,
                                       uint64_t Q, gfp_form form, gfp_word word,
                                       const void *CA_or_A, int64_t lda, const void *CB,
                                       int64_t ldb, void *C, int64_t ldc, int64_t kb,
                                       void *stream) {
    return gfp_gemm_compressed_vb(p, m, k, n, d, Q, form, word, p - 1, p - 1, CA_or_A, lda, CB, ldb, C,
                                  ldc, kb, stream);
}

GFP_API gfp_status gfp_gemm_compressed_compc(uint32_t p, int64_t m, int64_t k, int64_t n, int d, uint64_t Q,
                                             gfp_word word, const void *CA, int64_t lda, const void *CB,
                                             int64_t ldb, int64_t kb, int d_out, uint64_t Q_out, void *CC,
                                             int64_t ldcc, void *stream) {
    if (m < 0 || k < 0 || n < 0 || kb < 0 || d_out < 0) return GFP_EINVAL;
    if (word_bytes(word) == 0) return GFP_EINVAL;
    if (word != GFP_WORD_U64 && word != GFP_WORD_U32) return GFP_EUNSUPPORTED;
    gfp_status st = check_dqt(p, k, d, Q, GFP_FORM_DOT, word, kb);
    if (st != GFP_OK) return st;
    st = check_pack(p, d_out, Q_out, word);
    if (st != GFP_OK) return st;
    if (m == 0 || n == 0) return GFP_OK;
    const int64_t kc = cdiv(k, d + 1), wc = cdiv(n, d_out + 1);
    if (!CC || ldcc < wc) return GFP_EINVAL;
    if (kc > 0 && (!CA || !CB || lda < kc || ldb < n)) return GFP_EINVAL;
    const int64_t kbw = (kb > 0 && kb < k) ? kb / (d + 1) : 0;
    return launch_dot_compc(p, m, kc, n, d, log2_exact(Q), word, CA, lda, CB, ldb, kbw, d_out, log2_exact(Q_out),
                            CC, ldcc, (cudaStream_t)stream);
}

GFP_API gfp_status gfp_amax(int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx, uint32_t *out,
                            void *stream) {
    if (rows < 0 || cols < 0 || !out) return GFP_EINVAL;
    if (rows > 0 && cols > 0 && (!X || ldx < cols)) return GFP_EINVAL;
    return launch_amax(rows, cols, X, ldx, out, (cudaStream_t)stream);
}

GFP_API gfp_status gfp_gemm_compressed_vb(uint32_t p, int64_t m, int64_t k, int64_t n, int d,
                                          uint64_t Q, gfp_form form, gfp_word word, uint32_t amax_a,
                                          uint32_t amax_b, const void *CA_or_A, int64_t lda,
                                          const void *CB, int64_t ldb, void *C, int64_t ldc, int64_t kb,
                                          void *stream) {
    if (m < 0 || k < 0 || n < 0 || kb < 0) return GFP_EINVAL;
    if (form != GFP_FORM_DOT && form != GFP_FORM_MIXED && form != GFP_FORM_LEFT) return GFP_EINVAL;
    if (word_bytes(word) == 0) return GFP_EINVAL;
    gfp_status st = check_dqt_vb(p, k, d, Q, form, word, kb, amax_a, amax_b);
    if (st != GFP_OK) return st;
    if (m == 0 || n == 0) return GFP_OK;
    const int t = log2_exact(Q);
    cudaStream_t s = (cudaStream_t)stream;
    if (form == GFP_FORM_DOT) {
        const int64_t kc = cdiv(k, d + 1);
        if (!C || ldc < n) return GFP_EINVAL;
        if (kc > 0 && (!CA_or_A || !CB || lda < kc || ldb < n)) return GFP_EINVAL;
        const int64_t kbw = (kb > 0 && kb < k) ? kb / (d + 1) : 0;
        return launch_dot(p, m, kc, n, d, t, word, CA_or_A, lda, CB, ldb, (uint8_t *)C, ldc, kbw,
                          s);
    }
    if (form == GFP_FORM_LEFT) {
        const int64_t mc = cdiv(m, d + 1);
        if (!C || ldc < n) return GFP_EINVAL;
        if (k > 0 && (!CA_or_A || !CB || lda < k || ldb < n)) return GFP_EINVAL;
        return launch_left(p, mc, k, n, d, t, word, CA_or_A, lda, (const uint8_t *)CB, ldb, C, ldc, s);
    }
    const int64_t nc = cdiv(n, d + 1);
    if (!C || ldc < nc) return GFP_EINVAL;
    if (k > 0 && (!CA_or_A || !CB || lda < k || ldb < nc)) return GFP_EINVAL;
    return launch_mixed(p, m, k, nc, d, t, word, (const uint8_t *)CA_or_A, lda, CB, ldb, C, ldc, s);
}

GFP_API gfp_status gfp_selftest_wait_limit(void *workspace, size_t ws_bytes, uint32_t limit_ms, int *status,
                                           void *stream) {
    if (!status || limit_ms < 1 || limit_ms > 10000) return GFP_EINVAL;
    return tc_selftest_wait_limit(workspace, ws_bytes, (uint64_t)limit_ms * 1000000ull, status, (cudaStream_t)stream);
}

GFP_API gfp_status gfp_winograd_workspace_size(int64_t m, int64_t k, int64_t n, int d, int levels,
                                               size_t *bytes) {
    if (!bytes || m < 0 || k < 0 || n < 0 || d < 0 || levels < 0 || levels > 16) return GFP_EINVAL;
    *bytes = winograd_workspace_bytes(m, cdiv(k, d + 1), n, levels);
    return GFP_OK;
}

GFP_API gfp_status gfp_gemm_compressed_winograd(uint32_t p, int64_t m, int64_t k, int64_t n, int d, uint64_t Q,
                                                const void *CA, int64_t lda, const void *CB, int64_t ldb,
                                                uint8_t *C, int64_t ldc, int levels, void *workspace,
                                                size_t ws_bytes, void *stream) {
    if (m < 0 || k < 0 || n < 0 || levels < 0 || levels > 16) return GFP_EINVAL;
    gfp_status st = check_dqt(p, k, d, Q, GFP_FORM_DOT, GFP_WORD_U64, 0);
    if (st != GFP_OK) return st;
    if (m == 0 || n == 0) return GFP_OK;
    const int64_t kc = cdiv(k, d + 1);
    if (!C || ldc < n) return GFP_EINVAL;
    if (kc > 0 && (!CA || !CB || lda < kc || ldb < n)) return GFP_EINVAL;
    if (kc == 0) {
        const cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc, 0, (size_t)n, (size_t)m, (cudaStream_t)stream);
        return e == cudaSuccess ? GFP_OK : cuda_fail(e);
    }
    return launch_winograd_u64(p, m, kc, n, d, log2_exact(Q), static_cast<const uint64_t *>(CA), lda,
                               static_cast<const uint64_t *>(CB), ldb, C, ldc, levels, workspace, ws_bytes,
                               (cudaStream_t)stream);
}

GFP_API gfp_status gfp_gemm_full(uint32_t p, int64_t m, int64_t k, int64_t n, int dq, int dth,
                                 uint64_t Q, gfp_word word, const void *CA, int64_t lda,
                                 const void *CB, int64_t ldb, void *CC, int64_t ldc, void *stream) {
    if (m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    gfp_status st = check_full(p, k, dq, dth, Q, word);
    if (st != GFP_OK) return st;
    if (m == 0 || n == 0) return GFP_OK;
    const int64_t mc = cdiv(m, dq + 1), nc = cdiv(n, dth + 1);
    if (!CC || ldc < nc) return GFP_EINVAL;
    if (k > 0 && (!CA || !CB || lda < k || ldb < nc)) return GFP_EINVAL;
    return launch_full(p, mc, k, nc, dq, dth, log2_exact(Q), word, CA, lda, CB, ldb, CC, ldc,
                       (cudaStream_t)stream);
}

static gfp_status block_args(uint32_t p, int64_t rows, int64_t cols, int dq, int dth, uint64_t Q,
                             gfp_word word, int64_t ldx, int64_t ldw, bool have_x, bool have_w) {
    if (rows < 0 || cols < 0 || dq < 0 || dth < 0 || dq > 63 || dth > 63) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    const int t = log2_exact(Q);
    if (t < 0) return GFP_EQ;
    if (word != GFP_WORD_U64 && word != GFP_WORD_F64) return GFP_EUNSUPPORTED;
    if ((uint64_t)(p - 1) >= Q) return GFP_EBOUND;
    const int64_t bits = (int64_t)t * (dq + 1) * (dth + 1);
    if (bits > (word == GFP_WORD_F64 ? 52 : 64)) return GFP_EBOUND;
    if (rows == 0 || cols == 0) return GFP_OK;
    if (!have_x || !have_w || ldx < cols || ldw < cdiv(cols, dth + 1)) return GFP_EINVAL;
    return GFP_OK;
}

GFP_API gfp_status gfp_pack_block(uint32_t p, int64_t rows, int64_t cols, const uint8_t *X,
                                  int64_t ldx, int dq, int dth, uint64_t Q, gfp_word word, void *W,
                                  int64_t ldw, void *stream) {
    gfp_status st = block_args(p, rows, cols, dq, dth, Q, word, ldx, ldw, X != nullptr, W != nullptr);
    if (st != GFP_OK || rows == 0 || cols == 0) return st;
    return launch_block(true, rows, cols, X, nullptr, ldx, dq, dth, log2_exact(Q), word, nullptr, W, ldw,
                        (cudaStream_t)stream);
}

GFP_API gfp_status gfp_unpack_block(uint32_t p, int64_t rows, int64_t cols, const void *W,
                                    int64_t ldw, int dq, int dth, uint64_t Q, gfp_word word,
                                    uint8_t *X, int64_t ldx, void *stream) {
    gfp_status st = block_args(p, rows, cols, dq, dth, Q, word, ldx, ldw, X != nullptr, W != nullptr);
    if (st != GFP_OK || rows == 0 || cols == 0) return st;
    return launch_block(false, rows, cols, nullptr, X, ldx, dq, dth, log2_exact(Q), word, W, nullptr, ldw,
                        (cudaStream_t)stream);
}

}  // extern "C"
