// Conversions between residue matrices and Q-adic words (Section 2.1 INIT,
// Section 2.3 partial compression, Section 3 row compression; Table 2's
// INIT_e / EXTRACT_e).  Q = 2^t, so a word is built from shifts and adds and
// a coefficient is read back with a shift and a mask.
//
// Layouts, for a residue matrix X (rows x cols):
//   ROWS_REV: W[i][w] = sum_j X[i][w(d+1)+j] Q^(d-j)   (rows of A, reversed)
//   COLS    : W[w][j] = sum_s X[w(d+1)+s][j] Q^s       (columns of B)
//   ROWS    : W[i][v] = sum_j X[i][v(d+1)+j] Q^j       (rows, forward)
// Entries past the edge count as zero.
//
// These kernels move bytes: one thread per word, consecutive threads on
// consecutive words of a row, so both the residue reads and the word writes
// of a warp are contiguous.
#include <cstdint>
#include <type_traits>

#include "gfp_internal.h"

namespace gfp {
namespace {

// Words of type double hold integers below 2^53, so both conversions are exact.
template <class W>
__device__ __forceinline__ W to_word(uint64_t v) {
    return (W)v;
}

template <class W>
__device__ __forceinline__ uint64_t from_word(W w) {
    if constexpr (std::is_floating_point<W>::value) return __double2ull_rz(w);
    else return (uint64_t)w;
}

// Rows, reversed (REV) or forward: thread per word (i, w).
template <class W, bool REV>
__global__ void pack_rows_kernel(const uint8_t *__restrict__ X, int64_t ldx, int64_t rows,
                                 int64_t cols, int dp1, int t, W *__restrict__ out, int64_t ldw,
                                 int64_t wc) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= wc) return;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        const uint8_t *x = X + i * ldx + w * dp1;
        const int64_t rem = cols - w * dp1;
        const int n = rem < dp1 ? (int)rem : dp1;
        uint64_t acc = 0;
        for (int j = 0; j < n; ++j) {
            const int s = REV ? dp1 - 1 - j : j;
            acc += (uint64_t)x[j] << (t * s);
        }
        out[i * ldw + w] = to_word<W>(acc);
    }
}

// Columns: thread per word (w, j).
template <class W>
__global__ void pack_cols_kernel(const uint8_t *__restrict__ X, int64_t ldx, int64_t rows,
                                 int64_t cols, int dp1, int t, W *__restrict__ out, int64_t ldw,
                                 int64_t wr) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    for (int64_t w = blockIdx.y; w < wr; w += gridDim.y) {
        const int64_t rem = rows - w * dp1;
        const int n = rem < dp1 ? (int)rem : dp1;
        const uint8_t *x = X + (w * dp1) * ldx + j;
        uint64_t acc = 0;
        for (int s = 0; s < n; ++s) acc += (uint64_t)x[s * ldx] << (t * s);
        out[w * ldw + j] = to_word<W>(acc);
    }
}

template <class W, bool REV>
__global__ void unpack_rows_kernel(const W *__restrict__ Win, int64_t ldw, int64_t rows,
                                   int64_t cols, int dp1, int t, uint8_t *__restrict__ X,
                                   int64_t ldx, int64_t wc) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= wc) return;
    const uint64_t mask = (1ull << t) - 1;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        const uint64_t v = from_word<W>(Win[i * ldw + w]);
        const int64_t rem = cols - w * dp1;
        const int n = rem < dp1 ? (int)rem : dp1;
        uint8_t *x = X + i * ldx + w * dp1;
        for (int j = 0; j < n; ++j) {
            const int s = REV ? dp1 - 1 - j : j;
            x[j] = (uint8_t)((v >> (t * s)) & mask);
        }
    }
}

template <class W>
__global__ void unpack_cols_kernel(const W *__restrict__ Win, int64_t ldw, int64_t rows,
                                   int64_t cols, int dp1, int t, uint8_t *__restrict__ X,
                                   int64_t ldx, int64_t wr) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    const uint64_t mask = (1ull << t) - 1;
    for (int64_t w = blockIdx.y; w < wr; w += gridDim.y) {
        const uint64_t v = from_word<W>(Win[w * ldw + j]);
        const int64_t rem = rows - w * dp1;
        const int n = rem < dp1 ? (int)rem : dp1;
        uint8_t *x = X + (w * dp1) * ldx + j;
        for (int s = 0; s < n; ++s) x[s * ldx] = (uint8_t)((v >> (t * s)) & mask);
    }
}

// Section 4 result layout: W[u][v] = sum_i sum_j X[u(dq+1)+i][v(dth+1)+j]
// Q^(i + j(dq+1)); thread per word (u, v).
template <class W>
__global__ void pack_block_kernel(const uint8_t *__restrict__ X, int64_t ldx, int64_t rows,
                                  int64_t cols, int dq1, int dth1, int t, W *__restrict__ out,
                                  int64_t ldw, int64_t wcols, int64_t wrows) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= wcols) return;
    for (int64_t u = blockIdx.y; u < wrows; u += gridDim.y) {
        uint64_t acc = 0;
        for (int i = 0; i < dq1; ++i) {
            const int64_t r = u * dq1 + i;
            if (r >= rows) break;
            for (int j = 0; j < dth1; ++j) {
                const int64_t c = v * dth1 + j;
                if (c < cols) acc += (uint64_t)X[r * ldx + c] << (t * (i + j * dq1));
            }
        }
        out[u * ldw + v] = to_word<W>(acc);
    }
}

template <class W>
__global__ void unpack_block_kernel(const W *__restrict__ Win, int64_t ldw, int64_t rows,
                                    int64_t cols, int dq1, int dth1, int t, uint8_t *__restrict__ X,
                                    int64_t ldx, int64_t wcols, int64_t wrows) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= wcols) return;
    const uint64_t mask = (1ull << t) - 1;
    for (int64_t u = blockIdx.y; u < wrows; u += gridDim.y) {
        const uint64_t w = from_word<W>(Win[u * ldw + v]);
        for (int i = 0; i < dq1; ++i) {
            const int64_t r = u * dq1 + i;
            if (r >= rows) break;
            for (int j = 0; j < dth1; ++j) {
                const int64_t c = v * dth1 + j;
                if (c < cols) X[r * ldx + c] = (uint8_t)((w >> (t * (i + j * dq1))) & mask);
            }
        }
    }
}

constexpr int kThreads = 256;

dim3 grid_for(int64_t inner, int64_t outer) {
    const int64_t gx = (inner + kThreads - 1) / kThreads;
    const int64_t gy = outer < 65535 ? outer : 65535;
    return dim3((unsigned)gx, (unsigned)(gy > 0 ? gy : 1));
}

template <class W>
cudaError_t pack_t(int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx, int dp1, int t,
                   gfp_layout lay, void *Wp, int64_t ldw, cudaStream_t s) {
    W *out = static_cast<W *>(Wp);
    if (lay == GFP_LAYOUT_COLS) {
        const int64_t wr = (rows + dp1 - 1) / dp1;
        pack_cols_kernel<W><<<grid_for(cols, wr), kThreads, 0, s>>>(X, ldx, rows, cols, dp1, t,
                                                                      out, ldw, wr);
    } else {
        const int64_t wc = (cols + dp1 - 1) / dp1;
        if (lay == GFP_LAYOUT_ROWS_REV)
            pack_rows_kernel<W, true><<<grid_for(wc, rows), kThreads, 0, s>>>(X, ldx, rows, cols,
                                                                               dp1, t, out, ldw, wc);
        else
            pack_rows_kernel<W, false><<<grid_for(wc, rows), kThreads, 0, s>>>(
                X, ldx, rows, cols, dp1, t, out, ldw, wc);
    }
    return cudaGetLastError();
}

template <class W>
cudaError_t unpack_t(int64_t rows, int64_t cols, const void *Wp, int64_t ldw, int dp1, int t,
                     gfp_layout lay, uint8_t *X, int64_t ldx, cudaStream_t s) {
    const W *in = static_cast<const W *>(Wp);
    if (lay == GFP_LAYOUT_COLS) {
        const int64_t wr = (rows + dp1 - 1) / dp1;
        unpack_cols_kernel<W><<<grid_for(cols, wr), kThreads, 0, s>>>(in, ldw, rows, cols, dp1, t,
                                                                        X, ldx, wr);
    } else {
        const int64_t wc = (cols + dp1 - 1) / dp1;
        if (lay == GFP_LAYOUT_ROWS_REV)
            unpack_rows_kernel<W, true><<<grid_for(wc, rows), kThreads, 0, s>>>(
                in, ldw, rows, cols, dp1, t, X, ldx, wc);
        else
            unpack_rows_kernel<W, false><<<grid_for(wc, rows), kThreads, 0, s>>>(
                in, ldw, rows, cols, dp1, t, X, ldx, wc);
    }
    return cudaGetLastError();
}

}  // namespace

gfp_status launch_pack(uint32_t, int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx, int d,
                       int t, gfp_layout lay, gfp_word word, void *W, int64_t ldw,
                       cudaStream_t s) {
    cudaError_t e;
    if (word == GFP_WORD_F64)
        e = pack_t<double>(rows, cols, X, ldx, d + 1, t, lay, W, ldw, s);
    else if (word_bytes(word) == 8)
        e = pack_t<uint64_t>(rows, cols, X, ldx, d + 1, t, lay, W, ldw, s);
    else
        e = pack_t<uint32_t>(rows, cols, X, ldx, d + 1, t, lay, W, ldw, s);
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

gfp_status launch_unpack(int64_t rows, int64_t cols, const void *W, int64_t ldw, int d, int t,
                         gfp_layout lay, gfp_word word, uint8_t *X, int64_t ldx, cudaStream_t s) {
    cudaError_t e;
    if (word == GFP_WORD_F64)
        e = unpack_t<double>(rows, cols, W, ldw, d + 1, t, lay, X, ldx, s);
    else if (word_bytes(word) == 8)
        e = unpack_t<uint64_t>(rows, cols, W, ldw, d + 1, t, lay, X, ldx, s);
    else
        e = unpack_t<uint32_t>(rows, cols, W, ldw, d + 1, t, lay, X, ldx, s);
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

}  // namespace gfp

namespace gfp {

gfp_status launch_block(bool pack, int64_t rows, int64_t cols, const uint8_t *X, uint8_t *Xout,
                        int64_t ldx, int dq, int dth, int t, gfp_word word, const void *Win, void *Wout,
                        int64_t ldw, cudaStream_t s) {
    const int64_t wr = (rows + dq) / (dq + 1), wc = (cols + dth) / (dth + 1);
    const dim3 grid = grid_for(wc, wr);
    if (word == GFP_WORD_F64) {
        if (pack)
            pack_block_kernel<double><<<grid, kThreads, 0, s>>>(X, ldx, rows, cols, dq + 1, dth + 1, t,
                                                                static_cast<double *>(Wout), ldw, wc, wr);
        else
            unpack_block_kernel<double><<<grid, kThreads, 0, s>>>(static_cast<const double *>(Win), ldw,
                                                                  rows, cols, dq + 1, dth + 1, t, Xout,
                                                                  ldx, wc, wr);
    } else {
        if (pack)
            pack_block_kernel<uint64_t><<<grid, kThreads, 0, s>>>(X, ldx, rows, cols, dq + 1, dth + 1, t,
                                                                  static_cast<uint64_t *>(Wout), ldw, wc, wr);
        else
            unpack_block_kernel<uint64_t><<<grid, kThreads, 0, s>>>(static_cast<const uint64_t *>(Win),
                                                                    ldw, rows, cols, dq + 1, dth + 1, t,
                                                                    Xout, ldx, wc, wr);
    }
    return check_launch();
}

// Largest entry of a uint8 matrix (the amax bounds of the value-aware
// parameters): rows in a grid-stride loop, a warp maximum, one atomicMax per
// warp on the zeroed result.
__global__ void amax_kernel(const uint8_t *__restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                            uint32_t *out) {
    uint32_t mx = 0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const uint8_t *row = X + r * ldx;
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) mx = max(mx, (uint32_t)row[c]);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

gfp_status launch_amax(int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx, uint32_t *out,
                       cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (rows == 0 || cols == 0) return GFP_OK;
    const int64_t grid = rows < (int64_t)num_sms() * 8 ? rows : (int64_t)num_sms() * 8;
    amax_kernel<<<(unsigned)grid, 256, 0, s>>>(X, rows, cols, ldx, out);
    return check_launch();
}

}  // namespace gfp
