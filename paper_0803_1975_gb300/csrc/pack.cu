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
// These kernels move bytes.  Row layouts stage a chunk of up to 8 KB of a
// row's residues in shared memory per block, moved as aligned 16-byte blocks,
// and give a thread four consecutive words (vector loads and stores of words).
// Column layouts give a thread four adjacent columns, read or written as one
// 32-bit word of residues and stored as one 16-byte store of words.
#include <atomic>
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

constexpr int V = 4;   // words per thread

// Store N consecutive words at p: one vector store when N = 4, p is 16-byte
// aligned and all N are inside the row, else one by one.
template <class W, int N = V>
__device__ __forceinline__ void store_words(W *p, const W (&v)[N], int n) {
    if constexpr (N == 4) {
        if (n == N && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
            if constexpr (sizeof(W) == 8) {
                const unsigned long long *u = reinterpret_cast<const unsigned long long *>(v);
                reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(u[0], u[1]);
                reinterpret_cast<ulonglong2 *>(p)[1] = make_ulonglong2(u[2], u[3]);
            } else {
                *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
            }
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < N; ++e)
        if (e < n) p[e] = v[e];
}

// Load N consecutive words at p: one vector load when N = 4, p is 16-byte
// aligned and all N are inside the row, else one by one (zero past the row).
template <class W, int N = V>
__device__ __forceinline__ void load_words(const W *p, W (&v)[N], int n) {
    if constexpr (N == 4) {
        if (n == N && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
            if constexpr (sizeof(W) == 8) {
                const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2 *>(p));
                const ulonglong2 y = __ldg(reinterpret_cast<const ulonglong2 *>(p) + 1);
                const unsigned long long u[4] = {x.x, x.y, y.x, y.y};
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = __builtin_bit_cast(W, u[e]);
            } else {
                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
                const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = __builtin_bit_cast(W, u[e]);
            }
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = e < n ? __ldg(p + e) : W(0);
}

// Row layouts.  A block handles a chunk of up to ROW_WORDS consecutive words
// of a row (at most ROW_STAGE residues, staged in shared memory), V words per
// thread, and loops over rows; packing fetches the next row's residues while
// it builds the current row's words (the same for unpacking was measured
// slower: its sixteen words per thread stay in registers across the writes).
// The residues move as aligned 16-byte blocks (an aligned block that holds a
// byte of the row lies in the same page, so reading it cannot fault; on the
// write side only the blocks that lie inside the chunk are written whole, the
// two ragged ends byte by byte); up to ROW_LPT such loads per thread are
// issued back to back so that about 8 KB per block is in flight.
constexpr int ROW_THREADS = 256;
constexpr int ROW_STAGE = 8192;                                  // residues per chunk
constexpr int ROW_WORDS = 4096;                                  // words per chunk
constexpr int ROW_LPT = (ROW_STAGE / 16 + 2 + ROW_THREADS - 1) / ROW_THREADS;

// words per chunk with vw words per thread: short rows (one word per thread)
// need at most one word in each of V passes over the block
__host__ __device__ constexpr int row_words(int vw) { return vw == 1 ? V * ROW_THREADS : ROW_WORDS; }
// resident blocks the register budget aims at: all the rows of a small
// matrix in flight at once (one word per thread), one wave of long rows
__host__ __device__ constexpr int row_min_blocks(int vw, bool pack) { return vw == 1 ? 8 : pack ? 4 : 3; }

// Words per chunk: the row's wc words in equal chunks (a multiple of vw
// words each, at most what the stage and row_words allow), the count chosen
// to minimise chunks x passes of the block over a chunk -- a block waits at
// its barrier for its busiest thread, so a chunk of 1.3 passes costs two.
inline int row_chunk_words(int64_t wc, int dp1, int vw) {
    int64_t most = ROW_STAGE / dp1;
    most = most < row_words(vw) ? most : row_words(vw);
    most -= most % vw;
    if (most < vw) most = vw;
    const int64_t c0 = (wc + most - 1) / most, per_pass = (int64_t)vw * ROW_THREADS;
    int64_t best_w = most, best_cost = -1;
    for (int64_t c = c0 > 0 ? c0 : 1; c <= c0 + 8; ++c) {
        int64_t w = (wc + c - 1) / c;
        w = (w + vw - 1) / vw * vw;
        if (w > most) continue;
        const int64_t cost = c * ((w + per_pass - 1) / per_pass);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_w = w;
        }
    }
    return (int)best_w;
}

// Words per thread: V (vector loads and stores of words) for rows of at least
// V * ROW_THREADS words, one for shorter rows, whose chunk would otherwise
// leave most of the block idle.
inline int row_words_per_thread(int64_t wc) { return wc >= (int64_t)V * ROW_THREADS ? V : 1; }

// Rows, reversed (REV) or forward: a block packs words w0 .. w0 + nw - 1 of
// its rows from the residues staged in shared memory.
template <class W, bool REV, int VW, int DP1>
__global__ void __launch_bounds__(ROW_THREADS, row_min_blocks(VW, true))
pack_rows_kernel(const uint8_t *__restrict__ X, int64_t ldx, int64_t rows, int64_t cols, int dp1_arg, int t,
                 W *__restrict__ out, int64_t ldw, int64_t wc, int cw) {
    __shared__ uint4 sbuf[ROW_STAGE / 16 + 2];
    const int dp1 = DP1 > 0 ? DP1 : dp1_arg;      // residues per word (a constant when DP1 > 0)
    const int64_t whole = cols / dp1;            // words of dp1 residues; word `whole` holds the tail
    const int tail = (int)(cols - whole * dp1);
    const int64_t w0 = (int64_t)blockIdx.x * cw;
    const int nw = wc - w0 < cw ? (int)(wc - w0) : cw;
    const int64_t b0 = w0 * dp1, b1 = (w0 + nw) * dp1 < cols ? (w0 + nw) * dp1 : cols;
    // the aligned 16-byte blocks covering row i's chunk, into registers
    uint4 r[ROW_LPT];
    auto fetch = [&](int64_t i) {
        const uint8_t *row = X + i * ldx;
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(row + b0) & ~(uintptr_t)15;
        const int nq = (int)((reinterpret_cast<uintptr_t>(row + b1) + 15 - a0) / 16);
#pragma unroll
        for (int e = 0; e < ROW_LPT; ++e) {
            const int q = threadIdx.x + e * ROW_THREADS;
            if (q < nq) r[e] = __ldg(reinterpret_cast<const uint4 *>(a0) + q);
        }
    };
    // long rows (VW > 1): the next row's blocks are in flight while this row's
    // words are built; short rows have a block each and fetch as they go
    constexpr bool ahead = VW > 1;
    if (ahead && blockIdx.y < rows) fetch(blockIdx.y);
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        const uint8_t *row = X + i * ldx;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(row + b0), a0 = lo & ~(uintptr_t)15;
        const int nq = (int)((reinterpret_cast<uintptr_t>(row + b1) + 15 - a0) / 16);
        if (!ahead) fetch(i);
#pragma unroll
        for (int e = 0; e < ROW_LPT; ++e) {
            const int q = threadIdx.x + e * ROW_THREADS;
            if (q < nq) sbuf[q] = r[e];
        }
        __syncthreads();
        if (ahead && i + gridDim.y < rows) fetch(i + gridDim.y);
        const uint8_t *sb = reinterpret_cast<const uint8_t *>(sbuf) + (lo - a0);
#pragma unroll
        for (int g = 0; g < row_words(VW) / (VW * ROW_THREADS); ++g) {
            const int w = (threadIdx.x + g * ROW_THREADS) * VW;
            if (w >= nw) break;
            W v[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                // residues of word w0 + w + e inside the row (none past the last word)
                const int64_t word = w0 + w + e;
                const int n = word < whole ? dp1 : word == whole ? tail : 0;
                // Horner in base Q = 2^t, highest power first (each residue < Q)
                const uint8_t *src = sb + (w + e) * dp1;
                uint64_t acc = 0;
                if (DP1 > 0 && n == DP1) {
#pragma unroll
                    for (int j = 0; j < DP1; ++j) acc = (acc << t) | src[REV ? j : DP1 - 1 - j];
                } else if (REV) {
#pragma unroll 1
                    for (int j = 0; j < n; ++j) acc = (acc << t) | src[j];
                    if (n < dp1 && n > 0) acc <<= t * (dp1 - n);   // the missing residues are the low powers
                } else {
#pragma unroll 1
                    for (int j = n - 1; j >= 0; --j) acc = (acc << t) | src[j];
                }
                v[e] = to_word<W>(acc);
            }
            store_words<W, VW>(out + i * ldw + w0 + w, v, nw - w < VW ? nw - w : VW);
        }
        __syncthreads();
    }
}

// Columns: thread per V words (w, j0 .. j0+V-1), the residues of four
// adjacent columns read as one 32-bit word when aligned.
template <class W>
__global__ void pack_cols_kernel(const uint8_t *__restrict__ X, int64_t ldx, int64_t rows,
                                 int64_t cols, int dp1, int t, W *__restrict__ out, int64_t ldw,
                                 int64_t wr) {
    const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (j0 >= cols) return;
    const int nj = cols - j0 < V ? (int)(cols - j0) : V;
    // all four columns of every residue row in one aligned 32-bit load
    const bool vec = nj == V && ((reinterpret_cast<uintptr_t>(X + j0) | (uintptr_t)ldx) & 3) == 0;
    constexpr int MAXR = 8;   // residue rows per word held in registers (loads in flight together)
    for (int64_t w = blockIdx.y; w < wr; w += gridDim.y) {
        const int64_t rem = rows - w * dp1;
        const int n = rem < dp1 ? (int)rem : dp1;
        const uint8_t *x0 = X + w * dp1 * ldx + j0;
        // Horner in base Q = 2^t over the residue rows, highest power (row n-1) first
        uint64_t acc[V] = {0, 0, 0, 0};
        if (vec && n <= MAXR) {
            uint32_t q[MAXR];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r < n) q[r] = __ldg(reinterpret_cast<const uint32_t *>(x0 + r * ldx));
#pragma unroll
            for (int r = MAXR - 1; r >= 0; --r)
                if (r < n) {
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = (acc[e] << t) | ((q[r] >> (8 * e)) & 0xffu);
                }
        } else {
            for (int r = n - 1; r >= 0; --r) {
                const uint8_t *x = x0 + r * ldx;
                if (vec) {
                    const uint32_t q = __ldg(reinterpret_cast<const uint32_t *>(x));
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = (acc[e] << t) | ((q >> (8 * e)) & 0xffu);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (e < nj) acc[e] = (acc[e] << t) | __ldg(x + e);
                }
            }
        }
        W v[V];
#pragma unroll
        for (int e = 0; e < V; ++e) v[e] = to_word<W>(acc[e]);
        store_words<W>(out + w * ldw + j0, v, nj);
    }
}

template <class W, bool REV, int VW, int DP1>
__global__ void __launch_bounds__(ROW_THREADS, row_min_blocks(VW, false))
unpack_rows_kernel(const W *__restrict__ Win, int64_t ldw, int64_t rows, int64_t cols, int dp1_arg, int t,
                   uint8_t *__restrict__ X, int64_t ldx, int64_t wc, int cw) {
    __shared__ uint4 sbuf[ROW_STAGE / 16 + 2];
    const int dp1 = DP1 > 0 ? DP1 : dp1_arg;
    const int64_t whole = cols / dp1;
    const int tail = (int)(cols - whole * dp1);
    const int64_t w0 = (int64_t)blockIdx.x * cw;
    const int nw = wc - w0 < cw ? (int)(wc - w0) : cw;
    const int64_t b0 = w0 * dp1, b1 = (w0 + nw) * dp1 < cols ? (w0 + nw) * dp1 : cols;
    const uint64_t mask = (1ull << t) - 1;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        uint8_t *row = X + i * ldx;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(row + b0), hi = reinterpret_cast<uintptr_t>(row + b1);
        const uintptr_t a0 = lo & ~(uintptr_t)15;
        uint8_t *sb = reinterpret_cast<uint8_t *>(sbuf) + (lo - a0);
        // all of this thread's words first (their loads in flight together)
        constexpr int G = row_words(VW) / (VW * ROW_THREADS);
        W v[G][VW];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int w = (threadIdx.x + g * ROW_THREADS) * VW;
            if (w < nw) load_words<W, VW>(Win + i * ldw + w0 + w, v[g], nw - w < VW ? nw - w : VW);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int w = (threadIdx.x + g * ROW_THREADS) * VW;
            if (w >= nw) break;
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const int64_t word = w0 + w + e;
                const int n = word < whole ? dp1 : word == whole ? tail : 0;
                // digits peeled off the low end, lowest power first
                uint64_t x = from_word<W>(v[g][e]);
                uint8_t *dst = sb + (w + e) * dp1;
                if (DP1 > 0 && n == DP1) {
#pragma unroll
                    for (int j = 0; j < DP1; ++j, x >>= t) dst[REV ? DP1 - 1 - j : j] = (uint8_t)(x & mask);
                } else if (REV) {
                    if (n < dp1 && n > 0) x >>= t * (dp1 - n);      // the missing residues' powers
#pragma unroll 1
                    for (int j = n - 1; j >= 0; --j, x >>= t) dst[j] = (uint8_t)(x & mask);
                } else {
#pragma unroll 1
                    for (int j = 0; j < n; ++j, x >>= t) dst[j] = (uint8_t)(x & mask);
                }
            }
        }
        __syncthreads();
        // aligned 16-byte blocks inside [lo, hi) whole, the two ragged ends by bytes
        const int nq = (int)((((hi + 15) & ~(uintptr_t)15) - a0) / 16);
#pragma unroll
        for (int e = 0; e < ROW_LPT; ++e) {
            const int q = threadIdx.x + e * ROW_THREADS;
            if (q >= nq) break;
            const uintptr_t a = a0 + 16 * (uintptr_t)q;
            if (a >= lo && a + 16 <= hi) {
                *reinterpret_cast<uint4 *>(a) = sbuf[q];
            } else {
                const uint8_t *src = reinterpret_cast<const uint8_t *>(&sbuf[q]);
                for (int c = 0; c < 16; ++c)
                    if (a + c >= lo && a + c < hi) *reinterpret_cast<uint8_t *>(a + c) = src[c];
            }
        }
        __syncthreads();
    }
}

template <class W>
__global__ void unpack_cols_kernel(const W *__restrict__ Win, int64_t ldw, int64_t rows,
                                   int64_t cols, int dp1, int t, uint8_t *__restrict__ X,
                                   int64_t ldx, int64_t wr) {
    const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (j0 >= cols) return;
    const int nj = cols - j0 < V ? (int)(cols - j0) : V;
    const uint64_t mask = (1ull << t) - 1;
    for (int64_t w = blockIdx.y; w < wr; w += gridDim.y) {
        uint64_t v[V];
#pragma unroll
        for (int e = 0; e < V; ++e) v[e] = e < nj ? from_word<W>(__ldg(Win + w * ldw + j0 + e)) : 0;
        const int64_t rem = rows - w * dp1;
        const int n = rem < dp1 ? (int)rem : dp1;
        // digits peeled off the low end: residue row s holds the coefficient of Q^s
        for (int s = 0; s < n; ++s) {
            uint8_t *x = X + (w * dp1 + s) * ldx + j0;
            if (nj == V && (reinterpret_cast<uintptr_t>(x) & 3) == 0) {
                uint32_t q = 0;
#pragma unroll
                for (int e = 0; e < V; ++e) q |= (uint32_t)(v[e] & mask) << (8 * e);
                *reinterpret_cast<uint32_t *>(x) = q;
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (e < nj) x[e] = (uint8_t)(v[e] & mask);
            }
#pragma unroll
            for (int e = 0; e < V; ++e) v[e] >>= t;
        }
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

// Blocks of a staged row kernel: one per chunk of a row (row_chunk_words
// words) times as many row slices as the SMs hold resident blocks (the
// occupancy of the kernel, asked once) -- a single wave -- each block looping
// over rows.
template <class K>
dim3 rows_grid(K kernel, std::atomic<int> &per_sm, int64_t wc, int64_t rows, int cw) {
    int r = per_sm.load(std::memory_order_relaxed);
    if (r < 1) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kernel, ROW_THREADS, 0) != cudaSuccess || r < 1) {
            (void)cudaGetLastError();
            r = 1;
        }
        per_sm.store(r, std::memory_order_relaxed);
    }
    const int64_t gx = (wc + cw - 1) / cw;
    int64_t gy = (int64_t)num_sms() * r / gx;   // one wave: every block resident
    if (gy > rows) gy = rows;
    if (gy > 65535) gy = 65535;
    return dim3((unsigned)gx, (unsigned)(gy > 0 ? gy : 1));
}

template <class W, bool REV, int VW, int DP1>
cudaError_t launch_pack_rows(const uint8_t *X, int64_t ldx, int64_t rows, int64_t cols, int dp1, int t, W *out,
                             int64_t ldw, int64_t wc, cudaStream_t s) {
    static std::atomic<int> per_sm{0};
    const int cw = row_chunk_words(wc, dp1, VW);
    pack_rows_kernel<W, REV, VW, DP1><<<rows_grid(pack_rows_kernel<W, REV, VW, DP1>, per_sm, wc, rows, cw),
                                        ROW_THREADS, 0, s>>>(X, ldx, rows, cols, dp1, t, out, ldw, wc, cw);
    return cudaGetLastError();
}

// Long rows of 1 to 4 residues per word (the common word widths) get the
// kernel with that count as a constant: whole words unrolled, their shared-
// memory loads issued together (measured 25-30% faster than a loop over a
// run-time count at 16384^2).
template <class W, bool REV>
cudaError_t pack_rows_dispatch(const uint8_t *X, int64_t ldx, int64_t rows, int64_t cols, int dp1, int t, W *out,
                               int64_t ldw, int64_t wc, cudaStream_t s) {
    if (row_words_per_thread(wc) != V)
        return launch_pack_rows<W, REV, 1, 0>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
    switch (dp1) {
        case 1: return launch_pack_rows<W, REV, V, 1>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
        case 2: return launch_pack_rows<W, REV, V, 2>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
        case 3: return launch_pack_rows<W, REV, V, 3>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
        case 4: return launch_pack_rows<W, REV, V, 4>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
        default: return launch_pack_rows<W, REV, V, 0>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
    }
}

template <class W, bool REV, int VW, int DP1>
cudaError_t launch_unpack_rows(const W *in, int64_t ldw, int64_t rows, int64_t cols, int dp1, int t, uint8_t *X,
                               int64_t ldx, int64_t wc, cudaStream_t s) {
    static std::atomic<int> per_sm{0};
    const int cw = row_chunk_words(wc, dp1, VW);
    unpack_rows_kernel<W, REV, VW, DP1><<<rows_grid(unpack_rows_kernel<W, REV, VW, DP1>, per_sm, wc, rows, cw),
                                          ROW_THREADS, 0, s>>>(in, ldw, rows, cols, dp1, t, X, ldx, wc, cw);
    return cudaGetLastError();
}

template <class W, bool REV>
cudaError_t unpack_rows_dispatch(const W *in, int64_t ldw, int64_t rows, int64_t cols, int dp1, int t, uint8_t *X,
                                 int64_t ldx, int64_t wc, cudaStream_t s) {
    if (row_words_per_thread(wc) != V)
        return launch_unpack_rows<W, REV, 1, 0>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
    switch (dp1) {
        case 1: return launch_unpack_rows<W, REV, V, 1>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
        case 2: return launch_unpack_rows<W, REV, V, 2>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
        case 3: return launch_unpack_rows<W, REV, V, 3>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
        case 4: return launch_unpack_rows<W, REV, V, 4>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
        default: return launch_unpack_rows<W, REV, V, 0>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
    }
}

dim3 grid_for(int64_t inner, int64_t outer, int per_thread = 1) {
    const int64_t gx = (inner + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
    // about 16 blocks per SM in all, each looping over the outer index
    int64_t gy = ((int64_t)num_sms() * 16 + gx - 1) / gx;
    if (gy > outer) gy = outer;
    if (gy > 65535) gy = 65535;
    return dim3((unsigned)gx, (unsigned)(gy > 0 ? gy : 1));
}

template <class W>
cudaError_t pack_t(int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx, int dp1, int t,
                   gfp_layout lay, void *Wp, int64_t ldw, cudaStream_t s) {
    W *out = static_cast<W *>(Wp);
    if (lay == GFP_LAYOUT_COLS) {
        const int64_t wr = (rows + dp1 - 1) / dp1;
        pack_cols_kernel<W><<<grid_for(cols, wr, V), kThreads, 0, s>>>(X, ldx, rows, cols, dp1, t,
                                                                      out, ldw, wr);
    } else {
        const int64_t wc = (cols + dp1 - 1) / dp1;
        if (lay == GFP_LAYOUT_ROWS_REV)
            return pack_rows_dispatch<W, true>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
        return pack_rows_dispatch<W, false>(X, ldx, rows, cols, dp1, t, out, ldw, wc, s);
    }
    return cudaGetLastError();
}

template <class W>
cudaError_t unpack_t(int64_t rows, int64_t cols, const void *Wp, int64_t ldw, int dp1, int t,
                     gfp_layout lay, uint8_t *X, int64_t ldx, cudaStream_t s) {
    const W *in = static_cast<const W *>(Wp);
    if (lay == GFP_LAYOUT_COLS) {
        const int64_t wr = (rows + dp1 - 1) / dp1;
        unpack_cols_kernel<W><<<grid_for(cols, wr, V), kThreads, 0, s>>>(in, ldw, rows, cols, dp1, t,
                                                                        X, ldx, wr);
    } else {
        const int64_t wc = (cols + dp1 - 1) / dp1;
        if (lay == GFP_LAYOUT_ROWS_REV)
            return unpack_rows_dispatch<W, true>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
        return unpack_rows_dispatch<W, false>(in, ldw, rows, cols, dp1, t, X, ldx, wc, s);
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
