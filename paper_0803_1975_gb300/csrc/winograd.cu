// Strassen-Winograd recursion over the packed words of the Q-adic dot form
// (Section 5's remark on fast matrix multiplication: the gains of Table "gains"
// with exponent omega < 3).
//
// The dot form multiplies word matrices CA (m x kc) and CB (kc x n) and reads
// the coefficient of Q^d of every result word.  With 64-bit words that
// coefficient is exact modulo 2^64 when t(d+1) <= 64 (the u64 reading of the
// bounds), so only the word product mod 2^64 is needed -- and Winograd's
// 7-multiplication scheme is an identity over any ring, Z/2^64 included.  The
// recursion therefore runs on the words with wrapping 64-bit additions and
// subtractions, the base products are the raw word GEMM, and the digits are
// read once from the final words: exactly the words (and digits) of the
// classical product, with no bound beyond the dot form's own.
//
// One level, blocks X11 .. X22 of the operands split at ceil(dim / 2) (the
// last block row or column may be one shorter; missing entries count as 0):
//   S1 = A21 + A22   S2 = S1 - A11   S3 = A11 - A21   S4 = A12 - S2
//   T1 = B12 - B11   T2 = B22 - T1   T3 = B22 - B12   T4 = T2 - B21
//   P1 = A11 B11  P2 = A12 B21  P3 = S4 B22  P4 = A22 T4
//   P5 = S1 T1    P6 = S2 T2    P7 = S3 T3
//   C11 = P1 + P2          C12 = P1 + P6 + P5 + P3
//   C21 = P1 + P6 + P7 - P4   C22 = P1 + P6 + P7 + P5
// Products that involve an original block use its exact extent (P2, P3 and P4
// run over the shorter inner dimension, P3 has the shorter column count, P4
// the shorter row count), and the combination reads only what each defines.
#include <cstdint>

#include "gfp_internal.h"

namespace gfp {
namespace {

struct WView {               // a word matrix: rows x cols, leading dimension ld
    uint64_t *p;
    int64_t ld, rows, cols;
};

__device__ __forceinline__ uint64_t at(const uint64_t *X, int64_t ld, int64_t rows, int64_t cols, int64_t i,
                                       int64_t j) {
    return (i < rows && j < cols) ? X[i * ld + j] : 0ull;
}

// S1..S4 from the blocks of A (h1 x w1 each, contiguous, ld w1)
__global__ void wino_s_kernel(const uint64_t *__restrict__ A, int64_t lda, int64_t M, int64_t K, int64_t h1,
                              int64_t w1, uint64_t *__restrict__ S) {
    const int64_t area = h1 * w1;
    for (int64_t i = blockIdx.y; i < h1; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < w1; j += (int64_t)gridDim.x * blockDim.x) {
            const uint64_t a11 = A[i * lda + j];
            const uint64_t a12 = at(A + w1, lda, M, K - w1, i, j);
            const uint64_t a21 = at(A + h1 * lda, lda, M - h1, K, i, j);
            const uint64_t a22 = at(A + h1 * lda + w1, lda, M - h1, K - w1, i, j);
            const uint64_t s1 = a21 + a22, s2 = s1 - a11, s3 = a11 - a21, s4 = a12 - s2;
            const int64_t o = i * w1 + j;
            S[o] = s1;
            S[area + o] = s2;
            S[2 * area + o] = s3;
            S[3 * area + o] = s4;
        }
}

// T1..T4 from the blocks of B (h1 x w1 each)
__global__ void wino_t_kernel(const uint64_t *__restrict__ B, int64_t ldb, int64_t K, int64_t N, int64_t h1,
                              int64_t w1, uint64_t *__restrict__ T) {
    const int64_t area = h1 * w1;
    for (int64_t i = blockIdx.y; i < h1; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < w1; j += (int64_t)gridDim.x * blockDim.x) {
            const uint64_t b11 = B[i * ldb + j];
            const uint64_t b12 = at(B + w1, ldb, K, N - w1, i, j);
            const uint64_t b21 = at(B + h1 * ldb, ldb, K - h1, N, i, j);
            const uint64_t b22 = at(B + h1 * ldb + w1, ldb, K - h1, N - w1, i, j);
            const uint64_t t1 = b12 - b11, t2 = b22 - t1, t3 = b22 - b12, t4 = t2 - b21;
            const int64_t o = i * w1 + j;
            T[o] = t1;
            T[area + o] = t2;
            T[2 * area + o] = t3;
            T[3 * area + o] = t4;
        }
}

// C blocks from P1..P7 (m1 x n1 each, ld n1), clipped to the M x N result
__global__ void wino_combine_kernel(const uint64_t *__restrict__ P, int64_t m1, int64_t n1, uint64_t *__restrict__ C,
                                    int64_t ldc, int64_t M, int64_t N) {
    const int64_t area = m1 * n1;
    for (int64_t i = blockIdx.y; i < m1; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n1; j += (int64_t)gridDim.x * blockDim.x) {
            const int64_t o = i * n1 + j;
            const uint64_t p1 = P[o], p2 = P[area + o], p5 = P[4 * area + o], p6 = P[5 * area + o],
                           p7 = P[6 * area + o];
            const uint64_t u2 = p1 + p6, u3 = u2 + p7;
            C[i * ldc + j] = p1 + p2;
            const bool right = j + n1 < N, down = i + m1 < M;
            if (right) C[i * ldc + n1 + j] = u2 + p5 + P[2 * area + o];
            if (down) C[(m1 + i) * ldc + j] = u3 - P[3 * area + o];
            if (right && down) C[(m1 + i) * ldc + n1 + j] = u3 + p5;
        }
}

// The coefficient of Q^d of each word, reduced mod p
__global__ void digits_kernel(const uint64_t *__restrict__ W, int64_t ldw, int64_t M, int64_t N, uint32_t td,
                              uint64_t mask, uint32_t p, uint8_t *__restrict__ C, int64_t ldc) {
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
            C[i * ldc + j] = (uint8_t)(((W[i * ldw + j] >> td) & mask) % p);
}

dim3 grid2(int64_t rows, int64_t cols) {
    const int64_t gx = (cols + 255) / 256;
    return dim3((unsigned)(gx < 1024 ? (gx > 0 ? gx : 1) : 1024), (unsigned)(rows < 65535 ? (rows > 0 ? rows : 1) : 65535));
}

int64_t cdiv2(int64_t x) { return (x + 1) / 2; }

// Smallest side worth another level: below it the extra additions cost more
// than the eighth of the multiplications they save.
constexpr int64_t kCutoff = 256;

bool recurse(int levels, int64_t M, int64_t K, int64_t N) {
    return levels > 0 && M >= 2 * kCutoff && K >= 2 * kCutoff && N >= 2 * kCutoff;
}

// Words of scratch one level needs below this one (S, T, P and the levels
// under it), in 64-bit words.
int64_t scratch_words(int levels, int64_t M, int64_t K, int64_t N) {
    if (!recurse(levels, M, K, N)) return 0;
    const int64_t m1 = cdiv2(M), k1 = cdiv2(K), n1 = cdiv2(N);
    return 4 * m1 * k1 + 4 * k1 * n1 + 7 * m1 * n1 + scratch_words(levels - 1, m1, k1, n1);
}

gfp_status product(int levels, const WView &A, const WView &B, const WView &C, uint64_t *ws, cudaStream_t s) {
    const int64_t M = A.rows, K = A.cols, N = B.cols;
    if (M == 0 || N == 0) return GFP_OK;
    if (!recurse(levels, M, K, N))
        return launch_word_product_u64(A.p, A.ld, B.p, B.ld, C.p, C.ld, M, K, N, s);
    const int64_t m1 = cdiv2(M), k1 = cdiv2(K), n1 = cdiv2(N);
    const int64_t k2 = K - k1, m2 = M - m1, n2 = N - n1;
    uint64_t *S = ws, *T = S + 4 * m1 * k1, *P = T + 4 * k1 * n1, *rest = P + 7 * m1 * n1;
    wino_s_kernel<<<grid2(m1, k1), 256, 0, s>>>(A.p, A.ld, M, K, m1, k1, S);
    gfp_status st = check_launch();
    if (st != GFP_OK) return st;
    wino_t_kernel<<<grid2(k1, n1), 256, 0, s>>>(B.p, B.ld, K, N, k1, n1, T);
    st = check_launch();
    if (st != GFP_OK) return st;
    const int64_t aS = m1 * k1, aT = k1 * n1, aP = m1 * n1;
    auto Sv = [&](int i, int64_t cols) { return WView{S + (i - 1) * aS, k1, m1, cols}; };
    auto Tv = [&](int i, int64_t rows) { return WView{T + (i - 1) * aT, n1, rows, n1}; };
    auto Pv = [&](int i, int64_t rows, int64_t cols) { return WView{P + (i - 1) * aP, n1, rows, cols}; };
    const WView A11{A.p, A.ld, m1, k1}, A12{A.p + k1, A.ld, m1, k2}, A22{A.p + m1 * A.ld + k1, A.ld, m2, k2};
    const WView B11{B.p, B.ld, k1, n1}, B21{B.p + k1 * B.ld, B.ld, k2, n1}, B22{B.p + k1 * B.ld + n1, B.ld, k2, n2};
    struct Job { WView a, b, c; };
    const Job jobs[7] = {
        {A11, B11, Pv(1, m1, n1)},       {A12, B21, Pv(2, m1, n1)},
        {Sv(4, k2), B22, Pv(3, m1, n2)}, {A22, Tv(4, k2), Pv(4, m2, n1)},
        {Sv(1, k1), Tv(1, k1), Pv(5, m1, n1)}, {Sv(2, k1), Tv(2, k1), Pv(6, m1, n1)},
        {Sv(3, k1), Tv(3, k1), Pv(7, m1, n1)}};
    for (const Job &j : jobs) {
        st = product(levels - 1, j.a, j.b, j.c, rest, s);
        if (st != GFP_OK) return st;
    }
    wino_combine_kernel<<<grid2(m1, n1), 256, 0, s>>>(P, m1, n1, C.p, C.ld, M, N);
    return check_launch();
}

}  // namespace

size_t winograd_workspace_bytes(int64_t m, int64_t kc, int64_t n, int levels) {
    return (size_t)(m * n + scratch_words(levels, m, kc, n)) * sizeof(uint64_t);
}

gfp_status launch_winograd_u64(uint32_t p, int64_t m, int64_t kc, int64_t n, int d, int t, const uint64_t *CA,
                               int64_t lda, const uint64_t *CB, int64_t ldb, uint8_t *C, int64_t ldc, int levels,
                               void *ws, size_t ws_bytes, cudaStream_t s) {
    if (winograd_workspace_bytes(m, kc, n, levels) > ws_bytes || (!ws && m * n > 0)) return GFP_EWORKSPACE;
    if (m == 0 || n == 0) return GFP_OK;
    uint64_t *W = static_cast<uint64_t *>(ws);
    const WView A{const_cast<uint64_t *>(CA), lda, m, kc}, B{const_cast<uint64_t *>(CB), ldb, kc, n}, R{W, n, m, n};
    gfp_status st = product(levels, A, B, R, W + m * n, s);
    if (st != GFP_OK) return st;
    const uint64_t mask = t >= 64 ? ~0ull : ((1ull << t) - 1);
    digits_kernel<<<grid2(m, n), 256, 0, s>>>(W, n, m, n, (uint32_t)(t * d), mask, p, C, ldc);
    return check_launch();
}

}  // namespace gfp
