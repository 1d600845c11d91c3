// CUDA-core forms of C = A B mod p: the classical product, the Q-adic dot
// form of Section 2 in five machine words, and the right-compressed form of
// Section 3 with the simultaneous reduction REDQ.
#include <cstdint>

#include "gfp_internal.h"
#include "simt_gemm.cuh"

namespace gfp {
namespace {

// ---------------------------------------------------------------------------
// Classical product: one 32-bit multiply-add per term, one reduction per
// entry (exact while k (p-1)^2 < 2^32).
// ---------------------------------------------------------------------------
struct PlainP {
    using GA = uint8_t;
    using GB = uint8_t;
    using SA = uint32_t;
    using SB = uint32_t;
    using Acc = uint32_t;
    using GC = uint8_t;
    static constexpr bool kBlocked = false;
    struct Params {
        uint64_t M;
        uint32_t p;
        int64_t kbw;
        int64_t k;
    };
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                                    const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                                    const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
    __device__ static void mac(Acc &acc, SA a, SB b) { acc += a * b; }
    __device__ static uint32_t extract(Acc, const Params &) { return 0; }
    __device__ static GC finish(Acc acc, uint32_t, const Params &prm) {
        return (GC)fastmod_u32(acc, prm.M, prm.p);
    }
};

// Classical product on the byte dot-product instruction: each shared-memory
// element holds 4 consecutive k-entries of a row of A or a column of B.
struct Dp4aP : PlainP {
    // The loop runs over groups g < ceil(k/4); prm.k (the true k) guards
    // the entries of the last group.
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t g, int64_t M, int64_t,
                             const Params &prm) {
        uint32_t v = 0;
        if (i < M) {
            const int64_t k0 = 4 * g;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (k0 + q < prm.k) v |= (uint32_t)A[i * lda + k0 + q] << (8 * q);
        }
        return v;
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t g, int64_t j, int64_t, int64_t N,
                             const Params &prm) {
        uint32_t v = 0;
        if (j < N) {
            const int64_t k0 = 4 * g;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (k0 + q < prm.k) v |= (uint32_t)B[(k0 + q) * ldb + j] << (8 * q);
        }
        return v;
    }
    __device__ static void mac(Acc &acc, SA a, SB b) { acc = __dp4a(a, b, acc); }
};

// ---------------------------------------------------------------------------
// Q-adic dot form (Section 2): words CA[i][w] (reversed rows) and CB[w][j]
// (columns); the coefficient of Q^d of sum_w CA[i][w] CB[w][j] is the dot
// product (Section 2.2), exact under eq. (lower); it is read by a shift and a
// mask (Q = 2^t) and reduced mod p once (Section 2.5).
// ---------------------------------------------------------------------------
struct DotParams {
    uint64_t M;       // fastmod magic of p
    uint32_t p;
    uint32_t td;      // t * d: position of the coefficient of Q^d
    uint64_t mask;    // Q - 1
    double inv;       // 2^(-t d), exact
    int64_t kbw;      // words per k-block (blocked variants)
};

__device__ __forceinline__ uint32_t dot_reduce(uint64_t digit, uint32_t sum, const DotParams &prm,
                                               bool blocked) {
    if (blocked) return fastmod_u32(sum + (uint32_t)digit, prm.M, prm.p);
    if (digit <= 0xffffffffull) return fastmod_u32((uint32_t)digit, prm.M, prm.p);
    return (uint32_t)(digit % prm.p);
}

template <class W, class A_, bool BLK>
struct DotBase {
    using GA = W;
    using GB = W;
    using SA = W;
    using SB = W;
    using Acc = A_;
    using GC = uint8_t;
    using Params = DotParams;
    static constexpr bool kBlocked = BLK;
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                                    const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                                    const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
};

// 64-bit words, sums mod 2^64 (t(d+1) <= 64).
template <bool BLK>
struct DotU64 : DotBase<uint64_t, uint64_t, BLK> {
    __device__ static void mac(uint64_t &acc, uint64_t a, uint64_t b) { acc += a * b; }
    __device__ static uint64_t digit(uint64_t acc, const DotParams &prm) {
        return (acc >> prm.td) & prm.mask;
    }
    __device__ static uint32_t extract(uint64_t acc, const DotParams &prm) {
        return (uint32_t)digit(acc, prm);
    }
    __device__ static uint8_t finish(uint64_t acc, uint32_t s, const DotParams &prm) {
        return (uint8_t)dot_reduce(digit(acc, prm), s, prm, BLK);
    }
};

// 64-bit words, 128-bit accumulator (largest word < 2^64, t(d+1) <= 128).
template <bool BLK>
struct DotU64x128 : DotBase<uint64_t, unsigned __int128, BLK> {
    __device__ static void mac(unsigned __int128 &acc, uint64_t a, uint64_t b) {
        acc += (unsigned __int128)a * b;
    }
    __device__ static uint64_t digit(unsigned __int128 acc, const DotParams &prm) {
        return (uint64_t)(acc >> prm.td) & prm.mask;
    }
    __device__ static uint32_t extract(unsigned __int128 acc, const DotParams &prm) {
        return (uint32_t)digit(acc, prm);
    }
    __device__ static uint8_t finish(unsigned __int128 acc, uint32_t s, const DotParams &prm) {
        return (uint8_t)dot_reduce(digit(acc, prm), s, prm, BLK);
    }
};

// 32-bit words (largest word < 2^32) with a 64-bit accumulator.
template <bool BLK>
struct DotU32W : DotBase<uint32_t, uint64_t, BLK> {
    __device__ static void mac(uint64_t &acc, uint32_t a, uint32_t b) {
        acc += (uint64_t)a * (uint64_t)b;
    }
    __device__ static uint64_t digit(uint64_t acc, const DotParams &prm) {
        return (acc >> prm.td) & prm.mask;
    }
    __device__ static uint32_t extract(uint64_t acc, const DotParams &prm) {
        return (uint32_t)digit(acc, prm);
    }
    __device__ static uint8_t finish(uint64_t acc, uint32_t s, const DotParams &prm) {
        return (uint8_t)dot_reduce(digit(acc, prm), s, prm, BLK);
    }
};

// 32-bit words and accumulator (t(d+1) <= 32).
template <bool BLK>
struct DotU32 : DotBase<uint32_t, uint32_t, BLK> {
    __device__ static void mac(uint32_t &acc, uint32_t a, uint32_t b) { acc += a * b; }
    __device__ static uint32_t extract(uint32_t acc, const DotParams &prm) {
        return (acc >> prm.td) & (uint32_t)prm.mask;
    }
    __device__ static uint8_t finish(uint32_t acc, uint32_t s, const DotParams &prm) {
        return (uint8_t)dot_reduce(extract(acc, prm), s, prm, BLK);
    }
};

// Binary64 words holding exact integers, Q^(d+1) < 2^53 (eq. (upper)).  The
// accumulation rounds toward zero: the exact sum is c_H Q^d + c_L with
// 0 <= c_L < Q^d, and truncating to 53 bits never removes bits at or above
// Q^d while c_H < 2^53, nor makes the kept part of c_L reach Q^d.  The
// coefficient is read as in Section 2.5: multiply by the (exact) inverse of
// Q^d, truncate, keep the part below Q.
template <bool BLK>
struct DotF64 : DotBase<double, double, BLK> {
    __device__ static void mac(double &acc, double a, double b) { acc = __fma_rz(a, b, acc); }
    __device__ static uint64_t digit(double acc, const DotParams &prm) {
        return __double2ull_rz(acc * prm.inv) & prm.mask;
    }
    __device__ static uint32_t extract(double acc, const DotParams &prm) {
        return (uint32_t)digit(acc, prm);
    }
    __device__ static uint8_t finish(double acc, uint32_t s, const DotParams &prm) {
        return (uint8_t)dot_reduce(digit(acc, prm), s, prm, BLK);
    }
};

// ---------------------------------------------------------------------------
// Right-compressed form (Section 3): uncompressed A (bytes) times CB[l][v] =
// sum_j B[l][v(d+1)+j] Q^j.  The result word sum_l A[i][l] CB[l][v] holds the
// d+1 dot products as its coefficients (each < Q by eq. (lower)); REDQ
// reduces all of them mod p at once.
//
// REDQ (the paper cites it without giving it; derived here): for a word
// r = sum_j c_j Q^j with 0 <= c_j < Q, let q = floor(r / p), u_i = floor(r /
// Q^i) and v_i = floor(q / Q^i) = floor(u_i / p).  Then rho_i = u_i - p v_i =
// u_i mod p, and since c_i = u_i - Q u_{i+1},
//     c_i mod p = (rho_i + (p - Q mod p) rho_{i+1}) mod p,   rho_{d+1} = 0,
// one division by p per word and small reductions (< p^2) per coefficient.
// ---------------------------------------------------------------------------
struct MixedParams {
    uint64_t M;
    uint32_t p;
    uint32_t t;
    int d;
    uint32_t qc;      // p - (Q mod p)
    int64_t kbw;
};

__device__ __forceinline__ uint64_t redq(uint64_t r, const MixedParams &prm) {
    const uint64_t q = r / prm.p;
    uint32_t rho_next = 0;
    uint64_t out = 0;
    for (int i = prm.d; i >= 0; --i) {
        const uint32_t sh = prm.t * (uint32_t)i;
        const uint32_t u = (uint32_t)(r >> sh);
        const uint32_t v = (uint32_t)(q >> sh);
        const uint32_t rho = u - prm.p * v;    // u_i mod p, exact in 32 bits
        const uint32_t c = fastmod_u32(rho + prm.qc * rho_next, prm.M, prm.p);
        out |= (uint64_t)c << sh;
        rho_next = rho;
    }
    return out;
}

struct MixedU64 {
    using GA = uint8_t;
    using GB = uint64_t;
    using SA = uint32_t;
    using SB = uint64_t;
    using Acc = uint64_t;
    using GC = uint64_t;
    using Params = MixedParams;
    static constexpr bool kBlocked = false;
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                                    const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                                    const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
    __device__ static void mac(uint64_t &acc, uint32_t a, uint64_t b) { acc += (uint64_t)a * b; }
    __device__ static uint32_t extract(uint64_t, const Params &) { return 0; }
    __device__ static uint64_t finish(uint64_t acc, uint32_t, const Params &prm) {
        return redq(acc, prm);
    }
};

// Binary64 words: every partial sum is an integer below Q^(d+1) < 2^53, so
// the fused multiply-adds are exact in any rounding mode.
struct MixedF64 {
    using GA = uint8_t;
    using GB = double;
    using SA = double;
    using SB = double;
    using Acc = double;
    using GC = double;
    using Params = MixedParams;
    static constexpr bool kBlocked = false;
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                                    const Params &) {
        return (i < M && k < K) ? (double)A[i * lda + k] : 0.0;
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                                    const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
    __device__ static void mac(double &acc, double a, double b) { acc = __fma_rn(a, b, acc); }
    __device__ static uint32_t extract(double, const Params &) { return 0; }
    __device__ static double finish(double acc, uint32_t, const Params &prm) {
        return (double)redq(__double2ull_rz(acc), prm);
    }
};

// Tile shapes: L = 128 x 128 (8 x 8 per thread) for grids that fill the GPU,
// S = 64 x 64 (4 x 4 per thread) for smaller results.  256 threads either way.
template <class P>
cudaError_t run_simt(const typename P::GA *A, int64_t lda, const typename P::GB *B, int64_t ldb,
                     typename P::GC *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                     const typename P::Params &prm, cudaStream_t s, bool allow_large = true) {
    const int64_t tiles_l = ((M + 127) / 128) * ((N + 127) / 128);
    if (allow_large && tiles_l >= num_sms())
        return simt_gemm_launch<P, 128, 128, 8, 8, 8>(A, lda, B, ldb, C, ldc, M, N, K, prm, s);
    return simt_gemm_launch<P, 64, 64, 8, 4, 4>(A, lda, B, ldb, C, ldc, M, N, K, prm, s);
}

DotParams dot_params(uint32_t p, int d, int t, int64_t kbw) {
    DotParams prm;
    prm.M = fastmod_magic(p);
    prm.p = p;
    prm.td = (uint32_t)(t * d);
    prm.mask = (t >= 64) ? ~0ull : ((1ull << t) - 1);
    prm.inv = 1.0;
    for (int i = 0; i < t * d; ++i) prm.inv *= 0.5;
    prm.kbw = kbw;
    return prm;
}

template <template <bool> class P>
cudaError_t run_dot(const void *CA, int64_t lda, const void *CB, int64_t ldb, uint8_t *C,
                    int64_t ldc, int64_t m, int64_t n, int64_t kc, const DotParams &prm,
                    bool blocked, cudaStream_t s) {
    using W = typename P<false>::GA;
    const W *a = static_cast<const W *>(CA);
    const W *b = static_cast<const W *>(CB);
    if (blocked) {
        // 64-bit accumulators plus the 32-bit block sums need the small tile
        constexpr bool wide = sizeof(typename P<true>::Acc) > 4;
        return run_simt<P<true>>(a, lda, b, ldb, C, ldc, m, n, kc, prm, s, !wide);
    }
    // 128-bit accumulators do not fit the 8 x 8 register tile
    constexpr bool huge = sizeof(typename P<false>::Acc) > 8;
    return run_simt<P<false>>(a, lda, b, ldb, C, ldc, m, n, kc, prm, s, !huge);
}

}  // namespace

gfp_status launch_plain(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A, int64_t lda,
                        const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc, bool dp4a,
                        cudaStream_t s) {
    PlainP::Params prm{fastmod_magic(p), p, 0, k};
    cudaError_t e;
    if (dp4a) {
        e = run_simt<Dp4aP>(A, lda, B, ldb, C, ldc, m, n, (k + 3) / 4, prm, s);
    } else {
        e = run_simt<PlainP>(A, lda, B, ldb, C, ldc, m, n, k, prm, s);
    }
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

gfp_status launch_dot(uint32_t p, int64_t m, int64_t kc, int64_t n, int d, int t, gfp_word word,
                      const void *CA, int64_t lda, const void *CB, int64_t ldb, uint8_t *C,
                      int64_t ldc, int64_t kbw, cudaStream_t s) {
    const bool blocked = kbw > 0 && kbw < kc;
    const DotParams prm = dot_params(p, d, t, blocked ? kbw : 0);
    cudaError_t e = cudaErrorInvalidValue;
    switch (word) {
        case GFP_WORD_U64: e = run_dot<DotU64>(CA, lda, CB, ldb, C, ldc, m, n, kc, prm, blocked, s); break;
        case GFP_WORD_U64X128:
            e = run_dot<DotU64x128>(CA, lda, CB, ldb, C, ldc, m, n, kc, prm, blocked, s);
            break;
        case GFP_WORD_U32W: e = run_dot<DotU32W>(CA, lda, CB, ldb, C, ldc, m, n, kc, prm, blocked, s); break;
        case GFP_WORD_U32: e = run_dot<DotU32>(CA, lda, CB, ldb, C, ldc, m, n, kc, prm, blocked, s); break;
        case GFP_WORD_F64: e = run_dot<DotF64>(CA, lda, CB, ldb, C, ldc, m, n, kc, prm, blocked, s); break;
    }
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

gfp_status launch_mixed(uint32_t p, int64_t m, int64_t k, int64_t nc, int d, int t, gfp_word word,
                        const uint8_t *A, int64_t lda, const void *CB, int64_t ldb, void *CC,
                        int64_t ldc, cudaStream_t s) {
    MixedParams prm;
    prm.M = fastmod_magic(p);
    prm.p = p;
    prm.t = (uint32_t)t;
    prm.d = d;
    const uint32_t qmod = (uint32_t)((t >= 64 ? 0 : (1ull << t)) % p);
    prm.qc = p - qmod;
    prm.kbw = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (word == GFP_WORD_U64)
        e = run_simt<MixedU64>(A, lda, static_cast<const uint64_t *>(CB), ldb,
                               static_cast<uint64_t *>(CC), ldc, m, nc, k, prm, s);
    else if (word == GFP_WORD_F64)
        e = run_simt<MixedF64>(A, lda, static_cast<const double *>(CB), ldb,
                               static_cast<double *>(CC), ldc, m, nc, k, prm, s);
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

}  // namespace gfp
