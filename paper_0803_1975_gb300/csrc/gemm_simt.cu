// CUDA-core forms of C = A B mod p: the classical product, the Q-adic dot
// form of Section 2 in five machine words, and the right-compressed form of
// Section 3 with the simultaneous reduction REDQ.
// Every policy declares the whole interface the kernel template may use
// (extract, kSlowPipe, ...); an instantiation that does not use a member
// makes the front end note it, which says nothing here.
#pragma nv_diag_suppress 177
#include <cstdint>
#include <type_traits>

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
    static constexpr bool kAtomic = false;
    static constexpr bool kBKMajor = false;
    static constexpr bool kSlowPipe = false;
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
// element holds 4 consecutive k-entries of a row of A or a column of B.  B
// comes transposed (row j of the stored matrix is column j of B, zero past k,
// rows 4-byte aligned), so that both operands are read as one 32-bit word per
// group of 4 residues.  ALIGNED_A: A and its leading dimension are 4-byte
// aligned, so every group of A is one aligned word (the bytes of a last
// partial group past k meet B's zeros; an aligned word holding a byte of the
// row lies in the same page, so reading it cannot fault).
template <bool ALIGNED_A>
struct Dp4aT : PlainP {
    static constexpr bool kBKMajor = true;
    // The loop runs over groups g < ceil(k/4); prm.k (the true k) guards
    // the entries of the last group.
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t g, int64_t M, int64_t K,
                             const Params &prm) {
        if constexpr (ALIGNED_A) {
            return (i < M && g < K) ? __ldg(reinterpret_cast<const uint32_t *>(A + i * lda + 4 * g)) : 0u;
        } else {
            uint32_t v = 0;
            if (i < M) {
                const int64_t k0 = 4 * g;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (k0 + q < prm.k) v |= (uint32_t)A[i * lda + k0 + q] << (8 * q);
            }
            return v;
        }
    }
    // Bt: n rows of ldb bytes (ldb a multiple of 4, zero from k on); groups
    // g < K = ceil(k/4) lie inside the row
    __device__ static SB ldB(const GB *Bt, int64_t ldb, int64_t g, int64_t j, int64_t K, int64_t N,
                             const Params &) {
        return (g < K && j < N) ? __ldg(reinterpret_cast<const uint32_t *>(Bt + j * ldb + 4 * g)) : 0u;
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
    // ReduceAndCompress output (PackRowsRev): pd + 1 residues per word in
    // base 2^pt, out_words words per row, bn_eff columns per CTA (set at launch)
    int32_t pd;
    uint32_t pt;
    int64_t out_words;
    int64_t bn_eff;
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
    static constexpr bool kAtomic = false;
    static constexpr bool kBKMajor = false;
    static constexpr bool kSlowPipe = std::is_floating_point<W>::value;   // FP64 words: DFMA-bound
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                                    const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                                    const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
};

// A 64-bit word sum kept as two 32-bit halves, the carry out of the low
// half taken at every step: the word products are built from 32-bit
// multiply-adds only (the widening 32 x 32 -> 64 multiply-add issues at about
// a third of their rate on GB300, measured), which was 6% faster for the
// 64-bit dot form at 16384^3.
struct CarrySum {
    uint32_t lo, hi;
    __device__ CarrySum() {}
    __device__ CarrySum(int) : lo(0), hi(0) {}
    // += a b mod 2^64 for 64-bit a, b: the low half of aL bL with its carry,
    // its high half, and the two cross products aL bH, aH bL (mod 2^32)
    __device__ __forceinline__ void mad64(uint64_t a, uint64_t b) {
        asm("mad.lo.cc.u32 %0, %2, %4, %0;\n\t"
            "madc.hi.u32 %1, %2, %4, %1;\n\t"
            "mad.lo.u32 %1, %2, %5, %1;\n\t"
            "mad.lo.u32 %1, %3, %4, %1;"
            : "+r"(lo), "+r"(hi)
            : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)));
    }
    // += a b mod 2^64 for a 32-bit a and a 64-bit b
    __device__ __forceinline__ void mad32x64(uint32_t a, uint64_t b) {
        asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
            "madc.hi.u32 %1, %2, %3, %1;\n\t"
            "mad.lo.u32 %1, %2, %4, %1;"
            : "+r"(lo), "+r"(hi)
            : "r"(a), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)));
    }
    __device__ __forceinline__ uint64_t value() const { return ((uint64_t)hi << 32) | lo; }
};

// 64-bit words, sums mod 2^64 (t(d+1) <= 64).
template <bool BLK>
struct DotU64 : DotBase<uint64_t, CarrySum, BLK> {
    __device__ static void mac(CarrySum &acc, uint64_t a, uint64_t b) { acc.mad64(a, b); }
    __device__ static uint64_t digit(const CarrySum &acc, const DotParams &prm) {
        return (acc.value() >> prm.td) & prm.mask;
    }
    __device__ static uint32_t extract(const CarrySum &acc, const DotParams &prm) {
        return (uint32_t)digit(acc, prm);
    }
    __device__ static uint8_t finish(const CarrySum &acc, uint32_t s, const DotParams &prm) {
        return (uint8_t)dot_reduce(digit(acc, prm), s, prm, BLK);
    }
};

// 64-bit words, the raw word sums mod 2^64 as the result (the products of a
// Strassen-Winograd recursion over the ring Z/2^64, whose digits are read
// once at the end).
struct DotU64Raw : DotBase<uint64_t, CarrySum, false> {
    using GC = uint64_t;
    __device__ static void mac(CarrySum &acc, uint64_t a, uint64_t b) { acc.mad64(a, b); }
    __device__ static uint32_t extract(const CarrySum &, const DotParams &) { return 0; }
    __device__ static uint64_t finish(const CarrySum &acc, uint32_t, const DotParams &) { return acc.value(); }
};

// ReduceAndCompress fused into the dot form (procedure (compC) of Section
// 2.2, equation (1)): the product's residues, reduced mod p as the dot
// policy's finish gives them, are written as reversed-row words
// CC[i][w] = sum_s C[i][w(pd+1)+s] 2^(pt (pd - s)) (Section 2.1; missing
// entries of the last word are zero, Section 2.3) -- the left operand of the
// next product of a chain -- instead of bytes.
template <class Inner, class OutW>
struct PackRowsRev : Inner {
    using GC = OutW;
    static constexpr bool kPackOut = true;
};

// 64-bit words, 128-bit accumulator (largest word < 2^64, t(d+1) <= 128).
template <bool BLK>
struct DotU64x128 : DotBase<uint64_t, unsigned __int128, BLK> {
    __device__ static void mac(unsigned __int128 &acc, uint64_t a, uint64_t b) { mad_u64_u128(acc, a, b); }
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

// A sum of residue x 64-bit word terms mod 2^64, kept in two parts: the
// residues times the words' low halves (64-bit, by the widening multiply-add)
// and times their high halves (mod 2^32).  The two multiply-adds of a term are
// independent (no carry between them); the sum is lo + 2^32 hi mod 2^64.
// Measured 5-9% faster than the 64-bit multiply-add for these products.
template <bool PARTIAL>
struct MixedU64T {
    using GA = uint8_t;
    using GB = uint64_t;
    using SA = uint32_t;
    using SB = uint64_t;
    // split k slices (small results) keep one 64-bit sum: measured faster there
    using Acc = std::conditional_t<PARTIAL, uint64_t, CarrySum>;
    using GC = std::conditional_t<PARTIAL, unsigned long long, uint64_t>;
    using Params = MixedParams;
    static constexpr bool kBlocked = false;
    static constexpr bool kAtomic = PARTIAL;
    static constexpr bool kBKMajor = false;
    static constexpr bool kSlowPipe = std::is_floating_point<GB>::value;
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                                    const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                                    const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
    __device__ static void mac(Acc &acc, uint32_t a, uint64_t b) {
        if constexpr (PARTIAL) acc += (uint64_t)a * b;
        else acc.mad32x64(a, b);
    }
    __device__ static uint32_t extract(const Acc &, const Params &) { return 0; }
    __device__ static GC finish(const Acc &acc, uint32_t, const Params &prm) {
        if constexpr (PARTIAL) return (GC)acc;            // a slice's raw word sum
        else return redq(acc.value(), prm);
    }
};
using MixedU64 = MixedU64T<false>;

// Binary64 words: every partial sum is an integer below Q^(d+1) < 2^53, so
// the fused multiply-adds are exact in any rounding mode.
template <bool PARTIAL>
struct MixedF64T {
    using GA = uint8_t;
    using GB = double;
    using SA = double;
    using SB = double;
    using Acc = double;
    using GC = double;
    using Params = MixedParams;
    static constexpr bool kBlocked = false;
    static constexpr bool kAtomic = PARTIAL;
    static constexpr bool kBKMajor = false;
    static constexpr bool kSlowPipe = std::is_floating_point<GB>::value;
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
        if constexpr (PARTIAL) return acc;        // a slice's raw word sum, exact
        else return (double)redq(__double2ull_rz(acc), prm);
    }
};
using MixedF64 = MixedF64T<false>;

// In-place REDQ over a matrix of raw result words (after split-k slices were
// summed into it).
template <class W>
__global__ void redq_inplace_kernel(W *__restrict__ CC, int64_t ldc, int64_t rows, int64_t cols,
                                    MixedParams prm) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        W *w = CC + i * ldc + j;
        if constexpr (std::is_floating_point<W>::value) *w = (W)redq(__double2ull_rz(*w), prm);
        else *w = (W)redq((uint64_t)*w, prm);
    }
}

// ---------------------------------------------------------------------------
// Left compression (Table 2, "Left Comp."): A packed along m into column
// words CA[u][l] = sum_i A[u(d+1)+i][l] Q^i, times uncompressed B; the result
// word sum_l CA[u][l] B[l][j] holds the d+1 entries C[u(d+1)+i][j], reduced
// by REDQ (the right-compressed product with the outer dimensions exchanged).
//
// Full compression (Section 4): A packed along m in base Q (degree dq), B
// packed along n in base Theta = Q^(dq+1) (degree dth); the word product
// sum_l CA[u][l] CB[l][v] holds all (dq+1)(dth+1) entries of a block of C as
// base-Q coefficients, each below Q (eq. lower), so the whole word is exact
// while it fits (eq. dq); REDQ reduces all of them at once.
// ---------------------------------------------------------------------------
template <class W, bool PARTIAL>
struct LeftT {
    static constexpr bool FP = std::is_floating_point<W>::value;
    using GA = W;
    using GB = uint8_t;
    using SA = W;
    using SB = std::conditional_t<FP, double, uint32_t>;
    using Acc = std::conditional_t<FP, double, CarrySum>;
    using GC = std::conditional_t<PARTIAL && !FP, unsigned long long, W>;
    using Params = MixedParams;
    static constexpr bool kBlocked = false;
    static constexpr bool kAtomic = PARTIAL;
    static constexpr bool kBKMajor = false;
    static constexpr bool kSlowPipe = FP;
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                             const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                             const Params &) {
        return (k < K && j < N) ? (SB)B[k * ldb + j] : SB(0);
    }
    __device__ static void mac(Acc &acc, SA a, SB b) {
        if constexpr (FP) acc = __fma_rn(a, b, acc);
        else acc.mad32x64(b, a);                      // residue b times word a
    }
    __device__ static uint32_t extract(const Acc &, const Params &) { return 0; }
    __device__ static GC finish(const Acc &acc, uint32_t, const Params &prm) {
        if constexpr (FP) {
            if constexpr (PARTIAL) return (GC)acc;
            else return (GC)redq(__double2ull_rz(acc), prm);
        } else {
            if constexpr (PARTIAL) return (GC)acc.value();
            else return (GC)redq(acc.value(), prm);
        }
    }
};

template <class W, bool PARTIAL>
struct FullT {
    static constexpr bool FP = std::is_floating_point<W>::value;
    using GA = W;
    using GB = W;
    using SA = W;
    using SB = W;
    using Acc = W;
    using GC = std::conditional_t<PARTIAL && !FP, unsigned long long, W>;
    using Params = MixedParams;
    static constexpr bool kBlocked = false;
    static constexpr bool kAtomic = PARTIAL;
    static constexpr bool kBKMajor = false;
    static constexpr bool kSlowPipe = FP;
    __device__ static SA ldA(const GA *A, int64_t lda, int64_t i, int64_t k, int64_t M, int64_t K,
                             const Params &) {
        return ld_guarded<GA, SA>(A, lda, i, k, M, K);
    }
    __device__ static SB ldB(const GB *B, int64_t ldb, int64_t k, int64_t j, int64_t K, int64_t N,
                             const Params &) {
        return ld_guarded<GB, SB>(B, ldb, k, j, K, N);
    }
    __device__ static void mac(Acc &acc, SA a, SB b) {
        if constexpr (FP) acc = __fma_rn(a, b, acc);   // exact: every partial sum < 2^53
        else acc += a * b;                            // exact: the word stays < 2^64
    }
    __device__ static uint32_t extract(Acc, const Params &) { return 0; }
    __device__ static GC finish(Acc acc, uint32_t, const Params &prm) {
        if constexpr (PARTIAL) return (GC)acc;
        else if constexpr (FP) return (GC)redq(__double2ull_rz(acc), prm);
        else return (GC)redq(acc, prm);
    }
};

// Tile shapes, 256 threads each: L = 128 x 128 (8 x 8 per thread), M = 128 x
// 64 (8 x 4), S = 64 x 64 (4 x 4), XS = 32 x 32 (2 x 2).  Larger register
// tiles issue fewer shared-memory loads per multiply-add; smaller tiles
// balance better over the SMs and leave registers for more resident warps.
// The choice minimises (tiles on the busiest SM) x (tile area) / (issue
// efficiency of the tile), with the efficiencies measured on GB300 (products
// of 4096 and 16384 on a side) per class of policy:
//   byte operands, 32-bit accumulator (classical): L 1, M 0.95, S 0.86, XS 0.46
//   byte groups on dp4a, B k-major:                L 0.97, M 1, S 0.66, XS 0.46
//   32-bit words, 32-bit accumulator:              L 0.9, M 1, S 0.83, XS 0.5
//   32-bit words, 64-bit accumulator:              L 0.95, M 1, S 0.97, XS 0.83
//   64-bit words:                                  L 0.85, M 0.9, S 1, XS 0.9
//   128-bit accumulator:                           M 0.88, S 0.93, XS 1
//   a slow pipe (FP64 words, kSlowPipe):           1 for every shape
// L and M hold 32 to 64 accumulators per thread: not for accumulators wider
// than 64 bits (128-bit sums), nor for 64-bit ones beside the 32-bit block
// sums of a blocked product (they would spill), nor for the residue x word
// products of the mixed and left forms (measured slower).
enum class Tile { L, M, S, XS };

template <class P>
constexpr bool large_tiles_fit() {
    constexpr bool residue_word = (sizeof(typename P::GA) == 1 && sizeof(typename P::SB) == 8) ||
                                  (sizeof(typename P::GB) == 1 && sizeof(typename P::SA) == 8);
    return sizeof(typename P::Acc) <= 8 && !(P::kBlocked && sizeof(typename P::Acc) > 4) && !residue_word;
}

struct TileEff {
    double L, M, S, XS;
};

template <class P>
constexpr TileEff tile_eff() {
    if constexpr (P::kSlowPipe) return {1.0, 1.0, 1.0, 1.0};
    else if constexpr (std::is_same<typename P::Acc, unsigned __int128>::value) return {0.5, 0.88, 0.93, 1.0};
    else if constexpr (sizeof(typename P::SA) == 8 || sizeof(typename P::SB) == 8) return {0.85, 0.9, 1.0, 0.9};
    else if constexpr (P::kBKMajor) return {0.97, 1.0, 0.66, 0.46};
    else if constexpr (sizeof(typename P::GA) == 1 && sizeof(typename P::GB) == 1) return {1.0, 0.95, 0.86, 0.46};
    else if constexpr (sizeof(typename P::Acc) == 8) return {0.95, 1.0, 0.97, 0.83};
    else return {0.9, 1.0, 0.83, 0.5};
}

template <class P>
Tile choose_tile(int64_t M, int64_t N) {
    const int64_t sms = num_sms();
    constexpr TileEff eff = tile_eff<P>();
    auto tiles = [&](int bm, int bn) { return ((M + bm - 1) / bm) * ((N + bn - 1) / bn); };
    auto cost = [&](int bm, int bn, double e) {
        return (double)((tiles(bm, bn) + sms - 1) / sms) * bm * bn / e;
    };
    // a large tile runs one CTA (8 warps) per SM; in a grid of less than two
    // waves of them the cold operand reads are not hidden (measured: at 1024
    // on a side the 64 x 64 tiles, two CTAs per SM, are 15-20% faster)
    auto min_tiles = [&](Tile t) { return t == Tile::L || t == Tile::M ? 2 * sms : 0; };
    Tile best = Tile::S;
    double c = cost(64, 64, eff.S);
    auto consider = [&](Tile t, int bm, int bn, double e) {
        const double ct = cost(bm, bn, e);
        if (ct < c && tiles(bm, bn) >= min_tiles(t)) {
            best = t;
            c = ct;
        }
    };
    if constexpr (large_tiles_fit<P>()) {
        consider(Tile::L, 128, 128, eff.L);
        consider(Tile::M, 128, 64, eff.M);
    }
    consider(Tile::XS, 32, 32, eff.XS);
    return best;
}

template <class P>
cudaError_t run_simt(const typename P::GA *A, int64_t lda, const typename P::GB *B, int64_t ldb,
                     typename P::GC *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                     const typename P::Params &prm, cudaStream_t s, int splits = 1) {
    // k-slice depth: as deep as the 48 KB of static shared memory allows, so
    // the register prefetch of the next slice covers the global-load latency
    constexpr bool narrow = sizeof(typename P::SA) <= 4 && sizeof(typename P::SB) <= 4;
    const Tile tile = choose_tile<P>(M, N);
    if constexpr (large_tiles_fit<P>()) {
        if (tile == Tile::L)
            return simt_gemm_launch<P, 128, 128, narrow ? 16 : 8, 8, 8>(A, lda, B, ldb, C, ldc, M, N, K,
                                                                       prm, s, splits);
        if (tile == Tile::M)
            return simt_gemm_launch<P, 128, 64, narrow ? 16 : 8, 8, 4>(A, lda, B, ldb, C, ldc, M, N, K,
                                                                      prm, s, splits);
    }
    switch (tile) {
        case Tile::XS:
            return simt_gemm_launch<P, 32, 32, 16, 2, 2>(A, lda, B, ldb, C, ldc, M, N, K, prm, s, splits);
        default:
            return simt_gemm_launch<P, 64, 64, narrow ? 32 : 16, 4, 4>(A, lda, B, ldb, C, ldc, M, N, K,
                                                                      prm, s, splits);
    }
}

MixedParams redq_params(uint32_t p, int t, int digits_minus_1) {
    MixedParams prm;
    prm.M = fastmod_magic(p);
    prm.p = p;
    prm.t = (uint32_t)t;
    prm.d = digits_minus_1;
    const uint32_t qmod = (uint32_t)((t >= 64 ? 0 : (1ull << t)) % p);
    prm.qc = p - qmod;
    prm.kbw = 0;
    return prm;
}

// Products whose result words are reduced by REDQ: split k when the (narrow)
// result cannot fill the GPU -- slices add exactly because every coefficient
// of the full sum is below Q -- then REDQ in place.
template <class PF, class PP, class W>
gfp_status run_redq_form(const typename PF::GA *A, int64_t lda, const typename PF::GB *B, int64_t ldb,
                         W *C, int64_t ldc, int64_t M, int64_t N, int64_t K, const MixedParams &prm,
                         cudaStream_t s) {
    const int64_t sms = num_sms();
    const int64_t tiles = ((M + 63) / 64) * ((N + 63) / 64);
    int splits = 1;
    if (tiles < 2 * sms && K >= 512) {
        splits = (int)((2 * sms + tiles - 1) / tiles);
        const int maxs = (int)(K / 256);
        if (splits > maxs) splits = maxs;
        if (splits < 1) splits = 1;
    }
    cudaError_t e;
    if (splits > 1) {
        e = cudaMemset2DAsync(C, (size_t)ldc * sizeof(W), 0, (size_t)N * sizeof(W), (size_t)M, s);
        if (e != cudaSuccess) return cuda_fail(e);
        e = simt_gemm_launch<PP, 64, 64, 16, 4, 4>(A, lda, B, ldb, reinterpret_cast<typename PP::GC *>(C), ldc,
                                                  M, N, K, prm, s, splits);
        if (e != cudaSuccess) return cuda_fail(e);
        dim3 grid((unsigned)((N + 255) / 256), (unsigned)(M < 65535 ? M : 65535));
        redq_inplace_kernel<W><<<grid, 256, 0, s>>>(C, ldc, M, N, prm);
        return check_launch();
    }
    e = run_simt<PF>(A, lda, B, ldb, reinterpret_cast<typename PF::GC *>(C), ldc, M, N, K, prm, s);
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
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
    prm.pd = 0;
    prm.pt = 0;
    prm.out_words = 0;
    prm.bn_eff = 0;
    return prm;
}

template <template <bool> class P>
cudaError_t run_dot(const void *CA, int64_t lda, const void *CB, int64_t ldb, uint8_t *C,
                    int64_t ldc, int64_t m, int64_t n, int64_t kc, const DotParams &prm,
                    bool blocked, cudaStream_t s) {
    using W = typename P<false>::GA;
    const W *a = static_cast<const W *>(CA);
    const W *b = static_cast<const W *>(CB);
    if (blocked) return run_simt<P<true>>(a, lda, b, ldb, C, ldc, m, n, kc, prm, s);
    return run_simt<P<false>>(a, lda, b, ldb, C, ldc, m, n, kc, prm, s);
}

}  // namespace

size_t dp4a_workspace_bytes(int64_t k, int64_t n) {
    return 256 + (size_t)((n + 63) / 64 * 64) * (size_t)((k + 63) / 64 * 64);
}

gfp_status launch_plain(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A, int64_t lda,
                        const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc, bool dp4a, void *ws,
                        size_t ws_bytes, cudaStream_t s) {
    PlainP::Params prm{fastmod_magic(p), p, 0, k};
    cudaError_t e;
    if (dp4a) {
        // B transposed into the workspace (k-major rows of kp bytes, zero past k)
        const int64_t kp = (k + 63) / 64 * 64, np = (n + 63) / 64 * 64;
        if (!ws || ws_bytes < dp4a_workspace_bytes(k, n)) return GFP_EWORKSPACE;
        uint8_t *Bt = static_cast<uint8_t *>(ws) + 256;
        const gfp_status st = launch_transpose_bytes(B, ldb, k, n, Bt, kp, np, s);
        if (st != GFP_OK) return st;
        if (((reinterpret_cast<uintptr_t>(A) | (uintptr_t)lda) & 3) == 0)
            e = run_simt<Dp4aT<true>>(A, lda, Bt, kp, C, ldc, m, n, (k + 3) / 4, prm, s);
        else
            e = run_simt<Dp4aT<false>>(A, lda, Bt, kp, C, ldc, m, n, (k + 3) / 4, prm, s);
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

// The dot form with ReduceAndCompress in its epilogue: 64-bit or 32-bit
// words in (blocked or not), words of the same width out.
gfp_status launch_dot_compc(uint32_t p, int64_t m, int64_t kc, int64_t n, int d, int t, gfp_word word,
                            const void *CA, int64_t lda, const void *CB, int64_t ldb, int64_t kbw, int d_out,
                            int t_out, void *CC, int64_t ldcc, cudaStream_t s) {
    const bool blocked = kbw > 0 && kbw < kc;
    DotParams prm = dot_params(p, d, t, blocked ? kbw : 0);
    prm.pd = d_out;
    prm.pt = (uint32_t)t_out;
    prm.out_words = (n + d_out) / (d_out + 1);
    prm.bn_eff = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (word == GFP_WORD_U64) {
        auto a = static_cast<const uint64_t *>(CA);
        auto b = static_cast<const uint64_t *>(CB);
        auto c = static_cast<uint64_t *>(CC);
        e = blocked ? run_simt<PackRowsRev<DotU64<true>, uint64_t>>(a, lda, b, ldb, c, ldcc, m, n, kc, prm, s)
                    : run_simt<PackRowsRev<DotU64<false>, uint64_t>>(a, lda, b, ldb, c, ldcc, m, n, kc, prm, s);
    } else if (word == GFP_WORD_U32) {
        auto a = static_cast<const uint32_t *>(CA);
        auto b = static_cast<const uint32_t *>(CB);
        auto c = static_cast<uint32_t *>(CC);
        e = blocked ? run_simt<PackRowsRev<DotU32<true>, uint32_t>>(a, lda, b, ldb, c, ldcc, m, n, kc, prm, s)
                    : run_simt<PackRowsRev<DotU32<false>, uint32_t>>(a, lda, b, ldb, c, ldcc, m, n, kc, prm, s);
    } else {
        return GFP_EUNSUPPORTED;
    }
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

gfp_status launch_word_product_u64(const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb,
                                   uint64_t *C, int64_t ldc, int64_t m, int64_t kc, int64_t n,
                                   cudaStream_t s) {
    const DotParams prm = dot_params(2, 0, 1, 0);
    const cudaError_t e = run_simt<DotU64Raw>(A, lda, B, ldb, C, ldc, m, n, kc, prm, s);
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
    // The result m x ceil(n/(d+1)) is narrow: when its tiles cannot fill the
    // GPU, split k.  Each coefficient of a slice's word sum is below Q (eq.
    // (lower) holds for the whole k), so the slices' words add without carries:
    // zero CC, add the slices atomically, then REDQ in place.
    const int64_t sms = num_sms();
    const int64_t tiles = ((m + 63) / 64) * ((nc + 63) / 64);
    int splits = 1;
    if (tiles < 2 * sms && k >= 512) {
        splits = (int)((2 * sms + tiles - 1) / tiles);
        const int maxs = (int)(k / 256);
        if (splits > maxs) splits = maxs;
        if (splits < 1) splits = 1;
    }
    cudaError_t e = cudaErrorInvalidValue;
    const size_t wb = 8;
    if (splits > 1) {
        e = cudaMemset2DAsync(CC, (size_t)ldc * wb, 0, (size_t)nc * wb, (size_t)m, s);
        if (e != cudaSuccess) return cuda_fail(e);
        if (word == GFP_WORD_U64)
            e = simt_gemm_launch<MixedU64T<true>, 64, 64, 16, 4, 4>(
                A, lda, static_cast<const uint64_t *>(CB), ldb, static_cast<unsigned long long *>(CC),
                ldc, m, nc, k, prm, s, splits);
        else if (word == GFP_WORD_F64)
            e = simt_gemm_launch<MixedF64T<true>, 64, 64, 16, 4, 4>(
                A, lda, static_cast<const double *>(CB), ldb, static_cast<double *>(CC), ldc, m, nc, k,
                prm, s, splits);
        if (e != cudaSuccess) return cuda_fail(e);
        dim3 grid((unsigned)((nc + 255) / 256), (unsigned)(m < 65535 ? m : 65535));
        if (word == GFP_WORD_U64)
            redq_inplace_kernel<uint64_t><<<grid, 256, 0, s>>>(static_cast<uint64_t *>(CC), ldc, m, nc, prm);
        else
            redq_inplace_kernel<double><<<grid, 256, 0, s>>>(static_cast<double *>(CC), ldc, m, nc, prm);
        return check_launch();
    }
    if (word == GFP_WORD_U64)
        e = run_simt<MixedU64>(A, lda, static_cast<const uint64_t *>(CB), ldb,
                               static_cast<uint64_t *>(CC), ldc, m, nc, k, prm, s);
    else if (word == GFP_WORD_F64)
        e = run_simt<MixedF64>(A, lda, static_cast<const double *>(CB), ldb,
                               static_cast<double *>(CC), ldc, m, nc, k, prm, s);
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

}  // namespace gfp

namespace gfp {

gfp_status launch_left(uint32_t p, int64_t mc, int64_t k, int64_t n, int d, int t, gfp_word word,
                       const void *CA, int64_t lda, const uint8_t *B, int64_t ldb, void *CC,
                       int64_t ldc, cudaStream_t s) {
    const MixedParams prm = redq_params(p, t, d);
    if (word == GFP_WORD_U64)
        return run_redq_form<LeftT<uint64_t, false>, LeftT<uint64_t, true>, uint64_t>(
            static_cast<const uint64_t *>(CA), lda, B, ldb, static_cast<uint64_t *>(CC), ldc, mc, n, k, prm, s);
    if (word == GFP_WORD_F64)
        return run_redq_form<LeftT<double, false>, LeftT<double, true>, double>(
            static_cast<const double *>(CA), lda, B, ldb, static_cast<double *>(CC), ldc, mc, n, k, prm, s);
    return GFP_EUNSUPPORTED;
}

gfp_status launch_full(uint32_t p, int64_t mc, int64_t k, int64_t nc, int dq, int dth, int t,
                       gfp_word word, const void *CA, int64_t lda, const void *CB, int64_t ldb,
                       void *CC, int64_t ldc, cudaStream_t s) {
    const MixedParams prm = redq_params(p, t, (dq + 1) * (dth + 1) - 1);
    if (word == GFP_WORD_U64)
        return run_redq_form<FullT<uint64_t, false>, FullT<uint64_t, true>, uint64_t>(
            static_cast<const uint64_t *>(CA), lda, static_cast<const uint64_t *>(CB), ldb,
            static_cast<uint64_t *>(CC), ldc, mc, nc, k, prm, s);
    if (word == GFP_WORD_F64)
        return run_redq_form<FullT<double, false>, FullT<double, true>, double>(
            static_cast<const double *>(CA), lda, static_cast<const double *>(CB), ldb,
            static_cast<double *>(CC), ldc, mc, nc, k, prm, s);
    return GFP_EUNSUPPORTED;
}

}  // namespace gfp
