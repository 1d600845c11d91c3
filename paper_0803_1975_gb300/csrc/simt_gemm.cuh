// Register-tiled matrix product on the CUDA cores, shared by the plain, the
// Q-adic dot (Section 2) and the right-compressed (Section 3) forms.
//
// A CTA computes a BM x BN tile of the result from BK-deep slices of the
// operands staged in shared memory (double buffered: the next slice is read
// from global memory into registers while the current one is multiplied).
// Thread (tx, ty) owns TM rows and TN columns of the tile, in two halves
// (rows ty*TM/2 + i and BM/2 + ty*TM/2 + i, likewise for columns) so that
// its shared-memory reads are 16-byte vectors and a warp reads few banks.
//
// The arithmetic is a policy P:
//   GA, GB   operand element types in global memory
//   SA, SB   their types in shared memory and registers; P::ldA(A, lda, i, k,
//            M, K, prm) and P::ldB(B, ldb, k, j, K, N, prm) fetch one element
//            (zero outside the matrix) and convert it
//   Acc      accumulator, P::mac(acc, a, b) adds one term
//   GC       result element type, P::finish(acc, sum, prm) produces it
//   kBlocked when true, P::extract(acc) is called every prm.kbw steps of k
//            and its results are summed in a 32-bit register per entry; the
//            accumulator restarts from zero after each block.
//   kAtomic  when true the result is added atomically to C (split-k slices
//            of a linear accumulator; the caller zeroes C and finishes it).
//   kBKMajor when true B is stored k-contiguous (element (k, j) of the
//            product's B lies in row j of the stored matrix): its tile is
//            read along k like A's, consecutive threads on consecutive k.
//   kPackOut (optional, false when absent) when true the result residues
//            P::finish gives are packed, in the epilogue, into reversed-row
//            words of prm.pd + 1 residues in base 2^prm.pt (C then holds
//            words of type P::GC, prm.out_words per row): a CTA covers
//            prm.bn_eff = whole words' worth of columns, its residues pass
//            through shared memory and each word is built by Horner.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace gfp {

template <class P, class = void>
struct pack_out_of : std::false_type {};
template <class P>
struct pack_out_of<P, std::void_t<decltype(P::kPackOut)>> : std::integral_constant<bool, P::kPackOut> {};

// columns of the result one CTA covers
template <class P, int BN>
__host__ __device__ __forceinline__ int64_t tile_cols(const typename P::Params &prm) {
    if constexpr (pack_out_of<P>::value) return prm.bn_eff;
    else return BN;
}

// Read n contiguous elements of shared memory into registers with the widest
// vector loads the run allows (the run starts on a 16-byte boundary when its
// byte length is a multiple of 16, see the padding of the tiles).
template <class T, int n>
__device__ __forceinline__ void lds_run(T *r, const T *p) {
    constexpr int bytes = n * (int)sizeof(T);
    if constexpr (bytes % 16 == 0) {
#pragma unroll
        for (int v = 0; v < bytes / 16; ++v) {
            uint4 x = reinterpret_cast<const uint4 *>(p)[v];
            uint32_t w[4] = {x.x, x.y, x.z, x.w};
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) r[v * 4 + q] = __builtin_bit_cast(T, w[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    r[v * 2 + q] = __builtin_bit_cast(T, (uint64_t)w[2 * q] | ((uint64_t)w[2 * q + 1] << 32));
            }
        }
    } else if constexpr (bytes % 8 == 0 && sizeof(T) <= 8) {
#pragma unroll
        for (int v = 0; v < bytes / 8; ++v) {
            uint2 x = reinterpret_cast<const uint2 *>(p)[v];
            if constexpr (sizeof(T) == 4) {
                r[v * 2] = __builtin_bit_cast(T, x.x);
                r[v * 2 + 1] = __builtin_bit_cast(T, x.y);
            } else {
                r[v] = __builtin_bit_cast(T, (uint64_t)x.x | ((uint64_t)x.y << 32));
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < n; ++q) r[q] = p[q];
    }
}

template <class P, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
simt_gemm_kernel(const typename P::GA *__restrict__ A, int64_t lda,
                 const typename P::GB *__restrict__ B, int64_t ldb,
                 typename P::GC *__restrict__ C, int64_t ldc,
                 int64_t M, int64_t N, int64_t K, typename P::Params prm, int64_t kchunk) {
    constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
    constexpr int HM = TM / 2, HN = TN / 2;
    static_assert(TM % 2 == 0 && TN % 2 == 0, "rows and columns come in two halves");
    static_assert((BM * BK) % NT == 0 && (BK * BN) % NT == 0, "tile loads");
    using SA = typename P::SA;
    using SB = typename P::SB;
    using Acc = typename P::Acc;
    // pads keep rows 16-byte aligned and spread the transposing stores over banks
    constexpr int PADA = 16 / sizeof(SA), PADB = P::kBKMajor ? 16 / sizeof(SB) : 0;
    __shared__ __align__(16) SA As[2][BK][BM + PADA];
    __shared__ __align__(16) SB Bs[2][BK][BN + PADB];

    const int tid = threadIdx.x;
    const int tx = tid % NTX, ty = tid / NTX;
    // Tile order: with 64-bit word operands, groups of 16 tile-rows walk the
    // tile-columns together, so that the B panels a group shares are read
    // from DRAM once per group instead of once per tile-row (at 16384^3 the
    // row-major order read 185 GB per launch for 1.4 GB of operands, the
    // grouped one 23.5 GB; the right-compressed form ran 9% faster).  Byte
    // and 32-bit operands keep the row-major order, measured faster for them
    // (the classical product at 16384^3: 274 against 312 ms).
    int64_t by = blockIdx.y, bx = blockIdx.x;
    if constexpr (sizeof(SA) == 8 || sizeof(SB) == 8) {
        constexpr int64_t G = 16;
        const int64_t gxn = gridDim.x, gyn = gridDim.y;
        const int64_t lin = by * gxn + bx;
        const int64_t first = lin / (G * gxn) * G;
        const int64_t gsize = gyn - first < G ? gyn - first : G;
        const int64_t r = lin % (G * gxn);
        by = first + r % gsize;
        bx = r / gsize;
    }
    const int64_t m0 = by * BM;
    const int64_t n0 = bx * tile_cols<P, BN>(prm);
    // split k: slice z of the grid covers [kz0, kz1); the slices' raw sums
    // are added atomically (policies with kAtomic only)
    const int64_t kz0 = kchunk > 0 ? (int64_t)blockIdx.z * kchunk : 0;
    const int64_t kz1 = kchunk > 0 ? (kz0 + kchunk < K ? kz0 + kchunk : K) : K;

    constexpr int LA = BM * BK / NT, LB = BK * BN / NT;
    SA ra[LA];
    SB rb[LB];

    auto load = [&](int64_t k0) {
#pragma unroll
        for (int e = 0; e < LA; ++e) {
            const int idx = tid + e * NT;
            const int r = idx / BK, c = idx % BK;
            const int64_t gi = m0 + r, gk = k0 + c;
            ra[e] = P::ldA(A, lda, gi, gk, M, kz1, prm);
        }
#pragma unroll
        for (int e = 0; e < LB; ++e) {
            const int idx = tid + e * NT;
            const int r = P::kBKMajor ? idx % BK : idx / BN, c = P::kBKMajor ? idx / BK : idx % BN;
            const int64_t gk = k0 + r, gj = n0 + c;
            rb[e] = P::ldB(B, ldb, gk, gj, kz1, N, prm);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int e = 0; e < LA; ++e) {
            const int idx = tid + e * NT;
            As[buf][idx % BK][idx / BK] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < LB; ++e) {
            const int idx = tid + e * NT;
            if constexpr (P::kBKMajor) Bs[buf][idx % BK][idx / BK] = rb[e];
            else Bs[buf][idx / BN][idx % BN] = rb[e];
        }
    };

    Acc acc[TM][TN];
    uint32_t sum[P::kBlocked ? TM : 1][P::kBlocked ? TN : 1];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);
    if constexpr (P::kBlocked) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) sum[i][j] = 0;
    }
    int64_t countdown = P::kBlocked ? prm.kbw : 0;

    load(kz0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kz0; k0 < kz1; k0 += BK) {
        const bool more = k0 + BK < kz1;
        if (more) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            SA a[TM];
            SB b[TN];
            lds_run<SA, HM>(a, &As[buf][kk][ty * HM]);
            lds_run<SA, HM>(a + HM, &As[buf][kk][BM / 2 + ty * HM]);
            lds_run<SB, HN>(b, &Bs[buf][kk][tx * HN]);
            lds_run<SB, HN>(b + HN, &Bs[buf][kk][BN / 2 + tx * HN]);
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) P::mac(acc[i][j], a[i], b[j]);
            if constexpr (P::kBlocked) {
                if (--countdown == 0) {
                    countdown = prm.kbw;
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) {
                            sum[i][j] += P::extract(acc[i][j], prm);
                            acc[i][j] = Acc(0);
                        }
                }
            }
        }
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }

    if constexpr (pack_out_of<P>::value) {
        // ReduceAndCompress: the residues of the tile through shared memory
        // (the operand tiles are free now), then whole reversed-row words
        static_assert(sizeof(As) >= BM * BN, "the residue tile fits the A buffers");
        __syncthreads();
        uint8_t *res = reinterpret_cast<uint8_t *>(&As[0][0][0]);
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int r = i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM);
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int c = j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN);
                uint32_t sm = 0;
                if constexpr (P::kBlocked) sm = sum[i][j];
                res[r * BN + c] = (uint8_t)P::finish(acc[i][j], sm, prm);
            }
        }
        __syncthreads();
        const int dp1 = prm.pd + 1;
        const int W = (int)(prm.bn_eff / dp1);
        const int64_t w0 = n0 / dp1;
        for (int e = tid; e < BM * W; e += NT) {
            const int r = e / W, w = e % W;
            const int64_t gi = m0 + r, gw = w0 + w;
            if (gi >= M || gw >= prm.out_words) continue;
            uint64_t word = 0;
            for (int q = 0; q < dp1; ++q) {
                const int c = w * dp1 + q;
                const uint64_t v = n0 + c < N ? res[r * BN + c] : 0u;   // missing entries count as zero
                word = q ? (word << prm.pt) | v : v;
            }
            C[gi * ldc + gw] = (typename P::GC)word;
        }
    } else {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gi = m0 + (i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM));
            if (gi >= M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t gj = n0 + (j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN));
                if (gj < N) {
                    uint32_t s = 0;
                    if constexpr (P::kBlocked) s = sum[i][j];
                    if constexpr (P::kAtomic) atomicAdd(&C[gi * ldc + gj], P::finish(acc[i][j], s, prm));
                    else C[gi * ldc + gj] = P::finish(acc[i][j], s, prm);
                }
            }
        }
    }
}

template <class P, int BM, int BN, int BK, int TM, int TN>
cudaError_t simt_gemm_launch(const typename P::GA *A, int64_t lda, const typename P::GB *B,
                             int64_t ldb, typename P::GC *C, int64_t ldc, int64_t M, int64_t N,
                             int64_t K, const typename P::Params &prm, cudaStream_t s,
                             int splits = 1) {
    constexpr int NT = (BM / TM) * (BN / TN);
    typename P::Params prm2 = prm;
    if constexpr (pack_out_of<P>::value) {
        if (prm.pd < 0 || prm.pd + 1 > BN) return cudaErrorInvalidValue;
        prm2.bn_eff = BN / (prm.pd + 1) * (prm.pd + 1);     // whole words per CTA
    }
    const int64_t cols = tile_cols<P, BN>(prm2);
    const int64_t gx = (N + cols - 1) / cols, gy = (M + BM - 1) / BM;
    if (gx <= 0 || gy <= 0) return cudaSuccess;
    if (gx > 2147483647 || splits < 1 || splits > 65535) return cudaErrorInvalidConfiguration;
    int64_t kchunk = 0;
    if (splits > 1) kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    const unsigned gz = kchunk > 0 ? (unsigned)((K + kchunk - 1) / kchunk) : 1u;
    // a grid holds at most 65,535 row tiles: taller products run as several
    // launches over bands of rows (row i of A gives row i of C)
    constexpr int64_t band = (int64_t)65535 * BM;
    for (int64_t r0 = 0; r0 < M; r0 += band) {
        const int64_t rows = M - r0 < band ? M - r0 : band;
        simt_gemm_kernel<P, BM, BN, BK, TM, TN><<<dim3((unsigned)gx, (unsigned)((rows + BM - 1) / BM), gz), NT, 0, s>>>(
            A + r0 * lda, lda, B, ldb, C + r0 * ldc, ldc, rows, N, K, prm2, kchunk);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Default element fetch: a guarded load converted to the shared-memory type.
template <class G, class S>
__device__ __forceinline__ S ld_guarded(const G *X, int64_t ld, int64_t r, int64_t c, int64_t R,
                                        int64_t Cn) {
    return (r < R && c < Cn) ? (S)X[r * ld + c] : S(0);
}

// a mod p for 32-bit a (Lemire, Kaser, Kurz 2019), M = floor((2^64-1)/p) + 1.
__device__ __forceinline__ uint32_t fastmod_u32(uint32_t a, uint64_t M, uint32_t p) {
    return (uint32_t)__umul64hi(M * (uint64_t)a, (uint64_t)p);
}

// acc += a b for 64-bit a, b and a 128-bit accumulator held as four 32-bit
// limbs c0..c3: the four limb products a_i b_j, each added at limb i + j with
// its carries (low halves by mad.lo, high halves by madc.hi, carries rippled
// up).  Ten 32-bit multiply-adds and adds, slightly fewer issue slots than
// the 64 x 64 -> 128-bit multiply followed by a 128-bit add.
__device__ __forceinline__ void mad_u64_u128(unsigned __int128 &acc, uint64_t a, uint64_t b) {
    uint64_t lo = (uint64_t)acc, hi = (uint64_t)(acc >> 64);
    asm("{\n\t.reg .u32 a0, a1, b0, b1, c0, c1, c2, c3;\n\t"
        "mov.b64 {a0, a1}, %2;\n\t"
        "mov.b64 {b0, b1}, %3;\n\t"
        "mov.b64 {c0, c1}, %0;\n\t"
        "mov.b64 {c2, c3}, %1;\n\t"
        "mad.lo.cc.u32 c0, a0, b0, c0;\n\t"
        "madc.hi.cc.u32 c1, a0, b0, c1;\n\t"
        "madc.lo.cc.u32 c2, a1, b1, c2;\n\t"
        "madc.hi.u32 c3, a1, b1, c3;\n\t"
        "mad.lo.cc.u32 c1, a0, b1, c1;\n\t"
        "madc.hi.cc.u32 c2, a0, b1, c2;\n\t"
        "addc.u32 c3, c3, 0;\n\t"
        "mad.lo.cc.u32 c1, a1, b0, c1;\n\t"
        "madc.hi.cc.u32 c2, a1, b0, c2;\n\t"
        "addc.u32 c3, c3, 0;\n\t"
        "mov.b64 %0, {c0, c1};\n\t"
        "mov.b64 %1, {c2, c3};\n\t}"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
    acc = ((unsigned __int128)hi << 64) | lo;
}

}  // namespace gfp
