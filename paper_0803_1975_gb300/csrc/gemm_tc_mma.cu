// Exact C = A B mod p on the int8 tensor-core MMA (warp-level mma.sync,
// int8 x int8 -> int32).  No counterpart in the paper: this form replaces the
// packing of residues into machine words by the tensor cores' own packing.
//
// 1. Preprocess (HBM-bound): residues r in [0, p) become centred residues
//    c = r - p [r > (p-1)/2] in [-(p-1)/2, (p-1)/2], stored as int8 in the
//    workspace: A as Ac (mp x kp, row-major) and B transposed as Bt
//    (np x kp, row-major), zero padded to the tile multiples, so the main
//    loop has no edge tests.  For p = 2 the residues 0/1 are kept as they are.
// 2. Product: each |c| <= h = (p-1)/2, so a k-block of kb terms keeps the
//    int32 accumulator within kb h^2 + p; kb is chosen with kb h^2 + p < 2^30,
//    inside the int32 range with room for the non-negative shift of the
//    reduction.  After every k-block the accumulators are reduced to [0, p),
//    then the accumulation continues.  The last reduction gives C in [0, p).
//    (kb = whole k for every p <= 251 up to k = 68719.)
//
// Kernel layout: CTA tile 128 x 128, 8 warps as 2 (M) x 4 (N), warp tile
// 64 x 32 = 4 x 4 MMAs of m16n8k32.  The k dimension moves in 64-byte slices
// through a 4-stage cp.async ring in shared memory; rows of 64 bytes are
// stored with their four 16-byte chunks XOR-swizzled by (row >> 1) & 3 so
// that ldmatrix reads of 8 rows hit 8 distinct bank groups.
#include <cstdint>

#include "gfp_internal.h"

namespace gfp {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4, NT = 256;
constexpr int TILE_BYTES = BM * BK;   // one operand slice (BM == BN)

__device__ __forceinline__ uint32_t fastmod(uint32_t a, uint64_t M, uint32_t p) {
    return (uint32_t)__umul64hi(M * (uint64_t)a, (uint64_t)p);
}

// ---- preprocess -------------------------------------------------------------
// Four residue bytes centred at once: c = r - p where r > h, as int8 bytes
// (two's complement).  The byte-wise compare gives 0xFF where r > h; the
// byte-wise subtraction takes p off there (r - p >= -h: no borrow crosses a
// byte as the result wraps into the byte's own int8 value).
__device__ __forceinline__ uint32_t centre4(uint32_t w, uint32_t h4, uint32_t p4) {
    return __vsub4(w, __vcmpgtu4(w, h4) & p4);
}

// 16 consecutive residues as four words, zero outside [c0, limit) or when
// !row_ok: one 16-byte load when the run is inside the row and aligned.
__device__ __forceinline__ uint4 load16_bytes(const uint8_t *src, int64_t c0, int64_t limit, bool row_ok) {
    if (row_ok && c0 + 16 <= limit && (reinterpret_cast<uintptr_t>(src) & 15) == 0)
        return *reinterpret_cast<const uint4 *>(src);
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < 16; ++e)
        if (row_ok && c0 + e < limit) w[e >> 2] |= (uint32_t)src[e] << (8 * (e & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Ac[i][l] = centre(A[i][l]) for i < m, l < k; zero elsewhere in mp x kp
// (zero residues stay zero).  One thread per 16 consecutive values of a row.
__global__ void centre_rows_kernel(const uint8_t *__restrict__ A, int64_t lda, int64_t m,
                                   int64_t k, int8_t *__restrict__ Ac, int64_t kp, int64_t mp,
                                   uint32_t p, uint32_t h) {
    const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (l >= kp) return;
    const uint32_t h4 = h * 0x01010101u, p4 = p * 0x01010101u;
    for (int64_t i = blockIdx.y; i < mp; i += gridDim.y) {
        const uint4 v = load16_bytes(A + i * lda + l, l, k, i < m);
        *reinterpret_cast<uint4 *>(Ac + i * kp + l) =
            make_uint4(centre4(v.x, h4, p4), centre4(v.y, h4, p4), centre4(v.z, h4, p4), centre4(v.w, h4, p4));
    }
}

// Bt[j][l] = centre(B[l][j]) for l < k, j < n; zero elsewhere in np x kp.
// 64 x 64 byte tiles through shared memory, 256 threads, 16 values each way;
// CENTRE_TU column tiles per step of the grid-stride loop, all of their loads
// issued first.
constexpr int CENTRE_TU = 4;

__global__ void centre_transpose_kernel(const uint8_t *__restrict__ B, int64_t ldb, int64_t k,
                                        int64_t n, int8_t *__restrict__ Bt, int64_t kp, int64_t np,
                                        uint32_t p, uint32_t h) {
    __shared__ __align__(16) uint8_t tile[64][64 + 4];
    const int64_t l0 = (int64_t)blockIdx.x * 64;
    const int t = threadIdx.x, r = t >> 2, q = (t & 3) * 16;
    const int64_t l = l0 + r;
    const uint32_t h4 = h * 0x01010101u, p4 = p * 0x01010101u;
    for (int64_t jt = blockIdx.y; jt < np / 64; jt += CENTRE_TU * (int64_t)gridDim.y) {
        uint4 v[CENTRE_TU];
#pragma unroll
        for (int u = 0; u < CENTRE_TU; ++u) {
            const int64_t j0 = (jt + u * (int64_t)gridDim.y) * 64;
            v[u] = j0 < np ? load16_bytes(B + l * ldb + j0 + q, j0 + q, n, l < k) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < CENTRE_TU; ++u) {
            const int64_t j0 = (jt + u * (int64_t)gridDim.y) * 64;
            if (j0 >= np) break;   // the same in every thread of the block
            uint32_t *dst = reinterpret_cast<uint32_t *>(&tile[r][q]);
            dst[0] = centre4(v[u].x, h4, p4);
            dst[1] = centre4(v[u].y, h4, p4);
            dst[2] = centre4(v[u].z, h4, p4);
            dst[3] = centre4(v[u].w, h4, p4);
            __syncthreads();
            // row j0 + r of Bt, columns l0 + q .. l0 + q + 15 (np a multiple of 64: j < np)
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int e = 0; e < 16; ++e) w[e >> 2] |= (uint32_t)tile[q + e][r] << (8 * (e & 3));
            *reinterpret_cast<uint4 *>(Bt + (j0 + r) * kp + l0 + q) = make_uint4(w[0], w[1], w[2], w[3]);
            __syncthreads();   // the tile is refilled by the next column tile
        }
    }
}

// ---- product -----------------------------------------------------------------
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
    return (uint32_t)(row * BK + ((chunk ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t saddr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr));
}

__device__ __forceinline__ void mma_s8(int32_t (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Reduce an int32 accumulator |x| < 2^30 to [0, p): add off = p ceil(2^30 / p)
// (a multiple of p in [2^30, 2^30 + p)), which makes it a non-negative 32-bit
// value, then take a 32-bit remainder.
__device__ __forceinline__ int32_t reduce_acc(int32_t x, uint32_t off, uint64_t M, uint32_t p) {
    return (int32_t)fastmod((uint32_t)x + off, M, p);
}

struct MmaArgs {
    const int8_t *Ac;
    const int8_t *Bt;
    uint8_t *C;
    int64_t ldc, m, n, kp;
    int64_t kb_tiles;   // k-block in BK slices
    uint32_t p, off;
    uint64_t M;
    int64_t tile_m0;    // first row tile of this launch (grids hold at most 65,535 row tiles)
};

__global__ void __launch_bounds__(NT) mma_s8_kernel(MmaArgs g) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;           // 2 x 4 warps
    const int64_t m0 = ((int64_t)blockIdx.y + g.tile_m0) * BM, n0 = (int64_t)blockIdx.x * BN;
    const int8_t *Ag = g.Ac + m0 * g.kp;
    const int8_t *Bg = g.Bt + n0 * g.kp;
    const int64_t ktiles = g.kp / BK;

    // stage s: A slice at s * 2 * TILE_BYTES, B slice right after it
    auto load_stage = [&](int s, int64_t kt) {
        const uint32_t sa = sbase + s * 2 * TILE_BYTES, sb = sa + TILE_BYTES;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int idx = tid + e * NT;               // 512 chunks of 16 B per operand
            const int row = idx >> 2, ch = idx & 3;
            cp_async16(sa + swz(row, ch), Ag + row * g.kp + kt * BK + ch * 16);
            cp_async16(sb + swz(row, ch), Bg + row * g.kp + kt * BK + ch * 16);
        }
    };

    int32_t acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < ktiles) load_stage(s, s);
        cp_async_commit();
    }

    int64_t kb_left = g.kb_tiles;
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        {   // prefetch slice kt + STAGES - 1 into the stage freed last iteration
            const int64_t nk = kt + STAGES - 1;
            if (nk < ktiles) load_stage((int)(nk % STAGES), nk);
            cp_async_commit();
        }
        const int s = (int)(kt % STAGES);
        const uint32_t sa = sbase + s * 2 * TILE_BYTES, sb = sa + TILE_BYTES;
#pragma unroll
        for (int k32 = 0; k32 < 2; ++k32) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                // matrices: rows +0..7 / +8..15, k chunks 2*k32 / 2*k32 + 1
                const int row = wm * 64 + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int ch = k32 * 2 + (lane >> 4);
                ldmatrix_x4(af[mt], sa + swz(row, ch));
            }
#pragma unroll
            for (int np2 = 0; np2 < 2; ++np2) {
                // two n-tiles per x4: (n 0-7, k lo), (n 0-7, k hi), (n 8-15, k lo), (n 8-15, k hi)
                const int row = wn * 32 + np2 * 16 + (lane & 7) + (lane >> 4) * 8;
                const int ch = k32 * 2 + ((lane >> 3) & 1);
                uint32_t r[4];
                ldmatrix_x4(r, sb + swz(row, ch));
                bf[np2 * 2][0] = r[0];
                bf[np2 * 2][1] = r[1];
                bf[np2 * 2 + 1][0] = r[2];
                bf[np2 * 2 + 1][1] = r[3];
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_s8(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
        }
        if (--kb_left == 0 && kt + 1 < ktiles) {
            kb_left = g.kb_tiles;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][b][c] = reduce_acc(acc[a][b][c], g.off, g.M, g.p);
        }
    }
    cp_async_wait<0>();

    // epilogue: c0,c1 at (row lane/4, cols 2(lane%4) + {0,1}); c2,c3 at row + 8
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int64_t col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2;
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                const int64_t row = m0 + wm * 64 + mt * 16 + (lane >> 2) + hr * 8;
                if (row >= g.m) continue;
                const uint8_t v0 = (uint8_t)reduce_acc(acc[mt][nt][hr * 2], g.off, g.M, g.p);
                const uint8_t v1 = (uint8_t)reduce_acc(acc[mt][nt][hr * 2 + 1], g.off, g.M, g.p);
                uint8_t *c = g.C + row * g.ldc + col;
                if (col < g.n) c[0] = v0;
                if (col + 1 < g.n) c[1] = v1;
            }
        }
    }
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

int64_t tc_kblock_s32(uint32_t p) {
    const int64_t h = p == 2 ? 1 : (p - 1) / 2;
    // kb h^2 + p < 2^30 bounds every partial sum (after a reduction to [0, p))
    return ((int64_t(1) << 30) - 1 - p) / (h * h);
}

size_t tc_mma_workspace(int64_t m, int64_t k, int64_t n) {
    const int64_t kp = round_up(k > 0 ? k : 1, BK);
    return (size_t)(round_up(m, BM) + round_up(n, BN)) * (size_t)kp + 256;
}

gfp_status launch_tc_mma(uint32_t p, int64_t m, int64_t k, int64_t n, const uint8_t *A,
                         int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                         void *ws, size_t ws_bytes, cudaStream_t s) {
    const int64_t kp = round_up(k, BK), mp = round_up(m, BM), np = round_up(n, BN);
    if ((size_t)((mp + np) * kp) > ws_bytes) return GFP_EWORKSPACE;
    int8_t *Ac = static_cast<int8_t *>(ws);
    int8_t *Bt = Ac + mp * kp;
    const uint32_t h = p == 2 ? 1u : (p - 1) / 2;   // p = 2: residues stay 0/1
    {
        dim3 grid((unsigned)((kp / 16 + 255) / 256), (unsigned)(mp < 65535 ? mp : 65535));
        centre_rows_kernel<<<grid, 256, 0, s>>>(A, lda, m, k, Ac, kp, mp, p, h);
        const int64_t gy = (np / 64 + CENTRE_TU - 1) / CENTRE_TU;
        dim3 gt((unsigned)(kp / 64), (unsigned)(gy < 65535 ? gy : 65535));
        centre_transpose_kernel<<<gt, 256, 0, s>>>(B, ldb, k, n, Bt, kp, np, p, h);
    }
    MmaArgs g;
    g.Ac = Ac;
    g.Bt = Bt;
    g.C = C;
    g.ldc = ldc;
    g.m = m;
    g.n = n;
    g.kp = kp;
    int64_t kb = tc_kblock_s32(p) / BK;
    g.kb_tiles = kb > 0 ? kb : 1;
    g.p = p;
    g.off = (uint32_t)((((int64_t)1 << 30) + p - 1) / p * p);
    g.M = fastmod_magic(p);
    const int smem = STAGES * 2 * TILE_BYTES;
    static std::atomic<uint64_t> attr{0};
    const cudaError_t ea = smem_attr_once(reinterpret_cast<const void *>(mma_s8_kernel), smem, attr);
    if (ea != cudaSuccess) return cuda_fail(ea);
    // products taller than 65,535 row tiles run as several launches
    for (int64_t t0 = 0; t0 < mp / BM; t0 += 65535) {
        g.tile_m0 = t0;
        const int64_t rows = mp / BM - t0 < 65535 ? mp / BM - t0 : 65535;
        mma_s8_kernel<<<dim3((unsigned)(np / BN), (unsigned)rows), NT, smem, s>>>(g);
        const gfp_status st = check_launch();
        if (st != GFP_OK) return st;
    }
    return GFP_OK;
}

}  // namespace gfp
