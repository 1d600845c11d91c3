// Thousands of independent products C_i = A_i B_i mod p_i of uneven sizes in
// one persistent grouped launch (no counterpart in the paper; the workload is
// the strongly-regular-graph computations that motivate it, Section 1).
//
// Host side (gfp_batched_prepare): validate every problem, give each a tile
// kind, cut it into output tiles, and balance the tiles over a fixed grid of
// CTAs by longest-processing-time-first (tiles sorted by cost, each to the
// least loaded CTA).  The schedule -- problem table, tile list, per-CTA tile
// ranges, operand-conversion jobs -- is copied into the caller's workspace
// with one host-to-device copy.  gfp_batched_launch then runs, on the
// prepared workspace only (so it can be captured in a CUDA graph):
//   1. the operand conversion: every distinct (matrix, p, tile) operand of a
//      tensor-core tile becomes centred fp16, row-major, zero padded to
//      multiples of the tile (64 or 128) in both dimensions (A^2 problems
//      convert A once);
//   2. the one persistent grouped kernel over all tiles.
//
// Tile kinds (all 128 threads, 2 x 2 warps):
//   HMMA128 / HMMA64 / HMMA32 : 128 x 128 / 64 x 64 / 32 x 32 output tiles
//       (warp tiles 64 x 64 / 32 x 32 / 16 x 16) on the warp-level fp16
//       tensor-core MMA (m16n8k16, fp32 accumulation), operands streamed from
//       the converted copies with 16-byte cp.async through a 3-stage ring.
//       Every partial sum is an integer below 2^24 within a k-block kb with
//       kb h^2 + p < 2^24 (h = (p-1)/2), after which the accumulators are
//       reduced mod p.
//   DOT32 : 64 x 64 tiles of the Q-adic dot form (Section 2) in 32-bit words:
//       rows of A are packed reversed and columns of B forward into d+1
//       residues per word while they are staged (Section 2.1), the word
//       products accumulate mod 2^32 (t(d+1) <= 32), and the coefficient of
//       Q^d is extracted every kbw words (eq. (lower) for the k-block) and
//       summed, then reduced mod p once.  (t, d, kbw) are chosen per problem.
// The autotuner (gfp_batched_autotune) times the kinds per size bucket and
// fills the table GFP_ALGO_AUTO uses.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_fp16.h>

#include "gfp_internal.h"

namespace gfp {
namespace {

enum Kind : int32_t { KIND_HMMA64 = 0, KIND_HMMA32 = 1, KIND_DOT32 = 2, KIND_HMMA128 = 3, KIND_COUNT = 4 };

struct DevProblem {          // 96 bytes
    const uint8_t *A;
    const uint8_t *B;
    uint8_t *C;
    const __half *A16;       // converted operands of the tensor-core kinds
    const __half *B16;
    int32_t m, k, n, lda, ldb, ldc;
    int32_t ld16a, ld16b;    // leading dimensions of A16, B16 (fp16 elements)
    uint32_t p;
    int32_t kind;
    uint64_t M;              // fastmod magic
    int32_t kb_steps;        // HMMA: k-block in 32-wide k steps; DOT32: words per block
    uint16_t t, d;           // DOT32: Q = 2^t, d
};
static_assert(sizeof(DevProblem) == 96, "layout");

struct Item {                // 8 bytes: problem index, tile row, tile column
    int32_t prob;
    uint16_t tm, tn;
};

struct ConvJob {             // 48 bytes: one operand to convert
    const uint8_t *src;
    __half *dst;
    int32_t rows, cols, ld, dld, drows;
    uint32_t p;
    int32_t pad[2];
};
static_assert(sizeof(ConvJob) == 48, "layout");

struct ConvItem {            // 16 padded rows of one job
    int32_t job, row0;
};

struct Header {              // 128 bytes at the start of the workspace
    uint32_t magic;
    int32_t count;
    int32_t items;
    int32_t grid;
    int64_t off_probs, off_items, off_ranges, off_jobs, off_citems, off_ops;
    int64_t bytes;
    int32_t njobs, ncitems;
    int32_t pad[12];
};
static_assert(sizeof(Header) == 128, "layout");
constexpr uint32_t kMagic = 0x47465042u;   // "GFPB"
constexpr int NT = 128;
constexpr int CTAS_PER_SM = 2;
constexpr int PADQ = 64;                   // smallest padding quantum of converted operands
constexpr int HSTAGES = 3;

__device__ __forceinline__ uint32_t fmod32(uint32_t a, uint64_t M, uint32_t p) {
    return (uint32_t)__umul64hi(M * (uint64_t)a, (uint64_t)p);
}

__device__ __forceinline__ uint32_t s2u(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------- operand conversion
// c = r - p [r > h] as fp16, zero outside the matrix, 8 values per thread-step.
__global__ void __launch_bounds__(256) convert_kernel(const uint8_t *__restrict__ ws) {
    const Header *H = reinterpret_cast<const Header *>(ws);
    const ConvJob *jobs = reinterpret_cast<const ConvJob *>(ws + H->off_jobs);
    const ConvItem *items = reinterpret_cast<const ConvItem *>(ws + H->off_citems);
    for (int it = blockIdx.x; it < H->ncitems; it += gridDim.x) {
        const ConvItem ci = items[it];
        const ConvJob J = jobs[ci.job];
        const uint32_t h = J.p == 2 ? 1u : (J.p - 1) / 2;
        const int per_row = J.dld / 8;
        for (int idx = threadIdx.x; idx < 16 * per_row; idx += blockDim.x) {
            const int r = ci.row0 + idx / per_row, c = (idx % per_row) * 8;
            if (r >= J.drows) break;
            __align__(16) __half v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                int x = 0;
                if (r < J.rows && c + e < J.cols) {
                    const uint32_t q = J.src[(int64_t)r * J.ld + c + e];
                    x = (int)q - (q > h ? (int)J.p : 0);
                }
                v[e] = __int2half_rn(x);
            }
            *reinterpret_cast<uint4 *>(J.dst + (int64_t)r * J.dld + c) = *reinterpret_cast<const uint4 *>(v);
        }
    }
}

// ---------------------------------------------------------------- HMMA tiles
template <int BT>
struct HmmaSmem {
    __half As[HSTAGES][BT][32 + 8];   // [stage][m][k], 80-byte rows: 16-byte aligned, conflict-free ldmatrix
    __half Bs[HSTAGES][32][BT + 8];   // [stage][k][n]
};

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int BT>
__device__ void tile_hmma(const DevProblem &P, int tm, int tn, HmmaSmem<BT> &S) {
    constexpr int MT = BT / 32, NTL = BT / 16;      // per-warp m16 and n8 tiles
    constexpr int ACH = BT * 4, BCH = 32 * (BT / 8);  // 16-byte chunks per stage
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int64_t m0 = (int64_t)tm * BT, n0 = (int64_t)tn * BT;
    const uint32_t p = P.p;
    const int nk = (P.k + 31) / 32;
    float acc[MT][NTL][4];
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int b = 0; b < NTL; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const uint32_t off = (uint32_t)((((int64_t)1 << 24) + p - 1) / p * p);
    int kb_left = P.kb_steps;
    // padded operands: no edge tests
    auto load_stage = [&](int s, int kt) {
        const int64_t k0 = (int64_t)kt * 32;
        for (int c = tid; c < ACH; c += NT) {
            const int row = c >> 2, ch = c & 3;
            cp_async16(s2u(&S.As[s][row][ch * 8]), P.A16 + (m0 + row) * P.ld16a + k0 + ch * 8);
        }
        for (int c = tid; c < BCH; c += NT) {
            const int row = c / (BT / 8), ch = c % (BT / 8);
            cp_async16(s2u(&S.Bs[s][row][ch * 8]), P.B16 + (k0 + row) * P.ld16b + n0 + ch * 8);
        }
    };
#pragma unroll
    for (int s = 0; s < HSTAGES - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_wait<HSTAGES - 2>();
        __syncthreads();
        if (kt + HSTAGES - 1 < nk) load_stage((kt + HSTAGES - 1) % HSTAGES, kt + HSTAGES - 1);
        cp_commit();
        const int s = kt % HSTAGES;
#pragma unroll
        for (int ks = 0; ks < 32; ks += 16) {
            uint32_t af[MT][4], bf[NTL][2];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int row = wm * (BT / 2) + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int col = ks + (lane >> 4) * 8;
                asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                             : "=r"(af[mt][0]), "=r"(af[mt][1]), "=r"(af[mt][2]), "=r"(af[mt][3])
                             : "r"(s2u(&S.As[s][row][col])));
            }
#pragma unroll
            for (int np = 0; np < NTL; np += 2) {
                const int mi = lane >> 3;
                const int krow = ks + (lane & 7) + (mi & 1) * 8;
                const int ncol = wn * (BT / 2) + np * 8 + (mi >> 1) * 8;
                uint32_t r0, r1, r2, r3;
                asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                             : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                             : "r"(s2u(&S.Bs[s][krow][ncol])));
                bf[np][0] = r0;
                bf[np][1] = r1;
                bf[np + 1][0] = r2;
                bf[np + 1][1] = r3;
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NTL; ++nt)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
                        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]),
                          "+f"(acc[mt][nt][3])
                        : "r"(af[mt][0]), "r"(af[mt][1]), "r"(af[mt][2]), "r"(af[mt][3]),
                          "r"(bf[nt][0]), "r"(bf[nt][1]));
        }
        if (--kb_left == 0) {
            kb_left = P.kb_steps;
#pragma unroll
            for (int a = 0; a < MT; ++a)
#pragma unroll
                for (int b = 0; b < NTL; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[a][b][c] = (float)fmod32((uint32_t)__float2int_rn(acc[a][b][c]) + off, P.M, p);
        }
    }
    cp_wait<0>();
    __syncthreads();   // the next tile of this CTA reuses the ring
    // c0, c1 at (row g, cols 2t, 2t+1); c2, c3 at row g + 8
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NTL; ++nt) {
            const int64_t col = n0 + wn * (BT / 2) + nt * 8 + (lane & 3) * 2;
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                const int64_t row = m0 + wm * (BT / 2) + mt * 16 + (lane >> 2) + hr * 8;
                if (row >= P.m) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (col + e < P.n)
                        P.C[row * P.ldc + col + e] = (uint8_t)fmod32(
                            (uint32_t)__float2int_rn(acc[mt][nt][hr * 2 + e]) + off, P.M, p);
            }
        }
}

// ------------------------------------------------------ Q-adic dot form tile
struct DotSmem {
    uint32_t As[8][64 + 4];  // [word][row]
    uint32_t Bs[8][64];      // [word][col]
};

__device__ void tile_dot32(const DevProblem &P, int tm, int tn, DotSmem &S) {
    const int tid = threadIdx.x;
    const int tx = tid & 7, ty = tid >> 3;          // 8 x 16 threads, 4 x 8 outputs each
    const int64_t m0 = (int64_t)tm * 64, n0 = (int64_t)tn * 64;
    const int dp1 = P.d + 1, t = P.t;
    const uint32_t td = (uint32_t)(t * P.d), mask = (t >= 32) ? 0xffffffffu : ((1u << t) - 1u);
    const int64_t K = P.k, KW = (K + dp1 - 1) / dp1;
    uint32_t acc[4][8], sum[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = sum[i][j] = 0;
    int countdown = P.kb_steps;
    for (int64_t w0 = 0; w0 < KW; w0 += 8) {
        // pack 64 rows x 8 words of A (reversed) and 8 words x 64 columns of B
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT;          // 0 .. 511
            const int r = idx >> 3, w = idx & 7;
            const int64_t gi = m0 + r, gw = w0 + w;
            uint32_t word = 0;
            if (gi < P.m && gw < KW) {
                const uint8_t *a = P.A + gi * P.lda + gw * dp1;
                for (int j = 0; j < dp1; ++j)
                    if (gw * dp1 + j < K) word += (uint32_t)a[j] << (t * (dp1 - 1 - j));
            }
            S.As[w][r] = word;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * NT;
            const int w = idx >> 6, c = idx & 63;
            const int64_t gw = w0 + w, gj = n0 + c;
            uint32_t word = 0;
            if (gj < P.n && gw < KW) {
                const uint8_t *b = P.B + (gw * dp1) * P.ldb + gj;
                for (int s = 0; s < dp1; ++s)
                    if (gw * dp1 + s < K) word += (uint32_t)b[(int64_t)s * P.ldb] << (t * s);
            }
            S.Bs[w][c] = word;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint32_t a[4], b[8];
            const uint4 av = *reinterpret_cast<const uint4 *>(&S.As[w][ty * 4]);
            a[0] = av.x; a[1] = av.y; a[2] = av.z; a[3] = av.w;
            const uint4 b0 = *reinterpret_cast<const uint4 *>(&S.Bs[w][tx * 8]);
            const uint4 b1 = *reinterpret_cast<const uint4 *>(&S.Bs[w][tx * 8 + 4]);
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
            if (--countdown == 0) {
                countdown = P.kb_steps;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        sum[i][j] += (acc[i][j] >> td) & mask;
                        acc[i][j] = 0;
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = m0 + ty * 4 + i;
        if (row >= P.m) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t col = n0 + tx * 8 + j;
            if (col < P.n)
                P.C[row * P.ldc + col] = (uint8_t)fmod32(sum[i][j] + ((acc[i][j] >> td) & mask), P.M, P.p);
        }
    }
}

union BatchedSmem {
    HmmaSmem<128> h128;
    HmmaSmem<64> h64;
    HmmaSmem<32> h32;
    DotSmem dot;
};
constexpr int SMEM_BATCHED = (int)sizeof(BatchedSmem);

__global__ void __launch_bounds__(NT, CTAS_PER_SM) batched_kernel(const uint8_t *__restrict__ ws) {
    extern __shared__ __align__(128) uint8_t dsm[];
    BatchedSmem &S = *reinterpret_cast<BatchedSmem *>(dsm);
    const Header *H = reinterpret_cast<const Header *>(ws);
    const DevProblem *probs = reinterpret_cast<const DevProblem *>(ws + H->off_probs);
    const Item *items = reinterpret_cast<const Item *>(ws + H->off_items);
    const int32_t *ranges = reinterpret_cast<const int32_t *>(ws + H->off_ranges);
    if ((int)blockIdx.x >= H->grid) return;
    const int i0 = ranges[blockIdx.x], i1 = ranges[blockIdx.x + 1];
    for (int i = i0; i < i1; ++i) {
        const Item it = items[i];
        const DevProblem P = probs[it.prob];
        if (P.kind == KIND_HMMA128) tile_hmma<128>(P, it.tm, it.tn, S.h128);
        else if (P.kind == KIND_HMMA64) tile_hmma<64>(P, it.tm, it.tn, S.h64);
        else if (P.kind == KIND_HMMA32) tile_hmma<32>(P, it.tm, it.tn, S.h32);
        else tile_dot32(P, it.tm, it.tn, S.dot);
    }
}

// ------------------------------------------------------------------ host side
int tile_of(int kind) { return kind == KIND_HMMA32 ? 32 : kind == KIND_HMMA128 ? 128 : 64; }

double tile_cost(int kind, int64_t k, uint32_t p) {
    // relative cost of one tile: k steps of the tile's mainloop
    const double ksteps = (double)((k + 31) / 32);
    if (kind == KIND_HMMA128) return 12.0 * ksteps + 6.0;
    if (kind == KIND_HMMA64) return 4.0 * ksteps + 2.0;
    if (kind == KIND_HMMA32) return 1.4 * ksteps + 1.0;
    (void)p;
    return 10.0 * ksteps + 2.0;
}

// Autotuned kind per size bucket (bucket of max(m, k, n)); -1 = untuned.
constexpr int NBUCKETS = 7;
std::mutex g_tune_mu;
int g_tuned[NBUCKETS] = {-1, -1, -1, -1, -1, -1, -1};

int bucket_of(int64_t m, int64_t k, int64_t n) {
    const int64_t s = std::max(m, std::max(k, n));
    if (s <= 32) return 0;
    if (s <= 64) return 1;
    if (s <= 128) return 2;
    if (s <= 256) return 3;
    if (s <= 512) return 4;
    if (s <= 2048) return 5;
    return 6;
}

int default_kind(int64_t m, int64_t k, int64_t n) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int b = bucket_of(m, k, n);
    if (g_tuned[b] >= 0) return g_tuned[b];
    const int64_t s = std::max(m, n);
    return s <= 48 ? KIND_HMMA32 : s <= 160 ? KIND_HMMA64 : KIND_HMMA128;
}

// (t, d, words per block) of the 32-bit dot form for (p, k): the chooser of
// gfp_params with a k-block that maximises d + 1 under t(d+1) <= 32.
bool dot32_params(uint32_t p, int64_t k, int *t_out, int *d_out, int *kbw_out) {
    double best = 0;
    bool found = false;
    for (int t = 2; t <= 31; ++t) {
        const int d = 32 / t - 1;
        if (d < 0) continue;
        // largest kb with kb (p-1)^2 < 2^t, a multiple of d+1, at most k
        int64_t kb = (((int64_t)1 << t) - 1) / std::max<int64_t>(1, (int64_t)(p - 1) * (p - 1));
        if (p == 2) kb = ((int64_t)1 << t) - 1;
        kb = std::min<int64_t>(kb, ((k + d) / (d + 1)) * (d + 1));
        kb = kb / (d + 1) * (d + 1);
        if (kb < d + 1) continue;
        if (check_dqt(p, k, d, (uint64_t)1 << t, GFP_FORM_DOT, GFP_WORD_U32, kb >= k ? 0 : kb) != GFP_OK)
            continue;
        // useful multiply-adds per instruction: (d+1) per word, plus one
        // extraction per block of kb/(d+1) words
        const double words = (double)kb / (d + 1);
        const double score = (d + 1) * words / (words + 2.0);
        if (score > best) {
            best = score;
            *t_out = t;
            *d_out = d;
            *kbw_out = (int)std::min<int64_t>(words, 1 << 30);
            found = true;
        }
    }
    return found;
}

struct Plan {
    std::vector<DevProblem> probs;
    std::vector<Item> items;
    std::vector<int32_t> ranges;
    std::vector<ConvJob> jobs;               // dst holds the offset in the operand area
    std::vector<ConvItem> citems;
    std::vector<std::pair<int64_t, int64_t>> op_off;   // per problem: (A16, B16) offsets or -1
    int64_t ops_bytes = 0;
    int grid = 0;
};

int64_t round_to(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

gfp_status validate_problem(const gfp_problem &q) {
    if (!is_prime_small(q.p)) return GFP_EPRIME;
    if (q.m < 0 || q.k < 0 || q.n < 0 || q.reserved != 0) return GFP_EINVAL;
    if (q.m == 0 || q.n == 0) return GFP_OK;
    if (!q.C || q.ldc < q.n) return GFP_EINVAL;
    if (q.k > 0 && (!q.A || !q.B || q.lda < q.k || q.ldb < q.n)) return GFP_EINVAL;
    if ((q.m + 31) / 32 > 65535 || (q.n + 31) / 32 > 65535) return GFP_EUNSUPPORTED;
    return GFP_OK;
}

gfp_status make_plan(int64_t count, const gfp_problem *probs, gfp_algo algo, gfp_status *status,
                     const int *forced_kind, Plan &plan) {
    gfp_status first_bad = GFP_OK;
    plan = Plan();
    std::map<std::tuple<uintptr_t, int32_t, int32_t, int32_t, uint32_t, int>, int64_t> seen;
    std::vector<double> cost;
    for (int64_t i = 0; i < count; ++i) {
        const gfp_problem &q = probs[i];
        gfp_status st = validate_problem(q);
        int kind = -1;
        if (st == GFP_OK) {
            if (forced_kind) kind = *forced_kind;
            else if (algo == GFP_ALGO_AUTO) kind = default_kind(q.m, q.k, q.n);
            else if (algo == GFP_ALGO_TC_F16) {
                const int64_t sz = std::max(q.m, q.n);
                kind = sz <= 48 ? KIND_HMMA32 : sz <= 160 ? KIND_HMMA64 : KIND_HMMA128;
            }
            else if (algo == GFP_ALGO_DOT32) kind = KIND_DOT32;
            else st = GFP_EUNSUPPORTED;
        }
        DevProblem P{};
        if (st == GFP_OK && kind == KIND_DOT32) {
            int t = 0, d = 0, kbw = 0;
            if (!dot32_params(q.p, q.k, &t, &d, &kbw)) kind = KIND_HMMA64;
            else {
                P.t = (uint16_t)t;
                P.d = (uint16_t)d;
                P.kb_steps = kbw;
            }
        }
        if (status) status[i] = st;
        if (st != GFP_OK) {
            if (first_bad == GFP_OK) first_bad = st;
            continue;
        }
        if (q.m == 0 || q.n == 0) continue;
        P.A = q.A;
        P.B = q.B;
        P.C = q.C;
        P.m = q.m;
        P.k = q.k;
        P.n = q.n;
        P.lda = q.lda;
        P.ldb = q.ldb;
        P.ldc = q.ldc;
        P.p = q.p;
        P.kind = kind;
        P.M = fastmod_magic(q.p);
        if (kind != KIND_DOT32) {
            const int64_t h = q.p == 2 ? 1 : (q.p - 1) / 2;
            const int64_t kb = (((int64_t)1 << 24) - 1 - q.p) / (h * h);
            P.kb_steps = (int32_t)std::max<int64_t>(1, std::min<int64_t>(kb / 32, 1 << 30));
        }
        const int pi = (int)plan.probs.size();
        int64_t offA = -1, offB = -1;
        if (kind != KIND_DOT32 && q.k > 0) {
            // one converted copy per distinct (matrix, ld, shape, p); A^2 shares it
            const int pad = std::max(PADQ, tile_of(kind));
            auto job_for = [&](const uint8_t *src, int32_t rows, int32_t cols, int32_t ld) -> int64_t {
                const auto key = std::make_tuple((uintptr_t)src, ld, rows, cols, q.p, pad);
                auto it = seen.find(key);
                if (it != seen.end()) return it->second;
                ConvJob J{};
                J.src = src;
                J.rows = rows;
                J.cols = cols;
                J.ld = ld;
                J.dld = (int32_t)round_to(cols, pad);
                J.drows = (int32_t)round_to(rows, pad);
                J.p = q.p;
                const int64_t off = plan.ops_bytes;
                J.dst = reinterpret_cast<__half *>((uintptr_t)off);
                plan.ops_bytes += (int64_t)J.drows * J.dld * 2;
                const int jid = (int)plan.jobs.size();
                plan.jobs.push_back(J);
                for (int32_t r = 0; r < J.drows; r += 16) plan.citems.push_back(ConvItem{jid, r});
                seen[key] = off;
                return off;
            };
            offA = job_for(q.A, q.m, q.k, q.lda);
            offB = job_for(q.B, q.k, q.n, q.ldb);
            P.ld16a = (int32_t)round_to(q.k, pad);
            P.ld16b = (int32_t)round_to(q.n, pad);
        }
        plan.op_off.push_back({offA, offB});
        plan.probs.push_back(P);
        const int T = tile_of(kind);
        const int tmn = (int)((q.m + T - 1) / T), tnn = (int)((q.n + T - 1) / T);
        const double c = tile_cost(kind, q.k, q.p);
        for (int a = 0; a < tmn; ++a)
            for (int b = 0; b < tnn; ++b) {
                plan.items.push_back(Item{pi, (uint16_t)a, (uint16_t)b});
                cost.push_back(c);
            }
    }
    // longest processing time first onto the least loaded CTA
    const int grid = std::max(1, num_sms() * CTAS_PER_SM);
    plan.grid = grid;
    std::vector<int> order(plan.items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int>> per(grid);
    std::vector<std::pair<double, int>> heap;
    for (int g = 0; g < grid; ++g) heap.push_back({0.0, g});
    auto cmp = [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
        return a.first > b.first || (a.first == b.first && a.second > b.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (int idx : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto &top = heap.back();
        per[top.second].push_back(idx);
        top.first += cost[idx];
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    std::vector<Item> sorted;
    sorted.reserve(plan.items.size());
    plan.ranges.assign(grid + 1, 0);
    for (int g = 0; g < grid; ++g) {
        plan.ranges[g] = (int32_t)sorted.size();
        for (int idx : per[g]) sorted.push_back(plan.items[idx]);
    }
    plan.ranges[grid] = (int32_t)sorted.size();
    plan.items.swap(sorted);
    return first_bad;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t plan_bytes(int64_t nprobs, int64_t nitems, int grid, int64_t njobs, int64_t ncitems,
                  int64_t ops_bytes) {
    return align256(sizeof(Header)) + align256(nprobs * sizeof(DevProblem)) +
           align256(nitems * sizeof(Item)) + align256((grid + 1) * sizeof(int32_t)) +
           align256(njobs * sizeof(ConvJob)) + align256(ncitems * sizeof(ConvItem)) +
           align256((size_t)ops_bytes);
}

// Upper bound of the workspace: every problem cut into 32 x 32 tiles and both
// operands converted separately.
size_t bound_bytes(int64_t count, const gfp_problem *probs) {
    int64_t items = 0, ops = 0, citems = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t m = std::max<int64_t>(probs[i].m, 0), n = std::max<int64_t>(probs[i].n, 0);
        const int64_t k = std::max<int64_t>(probs[i].k, 0);
        items += ((m + 31) / 32) * ((n + 31) / 32);
        ops += (round_to(m, 128) * round_to(k, 128) + round_to(k, 128) * round_to(n, 128)) * 2;
        citems += (round_to(m, 128) + round_to(k, 128)) / 16;
    }
    return plan_bytes(count, items, std::max(1, num_sms() * CTAS_PER_SM), 2 * count, citems, ops);
}

gfp_status upload(Plan &plan, void *ws, size_t ws_bytes, cudaStream_t s) {
    const size_t need = plan_bytes((int64_t)plan.probs.size(), (int64_t)plan.items.size(), plan.grid,
                                   (int64_t)plan.jobs.size(), (int64_t)plan.citems.size(), plan.ops_bytes);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GFP_EWORKSPACE;
    Header H{};
    H.magic = kMagic;
    H.count = (int32_t)plan.probs.size();
    H.items = (int32_t)plan.items.size();
    H.grid = plan.grid;
    H.off_probs = (int64_t)align256(sizeof(Header));
    H.off_items = H.off_probs + (int64_t)align256(plan.probs.size() * sizeof(DevProblem));
    H.off_ranges = H.off_items + (int64_t)align256(plan.items.size() * sizeof(Item));
    H.off_jobs = H.off_ranges + (int64_t)align256(plan.ranges.size() * sizeof(int32_t));
    H.off_citems = H.off_jobs + (int64_t)align256(plan.jobs.size() * sizeof(ConvJob));
    H.off_ops = H.off_citems + (int64_t)align256(plan.citems.size() * sizeof(ConvItem));
    H.bytes = (int64_t)need;
    H.njobs = (int32_t)plan.jobs.size();
    H.ncitems = (int32_t)plan.citems.size();
    // operand offsets -> device addresses
    uint8_t *ops = static_cast<uint8_t *>(ws) + H.off_ops;
    for (size_t i = 0; i < plan.probs.size(); ++i) {
        if (plan.op_off[i].first >= 0) {
            plan.probs[i].A16 = reinterpret_cast<const __half *>(ops + plan.op_off[i].first);
            plan.probs[i].B16 = reinterpret_cast<const __half *>(ops + plan.op_off[i].second);
        }
    }
    for (auto &J : plan.jobs) J.dst = reinterpret_cast<__half *>(ops + (uintptr_t)J.dst);
    const size_t meta = (size_t)H.off_ops;   // the operand area itself is written by the launch
    std::vector<uint8_t> host(meta, 0);
    std::memcpy(host.data(), &H, sizeof(H));
    if (!plan.probs.empty())
        std::memcpy(host.data() + H.off_probs, plan.probs.data(), plan.probs.size() * sizeof(DevProblem));
    if (!plan.items.empty())
        std::memcpy(host.data() + H.off_items, plan.items.data(), plan.items.size() * sizeof(Item));
    std::memcpy(host.data() + H.off_ranges, plan.ranges.data(), plan.ranges.size() * sizeof(int32_t));
    if (!plan.jobs.empty())
        std::memcpy(host.data() + H.off_jobs, plan.jobs.data(), plan.jobs.size() * sizeof(ConvJob));
    if (!plan.citems.empty())
        std::memcpy(host.data() + H.off_citems, plan.citems.data(), plan.citems.size() * sizeof(ConvItem));
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(ws, host.data(), meta, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? GFP_OK : cuda_fail(e);
}

gfp_status launch_plan(void *ws, cudaStream_t s) {
    // operand conversion (a grid-stride loop over the jobs' 16-row items; it
    // reads their count from the workspace), then the grouped product
    convert_kernel<<<std::max(1, num_sms() * 4), 256, 0, s>>>(static_cast<const uint8_t *>(ws));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BATCHED);
        attr = true;
    }
    batched_kernel<<<std::max(1, num_sms() * CTAS_PER_SM), NT, SMEM_BATCHED, s>>>(
        static_cast<const uint8_t *>(ws));
    return check_launch();
}

gfp_status prepare_impl(int64_t count, const gfp_problem *probs, gfp_algo algo, gfp_status *status,
                        void *ws, size_t ws_bytes, cudaStream_t s, const int *forced) {
    if (count < 0 || (count > 0 && !probs)) return GFP_EINVAL;
    if (algo != GFP_ALGO_AUTO && algo != GFP_ALGO_TC_F16 && algo != GFP_ALGO_DOT32)
        return GFP_EUNSUPPORTED;
    Plan plan;
    gfp_status st = make_plan(count, probs, algo, status, forced, plan);
    gfp_status up = upload(plan, ws, ws_bytes, s);
    if (up != GFP_OK) return up;
    return st;
}

}  // namespace
}  // namespace gfp

using namespace gfp;

extern "C" {

GFP_API gfp_status gfp_batched_workspace_size(int64_t count, const gfp_problem *probs,
                                              size_t *bytes) {
    if (count < 0 || (count > 0 && !probs) || !bytes) return GFP_EINVAL;
    *bytes = bound_bytes(count, probs);
    return GFP_OK;
}

GFP_API gfp_status gfp_batched_prepare(int64_t count, const gfp_problem *probs, gfp_algo algo,
                                       gfp_status *status, void *workspace, size_t ws_bytes,
                                       void *stream) {
    return prepare_impl(count, probs, algo, status, workspace, ws_bytes, (cudaStream_t)stream, nullptr);
}

GFP_API gfp_status gfp_batched_launch(void *workspace, size_t ws_bytes, void *stream) {
    if (!workspace || ws_bytes < sizeof(Header) || ((uintptr_t)workspace & 255)) return GFP_EWORKSPACE;
    return launch_plan(workspace, (cudaStream_t)stream);
}

GFP_API gfp_status gfp_gemm_batched(int64_t count, const gfp_problem *probs, gfp_algo algo,
                                    gfp_status *status, void *workspace, size_t ws_bytes,
                                    void *stream) {
    gfp_status st = gfp_batched_prepare(count, probs, algo, status, workspace, ws_bytes, stream);
    if (st == GFP_EWORKSPACE || st == GFP_ECUDA || st == GFP_EINVAL && (count < 0 || !probs))
        return st;
    gfp_status l = launch_plan(workspace, (cudaStream_t)stream);
    return l != GFP_OK ? l : st;
}

GFP_API gfp_status gfp_batched_autotune(int64_t count, const gfp_problem *probs, void *workspace,
                                        size_t ws_bytes, void *stream, int *table, int table_len) {
    if (count < 0 || (count > 0 && !probs)) return GFP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int best[NBUCKETS];
    for (int b = 0; b < NBUCKETS; ++b) best[b] = -1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    gfp_status result = GFP_OK;
    for (int b = 0; b < NBUCKETS && result == GFP_OK; ++b) {
        std::vector<gfp_problem> sub;
        for (int64_t i = 0; i < count; ++i)
            if (validate_problem(probs[i]) == GFP_OK && bucket_of(probs[i].m, probs[i].k, probs[i].n) == b)
                sub.push_back(probs[i]);
        if (sub.empty()) continue;
        float best_ms = 1e30f;
        for (int kind = 0; kind < KIND_COUNT; ++kind) {
            gfp_status st = prepare_impl((int64_t)sub.size(), sub.data(), GFP_ALGO_AUTO, nullptr, workspace,
                                         ws_bytes, s, &kind);
            if (st != GFP_OK) {
                result = st;
                break;
            }
            float ms_sum = 0;
            for (int rep = 0; rep < 4; ++rep) {
                cudaEventRecord(e0, s);
                launch_plan(workspace, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_sum += ms;      // first run warms up
            }
            if (ms_sum < best_ms) {
                best_ms = ms_sum;
                best[b] = kind;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != GFP_OK) return result;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int b = 0; b < NBUCKETS; ++b)
            if (best[b] >= 0) g_tuned[b] = best[b];
    }
    if (table)
        for (int b = 0; b < table_len && b < NBUCKETS; ++b) table[b] = best[b];
    return GFP_OK;
}

GFP_API gfp_status gfp_batched_set_table(const int *table, int table_len) {
    if (!table || table_len < 0) return GFP_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int b = 0; b < NBUCKETS; ++b) {
        const int v = b < table_len ? table[b] : -1;
        if (v < -1 || v >= KIND_COUNT) return GFP_EINVAL;
        g_tuned[b] = v;
    }
    return GFP_OK;
}

}  // extern "C"
