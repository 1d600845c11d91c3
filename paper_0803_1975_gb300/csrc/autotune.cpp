// Autotuner of the Q-adic dot form for one product: which machine word and
// which k-block (and so which Q and d, by the bounds of Sections 2.4-2.5)
// run fastest on this GPU for (p, m, k, n).
//
// A smaller Q (a shorter k-block kb, eq. (lower) applied to kb) leaves room
// for more coefficients per word, but the coefficient of Q^d must then be
// extracted every kb terms; 32-bit words cost one multiply-add each, 64-bit
// words about three.  The candidates are the admissible (word, d, Q, kb)
// with no blocking and, for each Q = 2^t, the longest k-block eq. (lower)
// allows, keeping per (word, d) the longest k-block; each runs on the proxy
// shape min(m, 2048) x k x min(n, 2048) with zero operands (the kernels'
// speed does not depend on the values) in the caller's workspace, timed with
// CUDA events.  Not capturable in a graph (it waits for its timings).
#include <algorithm>
#include <cstring>
#include <vector>

#include "gfp_internal.h"

namespace gfp {
namespace {

constexpr int64_t kProxy = 2048;

struct Cand {
    gfp_word word;
    int d;
    uint64_t Q;
    int64_t kb;
};

std::vector<Cand> candidates(uint32_t p, int64_t m, int64_t k, int64_t n) {
    std::vector<Cand> out;
    const gfp_word words[3] = {GFP_WORD_U32, GFP_WORD_U32W, GFP_WORD_U64};
    for (gfp_word w : words) {
        // no blocking, then for each Q = 2^t the longest k-block eq. (lower)
        // allows: floor((2^t - 1) / (p-1)^2)
        const int64_t pp = p == 2 ? 1 : (int64_t)(p - 1) * (p - 1);
        for (int t = 0; t <= 40; ++t) {
            const int64_t req = t == 0 ? 0 : (((int64_t)1 << t) - 1) / pp;
            if (t != 0 && req < 1) continue;
            if (req >= k) break;
            int d = -1;
            uint64_t Q = 0;
            int64_t kb = req;
            if (gfp_params(p, m, k, n, GFP_FORM_DOT, w, &d, &Q, &kb) != GFP_OK) continue;
            // per (word, d) only the longest k-block (no blocking counts as the
            // longest): the same work per word with the fewest extractions
            bool placed = false;
            for (Cand &c : out) {
                if (c.word != w || c.d != d) continue;
                placed = true;
                const bool longer = c.kb != 0 && (kb == 0 || kb > c.kb);
                if (longer) c = Cand{w, d, Q, kb};
            }
            if (!placed) out.push_back(Cand{w, d, Q, kb});
        }
    }
    return out;
}

}  // namespace
}  // namespace gfp

using namespace gfp;

extern "C" {

GFP_API gfp_status gfp_dot_autotune_workspace_size(int64_t m, int64_t k, int64_t n, size_t *bytes) {
    if (!bytes || m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    const int64_t mp = std::min(m, kProxy), np = std::min(n, kProxy);
    // the widest candidate: 8-byte words, no compression (d = 0)
    *bytes = (size_t)(mp * k + k * np) * 8 + (size_t)(mp * np) + 256;
    return GFP_OK;
}

GFP_API gfp_status gfp_dot_autotune(uint32_t p, int64_t m, int64_t k, int64_t n, void *workspace,
                                    size_t ws_bytes, void *stream, gfp_dot_choice *best, gfp_dot_choice *all,
                                    int max_all, int *n_all) {
    if (!best || m < 1 || k < 1 || n < 1 || max_all < 0 || (max_all > 0 && !all)) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    size_t need = 0;
    gfp_dot_autotune_workspace_size(m, k, n, &need);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return GFP_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const std::vector<Cand> cands = candidates(p, m, k, n);
    if (cands.empty()) return GFP_EBOUND;
    const int64_t mp = std::min(m, kProxy), np = std::min(n, kProxy);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    cudaError_t e = cudaMemsetAsync(base, 0, need, s);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(e);
    }
    gfp_status st = GFP_OK;
    float best_ms = 0.f;
    int count = 0;
    for (const Cand &c : cands) {
        const int64_t kc = (k + c.d) / (c.d + 1);
        const size_t wb = word_bytes(c.word);
        uint8_t *CA = base + 256, *CB = CA + (size_t)mp * kc * wb, *C = CB + (size_t)kc * np * wb;
        const int t = log2_exact(c.Q);
        const int64_t kbw = c.kb > 0 ? c.kb / (c.d + 1) : 0;
        float ms = 0.f, runs[3];
        for (int r = -1; r < 3 && st == GFP_OK; ++r) {
            if (r >= 0) cudaEventRecord(ev[0], s);
            st = launch_dot(p, mp, kc, np, c.d, t, c.word, CA, kc, CB, np, C, np, kbw, s);
            if (st != GFP_OK) break;
            if (r >= 0) {
                cudaEventRecord(ev[1], s);
                if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) {
                    st = cuda_fail(e);
                    break;
                }
                cudaEventElapsedTime(&runs[r], ev[0], ev[1]);
            }
        }
        if (st != GFP_OK) break;
        std::sort(runs, runs + 3);
        ms = runs[1];
        const gfp_dot_choice ch{(int32_t)c.word, c.d, c.Q, c.kb, ms, 0};
        if (count < max_all) all[count] = ch;
        ++count;
        if (count == 1 || ms < best_ms) {
            best_ms = ms;
            *best = ch;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (n_all) *n_all = count;
    return st;
}

}  // extern "C"
