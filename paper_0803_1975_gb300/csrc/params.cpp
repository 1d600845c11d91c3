// Parameter validation and choice for the Q-adic forms (host only).
//
// Bounds (Dumas, Fousse, Salvy, arXiv 0803.1975):
//  * eq. (lower), Section 2.4: with delayed reduction every coefficient of
//    the accumulated word products stays below Q when k (p-1)^2 < Q (strict).
//    With a k-block kb the same bound applies to kb.  The argument only uses
//    that entries lie in [0, p-1]; with entries of A at most a and of B at
//    most b (0/1 adjacency matrices: a = b = 1) it gives k a b < Q, and the
//    packed words hold digits up to max(a, b).
//  * eq. (upper), Section 2.5: Q^(d+1) < 2^beta for a beta-bit mantissa.
//  * integer words: the coefficient of Q^d occupies bits [t d, t(d+1)); it
//    is exact when the accumulator keeps those bits (t(d+1) <= 64 for a
//    64-bit accumulator, <= 32 for a 32-bit one, <= 128 for 128 bits) and
//    the packed words fit their storage.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "gfp_internal.h"

namespace gfp {

bool is_prime_small(uint32_t p) {
    if (p < 2 || p > 251) return false;
    for (uint32_t q = 2; q * q <= p; ++q)
        if (p % q == 0) return false;
    return true;
}

int log2_exact(uint64_t Q) {
    if (Q < 2 || (Q & (Q - 1))) return -1;
    int t = 0;
    while ((Q >> t) != 1) ++t;
    return t;
}

// (p-1)(1 + Q + ... + Q^d) < 2^bits, with Q = 2^t, computed without overflow:
// the sum has its top set bit at t d + bitlen(p-1) - 1 at most, and equals
// (p-1) 2^(t d) + lower terms < (p-1) 2^(t d) + 2^(t d) = p 2^(t d).
bool amax_below_v(uint32_t v, int t, int d, int bits) {
    // exact test: v * sum_{s<=d} 2^(t s) < 2^bits
    // iterate with 128-bit integers while the value is small enough
    unsigned __int128 lim = 0;
    if (bits >= 128) return (int64_t)t * d + 9 <= 127;
    lim = (unsigned __int128)1 << bits;
    unsigned __int128 sum = 0;
    for (int s = 0; s <= d; ++s) {
        if ((int64_t)t * s >= bits) return false;
        sum += (unsigned __int128)1 << (t * s);
        if (sum * v >= lim) return false;
    }
    return sum * v < lim;
}

bool amax_below(uint32_t p, int t, int d, int bits) { return amax_below_v(p - 1, t, d, bits); }

size_t word_bytes(gfp_word w) {
    switch (w) {
        case GFP_WORD_U64:
        case GFP_WORD_U64X128:
        case GFP_WORD_F64: return 8;
        case GFP_WORD_U32W:
        case GFP_WORD_U32: return 4;
    }
    return 0;
}

// k a b < 2^t with a b = prod
static bool lower_ok_prod(uint64_t prod, int64_t k, int t) {
    if (k < 0) return false;
    unsigned __int128 lhs = (unsigned __int128)k * prod;
    if (t >= 100) return true;
    return lhs < ((unsigned __int128)1 << t);
}

static bool lower_ok(uint32_t p, int64_t k, int t) {   // k (p-1)^2 < 2^t
    return lower_ok_prod((uint64_t)(p - 1) * (p - 1), k, t);
}

// Storage bound of a packed word whose digits are at most v (needed by
// pack/unpack as well).
gfp_status check_pack_vb(uint32_t p, uint32_t v, int d, uint64_t Q, gfp_word word) {
    if (!is_prime_small(p)) return GFP_EPRIME;
    if (v > p - 1) return GFP_EINVAL;
    int t = log2_exact(Q);
    if (t < 0) return GFP_EQ;
    if (d < 0 || d > 255) return GFP_EINVAL;
    if (word_bytes(word) == 0) return GFP_EINVAL;
    if ((uint64_t)v >= Q) return GFP_EBOUND;   // an entry must be a digit
    int bits = word == GFP_WORD_F64 ? 53 : (int)(8 * word_bytes(word));
    if (!amax_below_v(v, t, d, bits)) return GFP_EBOUND;
    return GFP_OK;
}

gfp_status check_pack(uint32_t p, int d, uint64_t Q, gfp_word word) {
    return check_pack_vb(p, p - 1, d, Q, word);
}

gfp_status check_dqt(uint32_t p, int64_t k, int d, uint64_t Q, gfp_form form, gfp_word word,
                     int64_t kb) {
    return check_dqt_vb(p, k, d, Q, form, word, kb, p - 1, p - 1);
}

gfp_status check_dqt_vb(uint32_t p, int64_t k, int d, uint64_t Q, gfp_form form, gfp_word word,
                        int64_t kb, uint32_t va, uint32_t vb) {
    if (!is_prime_small(p)) return GFP_EPRIME;
    if (va > p - 1 || vb > p - 1) return GFP_EINVAL;
    const uint64_t prod = (uint64_t)va * vb;
    const uint32_t vmax = va > vb ? va : vb;
    int t = log2_exact(Q);
    if (t < 0) return GFP_EQ;
    if (k < 0 || d < 0 || d > 255 || kb < 0) return GFP_EINVAL;
    if (form != GFP_FORM_DOT && form != GFP_FORM_MIXED && form != GFP_FORM_LEFT) return GFP_EINVAL;
    if (word_bytes(word) == 0) return GFP_EINVAL;
    if (form != GFP_FORM_DOT && word != GFP_WORD_U64 && word != GFP_WORD_F64)
        return GFP_EUNSUPPORTED;
    const bool blocked = kb > 0 && kb < k;
    if (kb > 0) {
        if (form != GFP_FORM_DOT) return GFP_EUNSUPPORTED;
        if (kb % (d + 1) != 0) return GFP_EINVAL;
    }
    if (blocked) {
        // the extracted coefficients are summed in 32 bits
        unsigned __int128 tot = (unsigned __int128)k * prod;
        if (tot >= ((unsigned __int128)1 << 32)) return GFP_EBOUND;
    }
    if (!lower_ok_prod(prod, blocked ? kb : k, t)) return GFP_EBOUND;
    const int64_t td1 = (int64_t)t * (d + 1);
    if (form == GFP_FORM_DOT) {
        switch (word) {
            case GFP_WORD_U64:
                if (td1 > 64 || !amax_below_v(vmax, t, d, 64)) return GFP_EBOUND;
                break;
            case GFP_WORD_U64X128:
                if (td1 > 128 || !amax_below_v(vmax, t, d, 64)) return GFP_EBOUND;
                break;
            case GFP_WORD_U32W:
                if (td1 > 64 || !amax_below_v(vmax, t, d, 32)) return GFP_EBOUND;
                break;
            case GFP_WORD_U32:
                if (td1 > 32) return GFP_EBOUND;
                break;
            case GFP_WORD_F64:
                if (td1 > 52) return GFP_EBOUND;   // Q^(d+1) < 2^53 with Q = 2^t
                break;
        }
    } else {
        // right (MIXED) and left compression: every coefficient of a result
        // word is a full dot product < Q, so the word is below Q^(d+1)
        if (word == GFP_WORD_U64 && td1 > 64) return GFP_EBOUND;
        if (word == GFP_WORD_F64 && td1 > 52) return GFP_EBOUND;
    }
    return GFP_OK;
}

// Section 4 with Theta = Q^(dq+1): eq. (lower) for Q, and the whole word, with
// (dq+1)(dth+1) coefficients below Q, inside the word (eq. dq with beta = 64
// for uint64 words, 53 for binary64).
gfp_status check_full(uint32_t p, int64_t k, int dq, int dth, uint64_t Q, gfp_word word) {
    if (!is_prime_small(p)) return GFP_EPRIME;
    const int t = log2_exact(Q);
    if (t < 0) return GFP_EQ;
    if (k < 0 || dq < 0 || dth < 0 || dq > 63 || dth > 63) return GFP_EINVAL;
    if (word != GFP_WORD_U64 && word != GFP_WORD_F64) return GFP_EUNSUPPORTED;
    if (!lower_ok(p, k, t)) return GFP_EBOUND;
    const int64_t bits = (int64_t)t * (dq + 1) * (dth + 1);
    if (word == GFP_WORD_U64 && bits > 64) return GFP_EBOUND;
    if (word == GFP_WORD_F64 && bits > 52) return GFP_EBOUND;
    return GFP_OK;
}

}  // namespace gfp

using namespace gfp;

extern "C" {

GFP_API const char *gfp_status_string(gfp_status s) {
    switch (s) {
        case GFP_OK: return "ok";
        case GFP_EINVAL: return "invalid argument";
        case GFP_EPRIME: return "p is not a prime in [2, 251]";
        case GFP_EBOUND: return "parameters violate the bounds of the form";
        case GFP_EQ: return "Q is not a power of two";
        case GFP_EUNSUPPORTED: return "unsupported combination";
        case GFP_ECUDA: return "CUDA error";
        case GFP_EWORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

GFP_API size_t gfp_word_bytes(gfp_word word) { return word_bytes(word); }

GFP_API gfp_status gfp_params(uint32_t p, int64_t m, int64_t k, int64_t n, gfp_form form,
                              gfp_word word, int *d, uint64_t *Q, int64_t *kb) {
    return gfp_params_vb(p, m, k, n, form, word, p - 1, p - 1, d, Q, kb);
}

GFP_API gfp_status gfp_params_vb(uint32_t p, int64_t m, int64_t k, int64_t n, gfp_form form,
                                 gfp_word word, uint32_t amax_a, uint32_t amax_b, int *d, uint64_t *Q,
                                 int64_t *kb) {
    if (!d || !Q || !kb) return GFP_EINVAL;
    if (m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    if (form != GFP_FORM_DOT && form != GFP_FORM_MIXED && form != GFP_FORM_LEFT) return GFP_EINVAL;
    if (word_bytes(word) == 0) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    if (amax_a > p - 1 || amax_b > p - 1) return GFP_EINVAL;
    if (*d >= 0) return check_dqt_vb(p, k, *d, *Q, form, word, *kb, amax_a, amax_b);
    if (form != GFP_FORM_DOT && *kb > 0) return GFP_EUNSUPPORTED;
    // choose: the smallest Q for (lower), then the largest d the word admits
    const uint64_t prod = (uint64_t)amax_a * amax_b;
    const uint32_t vmax = amax_a > amax_b ? amax_a : amax_b;
    const int64_t kreq = (*kb > 0 && *kb < k) ? *kb : k;
    int t = 1;
    while (!lower_ok_prod(prod, kreq > 0 ? kreq : 1, t) || (uint64_t)vmax >= (1ull << t)) {
        if (++t > 62) return GFP_EBOUND;
    }
    const uint64_t QQ = 1ull << t;
    int best = -1;
    for (int dd = 0; dd <= 255; ++dd) {
        int64_t kbb = 0;
        if (*kb > 0 && *kb < k) {
            kbb = (*kb / (dd + 1)) * (dd + 1);
            if (kbb == 0) break;
        }
        if (check_dqt_vb(p, k, dd, QQ, form, word, kbb, amax_a, amax_b) == GFP_OK) best = dd;
    }
    if (best < 0) return form != GFP_FORM_DOT && word != GFP_WORD_U64 && word != GFP_WORD_F64
                             ? GFP_EUNSUPPORTED
                             : GFP_EBOUND;
    *d = best;
    *Q = QQ;
    *kb = (*kb > 0 && *kb < k) ? (*kb / (best + 1)) * (best + 1) : 0;
    return GFP_OK;
}

GFP_API gfp_status gfp_params_full(uint32_t p, int64_t m, int64_t k, int64_t n, gfp_word word,
                                   int *dq, int *dth, uint64_t *Q) {
    if (!dq || !dth || !Q || m < 0 || k < 0 || n < 0) return GFP_EINVAL;
    if (!is_prime_small(p)) return GFP_EPRIME;
    if (word != GFP_WORD_U64 && word != GFP_WORD_F64) return GFP_EUNSUPPORTED;
    if (*dq >= 0) return check_full(p, k, *dq, *dth, *Q, word);
    int t = 1;
    while (!lower_ok(p, k > 0 ? k : 1, t) || (uint64_t)(p - 1) >= (1ull << t)) {
        if (++t > 62) return GFP_EBOUND;
    }
    // the most coefficients per word, then the most balanced split (Section 5
    // compares full compression at equal degrees in both variables)
    int bq = -1, bt = -1;
    for (int a = 0; a < 64; ++a)
        for (int b = 0; b < 64; ++b) {
            if (check_full(p, k, a, b, 1ull << t, word) != GFP_OK) continue;
            const int cur = (a + 1) * (b + 1), best = (bq + 1) * (bt + 1);
            if (bq < 0 || cur > best || (cur == best && std::abs(a - b) < std::abs(bq - bt))) {
                bq = a;
                bt = b;
            }
        }
    if (bq < 0) return GFP_EBOUND;
    *dq = bq;
    *dth = bt;
    *Q = 1ull << t;
    return GFP_OK;
}

}  // extern "C"
