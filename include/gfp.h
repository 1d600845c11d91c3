/*
 * gfp.h -- exact dense matrix multiplication over a small prime field on one
 * GB300 (CUDA sm_103a).
 *
 * Method: J.-G. Dumas, L. Fousse, B. Salvy, "Compressed Modular Matrix
 * Multiplication" (arXiv 0803.1975).  Given a prime p, sizes m, k, n and a
 * machine word, the library computes C = A B mod p exactly, either plainly,
 * or with d+1 residues packed per word in base Q = 2^t (Sections 2-3), or on
 * the tensor cores from centred residues (no counterpart in the paper).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Residues are uint8 in the positive representation [0, p) (Section 2.4),
 *    so p <= 251 is the largest prime the storage admits.  Inputs outside
 *    [0, p) are a precondition violation: results are then unspecified but
 *    no call reads or writes outside the buffers it was given.
 *  - Matrices are row-major.  Leading dimensions (ld*) count ELEMENTS of the
 *    stored type (bytes for residues, words for packed matrices) and must be
 *    >= the row length.  All matrix pointers are DEVICE pointers owned by the
 *    caller; the library keeps no reference after the call is enqueued.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are asynchronous on it: they validate on the host,
 *    enqueue kernels and return.  They never synchronize the device.
 *  - The library allocates no device memory.  Calls that need scratch take a
 *    caller-provided workspace and report the size they need through a
 *    *_workspace_size query.
 *  - Every call returns a gfp_status.  All validation happens on the host
 *    before anything is launched: an invalid call launches nothing.  No
 *    kernel traps or asserts; a failed launch is reported as GFP_ECUDA with
 *    the CUDA error code available from gfp_last_cuda_error().
 *  - Sizes of zero are valid and launch nothing (an empty k gives C = 0).
 */
#ifndef GFP_H
#define GFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GFP_API __attribute__((visibility("default")))
#else
#define GFP_API
#endif

typedef enum gfp_status {
    GFP_OK = 0,
    GFP_EINVAL = 1,        /* null pointer, negative size, ld too small, bad enum value */
    GFP_EPRIME = 2,        /* p is not a prime in [2, 251] */
    GFP_EBOUND = 3,        /* (p, k, d, Q, kb) violate the bounds of the form and word */
    GFP_EQ = 4,            /* Q is not a power of two */
    GFP_EUNSUPPORTED = 5,  /* combination of form, word, algorithm and layout not provided */
    GFP_ECUDA = 6,         /* a CUDA runtime call or launch failed; see gfp_last_cuda_error() */
    GFP_EWORKSPACE = 7     /* workspace pointer missing, misaligned or smaller than required */
} gfp_status;

/* Compressed product forms.
 *  GFP_FORM_DOT   : Section 2, procedure (2) -- CA (rows of A packed reversed)
 *                   times CB (columns of B packed), the coefficient of Q^d of
 *                   each accumulated word is the dot product (delayed
 *                   reduction, Section 2.4), reduced mod p once.
 *  GFP_FORM_MIXED : Section 3, equation (LeftComp) -- uncompressed A times a
 *                   row-compressed right operand; each result word holds d+1
 *                   dot products, reduced simultaneously (REDQ).
 *  GFP_FORM_LEFT  : Table 2 "Left Comp." -- the same with the outer dimensions
 *                   exchanged: A packed along m (layout COLS) times
 *                   uncompressed B; each result word holds d+1 entries of a
 *                   column of C, reduced by REDQ.
 * Full compression (Section 4) has its own entry points (gfp_gemm_full). */
typedef enum gfp_form { GFP_FORM_DOT = 0, GFP_FORM_MIXED = 1, GFP_FORM_LEFT = 2 } gfp_form;

/* Machine words.  t = log2 Q.  Bounds (all require eq. (lower) of Section 2.4,
 * k (p-1)^2 < Q, with k replaced by the k-block kb when one is used):
 *  GFP_WORD_U64     : uint64 words, products and sums mod 2^64; t(d+1) <= 64.
 *  GFP_WORD_U64X128 : uint64 words (largest word < 2^64) with a 128-bit
 *                     accumulator; t(d+1) <= 128.  DOT form only.
 *  GFP_WORD_U32W    : uint32 words (largest word < 2^32), 64-bit accumulator.
 *                     DOT form only.
 *  GFP_WORD_U32     : uint32 words and accumulator, t(d+1) <= 32.  DOT only.
 *  GFP_WORD_F64     : IEEE binary64 words holding exact integers; eq. (upper)
 *                     of Section 2.5 with beta = 53, Q^(d+1) < 2^53.  The DOT
 *                     form accumulates with fused multiply-adds rounded
 *                     toward zero, which keeps the coefficient of Q^d exact
 *                     under eq. (upper) (round-to-nearest does not).
 * The largest word of a form is (p-1)(1 + Q + ... + Q^d). */
typedef enum gfp_word {
    GFP_WORD_U64 = 0,
    GFP_WORD_U64X128 = 1,
    GFP_WORD_U32W = 2,
    GFP_WORD_U32 = 3,
    GFP_WORD_F64 = 4
} gfp_word;

/* Packed layouts (Section 2.1, 2.3, 3).  For a residue matrix X (rows x cols)
 *  GFP_LAYOUT_ROWS_REV : W[i][w] = sum_{j=0..d} X[i][w(d+1)+j] Q^(d-j)
 *                        (rows x ceil(cols/(d+1)) words; left operand CA)
 *  GFP_LAYOUT_COLS     : W[w][j] = sum_{s=0..d} X[w(d+1)+s][j] Q^s
 *                        (ceil(rows/(d+1)) x cols words; right operand CB)
 *  GFP_LAYOUT_ROWS     : W[i][v] = sum_{j=0..d} X[i][v(d+1)+j] Q^j
 *                        (rows x ceil(cols/(d+1)) words; right operand of the
 *                        MIXED form and its compressed result CC)
 * Entries beyond the matrix edge count as zero (Section 2.3). */
typedef enum gfp_layout {
    GFP_LAYOUT_ROWS_REV = 0,
    GFP_LAYOUT_COLS = 1,
    GFP_LAYOUT_ROWS = 2
} gfp_layout;

/* Algorithms of gfp_gemm (uncompressed uint8 in and out).
 *  GFP_ALGO_PLAIN      : classical product, one 32-bit integer multiply-add
 *                        per term, 32-bit sums, one reduction per entry.
 *                        Needs k (p-1)^2 < 2^32.
 *  GFP_ALGO_DP4A       : classical product on the 4-way byte dot-product
 *                        instruction (same bound); B is first transposed into
 *                        the workspace (roundup(n, 64) x roundup(k, 64) bytes
 *                        after 256) so that both operands are read as one
 *                        32-bit word per 4 residues.
 *  GFP_ALGO_TC_MMA_S8  : centred residues c in [-(p-1)/2, (p-1)/2] as int8 on
 *                        the warp-level int8 tensor-core MMA with int32
 *                        accumulation; reduced mod p after every k-block kb
 *                        with kb ((p-1)/2)^2 < 2^31 (p = 2: residues 0/1).
 *  GFP_ALGO_TC_F16     : centred residues as fp16 on tcgen05 (kind::f16)
 *                        with fp32 accumulation, which is exact while every
 *                        partial sum is an integer of magnitude < 2^24: the
 *                        k-block is the largest kb with kb ((p-1)/2)^2 + p
 *                        < 2^24 (rounded down to a multiple of 128).  After the
 *                        call's kernels complete, the first 4 bytes of its
 *                        workspace hold the kernel's status: 0, or non-zero if
 *                        a bounded internal wait gave up (C is then invalid).
 *  GFP_ALGO_TC_F8      : as GFP_ALGO_TC_F16 with fp8 e4m3 operands on tcgen05
 *                        (kind::f8f6f4), which hold the centred residues of
 *                        p <= 31 exactly (|c| <= 15); twice the fp16 rate.
 *                        GFP_EUNSUPPORTED for p > 31.  Same status word.
 *  GFP_ALGO_TC_E2M1    : as GFP_ALGO_TC_F16 with fp4 e2m1 operands on the
 *                        block-scaled tcgen05 MMA (kind::mxf4, every scale
 *                        factor 1), which hold the centred residues of p <= 7
 *                        exactly (|c| <= 3): products are integers of
 *                        magnitude <= 9 and the k-block is the largest kb
 *                        with kb ((p-1)/2)^2 + p < 2^24 (a multiple of 256).
 *                        The workspace holds both operands packed two values
 *                        per byte.  GFP_EUNSUPPORTED for p > 7.  Same status
 *                        word.
 *  GFP_ALGO_AUTO       : GFP_ALGO_TC_E2M1 for p <= 7 when k >= 6144 and
 *                        m, n >= 4096; otherwise GFP_ALGO_TC_F8 for p <= 31,
 *                        else GFP_ALGO_TC_F16 (the fastest exact forms
 *                        measured on GB300). */
typedef enum gfp_algo {
    GFP_ALGO_AUTO = 0,
    GFP_ALGO_PLAIN = 1,
    GFP_ALGO_DP4A = 2,
    GFP_ALGO_TC_MMA_S8 = 3,
    GFP_ALGO_TC_F16 = 4,
    GFP_ALGO_DOT32 = 5,     /* batched only: Q-adic dot form in 32-bit words */
    GFP_ALGO_TC_F8 = 6,
    GFP_ALGO_TC_E2M1 = 7
} gfp_algo;

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

/* Short English name of a status code (static storage, never NULL). */
GFP_API const char *gfp_status_string(gfp_status s);

/* cudaError_t of the last GFP_ECUDA returned on the calling thread (0 if none). */
GFP_API int gfp_last_cuda_error(void);

/* Bytes of one packed word of `word` (8 or 4), or 0 for an invalid value. */
GFP_API size_t gfp_word_bytes(gfp_word word);

/* ------------------------------------------------------------------------ */
/* Parameters: validation and choice of (d, Q, kb)                          */
/* ------------------------------------------------------------------------ */

/* Section 1 (end) observes that p, the matrix sizes and the mantissa are
 * fixed by the problem and leave a constrained choice of Q and d; Sections
 * 2.4-2.5 give the bounds.  Host only, launches nothing, needs no GPU.
 *
 * p, m, k, n : the problem (m, n only checked for being >= 0).
 * form, word : the compressed form and machine word.
 * *d, *Q, *kb: in/out.  If *d < 0 on entry, the call CHOOSES: the smallest
 *              Q = 2^t satisfying eq. (lower) for k (or for *kb when
 *              *kb > 0 on entry), then the largest d the word admits; *kb is
 *              returned as 0 (whole k) or the k-block rounded down to a
 *              multiple of d+1.  If *d >= 0 the call VALIDATES the given
 *              (d, Q, kb) and leaves them unchanged.  kb = 0 means no
 *              k-blocking.  k-blocking is a DOT-form option: the coefficient
 *              of Q^d is extracted every kb terms and the extracted values
 *              are summed in 32 bits (needs k (p-1)^2 < 2^32).
 * Returns GFP_OK, GFP_EINVAL (null out-pointer, negative size, bad enum),
 * GFP_EPRIME, GFP_EQ, GFP_EBOUND or GFP_EUNSUPPORTED (word not offered for
 * the form). */
GFP_API gfp_status gfp_params(uint32_t p, int64_t m, int64_t k, int64_t n,
                              gfp_form form, gfp_word word,
                              int *d, uint64_t *Q, int64_t *kb);

/* Value-aware parameters (Section 2.4 with the operands' largest entries in
 * place of p-1).  The bound of eq. (lower) comes from the largest product of
 * two entries: with entries of A at most amax_a and of B at most amax_b it
 * reads k amax_a amax_b < Q (0/1 adjacency matrices: k < Q), and packed
 * words hold digits up to max(amax_a, amax_b).  A smaller Q leaves room for
 * more coefficients per word.  amax_a, amax_b <= p - 1 (gfp_params is the
 * case amax_a = amax_b = p - 1); that the entries respect them is a
 * precondition of the products made with the result, like entries < p for
 * every call (gfp_amax measures it).  Otherwise as gfp_params; additionally
 * GFP_EINVAL when amax_a or amax_b exceeds p - 1. */
GFP_API gfp_status gfp_params_vb(uint32_t p, int64_t m, int64_t k, int64_t n,
                                 gfp_form form, gfp_word word,
                                 uint32_t amax_a, uint32_t amax_b,
                                 int *d, uint64_t *Q, int64_t *kb);

/* Largest entry of a uint8 matrix X (rows x cols, leading dimension ldx
 * bytes), written to *out, a DEVICE pointer to one uint32 (0 for an empty
 * matrix).  Asynchronous on `stream`; no library counterpart in the paper:
 * it measures the amax bounds of gfp_params_vb.  Errors: GFP_EINVAL (null
 * pointer with a non-empty matrix, ldx < cols), GFP_ECUDA. */
GFP_API gfp_status gfp_amax(int64_t rows, int64_t cols, const uint8_t *X, int64_t ldx,
                            uint32_t *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Conversions (Section 2.1 INIT, Table 2 INIT_e / EXTRACT_e)                */
/* ------------------------------------------------------------------------ */

/* Pack a residue matrix X (rows x cols uint8, leading dimension ldx) into
 * words W of type `word` in layout `lay` (see gfp_layout), leading dimension
 * ldw in words.  W must hold ceil(cols/(d+1)) words per row for ROWS and
 * ROWS_REV and ceil(rows/(d+1)) rows of cols words for COLS.  Requires
 * 0 <= d, Q = 2^t with 1 <= t, and the largest word (p-1)(1+...+Q^d) to fit
 * the word (< 2^64, < 2^32, or < 2^53 for F64).  Errors: GFP_EINVAL,
 * GFP_EPRIME, GFP_EQ, GFP_EBOUND, GFP_ECUDA. */
GFP_API gfp_status gfp_pack(uint32_t p, int64_t rows, int64_t cols,
                            const uint8_t *X, int64_t ldx,
                            int d, uint64_t Q, gfp_layout lay, gfp_word word,
                            void *W, int64_t ldw, void *stream);

/* gfp_pack for entries at most amax (<= p - 1): the word bound becomes
 * amax (1+...+Q^d) and amax < Q (the parameters of gfp_params_vb). */
GFP_API gfp_status gfp_pack_vb(uint32_t p, uint32_t amax, int64_t rows, int64_t cols,
                               const uint8_t *X, int64_t ldx,
                               int d, uint64_t Q, gfp_layout lay, gfp_word word,
                               void *W, int64_t ldw, void *stream);

/* Inverse of gfp_pack: rows x cols residues X from the words W.  Every
 * coefficient of every word must be < Q (true of gfp_pack output and of the
 * MIXED form's result CC); coefficient values are written as they are
 * (they are already reduced for CC).  Errors as gfp_pack. */
GFP_API gfp_status gfp_unpack(uint32_t p, int64_t rows, int64_t cols,
                              const void *W, int64_t ldw,
                              int d, uint64_t Q, gfp_layout lay, gfp_word word,
                              uint8_t *X, int64_t ldx, void *stream);

/* ------------------------------------------------------------------------ */
/* Products                                                                  */
/* ------------------------------------------------------------------------ */

/* Bytes of workspace gfp_gemm needs for (algo, p, m, k, n); 0 when none.
 * GFP_ALGO_AUTO reports the need of the algorithm AUTO would pick. */
GFP_API gfp_status gfp_gemm_workspace_size(uint32_t p, int64_t m, int64_t k, int64_t n,
                                           gfp_algo algo, size_t *bytes);

/* C = A B mod p from uncompressed residues.  A: m x k (lda >= k), B: k x n
 * (ldb >= n), C: m x n (ldc >= n), all uint8 device memory.  C must not
 * overlap A or B.  workspace: device memory of at least the size
 * gfp_gemm_workspace_size reports (256-byte aligned), or NULL when that size
 * is 0.  The plain algorithms are the classical product against which
 * Section 2.2 measures the compressed one (whose gain is at most d+1); the
 * tensor-core algorithms are this library's exact extension.
 * Errors: GFP_EINVAL, GFP_EPRIME, GFP_EBOUND (k too large for the algorithm's
 * 32-bit sums), GFP_EWORKSPACE, GFP_EUNSUPPORTED, GFP_ECUDA. */
GFP_API gfp_status gfp_gemm(uint32_t p, int64_t m, int64_t k, int64_t n,
                            const uint8_t *A, int64_t lda,
                            const uint8_t *B, int64_t ldb,
                            uint8_t *C, int64_t ldc,
                            gfp_algo algo, void *workspace, size_t ws_bytes,
                            void *stream);

/* Size of the scratch buffer compiled into the library for gfp_gemm_noalloc. */
#define GFP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* C = A B mod p exactly as gfp_gemm(..., GFP_ALGO_TC_MMA_S8, ...), for callers
 * that cannot allocate device memory: a process with a fixed device-memory
 * budget, a framework whose allocator owns every device allocation, or a
 * latency-bound path where an allocation could synchronize the device.  They
 * cannot supply gfp_gemm's workspace, so this call allocates nothing and
 * takes no workspace; it uses a scratch array of GFP_NOALLOC_SCRATCH_BYTES
 * that the library holds on every GPU that loads it, until the process exits.
 * (No counterpart in the paper.)
 *  Arguments as gfp_gemm.  The problem must fit the scratch:
 *  (roundup(m, 128) + roundup(n, 128)) * roundup(k, 64) + 256 bytes <=
 *  GFP_NOALLOC_SCRATCH_BYTES (e.g. m = n = k = 2048); larger problems are
 *  rejected with GFP_EWORKSPACE before anything is launched.
 *  The first call on a device, with that device current, looks up the
 *  scratch's device address (one-time set-up); make that first call before
 *  any stream capture.  The address is kept with the context it was found
 *  in: after cudaDeviceReset the next call (again before any capture) looks
 *  it up anew.  Every call uses the same scratch, so calls whose
 *  kernels overlap on the GPU (other streams, other host threads) race on it
 *  and must be serialized by the caller.  Errors as gfp_gemm. */
GFP_API gfp_status gfp_gemm_noalloc(uint32_t p, int64_t m, int64_t k, int64_t n,
                                    const uint8_t *A, int64_t lda,
                                    const uint8_t *B, int64_t ldb,
                                    uint8_t *C, int64_t ldc, void *stream);

/* Compressed product.
 *  form = GFP_FORM_DOT (Section 2, procedure (2) after packing):
 *     CA_or_A : CA, m x ceil(k/(d+1)) words, layout ROWS_REV of A, lda words.
 *     CB      : ceil(k/(d+1)) x n words, layout COLS of B, ldb words.
 *     C       : m x n uint8 residues, ldc bytes:  C = A B mod p.
 *     Each entry is the coefficient of Q^d of sum_w CA[i][w] CB[w][j]
 *     (Section 2.2), reduced mod p once (Section 2.5); with kb > 0 it is
 *     extracted every kb terms (kb a multiple of d+1) and the extracted values
 *     are summed in 32 bits before the reduction.
 *  form = GFP_FORM_MIXED (Section 3, equation (LeftComp)):
 *     CA_or_A : A, m x k uint8 residues, lda bytes.
 *     CB      : k x ceil(n/(d+1)) words, layout ROWS of B, ldb words.
 *     C       : CC, m x ceil(n/(d+1)) words of type `word`, ldc words,
 *               layout ROWS of A B mod p: each word's d+1 coefficients are
 *               reduced mod p simultaneously (REDQ).  gfp_unpack(ROWS)
 *               gives the residues.  kb must be 0.
 *  form = GFP_FORM_LEFT (Table 2, left compression):
 *     CA_or_A : CA, ceil(m/(d+1)) x k words, layout COLS of A, lda words.
 *     CB      : B, k x n uint8 residues, ldb bytes.
 *     C       : CC, ceil(m/(d+1)) x n words, ldc words, layout COLS of
 *               A B mod p (coefficients reduced by REDQ).  kb must be 0.
 *  (d, Q, kb) must satisfy the bounds of gfp_params for (form, word).
 *  Errors: GFP_EINVAL, GFP_EPRIME, GFP_EQ, GFP_EBOUND, GFP_EUNSUPPORTED,
 *  GFP_ECUDA. */
GFP_API gfp_status gfp_gemm_compressed(uint32_t p, int64_t m, int64_t k, int64_t n,
                                       int d, uint64_t Q, gfp_form form, gfp_word word,
                                       const void *CA_or_A, int64_t lda,
                                       const void *CB, int64_t ldb,
                                       void *C, int64_t ldc, int64_t kb,
                                       void *stream);

/* ReduceAndCompress fused into the dot form: procedure (compC) of Section
 * 2.2, equation (1), CC = ReduceAndCompress(CA x CB), in one launch.  The
 * product is that of gfp_gemm_compressed(GFP_FORM_DOT, word) -- CA m x
 * ceil(k/(d+1)) words (ROWS_REV of A, lda words), CB ceil(k/(d+1)) x n words
 * (COLS of B, ldb words), (d, Q, kb) within the bounds of gfp_params -- and
 * its residues C = A B mod p, instead of being stored as bytes, are written
 * as reversed-row words of the same machine word (Section 2.1, missing
 * entries zero as in Section 2.3):
 *     CC[i][w] = sum_{s=0..d_out} C[i][w(d_out+1)+s] Q_out^(d_out-s),
 * m x ceil(n/(d_out+1)) words, ldcc words: the left operand (layout
 * ROWS_REV) of a further product with C on the left, e.g. the next power of
 * a chain A^l (a (d, Q) valid for every product of the chain may serve as
 * both (d, Q) and (d_out, Q_out)).  word: GFP_WORD_U64 or GFP_WORD_U32
 * (GFP_EUNSUPPORTED otherwise); (d_out, Q_out) must give words that `word`
 * holds (the rule of gfp_pack).  Nothing is allocated; one kernel launch.
 * Errors: GFP_EINVAL, GFP_EPRIME, GFP_EQ, GFP_EBOUND, GFP_EUNSUPPORTED,
 * GFP_ECUDA. */
GFP_API gfp_status gfp_gemm_compressed_compc(uint32_t p, int64_t m, int64_t k, int64_t n,
                                             int d, uint64_t Q, gfp_word word,
                                             const void *CA, int64_t lda,
                                             const void *CB, int64_t ldb, int64_t kb,
                                             int d_out, uint64_t Q_out,
                                             void *CC, int64_t ldcc, void *stream);

/* gfp_gemm_compressed with (d, Q, kb) validated against the value-aware bound
 * k amax_a amax_b < Q of gfp_params_vb (entries of A at most amax_a, of B at
 * most amax_b, a precondition).  The kernels are the same. */
GFP_API gfp_status gfp_gemm_compressed_vb(uint32_t p, int64_t m, int64_t k, int64_t n,
                                          int d, uint64_t Q, gfp_form form, gfp_word word,
                                          uint32_t amax_a, uint32_t amax_b,
                                          const void *CA_or_A, int64_t lda,
                                          const void *CB, int64_t ldb,
                                          void *C, int64_t ldc, int64_t kb,
                                          void *stream);

/* Self-test of failure detection (no counterpart in the paper).  Every wait
 * of the tcgen05 kernels (on a stage's copies, a free stage, an accumulator)
 * is bounded: when one runs out the kernel records which role gave up in a
 * status word (1 producer, 2 MMA issuer, 3 epilogue, 4 final drain), the
 * other roles stop, tensor memory is freed and the kernel returns, leaving
 * the context usable.  This call runs a 128 x 128 x 128 product whose first
 * copies are withheld, so a wait runs out after limit_ms (1 .. 10000), and
 * writes the status word to *status (host).  Workspace: >= 82,176 bytes,
 * 256-byte aligned, device.  Synchronizes the stream.  Errors: GFP_EINVAL,
 * GFP_EWORKSPACE, GFP_ECUDA. */
GFP_API gfp_status gfp_selftest_wait_limit(void *workspace, size_t ws_bytes, uint32_t limit_ms, int *status,
                                           void *stream);

/* Measured instruction rates of this GPU (no counterpart in the paper): the
 * ceilings against which the CUDA-core forms are reported.  rates[i]
 * receives operations per second of, in order: 0 the 32-bit multiply-add
 * (mad.lo.u32), 1 the widening 32 x 32 -> 64-bit multiply-add
 * (mad.wide.u32), 2 the 64-bit multiply-add keeping the low 64 bits
 * (mad.lo.u64 of full 64-bit operands, one step of the dot form in 64-bit
 * words), 3 the four-byte
 * dot product (dp4a), 4 the double-precision fused multiply-add (fma.rn.f64),
 * 5 the int8 warp MMA (mma.sync m16n8k32 s8, counted as 2 x 16 x 8 x 32
 * operations each); and, in flops per second, the dense rates of the
 * tcgen05 MMA kinds the tensor-core forms use -- 6 kind::f16 (fp16),
 * 7 kind::f8f6f4 (e4m3), 8 the block-scaled kind::mxf4 (e2m1, ue8m0 scale
 * factors per 32 values), 9 kind::mxf4nvf4 (e2m1, ue4m3 scale factors per 16
 * values) -- each measured with 128 x 256 MMAs issued back to back by one
 * thread per SM from fixed tiles in shared memory -- and 10, 11, 12 the
 * kinds of 6, 7, 8 on CTA pairs (256 x 256 MMAs, cta_group::2); 0 where a
 * bounded wait ran out.  The first min(n_rates, 13) are written.  Each is 8 independent chains of
 * the instruction per thread on 4 CTAs of 256 threads per SM, best of three
 * timed runs.  workspace: >= 256 bytes of device memory, 256-byte aligned
 * (a sink for the chains' values and a status word).  Synchronizes the
 * stream; takes about 0.1 s.  Errors: GFP_EINVAL, GFP_EWORKSPACE, GFP_ECUDA. */
GFP_API gfp_status gfp_pipe_rates(double *rates, int n_rates, void *workspace, size_t ws_bytes, void *stream);

/* Autotuner of the dot form for one product (no counterpart in the paper,
 * which fixes the word): a smaller Q -- the bound of eq. (lower) applied to
 * a k-block kb -- leaves room for more coefficients per word at the price of
 * an extraction every kb terms, and 32-bit words cost one multiply-add where
 * 64-bit words cost about three.  The admissible (word in U32, U32W, U64;
 * d, Q, kb) with no blocking and, for each Q = 2^t, the longest k-block
 * eq. (lower) allows -- per (word, d) the longest k-block, no
 * blocking counting as the longest -- are timed with
 * CUDA events on the proxy shape min(m, 2048) x k x min(n, 2048) with zero
 * operands in the caller's workspace (gfp_dot_autotune_workspace_size bytes,
 * 256-byte aligned; its contents are overwritten); *best receives the
 * fastest, all[0 .. min(*n_all, max_all)) every candidate with its median
 * time.  Waits for its timings: not capturable in a CUDA graph.  The choice
 * is valid for (p, m, k, n): pass it to gfp_pack and gfp_gemm_compressed.
 * Errors: GFP_EINVAL, GFP_EPRIME, GFP_EBOUND (no word admits k),
 * GFP_EWORKSPACE, GFP_ECUDA. */
typedef struct gfp_dot_choice {
    int32_t word;        /* gfp_word */
    int32_t d;
    uint64_t Q;
    int64_t kb;          /* 0: no k-blocking */
    float ms;            /* median of three timed runs on the proxy shape */
    int32_t reserved;
} gfp_dot_choice;

GFP_API gfp_status gfp_dot_autotune_workspace_size(int64_t m, int64_t k, int64_t n, size_t *bytes);
GFP_API gfp_status gfp_dot_autotune(uint32_t p, int64_t m, int64_t k, int64_t n,
                                    void *workspace, size_t ws_bytes, void *stream,
                                    gfp_dot_choice *best, gfp_dot_choice *all, int max_all,
                                    int *n_all);

/* Strassen-Winograd over the packed words of the dot form (the paper's
 * remark on fast matrix multiplication, Section 5).  With 64-bit words
 * (t(d+1) <= 64) the coefficient of Q^d is exact modulo 2^64, so only the
 * word product mod 2^64 matters, and Winograd's 7-multiplication scheme is
 * an identity over the ring Z/2^64: `levels` levels of it (stopping early
 * once a side falls below 512 words) on the words, with wrapping additions,
 * give the classical product's words and digits exactly.  Operands as
 * gfp_gemm_compressed(GFP_FORM_DOT, GFP_WORD_U64): CA m x ceil(k/(d+1))
 * words (ROWS_REV of A, lda words), CB ceil(k/(d+1)) x n words (COLS of B,
 * ldb words), C m x n uint8 (ldc bytes).  (d, Q) must satisfy the bounds of
 * gfp_params for (DOT, U64) without k-blocking.  The workspace (device,
 * caller-owned, gfp_winograd_workspace_size bytes) holds the m x n result
 * words and each level's sums and products; nothing is allocated, so the
 * call can be captured in a CUDA graph.  levels = 0 is the classical word
 * product with one digit pass.  Errors: GFP_EINVAL, GFP_EPRIME, GFP_EQ,
 * GFP_EBOUND, GFP_EWORKSPACE, GFP_ECUDA. */
GFP_API gfp_status gfp_winograd_workspace_size(int64_t m, int64_t k, int64_t n, int d, int levels,
                                               size_t *bytes);
GFP_API gfp_status gfp_gemm_compressed_winograd(uint32_t p, int64_t m, int64_t k, int64_t n,
                                                int d, uint64_t Q,
                                                const void *CA, int64_t lda,
                                                const void *CB, int64_t ldb,
                                                uint8_t *C, int64_t ldc, int levels,
                                                void *workspace, size_t ws_bytes,
                                                void *stream);

/* Full compression (Section 4): both outer dimensions packed.  With
 * Theta = Q^(dq+1) (the smallest Theta of eq. (qtheta)):
 *  CA : ceil(m/(dq+1)) x k words, layout COLS of A in base Q (degree dq),
 *       lda words (gfp_pack(..., d = dq, Q, GFP_LAYOUT_COLS, ...));
 *  CB : k x ceil(n/(dth+1)) words, layout ROWS of B in base Theta (degree
 *       dth), ldb words (gfp_pack(..., d = dth, Theta, GFP_LAYOUT_ROWS, ...));
 *  CC : ceil(m/(dq+1)) x ceil(n/(dth+1)) words, ldc words: word (u, v) holds
 *       C[u(dq+1)+i][v(dth+1)+j] mod p as its coefficient of Q^i Theta^j
 *       (gfp_unpack_block gives the residues).
 * Word products keep every coefficient, so the whole sum must fit the word:
 * eq. (lower) for Q and Q^((dq+1)(dth+1)) <= 2^64 (uint64, eq. (dq) with
 * beta = 64) or < 2^53 (binary64).  Words: GFP_WORD_U64 and GFP_WORD_F64.
 * Errors as gfp_gemm_compressed. */
GFP_API gfp_status gfp_gemm_full(uint32_t p, int64_t m, int64_t k, int64_t n, int dq, int dth,
                                 uint64_t Q, gfp_word word, const void *CA, int64_t lda,
                                 const void *CB, int64_t ldb, void *CC, int64_t ldc, void *stream);

/* Choose (*dq < 0 on entry) or validate (*dq >= 0) the parameters of
 * gfp_gemm_full: the smallest Q of eq. (lower), then the split with the most
 * coefficients per word, the most balanced one among equals.  Host only. */
GFP_API gfp_status gfp_params_full(uint32_t p, int64_t m, int64_t k, int64_t n, gfp_word word,
                                   int *dq, int *dth, uint64_t *Q);

/* The block layout of gfp_gemm_full's result for a residue matrix X (rows x
 * cols): W[u][v] = sum_{i<=dq} sum_{j<=dth} X[u(dq+1)+i][v(dth+1)+j]
 * Q^(i + j(dq+1)), entries past the edge zero; ceil(rows/(dq+1)) x
 * ceil(cols/(dth+1)) words, ldw words.  Requires Q > p - 1 and the word
 * bound of gfp_gemm_full.  Errors as gfp_pack. */
GFP_API gfp_status gfp_pack_block(uint32_t p, int64_t rows, int64_t cols, const uint8_t *X,
                                  int64_t ldx, int dq, int dth, uint64_t Q, gfp_word word, void *W,
                                  int64_t ldw, void *stream);
GFP_API gfp_status gfp_unpack_block(uint32_t p, int64_t rows, int64_t cols, const void *W,
                                    int64_t ldw, int dq, int dth, uint64_t Q, gfp_word word,
                                    uint8_t *X, int64_t ldx, void *stream);

/* One product of a batch: C = A B mod p with A m x k, B k x n, C m x n uint8
 * row-major device matrices.  (The batched workload of this library squares
 * adjacency matrices: A == B, m == k == n.)
 * flags: 0, or GFP_PROBLEM_B_IS_A_T when the caller knows that B equals the
 * transpose of A (n == m, B[l][j] == A[j][l]; e.g. B = A with A symmetric,
 * the square of an undirected graph's adjacency matrix).  The tensor-core
 * tiles then stage one copy of A and read it for both operands, with no
 * transpose, and since C = A A^T is symmetric they compute only the 128 x 128
 * tiles on and above the diagonal, writing each one above it twice (as
 * itself and transposed).  The flag is a precondition, not checked: if B is
 * not A^T the result is that of A A^T.  Any other bit: GFP_EINVAL. */
#define GFP_PROBLEM_B_IS_A_T 1
typedef struct gfp_problem {
    uint32_t p;
    int32_t m, k, n;
    const uint8_t *A;
    const uint8_t *B;
    uint8_t *C;
    int32_t lda, ldb, ldc;
    int32_t flags;
} gfp_problem;

/* Bytes of workspace gfp_gemm_batched needs for `count` problems. */
GFP_API gfp_status gfp_batched_workspace_size(int64_t count, const gfp_problem *probs,
                                              size_t *bytes);

/* Thousands of independent products of uneven sizes in one persistent
 * grouped launch (no counterpart in the paper; the workload is the
 * strongly-regular-graph computations of Section 1).
 *  probs       : HOST array of `count` problems; each is validated on the host.
 *  algo        : GFP_ALGO_AUTO   -- per size bucket (the largest of m, k, n),
 *                                   the tile kind gfp_batched_autotune chose;
 *                                   untuned buckets use the tcgen05 tiles
 *                                   (GFP_ALGO_TC_F8 below);
 *                GFP_ALGO_TC_F16 -- warp-level fp16 tensor-core MMA tiles
 *                                   (128 x 128 above m, n = 160, 64 x 64,
 *                                   32 x 32 for m, n <= 48) on
 *                                   centred residues, fp32 accumulation kept
 *                                   exact by k-blocks (kb h^2 + p < 2^24);
 *                GFP_ALGO_DOT32  -- the Q-adic dot form (Section 2) in 32-bit
 *                                   words, residues packed while staged, with
 *                                   (Q, d, k-block) chosen per problem;
 *                GFP_ALGO_TC_F8  -- tcgen05 128 x 128 tiles of a second
 *                                   grouped kernel: for p < 16 residue bytes
 *                                   read as e4m3 codes of r 2^-9 (exact while
 *                                   k (p-1)^2 < 2^24), for larger p centred
 *                                   fp16 (exact while k h^2 + p < 2^24, k <=
 *                                   32768); problems beyond those bounds fall
 *                                   back to the fp16 MMA tiles.
 *  status      : optional HOST array of `count` per-problem statuses.  A
 *                problem that fails validation is skipped (its C untouched)
 *                and the call returns the first failing status after
 *                launching the valid ones.
 *  workspace   : device memory of gfp_batched_workspace_size bytes (256-byte
 *                aligned).  It receives the schedule: problem table, tiles,
 *                and each CTA's range of tiles, balanced on the host
 *                (longest tile first onto the least loaded CTA).
 * Bytes 192 .. 195 of the workspace hold, once a launch's kernels complete,
 * the status of its bounded internal waits: 0, or non-zero if one gave up
 * (1-4 the tcgen05 tiles' roles, 6 an operand copy of the conversion; the
 * results are then invalid).
 * gfp_gemm_batched = gfp_batched_prepare + gfp_batched_launch.
 * gfp_batched_prepare writes the schedule with one host-to-device copy and
 * synchronizes `stream` (run it outside stream capture).  gfp_batched_launch
 * launches, on the prepared workspace, the operand conversion and the grouped
 * kernels the schedule uses (the mma.sync tiles, the tcgen05 tiles); it
 * allocates nothing and does not synchronize, so it can be captured in a CUDA
 * graph and replayed while the workspace and matrices stay in place.  Both
 * must run on the same device. */
GFP_API gfp_status gfp_gemm_batched(int64_t count, const gfp_problem *probs, gfp_algo algo,
                                    gfp_status *status, void *workspace, size_t ws_bytes,
                                    void *stream);

GFP_API gfp_status gfp_batched_prepare(int64_t count, const gfp_problem *probs, gfp_algo algo,
                                       gfp_status *status, void *workspace, size_t ws_bytes,
                                       void *stream);

GFP_API gfp_status gfp_batched_launch(void *workspace, size_t ws_bytes, void *stream);

/* Autotuner of the batched launch: for each size bucket present in `probs`
 * (largest of m, k, n in (0,32], (32,64], (64,128], (128,256], (256,512],
 * (512,2048], above) it times one grouped launch of that bucket's problems
 * with each tile kind (0 = fp16 MMA 64 x 64, 1 = fp16 MMA 32 x 32, 2 = Q-adic
 * 32-bit words with per-problem Q and d, 3 = fp16 MMA 128 x 128, 4 = tcgen05
 * 128 x 128, e4m3 for p < 16, fp16 above) and keeps the fastest; then it times the whole
 * batch with that table, with the default kinds (table -1) and with the
 * tcgen05 kind in every bucket (where it applies), and keeps the fastest
 * table -- mixing engines adds a grouped kernel that buckets timed alone do
 * not see.  The choice is stored in the library (used by GFP_ALGO_AUTO from
 * then on, process wide) and, if `table` is not NULL, written to
 * table[0 .. table_len) (-1: the default kind, or no problems).  It writes the problems' C matrices and uses
 * `workspace` (gfp_batched_workspace_size bytes); it synchronizes `stream`. */
GFP_API gfp_status gfp_batched_autotune(int64_t count, const gfp_problem *probs, void *workspace,
                                        size_t ws_bytes, void *stream, int *table, int table_len);

/* Install a tile-kind table (as written by gfp_batched_autotune, e.g. from a
 * cache file); -1 entries fall back to the default.  Host only. */
GFP_API gfp_status gfp_batched_set_table(const int *table, int table_len);

#ifdef __cplusplus
}
#endif

#endif /* GFP_H */
