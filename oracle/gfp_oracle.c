/*
 * Oracle for exact matrix multiplication over the prime field Z/pZ.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the GPU results with the plain
 * definition.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Section 1-2 of Dumas, Fousse, Salvy, "Compressed Modular
 * Matrix Multiplication"): every algorithm of the paper, compressed or not,
 * must return the classical product
 *
 *     C[i][j] = ( sum_{l=0}^{k-1} A[i][l] * B[l][j] ) mod p,
 *
 * with all residues in the positive representation [0, p) (Section 2.4).
 * The sum is formed exactly in a 64-bit unsigned accumulator: every entry
 * is < p <= 256, so k (p-1)^2 < 2^64 holds for any k below 2^48, and the
 * single reduction at the end is the definition itself.  Loops run in the
 * order of the definition (i, j, then l); the only concession to run time
 * is an OpenMP split of the independent rows i.
 */
#include <stdint.h>

/* Plain C = A*B mod p, all matrices row-major with leading dimensions in
 * elements.  A is m x k, B is k x n, C is m x n.  threads <= 0 means 1. */
void oracle_gemm_modp(uint32_t p, int64_t m, int64_t k, int64_t n,
                      const uint8_t *A, int64_t lda,
                      const uint8_t *B, int64_t ldb,
                      uint8_t *C, int64_t ldc, int threads)
{
    if (threads <= 0) threads = 1;
    #pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            uint64_t acc = 0;
            for (int64_t l = 0; l < k; ++l)
                acc += (uint64_t)A[i * lda + l] * (uint64_t)B[l * ldb + j];
            C[i * ldc + j] = (uint8_t)(acc % p);
        }
    }
}

/* The same definition for a chosen subset of rows: out[r][j] = C[rows[r]][j].
 * Used where the full product is too large to form on the host. */
void oracle_gemm_rows_modp(uint32_t p, int64_t nrows, const int64_t *rows,
                           int64_t k, int64_t n,
                           const uint8_t *A, int64_t lda,
                           const uint8_t *B, int64_t ldb,
                           uint8_t *out, int64_t ldo, int threads)
{
    if (threads <= 0) threads = 1;
    #pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        for (int64_t j = 0; j < n; ++j) {
            uint64_t acc = 0;
            for (int64_t l = 0; l < k; ++l)
                acc += (uint64_t)A[i * lda + l] * (uint64_t)B[l * ldb + j];
            out[r * ldo + j] = (uint8_t)(acc % p);
        }
    }
}
