"""The Strassen-Winograd schedule of the compressed dot form, checked on the
CPU with exact integers: one and two levels over Z/2^64, with the blocks split
at ceil(dim / 2), the missing entries of the shorter blocks taken as 0 and the
products that involve an original block run over its exact extent (the
convention of csrc/winograd.cu), equal the word product mod 2^64 -- for odd
and even sizes.  This pins the scheme the GPU path implements to the plain
definition; the GPU parity tests compare the digits with the oracle."""
import numpy as np
import pytest

M64 = 2 ** 64


def classical(A, B):
    return [[sum(A[i][l] * B[l][j] for l in range(len(B))) % M64 for j in range(len(B[0]) if B else 0)]
            for i in range(len(A))]


def block(X, r0, r1, c0, c1):
    return [row[c0:c1] for row in X[r0:r1]]


def padded(X, rows, cols):
    out = [[0] * cols for _ in range(rows)]
    for i, row in enumerate(X[:rows]):
        for j, v in enumerate(row[:cols]):
            out[i][j] = v
    return out


def ew(f, *Xs):
    return [[f(*vals) % M64 for vals in zip(*rows)] for rows in zip(*Xs)]


def winograd(A, B, levels):
    M, K, N = len(A), len(B), len(B[0])
    if levels == 0 or min(M, K, N) < 2:
        return classical(A, B)
    m1, k1, n1 = (M + 1) // 2, (K + 1) // 2, (N + 1) // 2
    A11, A12 = block(A, 0, m1, 0, k1), block(A, 0, m1, k1, K)
    A21, A22 = block(A, m1, M, 0, k1), block(A, m1, M, k1, K)
    B11, B12 = block(B, 0, k1, 0, n1), block(B, 0, k1, n1, N)
    B21, B22 = block(B, k1, K, 0, n1), block(B, k1, K, n1, N)
    a12, a21, a22 = padded(A12, m1, k1), padded(A21, m1, k1), padded(A22, m1, k1)
    b12, b21, b22 = padded(B12, k1, n1), padded(B21, k1, n1), padded(B22, k1, n1)
    S1 = ew(lambda x, y: x + y, a21, a22)
    S2 = ew(lambda x, y: x - y, S1, A11)
    S3 = ew(lambda x, y: x - y, A11, a21)
    S4 = ew(lambda x, y: x - y, a12, S2)
    T1 = ew(lambda x, y: x - y, b12, B11)
    T2 = ew(lambda x, y: x - y, b22, T1)
    T3 = ew(lambda x, y: x - y, b22, b12)
    T4 = ew(lambda x, y: x - y, T2, b21)
    k2, m2, n2 = K - k1, M - m1, N - n1
    P1 = winograd(A11, B11, levels - 1)
    P2 = winograd(A12, B21, levels - 1) if k2 else [[0] * n1 for _ in range(m1)]
    P3 = winograd([r[:k2] for r in S4], B22, levels - 1) if k2 and n2 else None
    P4 = winograd(A22, T4[:k2], levels - 1) if k2 and m2 else None
    P5 = winograd(S1, T1, levels - 1)
    P6 = winograd(S2, T2, levels - 1)
    P7 = winograd(S3, T3, levels - 1)
    C = [[0] * N for _ in range(M)]
    for i in range(m1):
        for j in range(n1):
            u2 = (P1[i][j] + P6[i][j]) % M64
            u3 = (u2 + P7[i][j]) % M64
            C[i][j] = (P1[i][j] + P2[i][j]) % M64
            if j < n2:
                C[i][n1 + j] = (u2 + P5[i][j] + P3[i][j]) % M64
            if i < m2:
                C[m1 + i][j] = (u3 - P4[i][j]) % M64
            if i < m2 and j < n2:
                C[m1 + i][n1 + j] = (u3 + P5[i][j]) % M64
    return C


@pytest.mark.parametrize("m,k,n,levels", [(4, 4, 4, 1), (5, 7, 3, 1), (9, 6, 11, 2), (8, 8, 8, 2), (7, 5, 9, 3)])
def test_winograd_schedule_equals_word_product_mod_2_64(m, k, n, levels):
    g = np.random.Generator(np.random.PCG64(m * 100 + k * 10 + n))
    A = [[int(x) for x in row] for row in g.integers(0, 2 ** 63, (m, k), dtype=np.uint64) * 2 + 1]
    B = [[int(x) for x in row] for row in g.integers(0, 2 ** 63, (k, n), dtype=np.uint64)]
    assert winograd(A, B, levels) == classical(A, B)
