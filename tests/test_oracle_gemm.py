"""Pins of the oracle's product C = A B mod p against things other than itself:
the paper's printed 2x2 example, a library matrix product, brute force and
the algebraic identities every matrix product over a field satisfies."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_examples():
    out = {}
    with open(os.path.join(GOLDEN, "worked_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, expr = line.split("=", 1)
            out[name.strip()] = expr.strip()
    return out


def test_worked_example_2x2_exhaustive_mod3():
    """Section 2.2 prints A B for the 2x2 matrices [[a,b],[c,d]], [[e,f],[g,h]];
    check the oracle on all 3^8 instances over F_3."""
    ex = load_examples()
    As, Bs, Cs = [], [], []
    for vals in itertools.product(range(3), repeat=8):
        env = dict(zip("abcdefgh", vals))
        As.append(eval(ex["A"], {}, env))
        Bs.append(eval(ex["B"], {}, env))
        Cs.append(eval(ex["C"], {}, env))
    for a, b, c in zip(As, Bs, Cs):
        C = oracle.gemm(3, np.asarray(a, np.uint8), np.asarray(b, np.uint8))
        assert (C == np.asarray(c) % 3).all()


@pytest.mark.parametrize("p,m,k,n", [(3, 17, 33, 9), (5, 64, 100, 31), (251, 20, 300, 40),
                                      (2, 5, 1, 7), (7, 1, 129, 1), (31, 33, 64, 65)])
def test_matches_numpy_int64(p, m, k, n):
    """numpy's int64 matrix product is exact here (k (p-1)^2 < 2^63), so
    (A @ B) % p is an independent value of the definition."""
    g = inputs.rng(90, p + m + k + n)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    ref = (A.astype(np.int64) @ B.astype(np.int64)) % p
    assert (oracle.gemm(p, A, B) == ref).all()
    assert (oracle.gemm(p, A, B, threads=4) == ref).all()


def test_brute_force_dot_products():
    """1 x k times k x 1: a plain Python sum of products."""
    g = inputs.rng(91, 0)
    for p in (2, 3, 5, 13, 251):
        for k in (1, 2, 3, 7, 64, 1000):
            a = inputs.residues(g, p, 1, k)
            b = inputs.residues(g, p, k, 1)
            s = sum(int(x) * int(y) for x, y in zip(a[0], b[:, 0])) % p
            assert int(oracle.gemm(p, a, b)[0, 0]) == s


def test_brute_force_3x3_mod2_exhaustive_rows():
    """All 2^9 matrices A over F_2 times a fixed B, entry by entry."""
    B = np.array([[1, 0, 1], [1, 1, 0], [0, 1, 1]], dtype=np.uint8)
    for bits in range(2 ** 9):
        A = np.array([(bits >> s) & 1 for s in range(9)], dtype=np.uint8).reshape(3, 3)
        C = oracle.gemm(2, A, B)
        for i in range(3):
            for j in range(3):
                assert C[i, j] == sum(int(A[i, l]) * int(B[l, j]) for l in range(3)) % 2


@pytest.mark.parametrize("p", [3, 5, 251])
def test_identities(p):
    g = inputs.rng(92, p)
    n = 24
    A = inputs.residues(g, p, n, 19)
    B = inputs.residues(g, p, 19, 23)
    Cm = inputs.residues(g, p, 23, 11)
    B2 = inputs.residues(g, p, 19, 23)
    I = np.eye(19, dtype=np.uint8)
    assert (oracle.gemm(p, A, I) == A).all()                       # A I = A
    assert (oracle.gemm(p, np.eye(n, dtype=np.uint8), A) == A).all()
    AB = oracle.gemm(p, A, B)
    assert (oracle.gemm(p, AB, Cm) == oracle.gemm(p, A, oracle.gemm(p, B, Cm))).all()  # (AB)C = A(BC)
    S = ((B.astype(np.int64) + B2) % p).astype(np.uint8)
    lhs = oracle.gemm(p, A, S)
    rhs = (oracle.gemm(p, A, B).astype(np.int64) + oracle.gemm(p, A, B2)) % p
    assert (lhs == rhs).all()                                      # A(B+B2) = AB + AB2
    assert (oracle.gemm(p, np.ascontiguousarray(B.T), np.ascontiguousarray(A.T)) == AB.T).all()
    Z = np.zeros((19, 23), dtype=np.uint8)
    assert (oracle.gemm(p, A, Z) == 0).all()


def test_rows_variant_matches_full():
    g = inputs.rng(93, 0)
    A = inputs.residues(g, 7, 40, 70)
    B = inputs.residues(g, 7, 70, 50)
    full = oracle.gemm(7, A, B)
    rows = [0, 3, 39, 17]
    assert (oracle.gemm_rows(7, rows, A, B) == full[rows]).all()


def test_empty_shapes():
    A = np.zeros((0, 5), np.uint8)
    B = np.zeros((5, 3), np.uint8)
    assert oracle.gemm(3, A, B).shape == (0, 3)
    A = np.zeros((4, 0), np.uint8)
    B = np.zeros((0, 3), np.uint8)
    assert (oracle.gemm(3, A, B) == 0).all()


def test_planted_mistake_is_caught():
    """A dropped term (here: the last l of each dot product) must be visible to
    the numpy pin; this guards the pin itself."""
    g = inputs.rng(94, 0)
    A = inputs.residues(g, 3, 8, 9)
    B = inputs.residues(g, 3, 9, 8)
    wrong = (A[:, :-1].astype(np.int64) @ B[:-1].astype(np.int64)) % 3
    assert not (oracle.gemm(3, A, B) == wrong).all()


# ---------------------------------------------------------------------------
# gemm_matmul: the definition with the sum formed by a binary64 matrix product
# ---------------------------------------------------------------------------
def test_matmul_form_worked_example_2x2_exhaustive_mod3():
    """Section 2.2's 2x2 example over all 3^8 instances, as for the triple loop."""
    ex = load_examples()
    for vals in itertools.product(range(3), repeat=8):
        env = dict(zip("abcdefgh", vals))
        a = np.asarray(eval(ex["A"], {}, env), np.uint8)
        b = np.asarray(eval(ex["B"], {}, env), np.uint8)
        c = np.asarray(eval(ex["C"], {}, env)) % 3
        assert (oracle.gemm_matmul(3, a, b) == c).all()


@pytest.mark.parametrize("p,m,k,n", [(3, 17, 33, 9), (5, 64, 100, 31), (251, 20, 3000, 40),
                                      (2, 5, 1, 7), (7, 1, 129, 1), (31, 133, 640, 65)])
def test_matmul_form_matches_triple_loop(p, m, k, n):
    g = inputs.rng(95, p + m + k + n)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    assert (oracle.gemm_matmul(p, A, B) == oracle.gemm(p, A, B, threads=4)).all()


def test_matmul_form_largest_sums_exact():
    """All entries p - 1 = 250 with k = 8192: every dot product is
    8192 * 250^2 = 512,000,000; its residue is computed with Python integers."""
    p, k = 251, 8192
    A = np.full((3, k), p - 1, np.uint8)
    B = np.full((k, 5), p - 1, np.uint8)
    assert (oracle.gemm_matmul(p, A, B) == (k * (p - 1) ** 2) % p).all()
    assert (oracle.gemm_rows(p, [0, 2], A, B) == (k * (p - 1) ** 2) % p).all()


def test_matmul_form_rejects_inexact_sizes():
    """k (p-1)^2 >= 2^53 is refused (zero-sized operands: nothing is allocated)."""
    k = -(-2 ** 53 // 250 ** 2)
    with pytest.raises(ValueError):
        oracle.gemm_matmul(251, np.zeros((0, k), np.uint8), np.zeros((k, 0), np.uint8))
    k -= 1
    assert oracle.gemm_matmul(251, np.zeros((0, k), np.uint8), np.zeros((k, 0), np.uint8)).shape == (0, 0)


def test_matmul_form_planted_mistake_is_caught():
    """A dropped term changes the matmul form's result; the comparison with
    the triple loop sees it."""
    g = inputs.rng(96, 0)
    A = inputs.residues(g, 5, 30, 40)
    B = inputs.residues(g, 5, 40, 20)
    wrong = oracle.gemm_matmul(5, A[:, :-1], B[:-1])
    assert not (wrong == oracle.gemm(5, A, B)).all()
