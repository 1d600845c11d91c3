"""Pins of the oracle's Q-adic packing, bounds and word-level emulation
against the paper's worked examples, Table 1, closed forms (byte order of
Q = 256 words) and exhaustive or worst-case emulation."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def examples():
    out = {}
    with open(os.path.join(GOLDEN, "worked_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=", 1)
                out[k.strip()] = v.strip()
    return out


EX = examples()


def _instances(p):
    for vals in itertools.product(range(p), repeat=8):
        yield dict(zip("abcdefgh", vals))


@pytest.mark.parametrize("t", [3, 4, 6])
def test_dot_form_worked_example_words_and_digits(t):
    """Section 2.2: rows of A become Qa+b, Qc+d; columns of B become e+Qg,
    f+Qh; the coefficient of Q in each word product is the dot product.
    Exhaustive over F_3^8 (k = 2, so (lower) needs Q > 8)."""
    Q = 2 ** t
    for env in _instances(3):
        env["Q"] = Q
        A = np.asarray(eval(EX["A"], {}, env), np.uint8)
        B = np.asarray(eval(EX["B"], {}, env), np.uint8)
        CA = eval(EX["CA"], {}, env)
        CB = eval(EX["CB"], {}, env)
        dig = eval(EX["DIGIT1"], {}, env)
        assert [int(x) for x in oracle.pack_rows_rev(A, 1, Q)[:, 0]] == CA
        assert [int(x) for x in oracle.pack_cols(B, 1, Q)[0, :]] == CB
        for i in range(2):
            for j in range(2):
                if oracle.lower_bound_holds(3, 2, Q):
                    assert (CA[i] * CB[j] // Q) % Q == dig[i][j]
                    assert oracle.dqt_dot(A[i], B[:, j], 3, 1, Q) == dig[i][j] % 3


def test_right_compressed_worked_example():
    """Section 3: B packed along rows as e+Qf, g+Qh; A times it gives
    (ae+bg) + Q(af+bh) per row.  Exhaustive over F_3^8 with Q = 16."""
    Q = 16
    for env in _instances(3):
        env["Q"] = Q
        A = np.asarray(eval(EX["A"], {}, env), np.uint8)
        B = np.asarray(eval(EX["B"], {}, env), np.uint8)
        CBR = eval(EX["CBR"], {}, env)
        CC = eval(EX["CC"], {}, env)
        assert [int(x) for x in oracle.pack_rows(B, 1, Q)[:, 0]] == CBR
        for i in range(2):
            assert sum(int(A[i, l]) * CBR[l] for l in range(2)) == CC[i]
            assert oracle.mixed_word(A[i], CBR, 3, 1, Q) == [(CC[i] // Q ** j) % Q % 3 for j in range(2)]


def test_full_compression_worked_example():
    """Section 4: [a+Qc, b+Qd] x [e+Theta f; g+Theta h] expands to the four
    dot products at 1, Q, Theta, Q Theta.  Theta = Q^2 (eq. qtheta, d_q = 1)."""
    Q = 16
    Theta = Q ** 2
    assert oracle.full_bounds_hold(3, 2, Q, 1, Theta, 1)
    for env in _instances(3):
        env.update(Q=Q, Theta=Theta)
        FA = eval(EX["FA"], {}, env)
        FB = eval(EX["FB"], {}, env)
        FULL = eval(EX["FULL"], {}, env)
        assert oracle.full_word(FA, FB, Q, Theta) == FULL
        # each of the four coefficients is recoverable (all < Q)
        digits = [(FULL // Theta ** jt // Q ** iq) % Q for jt in range(2) for iq in range(2)]
        C = eval(EX["C"], {}, env)
        assert digits == [C[0][0], C[1][0], C[0][1], C[1][1]]


def test_init3_horner_semantics():
    """Section 2.1's init3 builds a double by Horner's rule r = u; r = rQ+v;
    r = rQ+w.  For a block (u, v, w) this is the reversed word of pack_rows_rev
    with d = 2 (u gets Q^2), and the forward word of pack_cols for (w, v, u)."""
    g = inputs.rng(95, 0)
    for t in (5, 10, 17):
        Q = 2 ** t
        X = inputs.residues(g, 31, 50, 3)
        W = oracle.pack_rows_rev(X, 2, Q, dtype=np.float64)
        for i in range(50):
            r = float(X[i, 0])
            r *= Q
            r += float(X[i, 1])
            r *= Q
            r += float(X[i, 2])
            assert W[i, 0] == r
        Wc = oracle.pack_cols(np.ascontiguousarray(X[:, ::-1].T), 2, Q, dtype=np.float64)
        assert (Wc[0] == W[:, 0]).all()


def test_byte_order_closed_form():
    """With Q = 256 a word is a byte string: the reversed row word of 8 entries
    is their big-endian integer, the forward column/row word little-endian."""
    g = inputs.rng(95, 1)
    X = inputs.residues(g, 251, 6, 16)
    Wr = oracle.pack_rows_rev(X, 7, 256)
    Wf = oracle.pack_rows(X, 7, 256)
    Wc = oracle.pack_cols(np.ascontiguousarray(X.T), 7, 256)
    for i in range(6):
        for w in range(2):
            blk = bytes(X[i, 8 * w:8 * w + 8].tolist())
            assert int(Wr[i, w]) == int.from_bytes(blk, "big")
            assert int(Wf[i, w]) == int.from_bytes(blk, "little")
            assert int(Wc[w, i]) == int.from_bytes(blk, "little")


def test_partial_compression_tail():
    """Section 2.3: a short last block is zero padded; for the reversed word
    that multiplies the word of the remaining r entries by Q^(d+1-r)."""
    Q = 2 ** 7
    d = 2
    X = np.array([[1, 2, 0, 2, 1]], np.uint8)          # blocks (1,2,0), (2,1)
    W = oracle.pack_rows_rev(X, d, Q)
    assert int(W[0, 1]) == (2 * Q + 1) * Q ** (d + 1 - 2)
    Wc = oracle.pack_cols(np.ascontiguousarray(X.T), d, Q)
    assert int(Wc[1, 0]) == 2 + 1 * Q


@pytest.mark.parametrize("dtype", [np.uint64, np.float64])
@pytest.mark.parametrize("rows,cols,d,t", [(5, 13, 3, 13), (4, 12, 4, 10), (1, 1, 0, 3),
                                           (7, 9, 2, 17), (3, 64, 6, 7)])
def test_round_trip(dtype, rows, cols, d, t):
    Q = 2 ** t
    if dtype is np.float64 and not oracle.upper_bound_holds(Q, d):
        pytest.skip("word exceeds the mantissa")
    g = inputs.rng(96, rows * cols + d)
    X = inputs.residues(g, 3, rows, cols)
    assert (oracle.unpack_rows_rev(oracle.pack_rows_rev(X, d, Q, dtype), cols, d, Q) == X).all()
    assert (oracle.unpack_rows(oracle.pack_rows(X, d, Q, dtype), cols, d, Q) == X).all()
    Xt = np.ascontiguousarray(X.T)
    assert (oracle.unpack_cols(oracle.pack_cols(Xt, d, Q, dtype), cols, d, Q) == Xt).all()


def read_table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_mod3.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#") or line.startswith("t "):
                continue
            rows.append(line.split())
    return rows


def test_table1():
    """Table 1 (Section 2.6): for p = 3, beta = 53, Q = 2^t the compression
    e = floor(53/t), the degree d = e - 1, and the printed dimension equals
    Q/(p-1)^2.  Under the strict eq. (lower) the largest k is one less than
    the printed dimension (the table prints <=)."""
    for t, comp, d, dims in read_table1():
        r = oracle.table1_row(int(t))
        assert r["Q"] == 2 ** int(t)
        if comp != "?":
            assert r["e"] == int(comp)
        if d != "?":
            assert r["d"] == int(d)
        assert int(dims) == r["Q"] // 4
        assert r["kmax"] == int(dims) - 1
        assert oracle.lower_bound_holds(3, r["kmax"], r["Q"])
        assert not oracle.lower_bound_holds(3, int(dims), r["Q"])
        assert oracle.upper_bound_holds(r["Q"], r["d"]) and not oracle.upper_bound_holds(r["Q"], r["d"] + 1)


def test_size_regimes_narrative():
    """Section 2.6 text: below n = 256 the factor is 5, from there to 2048 it
    is 4, then 3 (p = 3, FP64).  With the strict bound the switch happens at
    256 and 2048 themselves."""
    def factor(n):
        d, Q = oracle.choose("dot", "f64", 3, n)
        return d + 1
    assert {factor(n) for n in range(65, 256)} == {5}
    assert {factor(n) for n in (256, 257, 1000, 2047)} == {4}
    assert {factor(n) for n in (2048, 4096, 10000, 32767)} == {3}


def test_lower_bound_strict_counterexample():
    """At p = 3, Q = 2^10, d = 3, k = Q/(p-1)^2 = 256 (the printed table bound)
    all-(p-1) inputs give a wrong digit; k = 255 is exact."""
    a = np.full(256, 2)
    assert oracle.dqt_dot(a, a, 3, 3, 2 ** 10) != (256 * 4) % 3
    assert oracle.dqt_dot(a[:255], a[:255], 3, 3, 2 ** 10) == (255 * 4) % 3


@pytest.mark.parametrize("p", [2, 3, 5, 7, 31])
def test_dqt_exact_inside_bounds(p):
    """Worst case (all p-1) and random inputs at the largest k the lower bound
    allows: the extracted digit equals the dot product mod p."""
    g = inputs.rng(97, p)
    for t in range(max(2, (p - 1).bit_length() * 2), 20):
        Q = 2 ** t
        kmax = (Q - 1) // (p - 1) ** 2
        if kmax < 1:
            continue
        for d in (0, 1, 3):
            for a, b in ((np.full(kmax, p - 1), np.full(kmax, p - 1)),
                         (g.integers(0, p, kmax), g.integers(0, p, kmax))):
                true = int(np.dot(a.astype(object), b.astype(object))) % p
                assert oracle.dqt_dot(a, b, p, d, Q) == true


def test_fp64_round_to_nearest_fails_toward_zero_holds():
    """Section 2.5 with FP64 words: at p = 3, Q = 2^10, d = 4 (Q^5 = 2^50 <
    2^53), k = 255, all-(p-1) inputs, round-to-nearest accumulation carries a
    rounded low part into the coefficient of Q^d; rounding toward zero does
    not (the library's FP64 form uses it)."""
    a = np.full(255, 2)
    true = (255 * 4) % 3
    assert oracle.dqt_dot_fp64(a, a, 3, 4, 2 ** 10, "rn") != true
    assert oracle.dqt_dot_fp64(a, a, 3, 4, 2 ** 10, "rz") == true


@pytest.mark.parametrize("p", [2, 3, 5, 7])
def test_fp64_toward_zero_sweep(p):
    """Every (t, d) with Q^(d+1) < 2^53 at the largest k of eq. (lower):
    round-toward-zero accumulation is exact on worst-case and random inputs."""
    g = inputs.rng(98, p)
    for t in range(2, 27):
        Q = 2 ** t
        kmax = (Q - 1) // (p - 1) ** 2
        if kmax < 1 or kmax > 5000:
            continue
        d = 0
        while oracle.upper_bound_holds(Q, d + 1):
            d += 1
        for a, b in ((np.full(kmax, p - 1), np.full(kmax, p - 1)),
                     (g.integers(p // 2, p, kmax), g.integers(p // 2, p, kmax))):
            true = int(np.dot(a.astype(object), b.astype(object))) % p
            assert oracle.dqt_dot_fp64(a, b, p, d, Q, "rz") == true


def test_u64_low_only_reading():
    """64-bit words kept mod 2^64: exact when t(d+1) <= 64, and a word one
    digit longer loses the coefficient of Q^d to the wrap."""
    p, t = 3, 16
    Q = 2 ** t
    k = (Q - 1) // 4 - 1                     # k (p-1)^2 not divisible by p
    a = np.full(k, 2)
    true = (k * 4) % p
    assert oracle.word_admissible("dot", "u64", p, k, 3, Q)          # t(d+1) = 64
    assert oracle.dqt_dot(a, a, p, 3, Q, modulus_bits=64) == true
    assert not oracle.word_admissible("dot", "u64", p, k, 4, Q)      # 80 bits
    assert oracle.dqt_dot(a, a, p, 4, Q, modulus_bits=64) != true
    # the 128-bit accumulator recovers d = 4 when the words still fit 64 bits
    assert oracle.amax(p, Q, 3) < 2 ** 64
    t2 = 13
    Q2 = 2 ** t2
    k2 = (Q2 - 1) // 4
    a2 = np.full(k2, 2)
    assert oracle.word_admissible("dot", "u64x128", p, k2, 4, Q2)
    assert not oracle.word_admissible("dot", "u64", p, k2, 4, Q2)
    assert oracle.dqt_dot(a2, a2, p, 4, Q2, modulus_bits=64) != (k2 * 4) % p
    assert oracle.dqt_dot(a2, a2, p, 4, Q2, modulus_bits=128) == (k2 * 4) % p


def test_u32_readings():
    p, t = 3, 8
    Q = 2 ** t
    k = 62                                   # k (p-1)^2 not divisible by p
    a = np.full(k, 2)
    true = (k * 4) % p
    assert oracle.word_admissible("dot", "u32", p, k, 3, Q)          # 32 bits
    assert oracle.dqt_dot(a, a, p, 3, Q, modulus_bits=32) == true
    assert not oracle.word_admissible("dot", "u32", p, k, 4, Q)
    assert oracle.dqt_dot(a, a, p, 4, Q, modulus_bits=32) != true
    # u32 words with a 64-bit accumulator: amax < 2^32 decides
    assert oracle.word_admissible("dot", "u32w", 3, 1024, 2, 2 ** 13)
    assert not oracle.word_admissible("dot", "u32w", 3, 1024, 3, 2 ** 13)
    assert oracle.amax(3, 2 ** 13, 3) >= 2 ** 32


@pytest.mark.parametrize("word,p,k,expect", [
    ("u64", 3, 256, 5), ("u64x128", 3, 256, 6), ("f64", 3, 256, 4), ("u32w", 3, 256, 3),
    ("u64", 3, 1024, 4), ("u64x128", 3, 1024, 5), ("f64", 3, 1024, 4), ("u32w", 3, 1024, 3),
    ("u64", 3, 8192, 4), ("f64", 3, 8192, 3), ("u64", 31, 8192, 2), ("u64x128", 31, 8192, 3),
    ("u64", 5, 16384, 3), ("u64x128", 5, 16384, 4), ("f64", 5, 16384, 2), ("u32", 3, 1024, 2),
])
def test_chooser_is_maximal_and_exact(word, p, k, expect):
    """choose() returns the largest d the word admits at the smallest Q of eq.
    (lower); emulating that (d, Q) on worst-case input of length k is exact,
    and d + 1 is rejected."""
    d, Q = oracle.choose("dot", word, p, k)
    assert d + 1 == expect
    assert oracle.lower_bound_holds(p, k, Q) and not oracle.lower_bound_holds(p, k, Q // 2)
    assert not oracle.word_admissible("dot", word, p, k, d + 1, Q)
    bits = {"u64": 64, "u64x128": 128, "u32w": 64, "u32": 32}.get(word)
    a = np.full(k, p - 1)
    true = (k * (p - 1) ** 2) % p
    if word == "f64":
        assert oracle.dqt_dot_fp64(a, a, p, d, Q, "rz") == true
    else:
        assert oracle.dqt_dot(a, a, p, d, Q, modulus_bits=bits) == true


def test_mixed_readings():
    """Right-compressed words: every coefficient is a full dot product < Q, so
    the word stays below Q^(d+1); u64 needs t(d+1) <= 64, f64 Q^(d+1) < 2^53."""
    p, k = 3, 1024
    d, Q = oracle.choose("mixed", "u64", p, k)
    assert (d, Q) == (3, 2 ** 13)
    d2, Q2 = oracle.choose("mixed", "f64", p, k)
    assert (d2, Q2) == (3, 2 ** 13)
    a = np.full(k, p - 1)
    words = [oracle.word_fwd([p - 1] * (d + 1), Q)] * k
    assert oracle.mixed_word(a, words, p, d, Q, modulus_bits=64) == [(k * 4) % p] * (d + 1)


def test_blocked_reading():
    """With a k-block kb the lower bound applies to kb: p = 5, t = 13 admits
    kb = 511 and d + 1 = 4 in u64, where the whole k = 16384 needs t = 19."""
    assert oracle.word_admissible("dot", "u64", 5, 16384, 3, 2 ** 13, kb=511)
    assert not oracle.word_admissible("dot", "u64", 5, 16384, 3, 2 ** 13, kb=512)
    assert oracle.choose("dot", "u64", 5, 16384) == (2, 2 ** 19)
    assert oracle.choose("dot", "u64", 5, 16384, kb=511) == (3, 2 ** 13)


def test_compression_factor():
    for t in range(2, 54):
        assert oracle.compression_factor(2 ** t) == 53 // t


def test_round53_against_binary64():
    """The rounding emulation used by dqt_dot_fp64, against the host's own
    binary64: float(int) rounds to nearest even; rounding toward zero gives a
    representable value z <= x whose next representable value exceeds x."""
    g = np.random.Generator(np.random.PCG64(3))
    cases = [2 ** 53 + 1, 2 ** 53 + 3, 2 ** 60 + 2 ** 7, 2 ** 60 + 3 * 2 ** 6, 2 ** 106 - 1, 0, 1, 2 ** 53]
    for _ in range(3000):
        hi = int(g.integers(1, 2 ** 62))
        cases.append((hi << int(g.integers(0, 60))) | int(g.integers(0, 2 ** 20)))
    for x in cases:
        assert oracle._round53(x, "rn") == int(float(x))
        z = oracle._round53(x, "rz")
        assert z <= x and int(float(z)) == z
        nxt = z + 1 if z < 2 ** 53 else int(math.nextafter(float(z), math.inf))
        assert nxt > x


def test_full_block_layout_worked_example():
    """Section 4: the 2x2 product packs into one word whose coefficients of
    1, Q, Theta, Q Theta are the four entries of C; pack_block of C gives it."""
    Q = 16
    for env in _instances(3):
        env.update(Q=Q, Theta=Q ** 2)
        C = np.asarray(eval(EX["C"], {}, env), dtype=np.uint8)
        FULL = eval(EX["FULL"], {}, env)
        W = oracle.pack_block(C, 1, 1, Q)
        assert W.shape == (1, 1) and int(W[0, 0]) == FULL
        assert (oracle.unpack_block(W, 2, 2, 1, 1, Q) == C).all()


@pytest.mark.parametrize("rows,cols,dq,dth,t", [(5, 7, 1, 2, 8), (4, 4, 0, 3, 10), (9, 3, 2, 0, 7),
                                               (1, 1, 1, 1, 12)])
def test_block_round_trip_and_special_cases(rows, cols, dq, dth, t):
    """Round trip; dth = 0 is the COLS layout, dq = 0 the ROWS layout."""
    Q = 2 ** t
    g = inputs.rng(99, rows * cols)
    X = inputs.residues(g, 5, rows, cols)
    W = oracle.pack_block(X, dq, dth, Q)
    assert (oracle.unpack_block(W, rows, cols, dq, dth, Q) == X).all()
    if dth == 0:
        assert (W == oracle.pack_cols(X, dq, Q)).all()
    if dq == 0:
        assert (W == oracle.pack_rows(X, dth, Q)).all()


def test_full_word_product_equals_block_of_C():
    """Section 4 on random data: sum_l (sum_i a_il Q^i)(sum_j b_lj Theta^j)
    equals pack_block(A B) when every coefficient stays below Q."""
    p, dq, dth, t = 3, 1, 2, 10
    Q = 2 ** t
    Theta = Q ** (dq + 1)
    g = inputs.rng(98, 7)
    A = inputs.residues(g, p, 4, 200)
    B = inputs.residues(g, p, 200, 6)
    assert oracle.full_admissible("u64", p, 200, dq, dth, Q)
    Aw = oracle.pack_cols(A, dq, Q)          # words along m
    Bw = oracle.pack_rows(B, dth, Theta)     # words along n, base Theta
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.uint64)
    want = oracle.pack_block(exact.astype(np.uint8) if exact.max() < 256 else exact, dq, dth, Q)
    for u in range(Aw.shape[0]):
        for v in range(Bw.shape[1]):
            w = oracle.full_word(Aw[u], Bw[:, v], Q, Theta)
            assert w == int(want[u, v])
            assert w < 2 ** 64
    assert not oracle.full_admissible("u64", p, 200, dq, dth + 1, Q)     # 10 * 2 * 4 = 80 bits


# ---- value-aware bounds (Section 2.4 with the entries' largest values) ----

def test_value_aware_bound_is_tight_for_0_1_inputs():
    """All-ones vectors (the largest 0/1 inputs): every coefficient of the
    accumulated word products is at most k, so k < Q is exact and k = Q
    carries into the next coefficient -- the bound k amax_a amax_b < Q is
    the tight one for amax = 1, where k (p-1)^2 < Q would ask for a Q
    (p-1)^2 times larger."""
    for p in (3, 5, 7):
        for t, d in ((6, 2), (9, 4), (11, 4)):
            Q = 2 ** t
            ones = np.ones(Q - 1, dtype=np.int64)
            assert oracle.lower_bound_holds(p, Q - 1, Q, 1, 1)
            assert not oracle.lower_bound_holds(p, Q - 1, Q)
            assert oracle.dqt_dot(ones, ones, p, d, Q) == (Q - 1) % p
            over = np.ones(Q, dtype=np.int64)
            assert not oracle.lower_bound_holds(p, Q, Q, 1, 1)
            assert oracle.dqt_dot(over, over, p, d, Q) != Q % p


def test_value_aware_bound_closed_form_and_mixed_bounds():
    """lower_bound_holds with amax_a, amax_b is k amax_a amax_b < Q; with
    amax = p - 1 it is eq. (lower); a matrix of (p-1) times a 0/1 matrix
    (the second product of a chain) needs k (p-1) < Q."""
    for p in (3, 7, 31):
        for k in (1, 5, 100, 1000):
            for t in range(1, 24):
                Q = 2 ** t
                assert oracle.lower_bound_holds(p, k, Q, 1, 1) == (k < Q)
                assert oracle.lower_bound_holds(p, k, Q, p - 1, 1) == (k * (p - 1) < Q)
                assert oracle.lower_bound_holds(p, k, Q, p - 1, p - 1) == oracle.lower_bound_holds(p, k, Q)
    # worst case of a residue matrix times a 0/1 matrix, exact at the bound
    p, t, d = 7, 12, 3
    Q = 2 ** t
    kmax = (Q - 1) // (p - 1)
    a = np.full(kmax, p - 1)
    b = np.ones(kmax, dtype=np.int64)
    assert oracle.dqt_dot(a, b, p, d, Q) == (kmax * (p - 1)) % p
    a2 = np.full(kmax + 1, p - 1)
    b2 = np.ones(kmax + 1, dtype=np.int64)
    assert kmax * (p - 1) < Q <= (kmax + 1) * (p - 1)
    assert oracle.dqt_dot(a2, b2, p, d, Q) != ((kmax + 1) * (p - 1)) % p


def test_value_aware_chooser_gains_compression():
    """0/1 inputs at p = 7, k = 1024: the smallest Q is 2^11 (k < Q) instead
    of 2^16 (36 k < Q), so 64-bit words hold 5 residues instead of 4 and
    FP64 words 4 instead of 3 (Q^(d+1) < 2^53)."""
    assert oracle.choose("dot", "u64", 7, 1024) == (3, 2 ** 16)
    assert oracle.choose("dot", "u64", 7, 1024, amax_a=1, amax_b=1) == (4, 2 ** 11)
    assert oracle.choose("dot", "f64", 7, 1024) == (2, 2 ** 16)
    assert oracle.choose("dot", "f64", 7, 1024, amax_a=1, amax_b=1) == (3, 2 ** 11)
    # brute force: the chosen Q is the smallest power of two above k amax_a amax_b
    for k in (1, 2, 3, 100, 1023, 1024, 5000):
        for a, b in ((1, 1), (6, 1), (1, 6), (2, 3)):
            d, Q = oracle.choose("dot", "u64", 7, k, amax_a=a, amax_b=b)
            t = Q.bit_length() - 1
            assert k * a * b < Q and max(a, b) < Q
            assert t == 1 or not (k * a * b < Q // 2 and max(a, b) < Q // 2)
            assert oracle.word_admissible("dot", "u64", 7, k, d, Q, amax_a=a, amax_b=b)
            assert not oracle.word_admissible("dot", "u64", 7, k, d + 1, Q, amax_a=a, amax_b=b)
