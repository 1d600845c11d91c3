"""Oracle for exact GF(p) matrix multiplication and the paper's Q-adic packing.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark import this package.  The product library
(`paper_0803_1975_gb300`) never imports it, and this package imports nothing
from the product: the two share no kernels, headers, helpers or tables.

Paper: J.-G. Dumas, L. Fousse, B. Salvy, "Compressed Modular Matrix
Multiplication" (arXiv 0803.1975).

Contents, each written from the cited passage:

* `gemm`, `gemm_rows`: the definition C = A B mod p, as a plain C triple loop
  (gfp_oracle.c); `gemm_matmul`, the same definition with the sum formed by a
  library matrix product in exact binary64 arithmetic, for the largest sizes.  Every form of the paper must reach this result exactly
  (Section 2.2: the compressed product recovers the same dot products).
* `pack_rows_rev`, `pack_cols`, `pack_rows` and their inverses: the Q-adic
  words of Section 2.1 (reversed rows of A, forward columns of B), the zero
  padding of Section 2.3, and the row-compressed right operand of Section 3.
* `lower_bound_holds`, `upper_bound_holds`, `compression_factor`,
  `full_bounds_hold`: equations (lower), (upper), (qtheta), (dq) and the
  compression factor e of Section 5.
* `word_admissible`, `choose`: the bounds read for each machine word the
  library offers (64-bit and 32-bit integers, FP64 mantissa); these readings
  are not printed in the paper and are stated next to each rule.
* `dqt_dot`, `dqt_dot_fp64`, `mixed_word`, `full_word`: the paper's steps on
  a single dot product carried out in exact integer arithmetic (and, for
  FP64, with the rounding of each fused multiply-add emulated exactly).  They
  are used to pin the readings, e.g. that the lower bound must be strict and
  that FP64 accumulation needs round-toward-zero.

All pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfp_oracle.c")
_SO = os.path.join(_HERE, "libgfp_oracle.so")
_lib = None


# --------------------------------------------------------------------------
# The C triple loop
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile gfp_oracle.c into libgfp_oracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64 = ctypes.c_int64
        lib.oracle_gemm_modp.argtypes = [ctypes.c_uint32, i64, i64, i64, u8p, i64, u8p, i64,
                                         u8p, i64, ctypes.c_int]
        lib.oracle_gemm_modp.restype = None
        lib.oracle_gemm_rows_modp.argtypes = [ctypes.c_uint32, i64, ctypes.POINTER(i64), i64, i64,
                                              u8p, i64, u8p, i64, u8p, i64, ctypes.c_int]
        lib.oracle_gemm_rows_modp.restype = None
        _lib = lib
    return _lib


def _u8(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _check_operands(p, A, B):
    if A.dtype != np.uint8 or B.dtype != np.uint8 or A.ndim != 2 or B.ndim != 2:
        raise TypeError("oracle operands are 2-D uint8 arrays")
    if A.shape[1] != B.shape[0]:
        raise ValueError("inner dimensions differ")
    if not (2 <= p <= 256):
        raise ValueError("p must fit the uint8 residue storage")


def gemm(p: int, A: np.ndarray, B: np.ndarray, threads: int = 1) -> np.ndarray:
    """C = A B mod p by the definition (triple loop, exact 64-bit sums)."""
    _check_operands(p, A, B)
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.uint8)
    if m and n:
        _load().oracle_gemm_modp(p, m, k, n, _u8(A), max(k, 1), _u8(B), max(n, 1), _u8(C),
                                 max(n, 1), threads)
    return C


def gemm_rows(p: int, rows, A: np.ndarray, B: np.ndarray, threads: int = 1) -> np.ndarray:
    """Rows `rows` of A B mod p, by the same definition."""
    _check_operands(p, A, B)
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    k = A.shape[1]
    n = B.shape[1]
    out = np.zeros((rows.size, n), dtype=np.uint8)
    if rows.size and n:
        _load().oracle_gemm_rows_modp(p, rows.size,
                                      rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      k, n, _u8(A), max(k, 1), _u8(B), max(n, 1), _u8(out),
                                      max(n, 1), threads)
    return out


def gemm_matmul(p: int, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The same definition with the sum formed by a library matrix product in
    binary64: every product A[i][l] B[l][j] and every partial sum is an
    integer below k (p-1)^2 + 1, so while k (p-1)^2 < 2^53 each one is exact
    in any order of summation, and C = (A B) mod p exactly.  It serves the
    sizes the triple loop cannot finish (8192^3 and beyond); the tests pin it
    to `gemm` and `gemm_rows`.  Raises where the bound fails."""
    _check_operands(p, A, B)
    m, k = A.shape
    n = B.shape[1]
    if k * (p - 1) ** 2 >= 2 ** 53:
        raise ValueError("k (p-1)^2 >= 2^53: binary64 sums would not be exact")
    S = np.matmul(A.astype(np.float64), B.astype(np.float64))
    return np.fmod(S, float(p)).astype(np.uint8).reshape(m, n)


# --------------------------------------------------------------------------
# Q-adic words (Section 2.1, 2.3, 3).  Q = 2^t throughout the library; the
# formulas below hold for any integer Q >= 2 and use exact arithmetic.
# --------------------------------------------------------------------------
def _check_word_range(d: int, Q: int, p: int | None = None):
    if d < 0 or Q < 2:
        raise ValueError("need d >= 0 and Q >= 2")


def _powers(d, Q, dtype):
    return [dtype(Q ** s) for s in range(d + 1)]


def pack_rows_rev(X: np.ndarray, d: int, Q: int, dtype=np.uint64) -> np.ndarray:
    """Section 2.1: a row block [a_0 .. a_d] is stored reversed, as
    abar = sum_i a_{d-i} Q^i, i.e. entry j of the block gets weight Q^(d-j).
    Section 2.3: a final block with r < d+1 entries is padded with zeros at
    its end, which multiplies the reversed word of the r entries by
    Q^(d+1-r).  Result: (rows, ceil(cols/(d+1))) words."""
    _check_word_range(d, Q)
    rows, cols = X.shape
    kc = -(-cols // (d + 1))
    W = np.zeros((rows, kc), dtype=dtype)
    pw = _powers(d, Q, dtype)
    for w in range(kc):
        for j in range(d + 1):
            l = w * (d + 1) + j
            if l < cols:
                W[:, w] += X[:, l].astype(dtype) * pw[d - j]
    return W


def pack_cols(X: np.ndarray, d: int, Q: int, dtype=np.uint64) -> np.ndarray:
    """Section 2.1: a column block [b_0 .. b_d] is stored forward, as
    bbar = sum_i b_i Q^i.  Missing entries of the last block are zero
    (Section 2.3: the forward word needs no adjustment for them).
    Result: (ceil(rows/(d+1)), cols) words."""
    _check_word_range(d, Q)
    rows, cols = X.shape
    kc = -(-rows // (d + 1))
    W = np.zeros((kc, cols), dtype=dtype)
    pw = _powers(d, Q, dtype)
    for w in range(kc):
        for s in range(d + 1):
            l = w * (d + 1) + s
            if l < rows:
                W[w, :] += X[l, :].astype(dtype) * pw[s]
    return W


def pack_rows(X: np.ndarray, d: int, Q: int, dtype=np.uint64) -> np.ndarray:
    """Section 3: the right operand of the right-compressed product is
    row-compressed, each word holding d+1 consecutive entries of a row:
    W[l][v] = sum_j X[l][v(d+1)+j] Q^j (missing entries zero).
    The compressed result CC of that product has the same layout.
    Result: (rows, ceil(cols/(d+1))) words."""
    _check_word_range(d, Q)
    rows, cols = X.shape
    nc = -(-cols // (d + 1))
    W = np.zeros((rows, nc), dtype=dtype)
    pw = _powers(d, Q, dtype)
    for v in range(nc):
        for j in range(d + 1):
            c = v * (d + 1) + j
            if c < cols:
                W[:, v] += X[:, c].astype(dtype) * pw[j]
    return W


def _digit(W: np.ndarray, s: int, Q: int) -> np.ndarray:
    """Coefficient of Q^s of words whose coefficients are all < Q."""
    if W.dtype == np.float64:
        Wi = W.astype(object)
        return np.vectorize(lambda x: (int(x) // Q ** s) % Q, otypes=[np.int64])(Wi)
    return (W // W.dtype.type(Q ** s)) % W.dtype.type(Q)


def unpack_rows_rev(W: np.ndarray, cols: int, d: int, Q: int) -> np.ndarray:
    """Inverse of pack_rows_rev: entry w(d+1)+j is the coefficient of Q^(d-j)."""
    rows = W.shape[0]
    X = np.zeros((rows, cols), dtype=np.uint8)
    for l in range(cols):
        w, j = divmod(l, d + 1)
        X[:, l] = _digit(W[:, w], d - j, Q).astype(np.uint8)
    return X


def unpack_cols(W: np.ndarray, rows: int, d: int, Q: int) -> np.ndarray:
    """Inverse of pack_cols: entry w(d+1)+s is the coefficient of Q^s."""
    cols = W.shape[1]
    X = np.zeros((rows, cols), dtype=np.uint8)
    for l in range(rows):
        w, s = divmod(l, d + 1)
        X[l, :] = _digit(W[w, :], s, Q).astype(np.uint8)
    return X


def unpack_rows(W: np.ndarray, cols: int, d: int, Q: int) -> np.ndarray:
    """Inverse of pack_rows: entry v(d+1)+j is the coefficient of Q^j."""
    rows = W.shape[0]
    X = np.zeros((rows, cols), dtype=np.uint8)
    for c in range(cols):
        v, j = divmod(c, d + 1)
        X[:, c] = _digit(W[:, v], j, Q).astype(np.uint8)
    return X


def pack_block(X: np.ndarray, dq: int, dth: int, Q: int, dtype=np.uint64) -> np.ndarray:
    """Section 4 result layout: with Theta = Q^(dq+1), the word of block
    (u, v) is sum_{i<=dq} sum_{j<=dth} X[u(dq+1)+i][v(dth+1)+j] Q^i Theta^j,
    i.e. the coefficient of position i + j(dq+1) in base Q.  Entries past the
    edge count as zero.  Result: (ceil(rows/(dq+1)), ceil(cols/(dth+1)))."""
    rows, cols = X.shape
    R = -(-rows // (dq + 1))
    Cc = -(-cols // (dth + 1))
    W = np.zeros((R, Cc), dtype=dtype)
    for i in range(dq + 1):
        for j in range(dth + 1):
            sub = np.zeros((R, Cc), dtype=np.uint64)
            part = X[i::dq + 1, j::dth + 1]
            sub[:part.shape[0], :part.shape[1]] = part
            W += (sub * np.uint64(Q ** (i + j * (dq + 1)))).astype(dtype)
    return W


def unpack_block(W: np.ndarray, rows: int, cols: int, dq: int, dth: int, Q: int) -> np.ndarray:
    """Inverse of pack_block."""
    X = np.zeros((rows, cols), dtype=np.uint8)
    for r in range(rows):
        u, i = divmod(r, dq + 1)
        for c in range(cols):
            v, j = divmod(c, dth + 1)
            X[r, c] = (int(W[u, v]) // Q ** (i + j * (dq + 1))) % Q
    return X


# --------------------------------------------------------------------------
# Bounds of the paper
# --------------------------------------------------------------------------
def lower_bound_holds(p: int, k: int, Q: int, amax_a: int | None = None, amax_b: int | None = None) -> bool:
    """Equation (lower), Section 2.4: with delayed reduction every
    coefficient of the accumulated word products stays below Q iff
    k (p-1)^2 < Q.  The inequality is strict, as the equation prints it
    (Table 1 prints the dimensions with <=; the strict form is the one that
    holds, see tests/test_oracle_dqt.py).

    The argument uses only that every entry lies in [0, p-1]; with entries
    of A at most amax_a and of B at most amax_b (value-aware reading, e.g.
    0/1 adjacency matrices) a coefficient is at most k amax_a amax_b, and
    the bound reads k amax_a amax_b < Q."""
    a = p - 1 if amax_a is None else amax_a
    b = p - 1 if amax_b is None else amax_b
    return k * a * b < Q


def upper_bound_holds(Q: int, d: int, beta: int = 53) -> bool:
    """Equation (upper), Section 2.5: Q^(d+1) < 2^beta, beta the mantissa."""
    return Q ** (d + 1) < 2 ** beta


def compression_factor(Q: int, beta: int = 53) -> int:
    """Section 5: e = floor(beta / log2 Q); the degree is d = e - 1."""
    return math.floor(beta / math.log2(Q))


def full_bounds_hold(p: int, k: int, Q: int, dq: int, Theta: int, dth: int,
                     beta: int = 53) -> bool:
    """Section 4: Q satisfies (lower), Q^(dq+1) <= Theta (eq. qtheta) and
    Q^((dq+1)(dth+1)) < 2^beta (eq. dq, which takes Theta = Q^(dq+1))."""
    return (lower_bound_holds(p, k, Q) and Q ** (dq + 1) <= Theta
            and Q ** ((dq + 1) * (dth + 1)) < 2 ** beta)


def amax(p: int, Q: int, d: int, v: int | None = None) -> int:
    """Largest packed word: all d+1 residues equal to p-1 (or to v, the
    largest entry of the packed matrix when it is known to be smaller)."""
    return (p - 1 if v is None else v) * sum(Q ** s for s in range(d + 1))


# Machine words offered by the library.  The paper gives the bounds for a
# floating-point mantissa of beta bits; for integer words the same argument
# reads as follows (each reading is pinned by an exact emulation in the
# tests):
#   u64   : 64-bit words, products and sums kept mod 2^64.  The coefficient
#           of Q^d sits in bits [t d, t(d+1)), exact mod 2^64 when
#           t(d+1) <= 64 (higher coefficients may wrap, they are not used).
#   u64x128: 64-bit words (amax < 2^64) with a 128-bit accumulator, so the
#           coefficient of Q^d is exact when t(d+1) <= 128.
#   u32w  : 32-bit words (amax < 2^32), 64-bit accumulator: t(d+1) <= 64.
#   u32   : 32-bit words and a 32-bit accumulator: t(d+1) <= 32.
#   f64   : eq. (upper) with beta = 53, Q^(d+1) < 2^53, accumulation by
#           fused multiply-add rounded toward zero (round-to-nearest is not
#           enough, see dqt_dot_fp64).
# For the right-compressed (mixed) product every coefficient of a result
# word is a full dot product < Q, so the word value is < Q^(d+1):
#   mixed u64 : t(d+1) <= 64;   mixed f64 : Q^(d+1) < 2^53.
# Left compression (Table 2, "Left Comp.") is the right-compressed product
# with the roles of the outer dimensions exchanged: the same readings apply.
# Full compression (Section 4) keeps every coefficient of the word, so the
# whole accumulated word must fit: t (dq+1)(dth+1) <= 64 for u64 (eq. dq with
# beta = 64 and Theta = Q^(dq+1)), Q^((dq+1)(dth+1)) < 2^53 for f64.
WORDS_DOT = ("u64", "u64x128", "u32w", "u32", "f64")
WORDS_MIXED = ("u64", "f64")


def word_admissible(form: str, word: str, p: int, k: int, d: int, Q: int,
                    kb: int | None = None, amax_a: int | None = None, amax_b: int | None = None) -> bool:
    """True when (p, k, d, Q) gives exact results for `form` ('dot' or
    'mixed') in `word`.  kb, when given, is the k-block after which the dot
    form extracts the coefficient of Q^d and restarts the word sum; the lower
    bound then applies to kb and the extracted coefficients are summed in
    32 bits, which needs k (p-1)^2 < 2^32.  amax_a, amax_b: the largest
    entries of A and B when known to be below p-1 (see lower_bound_holds);
    the packed words then hold digits up to max(amax_a, amax_b)."""
    if p < 2 or d < 0 or Q < 2 or Q & (Q - 1):
        return False
    a = p - 1 if amax_a is None else amax_a
    b = p - 1 if amax_b is None else amax_b
    v = max(a, b)
    t = Q.bit_length() - 1
    kk = k if kb is None else kb
    if kb is not None:
        if form != "dot" or kb < 1 or k * a * b >= 2 ** 32:
            return False
    if not lower_bound_holds(p, kk, Q, a, b):
        return False
    if form == "dot":
        if word == "u64":
            return t * (d + 1) <= 64 and amax(p, Q, d, v) < 2 ** 64
        if word == "u64x128":
            return amax(p, Q, d, v) < 2 ** 64 and t * (d + 1) <= 128
        if word == "u32w":
            return amax(p, Q, d, v) < 2 ** 32 and t * (d + 1) <= 64
        if word == "u32":
            return t * (d + 1) <= 32
        if word == "f64":
            return upper_bound_holds(Q, d, 53)
        return False
    if form in ("mixed", "left"):
        if word == "u64":
            return t * (d + 1) <= 64
        if word == "f64":
            return upper_bound_holds(Q, d, 53)
        return False
    return False


def full_admissible(word: str, p: int, k: int, dq: int, dth: int, Q: int) -> bool:
    """Section 4 with Theta = Q^(dq+1) (the smallest Theta of eq. qtheta):
    eq. (lower) for Q and the whole word within the word size (eq. dq)."""
    if p < 2 or dq < 0 or dth < 0 or Q < 2 or Q & (Q - 1):
        return False
    t = Q.bit_length() - 1
    if not lower_bound_holds(p, k, Q):
        return False
    if word == "u64":
        return t * (dq + 1) * (dth + 1) <= 64
    if word == "f64":
        return Q ** ((dq + 1) * (dth + 1)) < 2 ** 53
    return False


def choose(form: str, word: str, p: int, k: int, kb: int | None = None,
           amax_a: int | None = None, amax_b: int | None = None):
    """Smallest Q = 2^t that satisfies (lower) for k (or kb) and holds every
    entry as a digit, then the largest d the word admits for that Q.
    Returns (d, Q) or None."""
    a = p - 1 if amax_a is None else amax_a
    b = p - 1 if amax_b is None else amax_b
    kk = k if kb is None else kb
    t = 1
    while not lower_bound_holds(p, max(kk, 1), 2 ** t, a, b) or max(a, b) >= 2 ** t:
        t += 1
        if t > 64:
            return None
    Q = 2 ** t
    best = None
    for d in range(0, 64):
        if word_admissible(form, word, p, k, d, Q, kb, a, b):
            best = d
    return None if best is None else (best, Q)


def table1_row(t: int, p: int = 3, beta: int = 53):
    """One column of Table 1 (Section 2.6) for Q = 2^t: the compression
    factor e, the degree d = e - 1 and the largest k allowed by (lower)."""
    Q = 2 ** t
    e = compression_factor(Q, beta)
    kmax = (Q - 1) // (p - 1) ** 2
    while not lower_bound_holds(p, kmax, Q):
        kmax -= 1
    return {"Q": Q, "e": e, "d": e - 1, "kmax": kmax}


# --------------------------------------------------------------------------
# The paper's steps on one dot product, in exact arithmetic
# --------------------------------------------------------------------------
def _blocks(v, d):
    v = [int(x) for x in v]
    kc = -(-len(v) // (d + 1))
    return [v[w * (d + 1):(w + 1) * (d + 1)] + [0] * ((w + 1) * (d + 1) - min(len(v), (w + 1) * (d + 1)))
            for w in range(kc)]


def word_rev(block, Q):
    """abar of Section 2.1 for one block: sum_i a_{d-i} Q^i (exact int)."""
    d = len(block) - 1
    return sum(int(block[d - i]) * Q ** i for i in range(d + 1))


def word_fwd(block, Q):
    """bbar of Section 2.1 for one block: sum_i b_i Q^i (exact int)."""
    return sum(int(b) * Q ** i for i, b in enumerate(block))


def dqt_dot(a, b, p: int, d: int, Q: int, modulus_bits: int | None = None) -> int:
    """Sections 2.1-2.5 on one dot product sum_l a_l b_l mod p: pack a
    reversed and b forward in blocks of d+1 (zero padded), multiply the
    words and accumulate the products with no reduction, read the
    coefficient of Q^d and reduce it mod p.  `modulus_bits` keeps the
    accumulator mod 2^bits, as a machine word does."""
    acc = 0
    for ba, bb in zip(_blocks(a, d), _blocks(b, d)):
        acc += word_rev(ba, Q) * word_fwd(bb, Q)
        if modulus_bits is not None:
            acc %= 2 ** modulus_bits
    return ((acc // Q ** d) % Q) % p


def _round53(x: int, mode: str) -> int:
    """Round a non-negative integer to 53 significant bits ('rz' toward
    zero, 'rn' to nearest even), as IEEE binary64 does for integers."""
    if x < 0:
        raise ValueError("non-negative only")
    n = x.bit_length()
    if n <= 53:
        return x
    sh = n - 53
    q, r = x >> sh, x & ((1 << sh) - 1)
    if mode == "rn":
        half = 1 << (sh - 1)
        if r > half or (r == half and q & 1):
            q += 1
    elif mode != "rz":
        raise ValueError(mode)
    return q << sh


def dqt_dot_fp64(a, b, p: int, d: int, Q: int, mode: str) -> int:
    """dqt_dot with the words held in binary64 and accumulated by fused
    multiply-add, acc <- round(abar * bbar + acc), each rounding emulated
    exactly ('rz' or 'rn').  The coefficient of Q^d is then read as in
    Section 2.5: scale by the exact inverse 2^(-t d), truncate, keep the
    part below Q, reduce mod p.  Every word is an integer < 2^53, so the
    packed words themselves are exact."""
    acc = 0
    for ba, bb in zip(_blocks(a, d), _blocks(b, d)):
        wa, wb = word_rev(ba, Q), word_fwd(bb, Q)
        if wa >= 2 ** 53 or wb >= 2 ** 53:
            raise ValueError("word does not fit the mantissa")
        acc = _round53(wa * wb + acc, mode)
    return ((acc // Q ** d) % Q) % p


def mixed_word(a, bwords, p: int, d: int, Q: int, modulus_bits: int | None = None):
    """Section 3 on one result word: sum_l a_l * (sum_j b_lj Q^j) =
    sum_j (sum_l a_l b_lj) Q^j; returns the d+1 coefficients reduced mod p
    (what the simultaneous reduction REDQ delivers)."""
    acc = 0
    for al, wl in zip(a, bwords):
        acc += int(al) * int(wl)
        if modulus_bits is not None:
            acc %= 2 ** modulus_bits
    return [((acc // Q ** j) % Q) % p for j in range(d + 1)]


def full_word(awords, bwords, Q: int, Theta: int):
    """Section 4 on one result word: sum_l (sum_i a_il Q^i)(sum_j b_lj Theta^j);
    returns the exact integer."""
    return sum(int(x) * int(y) for x, y in zip(awords, bwords))
