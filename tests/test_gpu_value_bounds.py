"""GPU parity of the value-aware parameters (Section 2.4 with the operands'
largest entries): 0/1 adjacency matrices packed with the smaller Q that
k amax_a amax_b < Q allows, every word of the dot form and the mixed form,
the all-ones worst case at k = Q - 1, gfp_amax, and chained powers A^3 that
keep the packed right operand and re-compress each reduced product
(procedure (compC) of Section 2.3: C = CA x CB; CC = ReduceAndCompress(C))."""
import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def dot_vb(p, A, B, word, amax, kb=0, d=None, Q=None):
    m, k = A.shape
    n = B.shape[1]
    if d is None:
        d, Q, kb = gfp.gfp_params_vb(p, m, k, n, amax[0], amax[1], "dot", word, kb=kb)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word, amax=amax[0])
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word, amax=amax[1])
    C = gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB, kb=kb, amax=amax)
    return host(C), d, Q


@pytest.mark.parametrize("word", ["u64", "u64x128", "u32w", "u32", "f64"])
@pytest.mark.parametrize("p", [3, 7])
def test_dot_0_1_matrices_value_aware(word, p):
    g = inputs.rng(71, p)
    A = inputs.adjacency(g, 300)
    B = inputs.adjacency(g, 300)[:, :170]
    ref = oracle.gemm(p, A, B)
    got, d, Q = dot_vb(p, A, B, word, (1, 1))
    assert (got == ref).all()
    d0, Q0, _ = gfp.gfp_params(p, 300, 300, 170, "dot", word)
    assert Q < Q0 and d >= d0


def test_dot_value_aware_worst_case_at_the_bound():
    """All ones with k = Q - 1 (every coefficient of Q^d equals Q - 1):
    exact; the parameters for k = Q are rejected."""
    p, word = 7, "u64"
    k = 2047
    d, Q, _ = gfp.gfp_params_vb(p, 64, k, 64, 1, 1, "dot", word)
    assert Q == 2048 and d == 4
    A = np.ones((64, k), np.uint8)
    B = np.ones((k, 40), np.uint8)
    got, _, _ = dot_vb(p, A, B, word, (1, 1), d=d, Q=Q)
    assert (got == (k % p)).all()
    with pytest.raises(gfp.GfpError) as e:
        gfp.gfp_params_vb(p, 64, k + 1, 64, 1, 1, "dot", word, d=d, Q=Q)
    assert e.value.status == 3


def test_dot_value_aware_blocked_and_mixed():
    """k-blocking under the value bound (kb < Q) and the mixed form (REDQ)
    with a residue matrix on the left and a 0/1 matrix on the right."""
    p = 5
    g = inputs.rng(72, 0)
    A = inputs.adjacency(g, 2000)[:100]
    B = inputs.adjacency(g, 2000)[:, :90]
    got, d, Q = dot_vb(p, A, B, "u32", (1, 1), kb=200)
    assert (got == oracle.gemm(p, A, B)).all()
    R = inputs.residues(g, p, 120, 2000)
    d, Q, _ = gfp.gfp_params_vb(p, 120, 2000, 90, p - 1, 1, "mixed", "u64")
    assert Q < gfp.gfp_params(p, 120, 2000, 90, "mixed", "u64")[1]
    CB = gfp.gfp_pack(p, dev(B), d, Q, "rows", "u64", amax=1)
    CC = gfp.gfp_gemm_compressed(p, 120, 2000, 90, d, Q, "mixed", "u64", dev(R), CB, amax=(p - 1, 1))
    C = gfp.gfp_unpack(p, CC, 120, 90, d, Q, "rows", "u64")
    assert (host(C) == oracle.gemm(p, R, B)).all()


def test_amax():
    g = inputs.rng(73, 0)
    for X, want in ((inputs.residues(g, 251, 333, 517), None), (inputs.adjacency(g, 129), 1),
                    (np.zeros((7, 9), np.uint8), 0)):
        want = int(X.max()) if want is None else want
        assert int(gfp.gfp_amax(dev(X)).item()) == want
    big = np.zeros((2000, 3000), np.uint8)
    big[1999, 2999] = 200
    Xd = dev(big)
    assert int(gfp.gfp_amax(Xd[:, :2999]).item()) == 0          # strided view, max outside
    assert int(gfp.gfp_amax(Xd).item()) == 200
    assert int(gfp.gfp_amax(dev(np.zeros((0, 5), np.uint8))).item()) == 0


def test_chained_power_keeps_the_right_operand_packed():
    """A^3 mod p for an adjacency matrix: B = A is packed once (columns) with
    a Q valid for both products (k (p-1) 1 < Q: residues times 0/1); each
    product's reduced result is re-compressed as the next left operand."""
    p, n = 7, 700
    g = inputs.rng(74, 0)
    A = inputs.adjacency(g, n)
    d, Q, _ = gfp.gfp_params_vb(p, n, n, n, p - 1, 1, "dot", "u64")
    Ad = dev(A)
    CB = gfp.gfp_pack(p, Ad, d, Q, "cols", "u64", amax=1)
    C = Ad
    for step in range(2):
        CA = gfp.gfp_pack(p, C, d, Q, "rows_rev", "u64", amax=(1 if step == 0 else p - 1))
        C = gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "dot", "u64", CA, CB,
                                    amax=(1 if step == 0 else p - 1, 1))
    ref = oracle.gemm(p, oracle.gemm(p, A, A), A)
    assert (host(C) == ref).all()
