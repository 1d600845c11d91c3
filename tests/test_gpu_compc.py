"""ReduceAndCompress fused into the dot form (gfp_gemm_compressed_compc):
procedure (compC) of Section 2.2, equation (1).  The words it writes are
compared with the oracle's reversed-row packing (Section 2.1, zero padding of
Section 2.3) of the oracle's product, and chains A^l built from them with
the right operand packed once are compared with the oracle's powers."""
import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import THREADS, dev, ensure_built, words_np

pytestmark = pytest.mark.gpu

NP_WORD = {"u64": np.uint64, "u32": np.uint32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def compc(p, A, B, word, kb=0, out_params=None):
    m, k = A.shape
    n = B.shape[1]
    d, Q, kb = gfp.gfp_params(p, m, k, n, "dot", word, kb=kb)
    d_out, Q_out = out_params if out_params is not None else (d, Q)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word)
    W = gfp.gfp_gemm_compressed_compc(p, m, k, n, d, Q, word, CA, CB, d_out, Q_out, kb=kb)
    return words_np(W, word), d_out, Q_out


# shapes ragged against every tile (64 x 64 words of u64; 128 x 128 and 128 x 64
# of u32 from two waves on) and against the words of the output
CASES = [(3, 129, 300, 257), (5, 1000, 1000, 1001), (7, 4001, 200, 3999), (31, 70, 513, 66), (2, 33, 64, 95)]


@pytest.mark.parametrize("word,kb", [("u64", 0), ("u32", 0), ("u32", 60)])
@pytest.mark.parametrize("p,m,k,n", CASES)
def test_compc_matches_oracle_packing(p, m, k, n, word, kb):
    A, B = inputs.residues(inputs.rng(70, m), p, m, k), inputs.residues(inputs.rng(71, n), p, k, n)
    if word == "u32" and kb:
        kb = min(kb, k)
        try:
            gfp.gfp_params(p, m, k, n, "dot", word, kb=kb)
        except gfp.GfpError:
            pytest.skip("no u32 k-block for this p")
    try:
        W, d_out, Q_out = compc(p, A, B, word, kb=kb)
    except gfp.GfpError as e:
        if e.status == 3:
            pytest.skip("%s words do not admit k = %d for p = %d" % (word, k, p))
        raise
    C = oracle.gemm(p, A, B, threads=THREADS)
    assert (W == oracle.pack_rows_rev(C, d_out, Q_out, NP_WORD[word])).all()


@pytest.mark.parametrize("d_out", [0, 1, 2, 5])
def test_compc_output_degrees(d_out):
    """Output words of another degree (and base) than the input words."""
    p, m, k, n = 5, 300, 700, 333
    A, B = inputs.residues(inputs.rng(72, 0), p, m, k), inputs.residues(inputs.rng(72, 1), p, k, n)
    Q_out = 2 ** 8
    W, _, _ = compc(p, A, B, "u64", out_params=(d_out, Q_out))
    C = oracle.gemm(p, A, B, threads=THREADS)
    assert (W == oracle.pack_rows_rev(C, d_out, Q_out, np.uint64)).all()


@pytest.mark.parametrize("word", ["u64", "u32"])
@pytest.mark.parametrize("kind", ["adjacency", "residues"])
def test_chained_power_one_launch_per_product(word, kind):
    """A^4 mod p as A -> compC(A x A) -> compC(A^2 x A) -> A^3 x A: the right
    operand CB = CompressColumns(A) is packed once, each intermediate power
    stays packed (one launch per product), and one (d, Q) serves the chain."""
    p, n = 7, 1500
    g = inputs.rng(73, 0)
    A = inputs.adjacency(g, n) if kind == "adjacency" else inputs.residues(g, p, n, n)
    d, Q, _ = gfp.gfp_params(p, n, n, n, "dot", word)
    Ad = dev(A)
    CB = gfp.gfp_pack(p, Ad, d, Q, "cols", word)
    X = gfp.gfp_pack(p, Ad, d, Q, "rows_rev", word)
    for _ in range(2):
        X = gfp.gfp_gemm_compressed_compc(p, n, n, n, d, Q, word, X, CB, d, Q)
    C4 = gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "dot", word, X, CB)
    ref = A
    for _ in range(3):
        ref = oracle.gemm(p, ref, A, threads=THREADS)
    assert (C4.cpu().numpy() == ref).all()


def test_compc_full_size_16384():
    """p = 5, m = k = n = 16384 (the benchmark's shape) in 64-bit words:
    the packed result equals the oracle's packing of its product."""
    p, n = 5, 16384
    g = inputs.rng(5, 0)
    A = inputs.residues(g, p, n, n)
    B = inputs.residues(g, p, n, n)
    W, d_out, Q_out = compc(p, A, B, "u64")
    C = oracle.gemm_matmul(p, A, B)
    assert (W == oracle.pack_rows_rev(C, d_out, Q_out, np.uint64)).all()
