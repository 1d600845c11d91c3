"""GPU parity at the full sizes of the workloads, in the launch configurations
the benchmark uses, element by element against the oracle's full product.

The full products come from `oracle.gemm_matmul` (the definition with the
sum formed by a binary64 matrix product, exact while k (p-1)^2 < 2^53); at
each full size a few rows of the plain triple loop (`oracle.gemm_rows`) pin
that product too, so that the comparison rests on two independent forms of
the definition.

- tensor-core forms, p in {3, 31, 251}, m = k = n = 8192, and ragged sizes
  over the 256-column tiles;
- every form, p = 5, m = k = n = 16384."""
import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import THREADS, dev, ensure_built, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def full_oracle(p, A, B, pin_rows):
    """The oracle's whole product, with rows `pin_rows` of it checked against
    the triple loop."""
    C = oracle.gemm_matmul(p, A, B)
    assert (C[pin_rows] == oracle.gemm_rows(p, pin_rows, A, B, threads=THREADS)).all()
    return C


def assert_equal(name, got, ref):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError("%s: %d entries differ from the oracle, first at %s (got %d, want %d)"
                             % (name, len(bad), tuple(bad[0]), got[tuple(bad[0])], ref[tuple(bad[0])]))


def tc_algos(p):
    return [a for a in ("tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1")
            if a in gfp.ALGOS and {"tc_e2m1": p <= 7, "tc_f8": p <= 31}.get(a, True)]


@pytest.mark.parametrize("p", [3, 31, 251])
def test_tc_8192(p):
    n = 8192
    g = inputs.rng(3, p)
    A = inputs.residues(g, p, n, n)
    B = inputs.residues(g, p, n, n)
    ref = full_oracle(p, A, B, [0, 4097, 8191])
    Ad, Bd = dev(A), dev(B)
    for algo in tc_algos(p):
        assert_equal(algo, host(gfp.gfp_gemm(p, Ad, Bd, algo)), ref)


@pytest.mark.parametrize("p", [7, 31, 251])
def test_tc_ragged_256_column_tiles(p):
    """256-column tiles over an odd number (35) of 128-row tiles with ragged
    m, k and n: the last row tile and the last column tile are partial;
    p = 251 adds fp16 k-blocks."""
    m, k, n = 35 * 128 - 37, 1500, 4096 + 5
    g = inputs.rng(3, 100 + p)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    ref = full_oracle(p, A, B, [0, 128, m - 1])
    Ad, Bd = dev(A), dev(B)
    for algo in tc_algos(p):
        assert_equal(algo, host(gfp.gfp_gemm(p, Ad, Bd, algo)), ref)


def test_all_forms_16384():
    """p = 5, m = k = n = 16384: every form of the benchmark's step, each
    compared entry by entry with the oracle's product."""
    p, n = 5, 16384
    g = inputs.rng(5, 0)
    A = inputs.residues(g, p, n, n)
    B = inputs.residues(g, p, n, n)
    ref = full_oracle(p, A, B, [0, 5000, 16383])
    Ad, Bd = dev(A), dev(B)
    for algo in ("plain", "dp4a") + tuple(tc_algos(p)):
        assert_equal(algo, host(gfp.gfp_gemm(p, Ad, Bd, algo)), ref)
    best, _ = gfp.gfp_dot_autotune(p, n, n, n)
    for name, (word, d, Q, kb) in (("dot_u64", ("u64",) + gfp.gfp_params(p, n, n, n, "dot", "u64")),
                                   ("dot_tuned", (best["word"], best["d"], best["Q"], best["kb"]))):
        CA = gfp.gfp_pack(p, Ad, d, Q, "rows_rev", word)
        CB = gfp.gfp_pack(p, Bd, d, Q, "cols", word)
        assert_equal(name, host(gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "dot", word, CA, CB, kb=kb)), ref)
        del CA, CB
    d, Q, _ = gfp.gfp_params(p, n, n, n, "mixed", "u64")
    CB = gfp.gfp_pack(p, Bd, d, Q, "rows", "u64")
    CC = gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "mixed", "u64", Ad, CB)
    assert_equal("mixed_u64", host(gfp.gfp_unpack(p, CC, n, n, d, Q, "rows", "u64")), ref)
