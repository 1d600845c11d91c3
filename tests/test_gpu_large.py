"""GPU parity at the full sizes of the workloads, in the launch configurations
the benchmark uses: sampled rows against the oracle (which computes them one
by one) and Freivalds' test on the whole product (a property of any correct
product, independent of how it was computed).

- tensor-core forms, p in {3, 31, 251}, m = k = n = 8192, and ragged sizes
  over the 256-column tiles;
- every form, p = 5, m = k = n = 16384."""
import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import THREADS, dev, ensure_built, freivalds, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def check(p, A, B, C, rows, rounds=2):
    assert (C[rows] == oracle.gemm_rows(p, rows, A, B, threads=THREADS)).all()
    assert freivalds(p, A, B, C, rounds=rounds)


@pytest.mark.parametrize("p", [3, 31, 251])
def test_tc_8192(p):
    n = 8192
    g = inputs.rng(3, p)
    A = inputs.residues(g, p, n, n)
    B = inputs.residues(g, p, n, n)
    Ad, Bd = dev(A), dev(B)
    rows = [0, 1, 127, 128, 4095, 8191]
    for algo in ("tc_f16", "tc_mma_s8") + (("tc_f8",) if p <= 31 else ()):
        C = host(gfp.gfp_gemm(p, Ad, Bd, algo))
        check(p, A, B, C, rows)
        del C


@pytest.mark.parametrize("p", [7, 31, 251])
def test_tc_ragged_256_column_tiles(p):
    """256-column tiles over an odd number (35) of 128-row tiles with ragged
    m, k and n: the last row tile and the last column tile are partial;
    p = 251 adds fp16 k-blocks."""
    m, k, n = 35 * 128 - 37, 1500, 4096 + 5
    g = inputs.rng(3, 100 + p)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    Ad, Bd = dev(A), dev(B)
    rows = [0, 127, 128, 255, 256, 4095, 4096, m - 2, m - 1]
    for algo in ("tc_f16",) + (("tc_f8",) if p <= 31 else ()):
        C = host(gfp.gfp_gemm(p, Ad, Bd, algo))
        check(p, A, B, C, rows, rounds=3)


@pytest.fixture(scope="module")
def big5():
    n = 16384
    g = inputs.rng(5, 0)
    A = inputs.residues(g, 5, n, n)
    B = inputs.residues(g, 5, n, n)
    return A, B


def test_all_forms_16384(big5):
    p, n = 5, 16384
    A, B = big5
    Ad, Bd = dev(A), dev(B)
    rows = [0, 5000, 16383]
    results = {}
    for algo in ("plain", "tc_f16", "tc_f8", "tc_mma_s8"):
        results[algo] = host(gfp.gfp_gemm(p, Ad, Bd, algo))
    d, Q, _ = gfp.gfp_params(p, n, n, n, "dot", "u64")
    CA = gfp.gfp_pack(p, Ad, d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(p, Bd, d, Q, "cols", "u64")
    results["dot_u64"] = host(gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "dot", "u64", CA, CB))
    del CA, CB
    d, Q, _ = gfp.gfp_params(p, n, n, n, "mixed", "u64")
    CB = gfp.gfp_pack(p, Bd, d, Q, "rows", "u64")
    CC = gfp.gfp_gemm_compressed(p, n, n, n, d, Q, "mixed", "u64", Ad, CB)
    results["mixed_u64"] = host(gfp.gfp_unpack(p, CC, n, n, d, Q, "rows", "u64"))
    del CB, CC
    ref_rows = oracle.gemm_rows(p, rows, A, B, threads=THREADS)
    first = None
    for name, C in results.items():
        assert (C[rows] == ref_rows).all(), name
        if first is None:
            assert freivalds(p, A, B, C, rounds=2), name
            first = C
        else:
            assert (C == first).all(), name       # every form gives the same unique product
