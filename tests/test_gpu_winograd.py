"""GPU parity of Strassen-Winograd over Z/2^64 on the dot form's 64-bit words:
one and two levels at odd word counts (so the shorter blocks are exercised),
the early stop below 512 words, levels = 0, empty and k = 0 products, the
worst case (all entries p - 1 at the largest k of the bound), rejection of
a short workspace, and CUDA-graph capture."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, host

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def run(p, A, B, levels, d=None, Q=None):
    m, k = A.shape
    n = B.shape[1]
    if d is None:
        d, Q, _ = gfp.gfp_params(p, m, k, n, "dot", "u64")
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", "u64")
    return host(gfp.gfp_gemm_compressed_winograd(p, m, k, n, d, Q, CA, CB, levels=levels)), d, Q


@pytest.mark.parametrize("p,levels", [(3, 1), (3, 2), (5, 2), (2, 1)])
def test_winograd_matches_oracle_odd_sizes(p, levels):
    g = inputs.rng(81, p * 10 + levels)
    m, k, n = 1030, 4100, 1100          # p = 3: t = 15, d+1 = 4, kc = 1025 words (odd)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    got, d, Q = run(p, A, B, levels)
    assert (got == oracle.gemm(p, A, B, threads=THREADS)).all()


def test_winograd_levels_zero_and_early_stop_equal_dot_form():
    p = 7
    g = inputs.rng(82, 0)
    A = inputs.residues(g, p, 700, 900)
    B = inputs.residues(g, p, 900, 300)        # n = 300 < 512: no level applies
    ref = oracle.gemm(p, A, B, threads=THREADS)
    for levels in (0, 3):
        got, _, _ = run(p, A, B, levels)
        assert (got == ref).all(), levels


def test_winograd_worst_case_at_the_bound():
    """All entries p - 1 and k (p-1)^2 = Q - 1: every digit at its largest."""
    p, t = 3, 13
    k = (2 ** t - 1) // 4                     # 2047: k (p-1)^2 = 8188 < 2^13
    d = 64 // t - 1
    A = np.full((1024, k), p - 1, np.uint8)
    B = np.full((k, 1100), p - 1, np.uint8)
    got, _, _ = run(p, A, B, 1, d=d, Q=2 ** t)
    assert (got == (k * (p - 1) ** 2) % p).all()


def test_winograd_edges_and_rejections():
    p = 5
    d, Q, _ = gfp.gfp_params(p, 8, 100, 8, "dot", "u64")
    z = torch.zeros((0, 4), dtype=torch.int64, device="cuda")
    out = torch.empty((0, 7), dtype=torch.uint8, device="cuda")
    gfp.gfp_gemm_compressed_winograd(p, 0, 100, 7, d, Q, z, torch.zeros((25, 7), dtype=torch.int64, device="cuda"),
                                     levels=1, out=out)
    C = torch.full((6, 7), 9, dtype=torch.uint8, device="cuda")
    e = torch.zeros((6, 1), dtype=torch.int64, device="cuda")
    gfp.gfp_gemm_compressed_winograd(p, 6, 0, 7, d, Q, e, torch.zeros((1, 7), dtype=torch.int64, device="cuda"),
                                     levels=1, out=C)
    assert (host(C) == 0).all()
    g = inputs.rng(83, 0)
    A = inputs.residues(g, p, 600, 2100)
    B = inputs.residues(g, p, 2100, 600)
    d, Q, _ = gfp.gfp_params(p, 600, 2100, 600, "dot", "u64")
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", "u64")
    need = gfp.gfp_winograd_workspace_size(600, 2100, 600, d, 1)
    short = torch.empty(need - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(gfp.GfpError) as ei:
        gfp.gfp_gemm_compressed_winograd(p, 600, 2100, 600, d, Q, CA, CB, levels=1, workspace=short)
    assert ei.value.status == 7
    with pytest.raises(gfp.GfpError) as ei:
        gfp.gfp_gemm_compressed_winograd(p, 600, 2100, 600, d, Q * 2 ** 40, CA, CB, levels=1)
    assert ei.value.status == 3


def test_winograd_graph_capture():
    p = 3
    g = inputs.rng(84, 0)
    A = inputs.residues(g, p, 1040, 2100)
    B = inputs.residues(g, p, 2100, 1030)
    d, Q, _ = gfp.gfp_params(p, 1040, 2100, 1030, "dot", "u64")
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", "u64")
    ws = torch.empty(gfp.gfp_winograd_workspace_size(1040, 2100, 1030, d, 1), dtype=torch.uint8, device="cuda")
    C = torch.empty((1040, 1030), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gfp.gfp_gemm_compressed_winograd(p, 1040, 2100, 1030, d, Q, CA, CB, levels=1, out=C, workspace=ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gfp.gfp_gemm_compressed_winograd(p, 1040, 2100, 1030, d, Q, CA, CB, levels=1, out=C, workspace=ws)
    C.fill_(255)
    graph.replay()
    assert (host(C) == oracle.gemm(p, A, B, threads=THREADS)).all()
