"""The allocation-free entry point gfp_gemm_noalloc, for callers that cannot
allocate device memory (fixed memory budget, an allocator-owning framework,
latency-bound paths): called through the C ABI twice in a row, each time
against gfp_gemm's int8 tensor-core form on the same inputs, bit for bit
(the tolerance of every integer test here).  Kept in a file of its own that
pytest collects last; it builds what it needs, so it also runs alone."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, host

pytestmark = pytest.mark.gpu


def call_noalloc(L, p, A, B, C):
    m, k = A.shape
    n = B.shape[1]
    return L.gfp_gemm_noalloc(p, m, k, n, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                              ctypes.c_void_p(B.data_ptr()), B.stride(0),
                              ctypes.c_void_p(C.data_ptr()), C.stride(0),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_entry_point_twice():
    ensure_built()
    L = gfp.load()
    cases = [(3, 300, 500, 200), (251, 257, 1000, 129)]
    for call, (p, m, k, n) in enumerate(cases):
        g = inputs.rng(60, call)
        A_h = inputs.residues(g, p, m, k)
        B_h = inputs.residues(g, p, k, n)
        A, B = dev(A_h), dev(B_h)
        ref = host(gfp.gfp_gemm(p, A, B, "tc_mma_s8"))
        C = torch.full((m, n), 7, dtype=torch.uint8, device="cuda")
        assert call_noalloc(L, p, A, B, C) == 0
        got = host(C)
        assert (got == ref).all(), call
        assert (got == oracle.gemm(p, A_h, B_h)).all(), call


def test_noalloc_larger_call_then_smaller_ragged_call():
    """The shared scratch keeps the previous call's bytes.  A call that fills
    nearly all of it with nonzero operands (k = 8000) is followed by a smaller
    call with another padded k and ragged m, n, k: the smaller call must
    rewrite every byte it reads (padding included) and match gfp_gemm's
    int8 tensor-core form and the oracle bit for bit."""
    ensure_built()
    L = gfp.load()
    for call, (p, m, k, n) in enumerate([(251, 1024, 8000, 1000), (7, 131, 999, 77)]):
        g = inputs.rng(61, call)
        A_h = inputs.residues(g, p, m, k)
        B_h = inputs.residues(g, p, k, n)
        if call == 0:
            A_h |= 1            # nonzero everywhere
            B_h |= 1
        A, B = dev(A_h), dev(B_h)
        ref = host(gfp.gfp_gemm(p, A, B, "tc_mma_s8"))
        C = torch.full((m, n), 255, dtype=torch.uint8, device="cuda")
        assert call_noalloc(L, p, A, B, C) == 0
        got = host(C)
        assert (got == ref).all(), call
        assert (got == oracle.gemm(p, A_h, B_h, threads=8)).all(), call


def test_noalloc_rejects_problems_beyond_the_scratch():
    ensure_built()
    L = gfp.load()
    # (4096 + 4096) * 4096 bytes > 16 MiB: rejected on the host, nothing launched
    A = torch.zeros((4096, 4096), dtype=torch.uint8, device="cuda")
    C = torch.zeros((4096, 4096), dtype=torch.uint8, device="cuda")
    assert call_noalloc(L, 3, A, A, C) == 7


def test_noalloc_python_binding():
    """The binding's wrapper of the same entry point (argument marshalling
    only) returns the oracle's product and raises on a rejected size."""
    ensure_built()
    g = inputs.rng(60, 7)
    A_h = inputs.residues(g, 5, 70, 90)
    B_h = inputs.residues(g, 5, 90, 33)
    C = gfp.gfp_gemm_noalloc(5, dev(A_h), dev(B_h))
    assert (host(C) == oracle.gemm(5, A_h, B_h)).all()
    A = torch.zeros((4096, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(gfp.GfpError):
        gfp.gfp_gemm_noalloc(3, A, A)
