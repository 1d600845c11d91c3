"""Guard bytes around every output: each form writes its result into a view in
the middle of a larger buffer filled with a sentinel (unaligned column
offset, row stride wider than the result), and nothing outside the view may
change.  Covers the classical and tensor-core products, the dot form in every
word, Winograd, the mixed/left/full compressed outputs (word views) and the
batched launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, host

pytestmark = pytest.mark.gpu
SENT = 0xA5
PAD_R, PAD_C, EXTRA = 3, 13, 29


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def guarded(rows, cols, dtype=torch.uint8, fill=SENT):
    """A (rows x cols) view inside a sentinel-filled buffer, and the buffer."""
    buf = torch.full((rows + 2 * PAD_R, cols + PAD_C + EXTRA), fill, dtype=dtype, device="cuda")
    return buf[PAD_R:PAD_R + rows, PAD_C:PAD_C + cols], buf


def untouched(buf, rows, cols, fill=SENT):
    b = host(buf).copy()
    b[PAD_R:PAD_R + rows, PAD_C:PAD_C + cols] = fill
    return (b == fill).all()


SHAPES = [(3, 300, 257, 190), (31, 129, 1000, 257), (5, 1100, 700, 1030)]


@pytest.mark.parametrize("algo", ["plain", "dp4a", "tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"])
@pytest.mark.parametrize("p,m,k,n", SHAPES)
def test_gemm_writes_only_its_view(algo, p, m, k, n):
    if algo == "tc_e2m1" and p > 7:
        pytest.skip("e2m1 operands hold the centred residues of p <= 7 only")
    g = inputs.rng(95, m)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    C, buf = guarded(m, n)
    gfp.gfp_gemm(p, dev(A), dev(B), algo, out=C)
    assert (host(C) == oracle.gemm(p, A, B)).all()
    assert untouched(buf, m, n)


@pytest.mark.parametrize("word,kb", [("u64", 0), ("u64x128", 0), ("u32w", 0), ("u32", 0), ("f64", 0), ("u32", 60)])
def test_dot_writes_only_its_view(word, kb):
    p, m, k, n = 3, 333, 900, 271
    g = inputs.rng(96, 0)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    d, Q, kb = gfp.gfp_params(p, m, k, n, "dot", word, kb=kb)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word)
    C, buf = guarded(m, n)
    gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB, out=C, kb=kb)
    assert (host(C) == oracle.gemm(p, A, B)).all()
    assert untouched(buf, m, n)


def test_winograd_writes_only_its_view():
    p, m, k, n = 3, 1030, 2100, 1040
    g = inputs.rng(96, 1)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    d, Q, _ = gfp.gfp_params(p, m, k, n, "dot", "u64")
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", "u64")
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", "u64")
    C, buf = guarded(m, n)
    gfp.gfp_gemm_compressed_winograd(p, m, k, n, d, Q, CA, CB, levels=1, out=C)
    assert (host(C) == oracle.gemm(p, A, B)).all()
    assert untouched(buf, m, n)


WSENT = -0x5A5A5A5A5A5A5A5B


def test_packed_outputs_write_only_their_views():
    """mixed (CC rows), left (CC columns) and full (CC blocks) into guarded
    64-bit word views."""
    p, m, k, n = 5, 210, 400, 190
    g = inputs.rng(96, 2)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    ref = oracle.gemm(p, A, B)
    d, Q, _ = gfp.gfp_params(p, m, k, n, "mixed", "u64")
    CB = gfp.gfp_pack(p, dev(B), d, Q, "rows", "u64")
    nc = -(-n // (d + 1))
    CC, buf = guarded(m, nc, torch.int64, WSENT)
    gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "mixed", "u64", dev(A), CB, out=CC)
    assert (host(gfp.gfp_unpack(p, CC, m, n, d, Q, "rows", "u64")) == ref).all()
    assert untouched(buf, m, nc, WSENT)
    d, Q, _ = gfp.gfp_params(p, m, k, n, "left", "u64")
    CA = gfp.gfp_pack(p, dev(A), d, Q, "cols", "u64")
    mc = -(-m // (d + 1))
    CC, buf = guarded(mc, n, torch.int64, WSENT)
    gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "left", "u64", CA, dev(B), out=CC)
    assert (host(gfp.gfp_unpack(p, CC, m, n, d, Q, "cols", "u64")) == ref).all()
    assert untouched(buf, mc, n, WSENT)
    dq, dth, Q = gfp.gfp_params_full(p, m, k, n, "u64")
    CA = gfp.gfp_pack(p, dev(A), dq, Q, "cols", "u64")
    CBt = gfp.gfp_pack(p, dev(B), dth, Q ** (dq + 1), "rows", "u64")
    rows, cols = -(-m // (dq + 1)), -(-n // (dth + 1))
    CC, buf = guarded(rows, cols, torch.int64, WSENT)
    gfp.gfp_gemm_full(p, m, k, n, dq, dth, Q, "u64", CA, CBt, out=CC)
    assert (host(gfp.gfp_unpack_block(p, CC, m, n, dq, dth, Q, "u64")) == ref).all()
    assert untouched(buf, rows, cols, WSENT)


@pytest.mark.parametrize("algo", ["auto", "tc_f16", "tc_f8", "dot32"])
def test_batched_writes_only_its_views(algo):
    g = inputs.rng(97, 0)
    items, host_ops, bufs = [], [], []
    for p, m, k, n in ((3, 130, 200, 97), (5, 300, 64, 260), (7, 17, 513, 40), (251, 64, 100, 130),
                       (13, 257, 300, 129)):
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        C, buf = guarded(m, n)
        items.append((p, dev(A), dev(B), C))
        host_ops.append((p, A, B))
        bufs.append(buf)
    arr, cnt = gfp.make_problems(items)
    gfp.gfp_gemm_batched(arr, cnt, algo)
    for (p, A, B), (_, _, _, C), buf in zip(host_ops, items, bufs):
        assert (host(C) == oracle.gemm(p, A, B)).all()
        assert untouched(buf, C.shape[0], C.shape[1])
