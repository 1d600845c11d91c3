"""GPU parity of the batched grouped launch: every tile kind, uneven and
rectangular problems, invalid entries, CUDA-graph replay, the autotuner, and
the 4096-problem adjacency workload (sampled problems against the oracle,
Freivalds' check on every problem)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, freivalds, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def random_batch(seed, count, primes=(2, 3, 5, 7, 31, 251), smax=300):
    g = np.random.Generator(np.random.PCG64(seed))
    items, host_ops = [], []
    for _ in range(count):
        p = int(g.choice(primes))
        m, k, n = (int(x) for x in g.integers(1, smax, size=3))
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        items.append((p, dev(A), dev(B), torch.full((m, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A, B))
    return items, host_ops


@pytest.mark.parametrize("algo", ["tc_f16", "dot32", "tc_f8", "auto"])
def test_batched_rectangular_mixed_primes(algo):
    items, host_ops = random_batch(11, 120)
    arr, cnt = gfp.make_problems(items)
    gfp.gfp_gemm_batched(arr, cnt, algo)
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all()


def test_batched_worst_case_and_kblocks():
    """All entries p-1, and k beyond one fp16 k-block for p = 251."""
    items, refs = [], []
    for p, m, k, n in ((251, 70, 2500, 90), (7, 64, 512, 64), (3, 33, 1000, 31), (251, 5, 1100, 7)):
        A = np.full((m, k), p - 1, np.uint8)
        B = np.full((k, n), p - 1, np.uint8)
        items.append((p, dev(A), dev(B), torch.zeros((m, n), dtype=torch.uint8, device="cuda")))
        refs.append(oracle.gemm(p, A[:1], B)[0])
    for algo in ("tc_f16", "dot32", "tc_f8"):
        arr, cnt = gfp.make_problems(items)
        gfp.gfp_gemm_batched(arr, cnt, algo)
        for (p, A, B, C), ref in zip(items, refs):
            assert (host(C) == ref).all(), (algo, p)


def test_batched_invalid_entries_are_skipped():
    items, host_ops = random_batch(12, 6)
    arr, cnt = gfp.make_problems(items)
    arr[2].p = 4                       # not prime
    arr[4].lda = 0                     # ld too small
    ws, r, st = gfp.gfp_gemm_batched(arr, cnt, "auto", statuses=True)
    assert r == 2 and st[2] == 2 and st[4] == 1
    for i, ((p, A, B), (_, _, _, C)) in enumerate(zip(host_ops, items)):
        got = host(C)
        if i in (2, 4):
            assert (got == 255).all()
        else:
            assert (got == oracle.gemm(p, A, B)).all()


def test_batched_empty_and_degenerate():
    arr, cnt = gfp.make_problems([])
    gfp.gfp_gemm_batched(arr, 0, "auto")
    C = torch.full((3, 4), 9, dtype=torch.uint8, device="cuda")
    Z = torch.zeros((3, 0), dtype=torch.uint8, device="cuda")
    arr, cnt = gfp.make_problems([(5, Z, torch.zeros((0, 4), dtype=torch.uint8, device="cuda"), C)])
    gfp.gfp_gemm_batched(arr, cnt, "tc_f16")
    assert (host(C) == 0).all()


def test_batched_graph_replay():
    items, host_ops = random_batch(13, 40, smax=200)
    arr, cnt = gfp.make_problems(items)
    ws = torch.empty(gfp.gfp_batched_workspace_size(arr, cnt), dtype=torch.uint8, device="cuda")
    gfp.gfp_batched_prepare(arr, cnt, "auto", ws)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gfp.gfp_batched_launch(ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gfp.gfp_batched_launch(ws)
    for rep in range(2):
        for it in items:
            it[3].fill_(255)
        graph.replay()
        torch.cuda.synchronize()
        for (p, A, B), (_, _, _, C) in zip(host_ops, items):
            assert (host(C) == oracle.gemm(p, A, B)).all()


def test_autotune_then_auto():
    items, host_ops = random_batch(14, 60, primes=(3, 5, 7), smax=520)
    arr, cnt = gfp.make_problems(items)
    table = gfp.gfp_batched_autotune(arr, cnt)
    # per bucket a kind, or -1 when the whole-batch comparison kept the defaults
    assert len(table) == 7 and all(v in (-1, 0, 1, 2, 3, 4) for v in table)
    for it in items:
        it[3].fill_(255)
    gfp.gfp_gemm_batched(arr, cnt, "auto")
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all()
    gfp.gfp_batched_set_table([-1] * 7)


def test_adjacency_workload_4096():
    """The full batched workload: 4096 squares of symmetric 0/1 adjacency
    matrices, n log-uniform in [16, 512], p in {3, 5, 7}.  Every product is
    checked by Freivalds' test; 256 of them (and every one with n <= 40)
    against the oracle entry by entry."""
    probs = inputs.batched_problems()
    items = []
    for p, A in probs:
        Ad = dev(A)
        items.append((p, Ad, Ad, torch.empty(A.shape, dtype=torch.uint8, device="cuda")))
    arr, cnt = gfp.make_problems(items)
    gfp.gfp_gemm_batched(arr, cnt, "auto")
    torch.cuda.synchronize()
    g = np.random.Generator(np.random.PCG64(5))
    sample = set(g.choice(len(probs), size=256, replace=False).tolist())
    for i, ((p, A), it) in enumerate(zip(probs, items)):
        C = it[3].cpu().numpy()
        assert freivalds(p, A, A, C, rounds=4, seed=i)
        if i in sample or A.shape[0] <= 40:
            assert (C == oracle.gemm(p, A, A)).all(), i


def test_batched_tcgen05_tiles_graph_replay():
    """The grouped tcgen05 tiles (p < 16, raw e4m3 operands): square and
    rectangular problems around the 128-tile edges, replayed from a graph."""
    g = np.random.Generator(np.random.PCG64(21))
    items, host_ops = [], []
    for p, m, k, n in ((3, 128, 128, 128), (5, 129, 200, 127), (7, 300, 513, 260), (13, 97, 64, 400),
                       (2, 512, 512, 512), (11, 1, 700, 130)):
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        items.append((p, dev(A), dev(B), torch.full((m, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A, B))
    arr, cnt = gfp.make_problems(items)
    ws = torch.empty(gfp.gfp_batched_workspace_size(arr, cnt), dtype=torch.uint8, device="cuda")
    gfp.gfp_batched_prepare(arr, cnt, "tc_f8", ws)
    gfp.gfp_batched_launch(ws)
    torch.cuda.synchronize()
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all()
    assert int(ws[192:196].cpu().numpy().view(np.int32)[0]) == 0      # tcgen05 status word
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gfp.gfp_batched_launch(ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        gfp.gfp_batched_launch(ws)
    for it in items:
        it[3].fill_(255)
    graph.replay()
    torch.cuda.synchronize()
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all()


def test_batched_tcgen05_garbage_workspace():
    """Stacked tcgen05 operands are not padded: rows of neighbouring
    problems and unwritten columns share the 128 x 128 boxes.  A workspace
    filled with 0xFF (an e4m3 NaN code) before preparation must not change
    any stored output: k around multiples of 32 and 128, m and n around the
    tile edges, shared operands, several stride bins."""
    g = np.random.Generator(np.random.PCG64(22))
    items, host_ops = [], []
    shared = inputs.residues(g, 7, 140, 33)
    for p, m, k, n in ((3, 97, 1, 200), (5, 130, 31, 99), (7, 140, 33, 150), (13, 200, 129, 129),
                       (11, 255, 257, 97), (2, 128, 1000, 300), (3, 300, 96, 101), (5, 101, 160, 400),
                       (31, 130, 65, 99), (251, 200, 300, 129), (17, 97, 1, 140)):
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        items.append((p, dev(A), dev(B), torch.full((m, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A, B))
    Sd = dev(shared)
    for n in (97, 250):                               # one A, two products
        B = inputs.residues(g, 7, 33, n)
        items.append((7, Sd, dev(B), torch.full((140, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((7, shared, B))
    arr, cnt = gfp.make_problems(items)
    ws = torch.full((gfp.gfp_batched_workspace_size(arr, cnt),), 255, dtype=torch.uint8, device="cuda")
    gfp.gfp_batched_prepare(arr, cnt, "tc_f8", ws)
    gfp.gfp_batched_launch(ws)
    torch.cuda.synchronize()
    assert int(ws[192:196].cpu().numpy().view(np.int32)[0]) == 0
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all(), (p, A.shape, B.shape)


def test_batched_tcgen05_fp16_tiles():
    """p >= 16 on the grouped tcgen05 tiles: centred fp16 operands (kind::f16)
    in the same launch as raw e4m3 problems; ragged shapes; one matrix shared
    by products mod 31 and mod 251 (centred differently); the worst case at
    the fp16 bound (p = 251, k = 1073: every sum k h^2 below 2^24) and one
    past it (k = 1074, which falls back to the mma.sync tiles)."""
    g = np.random.Generator(np.random.PCG64(23))
    items, host_ops = [], []
    for p, m, k, n in ((17, 129, 200, 127), (31, 300, 513, 260), (101, 97, 64, 400), (251, 1, 700, 130),
                       (251, 256, 1000, 256), (3, 200, 300, 200), (19, 33, 17, 35)):
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        items.append((p, dev(A), dev(B), torch.full((m, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A, B))
    shared = inputs.residues(g, 31, 130, 150)       # one matrix, centred differently for p = 31 and 251
    for pp in (31, 251):
        Bs = inputs.residues(g, 31, 150, 90)
        items.append((pp, dev(shared), dev(Bs), torch.full((130, 90), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((pp, shared, Bs))
    for k in (1073, 1074):
        A = np.full((150, k), 125, np.uint8)          # centred +125
        B = np.full((k, 140), 126, np.uint8)          # centred -125
        items.append((251, dev(A), dev(B), torch.full((150, 140), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((251, A, B))
    arr, cnt = gfp.make_problems(items)
    ws = torch.full((gfp.gfp_batched_workspace_size(arr, cnt),), 255, dtype=torch.uint8, device="cuda")
    gfp.gfp_batched_prepare(arr, cnt, "tc_f8", ws)
    gfp.gfp_batched_launch(ws)
    torch.cuda.synchronize()
    assert int(ws[192:196].cpu().numpy().view(np.int32)[0]) == 0
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all(), (p, A.shape, B.shape)


def test_adjacency_workload_b_is_a_transpose_flag():
    """The same workload with each problem flagged B = A^T (true: A is
    symmetric and B = A): the tensor-core tiles stage one copy of A for both
    operands.  Every product equals the unflagged launch's bit for bit, and a
    sample equals the oracle's."""
    probs = inputs.batched_problems()
    runs = []
    for flags in (0, gfp.PROBLEM_B_IS_A_T):
        items = []
        for p, A in probs:
            Ad = dev(A)
            items.append((p, Ad, Ad, torch.full(A.shape, 255, dtype=torch.uint8, device="cuda")))
        arr, cnt = gfp.make_problems(items, flags=flags)
        gfp.gfp_gemm_batched(arr, cnt, "auto")
        torch.cuda.synchronize()
        runs.append([it[3].cpu().numpy() for it in items])
    for i, (C0, C1) in enumerate(zip(*runs)):
        assert (C0 == C1).all(), i
    for i in range(0, len(probs), 97):
        p, A = probs[i]
        assert (runs[1][i] == oracle.gemm(p, A, A)).all(), i


def test_b_is_a_transpose_flag_validation():
    """The flag needs n == m; unknown bits are rejected (per-problem status
    GFP_EINVAL); a flagged non-symmetric product gives A A^T, as documented."""
    g = np.random.Generator(np.random.PCG64(31))
    A = inputs.residues(g, 5, 40, 30)
    B = inputs.residues(g, 5, 30, 50)
    items = [(5, dev(A), dev(B), torch.empty((40, 50), dtype=torch.uint8, device="cuda"))]
    for flags in (gfp.PROBLEM_B_IS_A_T, 2):
        arr, cnt = gfp.make_problems(items, flags=flags)
        _, r, sts = gfp.gfp_gemm_batched(arr, cnt, "auto", statuses=True)
        torch.cuda.synchronize()
        assert r == 1 and sts == [1]
    At = np.ascontiguousarray(A.T)                  # B = A^T: 30 x 40, n = m = 40
    C = torch.empty((40, 40), dtype=torch.uint8, device="cuda")
    arr, cnt = gfp.make_problems([(5, dev(A), dev(At), C)], flags=gfp.PROBLEM_B_IS_A_T)
    gfp.gfp_gemm_batched(arr, cnt, "tc_f8")
    assert (host(C) == oracle.gemm(5, A, At)).all()


@pytest.mark.parametrize("algo", ["tc_f8", "auto"])
def test_b_is_a_transpose_symmetric_tiles(algo):
    """Flagged B = A^T with A not symmetric and k != m: C = A A^T is
    symmetric, so the tensor-core tiles compute only the tiles on and above
    the diagonal and store each one above it twice.  Ragged sizes of one to
    five 128-row tiles, raw e4m3 (p < 16) and centred fp16 (p >= 16) operands
    in one launch, C written into views with a wider row stride inside a
    sentinel-filled buffer; every entry against the oracle, nothing outside
    the views touched."""
    g = np.random.Generator(np.random.PCG64(37))
    items, host_ops, bufs = [], [], []
    for p, m, k in ((3, 129, 40), (5, 300, 513), (7, 513, 200), (31, 257, 300), (251, 640, 64),
                    (2, 128, 128), (5, 1, 7), (7, 255, 1)):
        A = inputs.residues(g, p, m, k)
        At = np.ascontiguousarray(A.T)
        buf = torch.full((m + 2, m + 19), 254, dtype=torch.uint8, device="cuda")
        C = buf[1:m + 1, 3:m + 3]
        items.append((p, dev(A), dev(At), C))
        host_ops.append((p, A, At))
        bufs.append(buf)
    arr, cnt = gfp.make_problems(items, flags=gfp.PROBLEM_B_IS_A_T)
    gfp.gfp_gemm_batched(arr, cnt, algo)
    torch.cuda.synchronize()
    for (p, A, At), (_, _, _, C), buf in zip(host_ops, items, bufs):
        ref = oracle.gemm(p, A, At)
        assert (ref == ref.T).all()
        assert (host(C) == ref).all(), (p, A.shape)
        out = host(buf).copy()
        out[1:A.shape[0] + 1, 3:A.shape[0] + 3] = 254
        assert (out == 254).all(), (p, A.shape)


@pytest.mark.parametrize("algo", ["tc_f8", "tc_f16", "dot32", "auto"])
def test_batched_strided_unaligned_operands(algo):
    """Operands given as views with a wider row stride at odd byte offsets
    (every row of A and B starts at another alignment), so that the operand
    staging joins misaligned 16-byte blocks and zero-fills row ends; raw e4m3,
    fp16 and word tiles in one launch; every entry against the oracle."""
    g = np.random.Generator(np.random.PCG64(41))
    items, host_ops, keep = [], [], []
    for p, m, k, n in ((3, 37, 1, 5), (5, 130, 17, 129), (7, 64, 300, 70), (31, 200, 129, 33),
                       (251, 90, 513, 140), (2, 257, 64, 1), (13, 1, 700, 300), (17, 45, 31, 400)):
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        bufA = dev(inputs.residues(g, p, m + 3, k + 21))
        bufB = dev(inputs.residues(g, p, k + 2, n + 13))
        Av = bufA[2:m + 2, 5:k + 5]
        Bv = bufB[1:k + 1, 7:n + 7]
        Av.copy_(dev(A))
        Bv.copy_(dev(B))
        items.append((p, Av, Bv, torch.full((m, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A, B))
        keep += [bufA, bufB]
    arr, cnt = gfp.make_problems(items)
    gfp.gfp_gemm_batched(arr, cnt, algo)
    torch.cuda.synchronize()
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all(), (p, A.shape, B.shape)


@pytest.mark.parametrize("algo", ["tc_f8", "tc_f16"])
def test_batched_row_staging_boundary(algo):
    """Rows of A around the largest that one bulk copy stages (k + 31 source
    bytes against the 18,368-byte limit, from any byte offset): k = 18,337
    fits, 18,338 goes through the per-warp row runs; both in one launch, as
    views at odd offsets, and against the oracle.  tc_f8 stages raw e4m3 rows
    (p < 16) and centred fp16 rows (p = 31); tc_f16 the padded fp16 copies of
    the mma.sync tiles."""
    g = np.random.Generator(np.random.PCG64(43))
    items, host_ops, keep = [], [], []
    for p, m, k, n in ((3, 5, 18337, 7), (3, 6, 18338, 9), (31, 3, 18337, 5), (5, 2, 18336, 3)):
        A = inputs.residues(g, p, m, k)
        B = inputs.residues(g, p, k, n)
        bufA = dev(inputs.residues(g, p, m + 1, k + 7))
        Av = bufA[1:m + 1, 3:k + 3]
        Av.copy_(dev(A))
        items.append((p, Av, dev(B), torch.full((m, n), 255, dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A, B))
        keep.append(bufA)
    arr, cnt = gfp.make_problems(items)
    ws = torch.full((gfp.gfp_batched_workspace_size(arr, cnt),), 255, dtype=torch.uint8, device="cuda")
    gfp.gfp_batched_prepare(arr, cnt, algo, ws)
    gfp.gfp_batched_launch(ws)
    torch.cuda.synchronize()
    assert int(ws[192:196].cpu().numpy().view(np.int32)[0]) == 0
    for (p, A, B), (_, _, _, C) in zip(host_ops, items):
        assert (host(C) == oracle.gemm(p, A, B)).all(), (p, A.shape, B.shape)
