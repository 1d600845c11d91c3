"""GPU parity: every form through the C ABI against the CPU oracle, bit for
bit, on seeded inputs.  Sizes span several tiles and ragged tails; adversarial
inputs (all p-1, k at the bound) and edge shapes are included."""
import numpy as np
import pytest
import torch

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import (THREADS, dev, ensure_built, freivalds, host, np_words_dtype, operands, oracle_product,
                     to_word_tensor, words_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# --------------------------------------------------------------------------- pack
PACK_CASES = [(3, 1024, 1024, 3, 13), (3, 37, 129, 3, 13), (5, 130, 67, 2, 19), (251, 9, 300, 1, 30),
              (2, 64, 64, 7, 8), (7, 1, 1, 0, 6),
              # rows of several staged chunks (a chunk holds up to 8192 residues)
              (3, 5, 20001, 3, 13), (251, 3, 9001, 0, 30), (5, 3, 10001, 1, 19), (3, 4, 12002, 2, 13),
              # long rows of more than four residues per word (the run-time digit count)
              (2, 3, 9000, 7, 8), (3, 2, 10007, 5, 10)]


@pytest.mark.parametrize("word", ["u64", "u32w", "f64"])
@pytest.mark.parametrize("p,rows,cols,d,t", PACK_CASES)
@pytest.mark.parametrize("layout", ["rows_rev", "cols", "rows"])
def test_pack_unpack(word, p, rows, cols, d, t, layout):
    Q = 2 ** t
    try:
        gfp.gfp_params(p, 1, 1, 1, "dot", "u64", d=d, Q=Q)   # (lower) with k = 1
    except gfp.GfpError:
        pytest.skip("not a valid (p, Q)")
    big = 53 if word == "f64" else (32 if word == "u32w" else 64)
    if oracle.amax(p, Q, d) >= 2 ** big:
        with pytest.raises(gfp.GfpError):
            gfp.gfp_pack(p, dev(np.zeros((rows, cols), np.uint8)), d, Q, layout, word)
        return
    g = inputs.rng(80, rows + cols + d)
    X = inputs.residues(g, p, rows, cols)
    W = gfp.gfp_pack(p, dev(X), d, Q, layout, word)
    dt = np_words_dtype(word)
    ref = {"rows_rev": oracle.pack_rows_rev, "cols": oracle.pack_cols,
           "rows": oracle.pack_rows}[layout](X, d, Q, dtype=np.uint64)
    got = words_np(W, word)
    assert got.shape == ref.shape
    assert (got.astype(np.uint64) == ref).all() if dt is not np.float64 else (got == ref.astype(np.float64)).all()
    back = gfp.gfp_unpack(p, W, rows, cols, d, Q, layout, word)
    assert (host(back) == X).all()


def test_pack_strided_views():
    """Leading dimensions larger than the row: pack a sub-matrix view."""
    g = inputs.rng(81, 0)
    X = inputs.residues(g, 3, 40, 100)
    Xd = dev(X)[:, 3:90]
    W = torch.zeros((40, 50), dtype=torch.int64, device="cuda")
    gfp.gfp_pack(3, Xd, 3, 2 ** 13, "rows_rev", "u64", out=W[:, :22])
    ref = oracle.pack_rows_rev(np.ascontiguousarray(X[:, 3:90]), 3, 2 ** 13)
    got = words_np(W, "u64")
    assert (got[:, :22] == ref).all() and (got[:, 22:] == 0).all()


@pytest.mark.parametrize("word", ["u64", "u32w", "f64"])
@pytest.mark.parametrize("layout", ["rows_rev", "rows"])
def test_pack_unpack_long_unaligned_rows(word, layout):
    """Rows of several chunks starting at odd byte addresses (a view with an
    odd leading dimension and column offset), unpacked into a strided view of a
    sentinel-filled buffer: only the view's bytes change."""
    p, t = 3, 13
    d = 2 if word == "u32w" else 3      # the largest 32-bit word holds three digits of 2^13
    Q = 2 ** t
    g = inputs.rng(82, len(word) + len(layout))
    big = inputs.residues(g, p, 7, 30011)
    X = np.ascontiguousarray(big[:, 5:29999])
    Xd = dev(big)[:, 5:29999]
    W = gfp.gfp_pack(p, Xd, d, Q, layout, word)
    ref = {"rows_rev": oracle.pack_rows_rev, "rows": oracle.pack_rows}[layout](X, d, Q, dtype=np.uint64)
    got = words_np(W, word)
    dt = np_words_dtype(word)
    assert (got.astype(np.uint64) == ref).all() if dt is not np.float64 else (got == ref.astype(np.float64)).all()
    sentinel = torch.full((9, 30017), 0xA5, dtype=torch.uint8, device="cuda")
    view = sentinel[1:8, 3:3 + X.shape[1]]
    gfp.gfp_unpack(p, W, X.shape[0], X.shape[1], d, Q, layout, word, out=view)
    out = host(sentinel)
    assert (out[1:8, 3:3 + X.shape[1]] == X).all()
    mask = np.ones(out.shape, bool)
    mask[1:8, 3:3 + X.shape[1]] = False
    assert (out[mask] == 0xA5).all()


def test_dp4a_aligned_rows_with_a_partial_last_group():
    """dp4a reads A four residues at a time when its rows are 4-byte aligned: with
    k = 1025 inside rows of 1028 bytes, the last group holds three bytes past k
    (real residues of the wider matrix), which must not reach C."""
    p, m, k, n = 7, 300, 1025, 260
    g = inputs.rng(83, 0)
    wide = inputs.residues(g, p, m, 1028)
    B = inputs.residues(g, p, k, n)
    C = gfp.gfp_gemm(p, dev(wide)[:, :k], dev(B), "dp4a")
    assert (host(C) == oracle.gemm(p, np.ascontiguousarray(wide[:, :k]), B, threads=THREADS)).all()


@pytest.mark.parametrize("algo", ["dp4a", "tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"])
def test_wider_than_the_grid_limit(algo):
    """n = 4,300,000 columns: more 64-column tiles of B^T (67,188) than a grid's y
    dimension holds (65,535); the operand transposes loop over them."""
    p, m, k, n = 5, 3, 5, 4_300_000
    A, B = operands(10, 1, p, m, k, n)
    C = gfp.gfp_gemm(p, dev(A), dev(B), algo)
    assert (host(C) == oracle.gemm(p, A, B, threads=THREADS)).all()


def test_taller_than_the_grid_limit():
    """m = 8,400,000 rows: more row tiles than a grid's y dimension holds
    (65,535 tiles of 128 rows, or of the CUDA-core kernels' tiles); the
    launches run over bands of rows.  Every uncompressed algorithm, the dot
    form in 32- and 64-bit words and the right-compressed form."""
    p, m, k, n = 5, 8_400_000, 5, 3
    A, B = operands(10, 2, p, m, k, n)
    ref = oracle.gemm(p, A, B, threads=THREADS)
    Ad, Bd = dev(A), dev(B)
    for algo in ALGOS:
        assert (host(gfp.gfp_gemm(p, Ad, Bd, algo)) == ref).all(), algo
    for word in ("u32", "u64"):
        d, Q, _ = gfp.gfp_params(p, m, k, n, "dot", word)
        CA = gfp.gfp_pack(p, Ad, d, Q, "rows_rev", word)
        CB = gfp.gfp_pack(p, Bd, d, Q, "cols", word)
        assert (host(gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB)) == ref).all(), word
        del CA, CB
    d, Q, _ = gfp.gfp_params(p, m, k, n, "mixed", "u64")
    CB = gfp.gfp_pack(p, Bd, d, Q, "rows", "u64")
    CC = gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "mixed", "u64", Ad, CB)
    assert (host(gfp.gfp_unpack(p, CC, m, n, d, Q, "rows", "u64")) == ref).all()


# Results spanning at least two waves of the 128 x 128 and 128 x 64 register tiles
# of the CUDA-core kernels (the only shapes that use them), ragged in both
# dimensions: at 4001 x 3999 the classical and dp4a products run on 128 x 128
# tiles, the 32-bit word products (whole and k-blocked) on 128 x 64.
@pytest.fixture(scope="module")
def wide_case():
    p, m, k, n = 3, 4001, 200, 3999
    A, B = operands(9, 1, p, m, k, n)
    return p, A, B, oracle.gemm(p, A, B, threads=THREADS)


@pytest.mark.parametrize("form", ["plain", "dp4a", "dot_u32", "dot_u32_kb60", "dot_u32w", "dot_u64"])
def test_large_register_tiles_ragged(wide_case, form):
    p, A, B, ref = wide_case
    m, k = A.shape
    n = B.shape[1]
    Ad, Bd = dev(A), dev(B)
    if form in ("plain", "dp4a"):
        C = gfp.gfp_gemm(p, Ad, Bd, form)
    else:
        word = form.split("_")[1]
        kb = 60 if form.endswith("kb60") else 0
        d, Q, kb = gfp.gfp_params(p, m, k, n, "dot", word, kb=kb)
        CA = gfp.gfp_pack(p, Ad, d, Q, "rows_rev", word)
        CB = gfp.gfp_pack(p, Bd, d, Q, "cols", word)
        C = gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB, kb=kb)
    assert (host(C) == ref).all()


# ------------------------------------------------------------------ plain / TC
GEMM_CASES = [(3, 256, 256, 256), (3, 1024, 1024, 1024), (5, 129, 300, 77), (251, 200, 513, 130),
              (2, 65, 64, 63), (7, 1, 1, 1), (31, 3, 1000, 5), (13, 128, 17, 128), (3, 300, 1, 299)]


ALGOS = ["plain", "dp4a", "tc_mma_s8", "tc_f16", "tc_f8", "tc_e2m1"]


def skip_unsupported(algo, p):
    limit = {"tc_f8": 31, "tc_e2m1": 7}.get(algo)
    if limit is not None and p > limit:
        with pytest.raises(gfp.GfpError) as e:
            gfp.gfp_gemm_workspace_size(p, 8, 8, 8, algo)
        assert e.value.status == 5
        pytest.skip("%s operands hold the centred residues of p <= %d only" % (algo, limit))


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("p,m,k,n", GEMM_CASES)
def test_gemm_matches_oracle(algo, p, m, k, n):
    skip_unsupported(algo, p)
    A, B = operands(2, 0, p, m, k, n)
    C = host(gfp.gfp_gemm(p, dev(A), dev(B), algo))
    assert (C == oracle_product(2, 0, p, m, k, n)).all()


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("p", [3, 7, 31, 251])
def test_gemm_worst_case(algo, p):
    """All entries p-1 (largest sums); for the centred form also the largest
    centred magnitude h = (p-1)/2 with both signs."""
    skip_unsupported(algo, p)
    m = k = n = 192
    h = (p - 1) // 2
    for fill_a, fill_b in ((p - 1, p - 1), (h, h), (h + 1, h), (h + 1, h + 1)):
        A = np.full((m, k), fill_a, np.uint8)
        B = np.full((k, n), fill_b, np.uint8)
        C = host(gfp.gfp_gemm(p, dev(A), dev(B), algo))
        assert (C == oracle.gemm(p, A, B)).all()


@pytest.mark.parametrize("algo", ALGOS)
def test_gemm_edges(algo):
    # empty inner dimension: C = 0
    C = torch.full((5, 7), 9, dtype=torch.uint8, device="cuda")
    gfp.gfp_gemm(3, torch.zeros((5, 0), dtype=torch.uint8, device="cuda"),
                 torch.zeros((0, 7), dtype=torch.uint8, device="cuda"), algo, out=C)
    assert (host(C) == 0).all()
    # strided views in and out
    A, B = operands(3, 1, 5, 70, 90, 60)
    Ad = dev(np.pad(A, ((0, 0), (0, 10))))[:, :90]
    Bd = dev(np.pad(B, ((0, 0), (0, 4))))[:, :60]
    Cd = torch.full((70, 64), 200, dtype=torch.uint8, device="cuda")
    gfp.gfp_gemm(5, Ad, Bd, algo, out=Cd[:, :60])
    got = host(Cd)
    assert (got[:, :60] == oracle.gemm(5, A, B)).all() and (got[:, 60:] == 200).all()


def tc_f16_status(ws: torch.Tensor) -> int:
    torch.cuda.synchronize()
    return int(ws[:4].cpu().numpy().view(np.int32)[0])


@pytest.mark.parametrize("algo,p", [("tc_f16", 3), ("tc_f16", 31), ("tc_f16", 251), ("tc_f8", 3),
                                    ("tc_f8", 31)])
def test_tc_exact_accumulation(algo, p):
    """fp32 accumulation in tensor memory is exact while partial sums are
    integers below 2^24.  Patterns at the k-block bound kb: all products +h^2
    (partial sums reach kb h^2), alternating signs, a large accumulator
    followed by small addends, and one k-block past the bound (blocked path)."""
    h = (p - 1) // 2
    kb = ((1 << 24) - 1 - p) // (h * h) // 128 * 128
    k = min(kb, 80000)                        # p = 31: 74560, p = 251: 1024
    m, n = 128, 256
    pos, neg = h, h + 1                       # residues whose centred values are +h, -h
    pats = {
        "all+": (np.full((m, k), pos, np.uint8), np.full((k, n), pos, np.uint8)),
        "all-+": (np.full((m, k), neg, np.uint8), np.full((k, n), pos, np.uint8)),
        "alt": (np.full((m, k), pos, np.uint8),
                np.where((np.arange(k) % 2)[:, None] == 0, pos, neg).astype(np.uint8).repeat(n, 1)),
    }
    big_then_small = np.full((m, k), pos, np.uint8)
    big_then_small[:, k // 2:] = 1
    pats["big-then-small"] = (big_then_small, np.full((k, n), pos, np.uint8))
    for name, (A, B) in pats.items():
        ws = torch.empty(gfp.gfp_gemm_workspace_size(p, m, k, n, algo), dtype=torch.uint8,
                         device="cuda")
        C = host(gfp.gfp_gemm(p, dev(A), dev(B), algo, workspace=ws))
        assert tc_f16_status(ws) == 0
        assert (C == oracle.gemm(p, A[:2], B)[0]).all(), name   # rows are identical


@pytest.mark.parametrize("p", [2, 3, 5, 7])
def test_tc_e2m1_exact_accumulation(p):
    """The block-scaled e2m1 MMA (unit scale factors) with fp32 accumulation at
    its k-block bound kb (kb h^2 + p < 2^24; h = 3 at p = 7: kb = 1,864,192):
    all products +h^2 (the sums reach kb h^2 ~ 2^24), products of both signs,
    a large accumulator followed by small addends, and one k-block and a
    ragged tail past the bound (the blocked path).  Every row and every column
    of each pattern is the same, so one oracle dot product is the expected
    value of all of C."""
    h = 1 if p == 2 else (p - 1) // 2
    kb = ((1 << 24) - 1 - p) // (h * h) // 256 * 256
    k = min(kb, 1 << 21)
    m, n = 128, 192
    pos, neg = h, (p - h if p > 2 else 1)      # centred +h and -h (p = 2: 0/1 only)
    pats = {
        "all+": (np.full((m, k), pos, np.uint8), np.full((k, n), pos, np.uint8)),
        "all-+": (np.full((m, k), neg, np.uint8), np.full((k, n), pos, np.uint8)),
        "alt": (np.full((m, k), pos, np.uint8),
                np.where((np.arange(k) % 2)[:, None] == 0, pos, neg).astype(np.uint8).repeat(n, 1)),
    }
    big_then_small = np.full((m, k), pos, np.uint8)
    big_then_small[:, k // 2:] = 1
    pats["big-then-small"] = (big_then_small, np.full((k, n), pos, np.uint8))
    if kb <= 1 << 21:                          # p = 7: the bound itself is in reach
        k2 = kb + 300
        pats["past-the-block"] = (np.full((m, k2), pos, np.uint8), np.full((k2, n), pos, np.uint8))
    for name, (A, B) in pats.items():
        mk, kk = A.shape
        ws = torch.empty(gfp.gfp_gemm_workspace_size(p, mk, kk, n, "tc_e2m1"), dtype=torch.uint8,
                         device="cuda")
        C = host(gfp.gfp_gemm(p, dev(A), dev(B), "tc_e2m1", workspace=ws))
        assert tc_f16_status(ws) == 0
        want = oracle.gemm(p, A[:1], np.ascontiguousarray(B[:, :1]))[0, 0]
        assert (C == want).all(), name
        del ws, C


@pytest.mark.parametrize("algo,p", [("tc_f16", 251), ("tc_f8", 31), ("tc_e2m1", 7)])
def test_tc_pairs_exact_accumulation(algo, p):
    """The CTA-pair kernels (chosen when the 256-row tiles give every pair of
    SMs a tile: here m = 256, n = 19456) with fp32 accumulation at the k-block
    bound kb: all products +h^2, products of both signs, a large accumulator
    followed by small addends; fp16 at p = 251 also runs two k-blocks and a
    ragged tail (the blocked path).  Operands are built on the GPU (B is up to
    36 GB for e2m1 at p = 7, kb = 1,864,192); every entry of C has the same
    expected value, one oracle dot product."""
    h = (p - 1) // 2
    step = 256 if algo == "tc_e2m1" else 128
    kb = ((1 << 24) - 1 - p) // (h * h) // step * step
    k = 2 * kb + 300 if algo == "tc_f16" else kb
    m, n = 256, 19456
    pos, neg = h, h + 1                       # centred +h and -h
    col = {"all+": np.full(k, pos, np.uint8), "alt": np.where(np.arange(k) % 2 == 0, pos, neg).astype(np.uint8)}
    row = {"all+": np.full(k, pos, np.uint8), "alt": np.full(k, pos, np.uint8),
           "big-then-small": np.where(np.arange(k) < k // 2, pos, 1).astype(np.uint8)}
    for name, bname in (("all+", "all+"), ("alt", "alt"), ("big-then-small", "all+")):
        A = dev(row[name])[None, :].expand(m, k).contiguous()
        B = dev(col[bname])[:, None].expand(k, n).contiguous()
        ws = torch.empty(gfp.gfp_gemm_workspace_size(p, m, k, n, algo), dtype=torch.uint8, device="cuda")
        C = host(gfp.gfp_gemm(p, A, B, algo, workspace=ws))
        assert tc_f16_status(ws) == 0, name
        want = oracle.gemm(p, row[name][None, :], col[bname][:, None])[0, 0]
        assert (C == want).all(), name
        del A, B, ws
        torch.cuda.empty_cache()


def test_tc_f16_blocked_path():
    """p = 251 beyond one fp32 k-block (kb = 1024): running residues across
    k-blocks, random and worst-case inputs."""
    p, m, k, n = 251, 200, 3 * 1024 + 64 + 17, 300
    A, B = operands(5, 0, p, m, k, n)
    ws = torch.empty(gfp.gfp_gemm_workspace_size(p, m, k, n, "tc_f16"), dtype=torch.uint8, device="cuda")
    C = host(gfp.gfp_gemm(p, dev(A), dev(B), "tc_f16", workspace=ws))
    assert tc_f16_status(ws) == 0
    assert (C == oracle.gemm(p, A, B, threads=8)).all()
    A = np.full((m, k), 126, np.uint8)        # centred -125
    B = np.full((k, n), 125, np.uint8)        # centred +125
    C = host(gfp.gfp_gemm(p, dev(A), dev(B), "tc_f16", workspace=ws))
    assert (C == oracle.gemm(p, A[:1], B)[0]).all()


def test_tc_kblock_reduction():
    """k beyond one int32 k-block for p = 251 (kb = 68672): the blocked
    reduction path, checked on sampled rows."""
    p, m, k, n = 251, 128, 70000, 128
    g = inputs.rng(33, 0)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    C = host(gfp.gfp_gemm(p, dev(A), dev(B), "tc_mma_s8"))
    rows = [0, 1, 63, 64, 127]
    assert (C[rows] == oracle.gemm_rows(p, rows, A, B, threads=8)).all()


# --------------------------------------------------------------- compressed dot
DOT_CASES = [(3, 1024, 1024, 1024), (3, 100, 333, 70), (5, 64, 1000, 200), (31, 40, 8, 50),
             (2, 129, 257, 65), (251, 33, 40, 33),
             (7, 1, 1, 1), (3, 1, 500, 1), (5, 300, 1, 2), (3, 2, 3, 1)]


@pytest.mark.parametrize("word", ["u64", "u64x128", "u32w", "u32", "f64"])
@pytest.mark.parametrize("p,m,k,n", DOT_CASES)
def test_dot_matches_oracle(word, p, m, k, n):
    """Procedure (2) of Section 2.2: CompressRows(A), CompressColumns(B), CA x CB."""
    try:
        d, Q, _ = gfp.gfp_params(p, m, k, n, "dot", word)
    except gfp.GfpError:
        pytest.skip("no admissible (d, Q)")
    A, B = operands(2, 1, p, m, k, n)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word)
    C = host(gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB))
    assert (C == oracle_product(2, 1, p, m, k, n)).all()


@pytest.mark.parametrize("word", ["u64", "u64x128", "u32w", "u32", "f64"])
def test_dot_at_the_bound(word):
    """All entries p-1 at the largest k of eq. (lower) for the chosen Q."""
    p = 3
    d, Q, _ = gfp.gfp_params(p, 64, 1024, 64, "dot", word)
    k = (Q - 1) // 4
    d, Q2, _ = gfp.gfp_params(p, 64, k, 64, "dot", word, d=d, Q=Q)
    A = np.full((70, k), 2, np.uint8)
    B = np.full((k, 66), 2, np.uint8)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word)
    C = host(gfp.gfp_gemm_compressed(p, 70, k, 66, d, Q, "dot", word, CA, CB))
    assert (C == (k * 4) % 3).all()


def test_dot_f64_round_toward_zero_case():
    """The case where round-to-nearest FP64 accumulation loses the digit
    (p = 3, Q = 2^10, d = 4, k = 255, all entries 2) is exact here."""
    p, d, Q, k = 3, 4, 2 ** 10, 255
    A = np.full((33, k), 2, np.uint8)
    B = np.full((k, 35), 2, np.uint8)
    assert oracle.dqt_dot_fp64(A[0], B[:, 0], p, d, Q, "rn") != (k * 4) % 3
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", "f64")
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", "f64")
    C = host(gfp.gfp_gemm_compressed(p, 33, k, 35, d, Q, "dot", "f64", CA, CB))
    assert (C == (k * 4) % 3).all()


@pytest.mark.parametrize("word", ["u64", "u64x128", "u32w", "u32", "f64"])
@pytest.mark.parametrize("p,k,kb", [(3, 1024, 60), (5, 1000, 48), (3, 777, 28), (7, 500, 10)])
def test_dot_blocked(word, p, k, kb):
    """k-blocked extraction: the lower bound holds for kb only."""
    m, n = 96, 80
    d, Q, kbr = gfp.gfp_params(p, m, k, n, "dot", word, kb=kb)
    A, B = operands(4, kb, p, m, k, n)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word)
    C = host(gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB, kb=kbr))
    assert (C == oracle.gemm(p, A, B)).all()
    # worst case within each block
    A = np.full((m, k), p - 1, np.uint8)
    B = np.full((k, n), p - 1, np.uint8)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", word)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", word)
    C = host(gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", word, CA, CB, kb=kbr))
    assert (C == (k * (p - 1) ** 2) % p).all()


# ------------------------------------------------------------------------ mixed
MIXED_CASES = [(3, 1024, 1024, 1024), (3, 77, 300, 101), (5, 64, 200, 64), (251, 20, 30, 41),
               (2, 65, 129, 67), (7, 1, 1, 1), (3, 1, 500, 1), (5, 300, 1, 2), (3, 2, 3, 1)]


@pytest.mark.parametrize("word", ["u64", "f64"])
@pytest.mark.parametrize("p,m,k,n", MIXED_CASES)
def test_mixed_matches_oracle(word, p, m, k, n):
    """Equation (LeftComp) of Section 3: A x CB then REDQ; CC holds the
    residues of A B packed along rows, its unpacking is A B mod p."""
    d, Q, _ = gfp.gfp_params(p, m, k, n, "mixed", word)
    A, B = operands(2, 2, p, m, k, n)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "rows", word)
    CC = gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "mixed", word, dev(A), CB)
    ref = oracle_product(2, 2, p, m, k, n)
    got = words_np(CC, word)
    want = oracle.pack_rows(ref, d, Q, dtype=np.uint64)
    if word == "f64":
        assert (got == want.astype(np.float64)).all()
    else:
        assert (got == want).all()
    C = host(gfp.gfp_unpack(p, CC, m, n, d, Q, "rows", word))
    assert (C == ref).all()


@pytest.mark.parametrize("word", ["u64", "f64"])
def test_mixed_worst_case(word):
    p = 3
    k = 2047
    d, Q, _ = gfp.gfp_params(p, 8, k, 8, "mixed", word)
    A = np.full((40, k), 2, np.uint8)
    B = np.full((k, 50), 2, np.uint8)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "rows", word)
    CC = gfp.gfp_gemm_compressed(p, 40, k, 50, d, Q, "mixed", word, dev(A), CB)
    C = host(gfp.gfp_unpack(p, CC, 40, 50, d, Q, "rows", word))
    assert (C == (k * 4) % 3).all()


# ------------------------------------------------------ left / full compression
LEFT_CASES = [(3, 1024, 1024, 1024), (3, 77, 300, 101), (5, 64, 200, 64), (251, 41, 30, 20),
              (2, 67, 129, 65), (7, 1, 1, 1), (3, 1, 500, 1), (5, 300, 1, 2), (3, 2, 3, 1)]


@pytest.mark.parametrize("word", ["u64", "f64"])
@pytest.mark.parametrize("p,m,k,n", LEFT_CASES)
def test_left_matches_oracle(word, p, m, k, n):
    """Table 2 left compression: A packed along m (COLS) times uncompressed B;
    the result words are the COLS packing of A B mod p."""
    d, Q, _ = gfp.gfp_params(p, m, k, n, "left", word)
    A, B = operands(2, 3, p, m, k, n)
    CA = gfp.gfp_pack(p, dev(A), d, Q, "cols", word)
    CC = gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "left", word, CA, dev(B))
    ref = oracle_product(2, 3, p, m, k, n)
    want = oracle.pack_cols(ref, d, Q, dtype=np.uint64)
    got = words_np(CC, word)
    assert (got == (want.astype(np.float64) if word == "f64" else want)).all()
    assert (host(gfp.gfp_unpack(p, CC, m, n, d, Q, "cols", word)) == ref).all()


FULL_CASES = [(3, 1024, 1024, 1024), (3, 77, 300, 101), (5, 64, 200, 64), (7, 33, 40, 17),
              (2, 65, 129, 67), (7, 1, 1, 1), (3, 1, 500, 1), (5, 300, 1, 2), (3, 2, 3, 1)]


@pytest.mark.parametrize("word", ["u64", "f64"])
@pytest.mark.parametrize("p,m,k,n", FULL_CASES)
def test_full_matches_oracle(word, p, m, k, n):
    """Section 4: A packed along m in base Q, B along n in base Theta =
    Q^(dq+1); every result word is the block packing of A B mod p."""
    dq, dth, Q = gfp.gfp_params_full(p, m, k, n, word)
    Theta = Q ** (dq + 1)
    A, B = operands(2, 4, p, m, k, n)
    CA = gfp.gfp_pack(p, dev(A), dq, Q, "cols", word)
    CB = gfp.gfp_pack(p, dev(B), dth, Theta, "rows", word)
    CC = gfp.gfp_gemm_full(p, m, k, n, dq, dth, Q, word, CA, CB)
    ref = oracle_product(2, 4, p, m, k, n)
    want = oracle.pack_block(ref, dq, dth, Q)
    got = words_np(CC, word)
    assert (got == (want.astype(np.float64) if word == "f64" else want)).all()
    assert (host(gfp.gfp_unpack_block(p, CC, m, n, dq, dth, Q, word)) == ref).all()
    # the block layout written directly from the residues agrees
    assert (words_np(gfp.gfp_pack_block(p, dev(ref), dq, dth, Q, word), word) == got).all()


@pytest.mark.parametrize("word", ["u64", "f64"])
def test_full_worst_case(word):
    p, k = 3, 2047
    dq, dth, Q = gfp.gfp_params_full(p, 8, k, 8, word)
    A = np.full((30, k), 2, np.uint8)
    B = np.full((k, 40), 2, np.uint8)
    CA = gfp.gfp_pack(p, dev(A), dq, Q, "cols", word)
    CB = gfp.gfp_pack(p, dev(B), dth, Q ** (dq + 1), "rows", word)
    CC = gfp.gfp_gemm_full(p, 30, k, 40, dq, dth, Q, word, CA, CB)
    assert (host(gfp.gfp_unpack_block(p, CC, 30, 40, dq, dth, Q, word)) == (k * 4) % 3).all()


@pytest.mark.parametrize("p", [2, 5, 13])
def test_tc_f8_raw_operands(p):
    """fp8 form with p < 16 reads A straight from the caller's matrix (the byte
    r is the e4m3 code of r 2^-9) when A and lda are 16-byte aligned: strided A
    (lda = 160 > k = 150, k not a multiple of 128), m off the tile grid,
    random and all-(p-1) entries."""
    m, k, n = 200, 150, 300
    g = inputs.rng(35, p)
    for A in (inputs.residues(g, p, m, k), np.full((m, k), p - 1, np.uint8)):
        B = inputs.residues(g, p, k, n)
        Ad = torch.zeros((m, 160), dtype=torch.uint8, device="cuda")
        Ad[:, :k] = dev(A)
        C = host(gfp.gfp_gemm(p, Ad[:, :k], dev(B), "tc_f8"))
        assert (C == oracle.gemm(p, A, B)).all()
