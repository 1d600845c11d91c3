"""Host-side tests of the C ABI (no GPU): the library loads, exports every
function include/gfp.h declares, and its parameter logic agrees with the
oracle's reading of the paper's bounds.  Calls that fail validation launch
nothing, so they are safe without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import build as gbuild
from paper_0803_1975_gb300 import gfp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    return gfp.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"GFP_API\s+[\w\s\*]+?\b(gfp_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(gfp.EXPORTS) <= set(names)


def test_status_strings(L):
    for s in range(8):
        assert L.gfp_status_string(s)
    assert L.gfp_word_bytes(0) == 8 and L.gfp_word_bytes(3) == 4 and L.gfp_word_bytes(9) == 0


@pytest.mark.parametrize("form,words", [("dot", oracle.WORDS_DOT), ("mixed", oracle.WORDS_MIXED)])
def test_chooser_matches_oracle(L, form, words):
    for word in words:
        for p in (2, 3, 5, 7, 31, 251):
            for k in (1, 2, 17, 256, 1000, 1024, 8192, 16384):
                ref = oracle.choose(form, word, p, k)
                d, Q, kb = gfp.gfp_params(p, 8, k, 8, form, word)
                assert ref == (d, Q), (form, word, p, k)
                assert kb == 0


@pytest.mark.parametrize("word", ["u64", "u32", "u32w", "f64", "u64x128"])
def test_blocked_chooser_matches_oracle(L, word):
    for p, k, kb in ((3, 1024, 60), (5, 16384, 511), (3, 8192, 255), (7, 4096, 100)):
        d, Q, kbr = gfp.gfp_params(p, 8, k, 8, "dot", word, kb=kb)
        ref = oracle.choose("dot", word, p, k, kb=kbr)
        assert (d, Q) == ref
        assert kbr % (d + 1) == 0 and 0 < kbr <= kb
        assert oracle.word_admissible("dot", word, p, k, d, Q, kb=kbr)


def test_validator_matches_oracle_sweep(L):
    """Every (form, word, p, k, d, t) in a sweep: gfp_params accepts exactly
    what the oracle admits."""
    for form, words in (("dot", oracle.WORDS_DOT), ("mixed", oracle.WORDS_MIXED)):
        for word in words:
            for p in (2, 3, 5, 31):
                for k in (1, 7, 255, 256, 2047, 2048):
                    for t in (4, 8, 10, 11, 13, 16, 20, 26):
                        for d in (0, 1, 2, 3, 4, 5, 7):
                            ok = oracle.word_admissible(form, word, p, k, d, 2 ** t)
                            try:
                                gfp.gfp_params(p, 4, k, 4, form, word, d=d, Q=2 ** t)
                                got = True
                            except gfp.GfpError as e:
                                assert e.status == 3, (form, word, p, k, d, t, e)
                                got = False
                            assert got == ok, (form, word, p, k, d, t)


def test_rejections(L):
    def status(**kw):
        args = dict(p=3, m=4, k=1024, n=4, form="dot", word="u64", d=3, Q=2 ** 13, kb=0)
        args.update(kw)
        try:
            gfp.gfp_params(args["p"], args["m"], args["k"], args["n"], args["form"], args["word"],
                           d=args["d"], Q=args["Q"], kb=args["kb"])
            return 0
        except gfp.GfpError as e:
            return e.status
    assert status() == 0
    assert status(p=4) == 2 and status(p=1) == 2 and status(p=257) == 2 and status(p=253) == 2
    assert status(Q=3 * 2 ** 12) == 4
    assert status(k=2048) == 3                   # k (p-1)^2 = Q: the strict bound
    assert status(d=4) == 3                      # t(d+1) = 65 > 64
    assert status(word="u64x128", d=4) == 0      # ... allowed with 128-bit sums
    assert status(word="f64", d=4, Q=2 ** 10, k=255) == 0    # Q^5 = 2^50
    assert status(word="f64", d=5, Q=2 ** 10, k=255) == 3    # Q^6 = 2^60
    assert status(m=-1) == 1
    assert status(form="mixed", word="u32") == 5
    assert status(kb=102) == 1                   # kb not a multiple of d+1
    assert status(kb=102, d=3, Q=2 ** 8, word="u32") == 1
    assert status(kb=60, d=3, Q=2 ** 8, word="u32") == 0
    assert status(kb=64, d=3, Q=2 ** 8, word="u32") == 3     # 64 * 4 = Q


def test_invalid_calls_launch_nothing(L):
    """Host validation rejects these before any CUDA call (no GPU needed)."""
    null = ctypes.c_void_p(0)
    # p not prime
    assert L.gfp_pack(4, 2, 2, null, 2, 1, 16, 0, 0, null, 1, null) == 2
    # null pointers with non-empty shapes
    assert L.gfp_pack(3, 2, 2, null, 2, 1, 16, 0, 0, null, 1, null) == 1
    # bad layout
    assert L.gfp_pack(3, 2, 2, null, 2, 1, 16, 7, 0, null, 1, null) == 1
    # word too small for the packed value
    assert L.gfp_pack(3, 2, 64, null, 64, 7, 2 ** 13, 0, 3, null, 8, null) == 3
    # ld too small
    a = ctypes.c_void_p(0x1000)
    assert L.gfp_gemm(3, 4, 4, 4, a, 3, a, 4, a, 4, 1, null, 0, null) == 1
    # plain product whose 32-bit sums would overflow: k (p-1)^2 >= 2^32
    assert L.gfp_gemm(251, 4, 70000, 4, a, 70000, a, 4, a, 4, 1, null, 0, null) == 3
    # tensor-core product without its workspace
    assert L.gfp_gemm(3, 64, 64, 64, a, 64, a, 64, a, 64, 3, null, 0, null) == 7
    # compressed product outside the bounds
    assert L.gfp_gemm_compressed(3, 4, 2048, 4, 3, 2 ** 13, 0, 0, a, 512, a, 4, a, 4, 0, null) == 3
    # empty shapes are valid and launch nothing
    assert L.gfp_gemm(3, 0, 4, 4, null, 4, null, 4, null, 4, 1, null, 0, null) == 0
    assert L.gfp_gemm_compressed(3, 0, 4, 4, 1, 2 ** 5, 0, 0, null, 2, null, 4, null, 4, 0, null) == 0


def test_workspace_sizes(L):
    assert gfp.gfp_gemm_workspace_size(3, 256, 256, 256, "plain") == 0
    ws = gfp.gfp_gemm_workspace_size(3, 100, 70, 200, "tc_mma_s8")
    assert ws >= (128 + 256) * 128
    # dp4a: B transposed into k-major rows, both dimensions padded to 64, after 256 bytes
    assert gfp.gfp_gemm_workspace_size(3, 100, 70, 200, "dp4a") == 256 + 256 * 128
    assert gfp.gfp_gemm_workspace_size(3, 5, 64, 64, "dp4a") == 256 + 64 * 64


def test_dp4a_requires_its_workspace(L):
    # rejected on the host before any launch (the pointers are never read)
    A = ctypes.c_void_p(256)
    need = gfp.gfp_gemm_workspace_size(3, 8, 8, 8, "dp4a")
    assert L.gfp_gemm(3, 8, 8, 8, A, 8, A, 8, A, 8, gfp.ALGOS["dp4a"], None, 0, None) == 7   # GFP_EWORKSPACE
    assert L.gfp_gemm(3, 8, 8, 8, A, 8, A, 8, A, 8, gfp.ALGOS["dp4a"], A, need - 1, None) == 7


def test_left_chooser_matches_oracle(L):
    for word in oracle.WORDS_MIXED:
        for p in (2, 3, 5, 31, 251):
            for k in (1, 100, 1024, 16384):
                assert gfp.gfp_params(p, 8, k, 8, "left", word)[:2] == oracle.choose("left", word, p, k)


def test_full_params_match_oracle(L):
    """gfp_params_full picks an admissible (dq, dth, Q) of Section 4 with the
    most coefficients per word; validation agrees with the oracle's reading."""
    for word in ("u64", "f64"):
        for p in (2, 3, 5, 7, 31):
            for k in (1, 64, 1024, 8192):
                dq, dth, Q = gfp.gfp_params_full(p, 8, k, 8, word)
                assert oracle.full_admissible(word, p, k, dq, dth, Q)
                assert not oracle.lower_bound_holds(p, k, Q // 2) or Q == 2
                best = max((a + 1) * (b + 1) for a in range(64) for b in range(64)
                           if oracle.full_admissible(word, p, k, a, b, Q))
                assert (dq + 1) * (dth + 1) == best
                for a in range(5):
                    for b in range(5):
                        ok = oracle.full_admissible(word, p, k, a, b, Q)
                        try:
                            gfp.gfp_params_full(p, 8, k, 8, word, dq=a, dth=b, Q=Q)
                            got = True
                        except gfp.GfpError as e:
                            assert e.status == 3
                            got = False
                        assert got == ok, (word, p, k, a, b)


def test_value_aware_chooser_and_validator_match_oracle(L):
    """gfp_params_vb chooses what the oracle chooses for every (form, word,
    p, k, amax_a, amax_b) of a sweep and accepts exactly what it admits;
    amax = p - 1 is gfp_params; amax above p - 1 is GFP_EINVAL."""
    for form, words in (("dot", oracle.WORDS_DOT), ("mixed", oracle.WORDS_MIXED)):
        for word in words:
            for p in (3, 7, 31):
                for k in (1, 17, 1024, 8192):
                    for a, b in ((1, 1), (p - 1, 1), (1, p - 1), (p - 1, p - 1), (2, 2)):
                        ref = oracle.choose(form, word, p, k, amax_a=a, amax_b=b)
                        d, Q, kb = gfp.gfp_params_vb(p, 8, k, 8, a, b, form, word)
                        assert ref == (d, Q), (form, word, p, k, a, b)
                        for dd in (d - 1, d, d + 1):
                            for QQ in (Q // 2, Q, 2 * Q):
                                if dd < 0 or QQ < 2:
                                    continue
                                ok = oracle.word_admissible(form, word, p, k, dd, QQ, amax_a=a, amax_b=b)
                                try:
                                    gfp.gfp_params_vb(p, 8, k, 8, a, b, form, word, d=dd, Q=QQ)
                                    got = True
                                except gfp.GfpError as e:
                                    assert e.status == 3
                                    got = False
                                assert got == ok, (form, word, p, k, a, b, dd, QQ)
    assert gfp.gfp_params_vb(5, 8, 1000, 8, 4, 4) == gfp.gfp_params(5, 8, 1000, 8)
    for a, b in ((5, 1), (1, 5)):
        with pytest.raises(gfp.GfpError) as e:
            gfp.gfp_params_vb(5, 8, 1000, 8, a, b)
        assert e.value.status == 1


def test_e2m1_workspace_and_prime_limit(L):
    # both operands packed two values per byte, k padded to 256, after 256 bytes
    assert gfp.gfp_gemm_workspace_size(7, 100, 70, 200, "tc_e2m1") == 256 + (128 + 256) * 128
    assert gfp.gfp_gemm_workspace_size(2, 129, 300, 257, "tc_e2m1") == 256 + (256 + 512) * 256
    # e2m1 holds the centred residues of p <= 7 only: rejected before any launch
    a = ctypes.c_void_p(0x1000)
    for p in (11, 13, 31, 251):
        with pytest.raises(gfp.GfpError) as e:
            gfp.gfp_gemm_workspace_size(p, 8, 8, 8, "tc_e2m1")
        assert e.value.status == 5
        assert L.gfp_gemm(p, 8, 8, 8, a, 8, a, 8, a, 8, gfp.ALGOS["tc_e2m1"], a, 1 << 20, None) == 5
    # without its workspace
    assert L.gfp_gemm(5, 64, 64, 64, a, 64, a, 64, a, 64, gfp.ALGOS["tc_e2m1"], None, 0, None) == 7


def test_pipe_rates_rejects_bad_arguments(L):
    # host-side checks, before any CUDA call
    out = (ctypes.c_double * 5)()
    assert L.gfp_pipe_rates(None, 5, ctypes.c_void_p(256), 256, None) == 1          # GFP_EINVAL
    assert L.gfp_pipe_rates(out, 0, ctypes.c_void_p(256), 256, None) == 1
    assert L.gfp_pipe_rates(out, 5, None, 256, None) == 7                            # GFP_EWORKSPACE
    assert L.gfp_pipe_rates(out, 5, ctypes.c_void_p(256), 255, None) == 7
    assert L.gfp_pipe_rates(out, 5, ctypes.c_void_p(257), 256, None) == 7


def test_compc_rejects_before_any_launch(L):
    """ReduceAndCompress entry point: host-side checks only (no GPU here)."""
    a = ctypes.c_void_p(0x1000)
    d, Q, _ = gfp.gfp_params(5, 64, 64, 64, "dot", "u64")
    W = gfp.WORDS
    # words other than u64 / u32
    for word in ("u32w", "u64x128", "f64"):
        assert L.gfp_gemm_compressed_compc(5, 64, 64, 64, d, Q, W[word], a, 64, a, 64, 0, d, Q, a, 64, None) == 5
    # output words that do not fit the word (50 residues of 13 bits), Q_out not a power of two
    assert L.gfp_gemm_compressed_compc(5, 64, 64, 64, d, Q, W["u64"], a, 64, a, 64, 0, 49, 2 ** 13, a, 64, None) == 3
    assert L.gfp_gemm_compressed_compc(5, 64, 64, 64, d, Q, W["u64"], a, 64, a, 64, 0, d, 1000, a, 64, None) == 4
    # input parameters outside eq. (lower)
    assert L.gfp_gemm_compressed_compc(5, 64, 4096, 64, 1, 2 ** 10, W["u64"], a, 4096, a, 64, 0, 1, 2 ** 10, a, 64,
                                       None) == 3
    # output leading dimension below ceil(n / (d_out + 1)), null output
    assert L.gfp_gemm_compressed_compc(5, 64, 64, 64, d, Q, W["u64"], a, 64, a, 64, 0, 1, 2 ** 13, a, 31, None) == 1
    assert L.gfp_gemm_compressed_compc(5, 64, 64, 64, d, Q, W["u64"], a, 64, a, 64, 0, 1, 2 ** 13, None, 64, None) == 1
    # empty products launch nothing
    assert L.gfp_gemm_compressed_compc(5, 0, 64, 64, d, Q, W["u64"], None, 64, None, 64, 0, d, Q, None, 64, None) == 0


def test_auto_algorithm_choice(L):
    """GFP_ALGO_AUTO resolves on the host: its workspace is that of the form it
    picks (e2m1 for large products with p <= 7 and k >= 6144, else e4m3 for
    p <= 31, else fp16)."""
    ws = gfp.gfp_gemm_workspace_size
    assert ws(5, 8192, 8192, 8192, "auto") == ws(5, 8192, 8192, 8192, "tc_e2m1")
    assert ws(5, 8192, 4096, 8192, "auto") == ws(5, 8192, 4096, 8192, "tc_f8")
    assert ws(11, 8192, 8192, 8192, "auto") == ws(11, 8192, 8192, 8192, "tc_f8")
    assert ws(251, 8192, 8192, 8192, "auto") == ws(251, 8192, 8192, 8192, "tc_f16")
    assert ws(3, 1024, 8192, 1024, "auto") == ws(3, 1024, 8192, 1024, "tc_f8")
