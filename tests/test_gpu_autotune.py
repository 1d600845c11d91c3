"""The dot-form autotuner: every candidate it times is admissible for the
real (p, k) by the oracle's bounds, the choice is the fastest of them, and
the product made with the choice equals the oracle's."""
import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("p,m,k,n", [(3, 1024, 1024, 1024), (5, 700, 3000, 900), (251, 300, 400, 200)])
def test_autotune_choice_is_admissible_fastest_and_exact(p, m, k, n):
    best, cands = gfp.gfp_dot_autotune(p, m, k, n)
    assert cands and best in cands
    for c in cands:
        kb = c["kb"] or None
        assert oracle.word_admissible("dot", c["word"], p, k, c["d"], c["Q"], kb=kb), c
        assert c["ms"] > 0
    assert best["ms"] == min(c["ms"] for c in cands)
    g = inputs.rng(91, p)
    A = inputs.residues(g, p, m, k)
    B = inputs.residues(g, p, k, n)
    d, Q, kb, w = best["d"], best["Q"], best["kb"], best["word"]
    CA = gfp.gfp_pack(p, dev(A), d, Q, "rows_rev", w)
    CB = gfp.gfp_pack(p, dev(B), d, Q, "cols", w)
    C = gfp.gfp_gemm_compressed(p, m, k, n, d, Q, "dot", w, CA, CB, kb=kb)
    assert (host(C) == oracle.gemm(p, A, B)).all()


def test_autotune_offers_blocked_words_with_more_coefficients():
    """At p = 5, k = 16384 the unblocked 32-bit word holds one residue; the
    candidates include blocked 32-bit words with 3 or 4."""
    _, cands = gfp.gfp_dot_autotune(5, 512, 16384, 512)
    u32 = [c for c in cands if c["word"] == "u32"]
    assert any(c["kb"] == 0 and c["d"] == 0 for c in u32)
    assert any(c["kb"] > 0 and c["d"] + 1 >= 3 for c in u32)


def test_tuning_cache_round_trip(tmp_path):
    """The JSON cache with the real tuners: a second process-level cache on
    the same file reuses both choices, and the installed batched table gives
    exact products."""
    from paper_0803_1975_gb300.tuning_cache import TuningCache
    import torch
    path = str(tmp_path / "tune.json")
    c = TuningCache(path)
    w = c.dot(3, 512, 1024, 512)
    g = inputs.rng(92, 0)
    items, host_ops = [], []
    for p, n in ((3, 40), (5, 200), (7, 300), (251, 90)):
        A = inputs.adjacency(g, n)
        items.append((p, dev(A), dev(A), torch.empty((n, n), dtype=torch.uint8, device="cuda")))
        host_ops.append((p, A))
    arr, cnt = gfp.make_problems(items)
    table = c.batched(arr, cnt)
    c2 = TuningCache(path)
    assert c2.reused and c2.dot(3, 512, 1024, 512) == w and c2.batched(arr, cnt) == table
    gfp.gfp_gemm_batched(arr, cnt, "auto")
    for (p, A), it in zip(host_ops, items):
        assert (host(it[3]) == oracle.gemm(p, A, A)).all()
    gfp.gfp_batched_set_table([-1] * 7)
