"""Failure detection without a GPU fault: a tcgen05 kernel whose first
operand copies are withheld waits on a stage that never fills; the bounded
wait runs out after the given limit, the kernel records which role gave up in
its status word, stops every role, frees tensor memory and returns -- and the
context stays usable (a normal product runs right after and is exact)."""
import time

import numpy as np
import pytest

import oracle
from paper_0803_1975_gb300 import gfp, inputs

from helpers import dev, ensure_built, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("limit_ms", [50, 300])
def test_wait_runs_out_and_the_context_survives(limit_ms):
    t0 = time.time()
    status = gfp.gfp_selftest_wait_limit(limit_ms)
    dt = time.time() - t0
    assert status in (1, 2, 3, 4), status        # which role gave up; 0 would mean nothing ran out
    assert dt >= limit_ms / 1000.0 * 0.9
    assert dt < limit_ms / 1000.0 + 5.0
    g = inputs.rng(98, limit_ms)
    A = inputs.residues(g, 7, 300, 500)
    B = inputs.residues(g, 7, 500, 200)
    for algo in ("tc_f16", "tc_f8"):
        assert (host(gfp.gfp_gemm(7, dev(A), dev(B), algo)) == oracle.gemm(7, A, B)).all()


def test_selftest_rejects_bad_arguments():
    L = gfp.load()
    import ctypes
    st = ctypes.c_int(0)
    assert L.gfp_selftest_wait_limit(None, 0, 100, ctypes.byref(st), None) == 7
    assert L.gfp_selftest_wait_limit(None, 0, 0, ctypes.byref(st), None) == 1
    assert L.gfp_selftest_wait_limit(None, 0, 20000, ctypes.byref(st), None) == 1
