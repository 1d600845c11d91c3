"""The instruction-rate probe (gfp_pipe_rates) gives the measured ceilings
the benchmark reports the CUDA-core forms against: every rate is positive,
below the SM count x 128 lanes x the maximum clock (no instruction here
issues faster than the FP32 lanes), and double precision is far slower than
the 32-bit integer multiply-add on GB300."""
import pytest
import torch

from paper_0803_1975_gb300 import gfp

from helpers import ensure_built

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    ensure_built()
    r = gfp.gfp_pipe_rates()
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 128 * 2.2e9
    for name, v in r.items():
        if name != "mma_s8" and not name.startswith("tc_"):
            assert 0 < v < ceiling, (name, v)
    assert 0 < r["mma_s8"] < 2.25e15
    # dense tcgen05 rates: below GB300's nominal dense peaks (2.25 / 4.5 / 13.5
    # PFLOP/s at the boost clock), each kind faster than the one before
    assert 0 < r["tc_f16"] < 2.5e15 and r["tc_f16"] < r["tc_f8"] < 5e15 and r["tc_f8"] < r["tc_e2m1"] < 15e15
    assert r["dfma"] < r["imad"] / 4
    assert r["mad64"] < r["imad"]
