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
        if name != "mma_s8":
            assert 0 < v < ceiling, (name, v)
    assert 0 < r["mma_s8"] < 2.25e15
    assert r["dfma"] < r["imad"] / 4
    assert r["mad64"] < r["imad"]
