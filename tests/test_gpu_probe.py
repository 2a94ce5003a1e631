"""The measured rates the roofline figures are quoted against
(mrrr_probe_peak), and the two facts of the FP64 cost model the interval
engine is designed around: a warp instruction on the FP64 pipe costs the
same whatever its number of active lanes, and a dependent FP64 FMA takes
tens of cycles (so a lone warp cannot keep the pipe busy)."""
import math

import pytest

from paper_1205_2107_gb300 import api

pytestmark = pytest.mark.gpu


def test_rates_are_positive_and_ordered():
    r = {k: api.probe_peak(k) for k in api.PEAK_KINDS}
    for k, v in r.items():
        assert math.isfinite(v) and v > 0, k
    # FP32 FMA far above FP64 FMA; a division costs several FMAs
    assert r["ffma"] > 10 * r["dfma"]
    assert r["ddiv"] < r["dfma"] / 2 / 4
    # one active lane per warp: the same warp-instruction rate as 32 lanes
    full_warp_instr = r["dfma"] / 2 / 32
    assert 0.7 * full_warp_instr <= r["dfma_one_lane"] <= 1.3 * full_warp_instr
    assert 8 <= r["dfma_latency"] <= 1000
    assert r["ddiv_latency"] > r["dfma_latency"]
