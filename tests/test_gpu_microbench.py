"""The microbenchmarks (chm_microbench) run and give physically sane numbers
on the GPU; their values are printed (the design notes quote them)."""
from __future__ import annotations

import pytest
import torch

from paper_1011_1173_gb300 import chm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)


def test_microbenchmarks():
    fp64, fp64_sm = chm.microbench("fp64_rate")
    fp32, fp32_sm = chm.microbench("fp32_rate")
    issue, lat = chm.microbench("fp64_warp")
    conv, split = chm.microbench("shfl_split")
    hbm, ms = chm.microbench("hbm_copy")
    rt, failed = chm.microbench("flag_round_trip")
    one_lane, four_warps = chm.microbench("fp64_lanes")
    print("FP64 %.3f T FMA/s (%.2f G/SM); FP32 %.2f T FMA/s; one warp: %.1f cycles per independent FP64 FMA, "
          "%.1f per dependent, %.1f with one active lane, %.1f each for four warps of one SM; 32 shuffles %d "
          "cycles converged, %d after a lane-0 wait; HBM copy %.0f GB/s; flag round trip %.2f us"
          % (fp64, fp64_sm * 1e3, fp32, issue, lat, one_lane, four_warps, conv, split, hbm, rt))
    assert one_lane >= 1.0 and four_warps >= 1.0
    assert 0.05 < fp64 < 10.0
    assert fp32 > 5 * fp64
    assert issue >= 1.0 and lat >= 4.0
    assert conv > 0 and split > 0
    assert 500.0 < hbm < 20000.0
    assert failed == 0.0 and 0.05 < rt < 100.0
