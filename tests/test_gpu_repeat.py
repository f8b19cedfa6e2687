"""Many launches in a row must all finish without a device-side error.

The launch schedules sweep tasks from per-group ticket words while the
groups take (factor, wave) pairs in order; a lost ticket or a task taken in
an order that waits on its own warp's next pair would stall the launch until
its bounded waits run out (CHM_ERR_TIMEOUT).  Such races are rare per
launch, so this runs a few hundred launches of shapes with many pairs per
launch and checks every status, and that an even number of alternating
update/downdate launches returns close to the start."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1011_1173_gb300 import chm, inputs
from tests.common import colscaled_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)


@pytest.mark.parametrize("n,k,dtype,reps", [(3000, 64, torch.float64, 120), (20000, 16, torch.float32, 60),
                                            (700, 40, torch.float64, 200)])
def test_repeated_launches_all_finish(n, k, dtype, reps):
    L0 = inputs.random_factor(n, 13, device="cuda", dtype=dtype)
    V = inputs.update_block(n, k, 13, device="cuda", scale=0.3 / np.sqrt(n * k)).to(dtype)
    L = L0.clone()
    bad = []
    for r in range(reps):
        assert chm.modify(L, V, 1 if r % 2 == 0 else -1) == chm.CHM_OK
        st, info = chm.status_sync()
        if st != chm.CHM_OK:
            bad.append((r, st, info))
    assert not bad, bad[:5]
    tol = 1e-9 if dtype == torch.float64 else 1e-3
    m = min(n, 512)
    assert colscaled_err(L[:m, :m].double().cpu().numpy(), L0[:m, :m].double().cpu().numpy()) <= tol
