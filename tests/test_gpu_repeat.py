"""Many launches in a row must all finish without a device-side error.

The launch hands out sweep tasks from per-pair ticket words while SM groups
take (factor, wave) pairs in order; a lost ticket, or warps filling up with
tasks of a pair whose previous wave's tasks then find no warp, would stall
the launch until its bounded waits run out (CHM_ERR_TIMEOUT).  Such a stall
depends on timing and shows in some launches only, so this runs a few
hundred launches of single factors and of many-factor batches and checks
every status, and that an even number of alternating update/downdate
launches returns close to the start."""
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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_repeated_many_factor_batches_all_finish(dtype):
    """The batched workload's shape (many factors of uneven order in one
    launch, the default many-group configuration): every execution of a
    run of update and downdate batches must finish."""
    rng = np.random.default_rng(31)
    count = 256
    ns = np.exp(rng.uniform(np.log(64), np.log(4096), count)).astype(int).tolist()
    ks = rng.choice([1, 4, 16], count).tolist()
    Ls = [inputs.random_factor(n, 900 + i, device="cuda", dtype=dtype) for i, n in enumerate(ns)]
    Vs = [inputs.update_block(n, k, 900 + i, device="cuda", scale=0.3 / np.sqrt(n * k)).to(dtype)
          for i, (n, k) in enumerate(zip(ns, ks))]
    code = chm.CHM_F64 if dtype == torch.float64 else chm.CHM_F32_MIXED
    up = chm.BatchPlan(ns, ns, ks, [1] * count, code)
    down = chm.BatchPlan(ns, ns, ks, [-1] * count, code)
    bad = []
    for r in range(24):
        plan = up if r % 2 == 0 else down
        assert plan.execute(Ls, Vs) == chm.CHM_OK
        st, infos = plan.status()
        if st != chm.CHM_OK:
            bad.append((r, st, sorted(set(tuple(x) for x in infos))[:4]))
    up.close()
    down.close()
    assert not bad, bad[:3]
