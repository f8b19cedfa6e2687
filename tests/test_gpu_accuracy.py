"""The paper's accuracy experiment (Sec. 5) on the GPU path: B and V with
i.i.d. U[0, 1] entries, A = B^T B + I (update test) or A = B^T B + I + V V^T
(downdate test), and the paper's error metric max |A~ - L~^T L~| for the
float64 path and the mixed-precision path, beside the oracle's own error.
The float64 path must be as accurate as the oracle (within a small factor);
the mixed path is reported and bounded by float rounding."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs

pytestmark = pytest.mark.gpu

CASES = [(1000, 1), (1000, 16), (2000, 1), (2000, 16), (5000, 1), (5000, 16)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)


def residual(L_cm, A_new):
    """max |A~ - L^T L| with L in (n, n) storage (row j = column j of L), float64 on the GPU."""
    Lt = L_cm.double()            # Lt[j, i] = L[i, j]: Lt = L^T
    return float((A_new - Lt @ Lt.T).abs().max())


@pytest.mark.parametrize("down", [False, True])
@pytest.mark.parametrize("n,k", CASES)
def test_paper_uniform_experiment(n, k, down):
    L_cm, V_cm, A = inputs.paper_uniform_problem(n, k, 3000 + n + k, downdate=down, device="cuda")
    sigma = -1 if down else 1
    A_new = A + sigma * (V_cm.T @ V_cm)
    scale = float(A_new.abs().max())
    # float64 path
    L = L_cm.clone().contiguous()
    assert chm.modify(L, V_cm.contiguous(), sigma) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    err_gpu = residual(L, A_new)
    # oracle
    ref = L_cm.cpu().numpy().copy()
    assert oracle.modify_b(ref, V_cm.cpu().numpy(), sigma)[0] == 0
    err_orc = residual(torch.as_tensor(ref, device="cuda"), A_new)
    # mixed precision
    Lf = L_cm.float().contiguous()
    assert chm.modify(Lf, V_cm.float().contiguous(), sigma) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    err_mix = residual(Lf, A_new)
    print("n=%d k=%d %s: max|A~ - L~^T L~| float64 %.3e (oracle %.3e), mixed %.3e; max|A~| %.3e"
          % (n, k, "downdate" if down else "update", err_gpu, err_orc, err_mix, scale))
    assert err_gpu <= 10 * err_orc + 1e-13 * scale
    assert err_mix <= 1e-5 * scale
