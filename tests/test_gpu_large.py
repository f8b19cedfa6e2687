"""Full-size parity for the large single-factor configuration: n = 32768,
k in {1, 4, 16, 64}, an update by U followed by the downdate by 0.9 U (a
cancellation-stressed downdate), float64 and float32 storage with float64
Compute, through the same C ABI call the benchmark times.

The oracle cannot run all n rows at this size, so two checks cover the
factor:
  * sampled outputs: the leading 48 rows of the result (all 32768 columns),
    which depend only on the leading rows of L and on V, are compared with
    the oracle's truncated run (CholeskyModifyB with m_rows = 48; the oracle
    pins a truncated run equal to the full run bit for bit);
  * a property at every size: sampled entries (i, j) spread over the whole
    factor satisfy (L~^T L~)_ij = (L^T L)_ij + 0.19 (U U^T)_ij to the
    rounding bound of a backward-stable factorisation.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64

pytestmark = pytest.mark.gpu

N = 32768
M_ROWS = 48
SEED = inputs.config_seed(2)
# Mixed precision against its float emulation, leading rows (few rotations each).
TOL_MIXED_LEAD = 1e-4
# Residual of sampled entries relative to sqrt(A~_ii A~_jj): c * n * u with c ~ 30.
TOL_RESID_F64 = 1e-10
TOL_RESID_F32 = 3e-3


@pytest.fixture(scope="module")
def factor():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    L0 = inputs.spd_factor(N, SEED, device="cuda")           # float64 (n, n)
    host = L0.cpu().numpy()                                   # oracle input, 8.6 GB
    lead = host[:, :M_ROWS].copy()                            # what a truncated run modifies
    return L0, host, lead


def lead_err(got, ref):
    """Column-scaled error over the leading rows: storage row j, entries i < M_ROWS, i <= j."""
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    n, m = r.shape
    mask = np.arange(m)[None, :] <= np.arange(n)[:, None]
    colmax = np.max(np.where(mask, np.abs(r), 0.0), axis=1, keepdims=True)
    scale = np.maximum(np.abs(r), colmax)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.where(mask, np.abs(g - r) / scale, 0.0).max())


def sampled_residual(L0, L1, U, coef, count=256, seed=11):
    """max |(L1^T L1 - L0^T L0 - coef U U^T)_ij| / sqrt(A1_ii A1_jj) over sampled i <= j,
    in float64 (column x of L is storage row x, entries 0..x)."""
    rng = np.random.default_rng(seed)
    ii = rng.integers(0, N, count)
    jj = rng.integers(0, N, count)
    worst = 0.0
    Ud = U.double()
    for i, j in zip(np.minimum(ii, jj).tolist(), np.maximum(ii, jj).tolist()):
        a0 = torch.dot(L0[i, :i + 1].double(), L0[j, :i + 1].double())
        a1 = torch.dot(L1[i, :i + 1].double(), L1[j, :i + 1].double())
        d_i = torch.dot(L1[i, :i + 1].double(), L1[i, :i + 1].double())
        d_j = torch.dot(L1[j, :j + 1].double(), L1[j, :j + 1].double())
        uu = torch.dot(Ud[:, i], Ud[:, j])
        worst = max(worst, float((a1 - a0 - coef * uu).abs() / torch.sqrt(d_i * d_j)))
    return worst


@pytest.mark.parametrize("k", [1, 4, 16, 64])
def test_n32768_f64_update_then_downdate(factor, k):
    L0, host, lead = factor
    U = inputs.update_block(N, k, SEED)
    Ud = U.cuda()
    L = L0.clone()
    assert chm.modify(L, Ud, 1) == chm.CHM_OK
    assert chm.modify(L, (0.9 * Ud).contiguous(), -1) == chm.CHM_OK
    st, info = chm.status_sync()
    assert st == chm.CHM_OK, info
    # oracle on the leading rows (restored afterwards for the next case)
    Un = U.numpy()
    try:
        assert oracle.modify_b(host, Un, 1, m_rows=M_ROWS)[0] == 0
        assert oracle.modify_b(host, np.ascontiguousarray(0.9 * Un), -1, m_rows=M_ROWS)[0] == 0
        ref = host[:, :M_ROWS].copy()
    finally:
        host[:, :M_ROWS] = lead
    got = L[:, :M_ROWS].cpu().numpy()
    assert lead_err(got, ref) <= TOL_F64
    assert sampled_residual(L0, L, Ud, 1.0 - 0.81) <= TOL_RESID_F64
    del L


@pytest.mark.parametrize("k", [1, 16, 64])
def test_n32768_mixed_update_then_downdate(factor, k):
    L0, host, lead = factor
    U = inputs.update_block(N, k, SEED)
    U32 = U.float()
    L = L0.float().contiguous()
    Lf0 = L.clone()
    assert chm.modify(L, U32.cuda(), 1) == chm.CHM_OK
    assert chm.modify(L, (0.9 * U32).cuda().contiguous(), -1) == chm.CHM_OK
    st, info = chm.status_sync()
    assert st == chm.CHM_OK, info
    got = L[:, :M_ROWS].cpu().numpy()
    # float emulation of the same operations on the leading rows
    h32 = Lf0.cpu().numpy()
    u32 = U32.numpy()
    assert oracle.modify_mixed32(h32, u32, 1, m_rows=M_ROWS)[0] == 0
    assert oracle.modify_mixed32(h32, np.ascontiguousarray(0.9 * u32), -1, m_rows=M_ROWS)[0] == 0
    assert lead_err(got, h32[:, :M_ROWS]) <= TOL_MIXED_LEAD
    # error against the float64 oracle (reported; float storage bounds it)
    try:
        assert oracle.modify_b(host, U.numpy(), 1, m_rows=M_ROWS)[0] == 0
        assert oracle.modify_b(host, np.ascontiguousarray(0.9 * U.numpy()), -1, m_rows=M_ROWS)[0] == 0
        ref64 = host[:, :M_ROWS].copy()
    finally:
        host[:, :M_ROWS] = lead
    err64 = lead_err(got, ref64)
    print("n=%d k=%d mixed precision: leading-row error vs float64 oracle %.3e" % (N, k, err64))
    assert err64 <= 1e-4
    assert sampled_residual(Lf0, L, U32.cuda(), 1.0 - 0.81) <= TOL_RESID_F32
    del L
