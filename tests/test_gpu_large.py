"""Full-size parity for the large single-factor configuration: n = 32768,
k in {1, 4, 16, 64}, an update by U followed by the downdate by 0.9 U (a
cancellation-stressed downdate), float64 and float32 storage with float64
Compute, through the same C ABI call the benchmark times.

Checks:
  * float64, k = 1 and 4: the whole factor against the oracle run on all
    32768 rows (update, then downdate), elementwise;
  * float64, k = 16 and 64, and mixed precision: the leading 48 rows of the
    result (all 32768 columns), which depend only on the leading rows of L
    and on V, against the oracle's truncated run (CholeskyModifyB with
    m_rows = 48; the oracle pins a truncated run equal to the full run bit
    for bit), for mixed precision against its emulation with the path's
    group of vectors, within the derived float bound;
  * a property at every size: sampled entries (i, j) spread over the whole
    factor satisfy (L~^T L~)_ij = (L^T L)_ij + 0.19 (U U^T)_ij to the
    rounding bound of a backward-stable factorisation.
Each case runs on the path the automatic rule picks (as the benchmark's).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, accuracy_as_serial, colscaled_err, elementwise_rel_err, tol_mixed

pytestmark = pytest.mark.gpu

N = 32768
M_ROWS = 48
SEED = inputs.config_seed(2)
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


@pytest.mark.parametrize("k", [1, 4])
def test_n32768_f64_full_factor(factor, k):
    """Every row of the order-32768 factor against the oracle's full run."""
    L0, host, lead = factor
    U = inputs.update_block(N, k, SEED)
    Ud = U.cuda()
    L = L0.clone()
    assert chm.modify(L, Ud, 1) == chm.CHM_OK
    assert chm.modify(L, (0.9 * Ud).contiguous(), -1) == chm.CHM_OK
    st, info = chm.status_sync()
    assert st == chm.CHM_OK, info
    got = L.cpu().numpy()
    ref = host.copy()
    Un = U.numpy()
    assert oracle.modify_b(ref, Un, 1)[0] == 0
    assert oracle.modify_b(ref, np.ascontiguousarray(0.9 * Un), -1)[0] == 0
    e_col = colscaled_err(got, ref)
    print("n=%d k=%d float64 (path %d), all rows: column-scaled %.3g, elementwise relative %.3g"
          % (N, k, chm.path_for(N, k, chm.CHM_F64), e_col, elementwise_rel_err(got, ref)))
    assert e_col <= TOL_F64
    assert sampled_residual(L0, L, Ud, 1.0 - 0.81) <= TOL_RESID_F64
    del L, got, ref


@pytest.mark.parametrize("k", [16, 64])
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
    # float emulation of the same operations on the leading rows, with the
    # path's group of vectors per launch or pass
    path = chm.path_for(N, k, chm.CHM_F32_MIXED)
    group = min(k, chm.config_get("pass_kb_f32")) if path == chm.PATH_PASS else min(k, 64)
    h32 = Lf0.cpu().numpy()
    u32 = U32.numpy()
    assert oracle.modify_mixed32(h32, u32, 1, m_rows=M_ROWS, group=group)[0] == 0
    assert oracle.modify_mixed32(h32, np.ascontiguousarray(0.9 * u32), -1, m_rows=M_ROWS, group=group)[0] == 0
    d = lead_err(got, h32[:, :M_ROWS])
    # error against the float64 oracle on the same float inputs
    h64 = Lf0.cpu().numpy().astype(np.float64)
    u64 = u32.astype(np.float64)
    assert oracle.modify_b(h64, u64, 1, m_rows=M_ROWS)[0] == 0
    assert oracle.modify_b(h64, np.ascontiguousarray((0.9 * u32).astype(np.float64)), -1, m_rows=M_ROWS)[0] == 0
    e_gpu, e_emu = lead_err(got, h64[:, :M_ROWS]), lead_err(h32[:, :M_ROWS], h64[:, :M_ROWS])
    # against the float64 problem itself (float storage of L and U bounds it)
    try:
        assert oracle.modify_b(host, U.numpy(), 1, m_rows=M_ROWS)[0] == 0
        assert oracle.modify_b(host, np.ascontiguousarray(0.9 * U.numpy()), -1, m_rows=M_ROWS)[0] == 0
        ref64 = host[:, :M_ROWS].copy()
    finally:
        host[:, :M_ROWS] = lead
    err64 = lead_err(got, ref64)
    print("n=%d k=%d mixed (path %d): |gpu-emu| %.3g (bound %.3g); vs float64 oracle on the float inputs: "
          "gpu %.3g, emulation %.3g; vs the float64 problem %.3g"
          % (N, k, path, d, tol_mixed(M_ROWS, 2 * k), e_gpu, e_emu, err64))
    assert d <= tol_mixed(M_ROWS, 2 * k)
    assert accuracy_as_serial(e_gpu, e_emu)
    assert err64 <= 1e-4
    assert sampled_residual(Lf0, L, U32.cuda(), 1.0 - 0.81) <= TOL_RESID_F32
    del L
