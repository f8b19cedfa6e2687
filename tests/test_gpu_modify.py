"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on
both paths of the single-factor entry points (wave kernel, pass kernels).

Float64: elementwise, column-scaled relative error <= 1e-11 (see
``tests/common.py``).  Mixed precision (float storage and Apply, double
Compute): against the oracle's mixed-precision emulation, which rounds the
same quantities to float but evaluates Apply with division where the kernel
multiplies by 1/c, so the two agree to float rounding, not bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, colscaled_err

pytestmark = pytest.mark.gpu

# Mixed precision against its emulation: float rounding differences grow
# with the number of rotations a column goes through (~n k).
TOL_MIXED = 1e-4


@pytest.fixture(scope="module", autouse=True, params=["wave", "pass"])
def _device(request):
    """Every test of this file runs once on each path of the single-factor
    entry points (the wave kernel and the pass kernels)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    chm.config_set("path", chm.PATH_WAVE if request.param == "wave" else chm.PATH_PASS)
    yield request.param
    chm.config_set("path", chm.PATH_AUTO)


def gpu_modify(L_cm, V_cm, sigma, dtype=torch.float64, n=None):
    Ld = torch.as_tensor(L_cm).to("cuda", dtype).contiguous()
    Vd = torch.as_tensor(V_cm).to("cuda", dtype).contiguous()
    st = chm.modify(Ld, Vd, sigma, n=n)
    assert st == chm.CHM_OK
    st, info = chm.status_sync()
    return st, info, Ld.cpu().numpy()


def oracle_modify(L_cm, V_cm, sigma, n=None):
    L = np.array(L_cm, dtype=np.float64, copy=True)
    st, info = oracle.modify_b(L, np.ascontiguousarray(V_cm, dtype=np.float64), sigma, n=n)
    return st, info, L


def oracle_mixed(L_cm, V_cm, sigma):
    L = np.array(L_cm, dtype=np.float32, copy=True)
    st, info = oracle.modify_mixed32(L, np.ascontiguousarray(V_cm, dtype=np.float32), sigma)
    return st, info, L


def problem(n, k, seed, ld=None, scale=None):
    L = inputs.spd_factor(n, seed, ld=ld).numpy()
    V = inputs.update_block(n, k, seed, scale=scale).numpy()
    return L, V


def test_plain_rank1_update_then_downdate_n512():
    n, k = 512, 1
    L, V = problem(n, k, inputs.config_seed(0))
    st, info, g_up = gpu_modify(L, V, 1)
    ost, oinfo, o_up = oracle_modify(L, V, 1)
    assert st == ost == 0
    assert colscaled_err(g_up, o_up) <= TOL_F64
    st, info, g_down = gpu_modify(g_up, V, -1)
    ost, oinfo, o_down = oracle_modify(o_up, V, -1)
    assert st == ost == 0
    assert colscaled_err(g_down, o_down) <= TOL_F64
    assert colscaled_err(g_down, L) <= TOL_F64


SHAPES = [(1, 1, 0), (2, 3, 1), (31, 2, 0), (32, 1, 0), (33, 5, 2), (63, 16, 0), (64, 17, 3),
          (65, 1, 1), (100, 33, 0), (257, 7, 5), (300, 70, 0), (129, 16, 31)]


@pytest.mark.parametrize("n,k,pad", SHAPES)
def test_random_shapes_f64(n, k, pad):
    seed = 1000 + n * 7 + k
    L, V = problem(n, k, seed, ld=n + pad, scale=0.5 / np.sqrt(max(n, 1) * k))
    sig = inputs.sigma_vector(k, seed).numpy()
    st, info, g = gpu_modify(L, V, sig)
    ost, oinfo, o = oracle_modify(L, V, sig)
    assert ost == 0 and st == 0, (st, info)
    assert colscaled_err(g, o) <= TOL_F64


def test_lower_triangle_and_padding_untouched():
    n, ld, k = 150, 157, 9
    L, V = problem(n, k, 7, ld=ld)
    sentinel = L.copy()
    lower = np.triu(np.ones((n, ld), dtype=bool), 1)
    sentinel[lower] = np.nan
    st, info, g = gpu_modify(sentinel, V, 1)
    assert st == 0
    assert np.all(np.isnan(g[lower]))
    ost, oinfo, o = oracle_modify(sentinel, V, 1)
    assert colscaled_err(np.where(lower, 0, g), np.where(lower, 0, o)) <= TOL_F64


def test_zero_update_bitwise_identity():
    n, k = 97, 16
    L, _ = problem(n, k, 8)
    st, info, g = gpu_modify(L, np.zeros((k, n)), 1)
    assert st == 0 and np.array_equal(g, L)


def test_headline_shape_n5000_k16_update_then_downdate():
    n, k = 5000, 16
    L, V = problem(n, k, inputs.config_seed(1))
    st, info, g_up = gpu_modify(L, V, 1)
    ost, oinfo, o_up = oracle_modify(L, V, 1)
    assert st == ost == 0
    assert colscaled_err(g_up, o_up) <= TOL_F64
    st, info, g_dn = gpu_modify(g_up, V, -1)
    ost, oinfo, o_dn = oracle_modify(o_up, V, -1)
    assert st == ost == 0
    assert colscaled_err(g_dn, o_dn) <= TOL_F64


def test_headline_shape_n5000_k1():
    n, k = 5000, 1
    L, V = problem(n, k, inputs.config_seed(1) + 50)
    for sig in (1, -1):
        st, info, g = gpu_modify(L, V, sig)
        ost, oinfo, o = oracle_modify(L, V, sig)
        assert st == ost == 0
        assert colscaled_err(g, o) <= TOL_F64


@pytest.mark.parametrize("n,k", [(1, 1), (33, 3), (200, 16), (301, 20)])
def test_mixed_precision_against_emulation(n, k):
    L, V = problem(n, k, 2000 + n, scale=0.5 / np.sqrt(n * k))
    sig = inputs.sigma_vector(k, 2000 + n).numpy()
    L32 = L.astype(np.float32)
    V32 = V.astype(np.float32)
    st, info, g = gpu_modify(L32, V32, sig, dtype=torch.float32)
    ost, oinfo, o = oracle_mixed(L32, V32, sig)
    assert st == ost == 0
    assert g.dtype == np.float32
    assert colscaled_err(g, o) <= TOL_MIXED
    # and it is a float-accurate answer to the float64 problem
    o64 = oracle_modify(L32.astype(np.float64), V32.astype(np.float64), sig)[2]
    assert colscaled_err(g, o64) <= 1e-3


def test_not_positive_definite_reported():
    n = 100
    V = np.zeros((1, n))
    V[0, 50] = 1.5
    st, info, g = gpu_modify(np.eye(n), V, -1)
    assert st == chm.CHM_ERR_NOT_PD and info == 50
    ost, oinfo, _ = oracle_modify(np.eye(n), V, -1)
    assert ost == oracle.ERR_NOT_PD and oinfo == 50
    V = np.zeros((2, n))
    V[1, 0] = 1.0
    st, info, g = gpu_modify(np.eye(n), V, [1, -1])  # 1 - 1 = 0 at row 0
    assert st == chm.CHM_ERR_NOT_PD and info == 0
    # the status word is cleared by the read
    st, info = chm.status_sync()
    assert st == chm.CHM_OK


def test_device_info_per_call():
    n = 70
    Ld = torch.eye(n, dtype=torch.float64, device="cuda")
    V = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    V[0, 40] = 2.0
    d_info = torch.full((2,), 77, dtype=torch.int64, device="cuda")
    assert chm.modify(Ld, V, -1, d_info=d_info) == chm.CHM_OK
    torch.cuda.synchronize()
    assert d_info.tolist() == [chm.CHM_ERR_NOT_PD, 40]
    chm.status_sync()
    Ld = torch.eye(n, dtype=torch.float64, device="cuda")
    assert chm.modify(Ld, V * 0.25, -1, d_info=d_info) == chm.CHM_OK
    torch.cuda.synchronize()
    assert d_info.tolist() == [chm.CHM_OK, -1]


def test_short_forms_and_streams():
    n, k = 120, 4
    L, V = problem(n, k, 9)
    o = oracle_modify(L, V, 1)[2]
    s = torch.cuda.Stream()
    Ld = torch.as_tensor(L).cuda()
    Vd = torch.as_tensor(V).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert chm.update(Ld, Vd) == chm.CHM_OK
        st, info = chm.status_sync()
    assert st == chm.CHM_OK
    assert colscaled_err(Ld.cpu().numpy(), o) <= TOL_F64
    with torch.cuda.stream(s):
        assert chm.downdate(Ld, Vd) == chm.CHM_OK
        st, info = chm.status_sync()
    assert colscaled_err(Ld.cpu().numpy(), L) <= TOL_F64
