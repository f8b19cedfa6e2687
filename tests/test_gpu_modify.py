"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on
both paths of the single-factor entry points (wave kernel, pass kernels).

Float64: elementwise, column-scaled relative error <= 1e-11 (see
``tests/common.py``).  Mixed precision (float storage and Apply, double
Compute): against the oracle's mixed-precision emulation with the path's
group of vectors (a launch of the wave kernel: up to 64; a pass: up to 16),
within the derived float bound ``tol_mixed``, at least as accurate as the
emulation against the float64 oracle (``accuracy_as_serial``), and equal bit
for bit where the result is a single rounding of a double value (n = 1).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, U_F32, accuracy_as_serial, colscaled_err, elementwise_rel_err, tol_mixed

pytestmark = pytest.mark.gpu


def mixed_group(k):
    """Vectors whose diagonals the current path carries in double at once."""
    path = chm.config_get("path")
    if path == chm.PATH_PASS:
        return min(k, chm.config_get("pass_kb_f32"))
    return min(k, 64)


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


def oracle_mixed(L_cm, V_cm, sigma, group=None):
    L = np.array(L_cm, dtype=np.float32, copy=True)
    st, info = oracle.modify_mixed32(L, np.ascontiguousarray(V_cm, dtype=np.float32), sigma, group=group)
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


@pytest.mark.parametrize("n,k", [(1, 1), (33, 3), (200, 16), (301, 20), (1000, 5), (2100, 17)])
def test_mixed_precision_against_emulation(n, k):
    L, V = problem(n, k, 2000 + n, scale=0.5 / np.sqrt(n * k))
    sig = inputs.sigma_vector(k, 2000 + n).numpy()
    L32 = L.astype(np.float32)
    V32 = V.astype(np.float32)
    st, info, g = gpu_modify(L32, V32, sig, dtype=torch.float32)
    ost, oinfo, o = oracle_mixed(L32, V32, sig, group=mixed_group(k))
    assert st == ost == 0
    assert g.dtype == np.float32
    d = colscaled_err(g, o)
    # accuracy against the float64 oracle on the same (float) inputs
    o64 = oracle_modify(L32.astype(np.float64), V32.astype(np.float64), sig)[2]
    e_gpu, e_emu = colscaled_err(g, o64), colscaled_err(o, o64)
    print("mixed n=%d k=%d: |gpu-emu| %.3g (bound %.3g), error vs float64 oracle: gpu %.3g, emulation %.3g"
          % (n, k, d, tol_mixed(n, k), e_gpu, e_emu))
    assert d <= tol_mixed(n, k)
    assert accuracy_as_serial(e_gpu, e_emu)


def test_mixed_diagonal_carried_in_double():
    """n = 1, three vectors of 2^-12: the diagonal carried in double rounds
    once to 1 + 2^-23 (rounded after each vector it would stay 1); the same
    hand-derived value as the emulation's pin (tests/golden/mixed_examples.json)."""
    L = np.ones((1, 1), np.float32)
    V = np.full((3, 1), 2.0 ** -12, np.float32)
    st, info, g = gpu_modify(L, V, 1, dtype=torch.float32)
    assert st == 0
    assert g[0, 0] == np.float32(1.0 + 2.0 ** -23)
    assert oracle_mixed(L, V, 1, group=3)[2][0, 0] == g[0, 0]


def test_f64_elementwise_relative_error_reported():
    """Besides the column-scaled check, the plain elementwise relative error
    of the float64 path (the spec reading of 1e-11) on a full factor."""
    n, k = 2000, 16
    L, V = problem(n, k, 4321)
    st, info, g = gpu_modify(L, V, 1)
    ost, oinfo, o = oracle_modify(L, V, 1)
    assert st == ost == 0
    e_col, e_elt = colscaled_err(g, o), elementwise_rel_err(g, o)
    # entries at least 1e-4 of their column's largest: plain relative error
    keep = np.abs(o[:n, :n]) >= 1e-4 * np.max(np.abs(np.tril(o[:n, :n])), axis=1, keepdims=True)
    e_big = float(np.max(np.where(np.tril(keep), np.abs(g[:n, :n] - o[:n, :n]) / np.abs(np.where(keep, o[:n, :n], 1.0)), 0.0)))
    print("f64 n=%d k=%d: column-scaled %.3g, elementwise relative %.3g (entries >= 1e-4 of their column: %.3g)"
          % (n, k, e_col, e_elt, e_big))
    assert e_col <= TOL_F64
    assert e_big <= TOL_F64


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
