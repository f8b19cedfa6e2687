"""The pass kernels (one sweep of the factor per block of up to 16 vectors)
against the CPU oracle, through the C ABI, over their own parameters: the
vectors per pass, the lookahead of the forward-substitution chain, several
passes per call, ragged shapes, the first failing row, and the full-size
factor of order 32768.

Float64 parity: elementwise, column-scaled relative error <= 1e-11.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, accuracy_as_serial, colscaled_err, tol_mixed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    chm.config_set("path", chm.PATH_PASS)
    yield
    chm.config_set("path", chm.PATH_AUTO)
    chm.config_set("pass_kb", 0)
    chm.config_set("pass_d", 0)
    chm.config_set("pass_seg", 0)


def run(L, V, sig, dtype=torch.float64):
    Ld = torch.as_tensor(L).to("cuda", dtype).contiguous()
    Vd = torch.as_tensor(V).to("cuda", dtype).contiguous()
    assert chm.modify(Ld, Vd, sig, n=L.shape[0]) == chm.CHM_OK
    st, info = chm.status_sync()
    return st, info, Ld.cpu().numpy()


def ref(L, V, sig):
    o = np.array(L, dtype=np.float64, copy=True)
    st, info = oracle.modify_b(o, np.ascontiguousarray(V, dtype=np.float64), sig, n=L.shape[0])
    return st, info, o


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("kb", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("d", [2, 3, 8])
def test_vectors_per_pass_and_lookahead(kb, d, fused):
    """Both forms of a pass: fused (the substitution kernel's workers form
    the coefficients and sweep as their inputs arrive; up to 8 vectors per
    pass) and the six-kernel sequence; float64 against the oracle, float
    storage against the emulation."""
    chm.config_set("pass_kb", kb)
    chm.config_set("pass_d", d)
    chm.config_set("pass_fused", fused)
    try:
        for n, k, pad in [(33, 5, 1), (200, 16, 0), (611, 19, 3)]:
            seed = 77 + n + k + kb
            L = inputs.spd_factor(n, seed, ld=n + pad).numpy()
            V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(n * k)).numpy()
            sig = inputs.sigma_vector(k, seed).numpy()
            st, info, g = run(L, V, sig)
            ost, _, o = ref(L, V, sig)
            assert st == ost == 0
            assert colscaled_err(g, o) <= TOL_F64, (n, k, kb, d)
            L32, V32 = L.astype(np.float32), V.astype(np.float32)
            st, info, g32 = run(L32, V32, sig, dtype=torch.float32)
            o32 = np.array(L32, copy=True)
            assert oracle.modify_mixed32(o32, np.ascontiguousarray(V32), sig, n=n, group=kb)[0] == 0
            o64 = np.array(L32, dtype=np.float64, copy=True)
            assert oracle.modify_b(o64, np.ascontiguousarray(V32, dtype=np.float64), sig, n=n)[0] == 0
            dm = colscaled_err(g32, o32, n=n)
            assert st == 0 and dm <= tol_mixed(n, k), (n, k, kb, d, dm)
            assert accuracy_as_serial(colscaled_err(g32, o64, n=n), colscaled_err(o32, o64, n=n))
    finally:
        chm.config_set("pass_kb", 0)
        chm.config_set("pass_d", 0)
        chm.config_set("pass_fused", 1)


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("seg", [1, 2, 5])
@pytest.mark.parametrize("kb,d", [(1, 2), (3, 4), (16, 3)])
def test_sweep_segments_restart_from_residuals(seg, kb, d, fused):
    """Short sweep segments (every seg row blocks a column's carry is rebuilt
    from the substitution's partial residual and the prefix Gram's LDL^T
    there), so that most tiles of these shapes lie in restarted segments:
    float64 against the oracle, float storage against the emulation."""
    chm.config_set("pass_seg", seg)
    chm.config_set("pass_kb", kb)
    chm.config_set("pass_d", d)
    chm.config_set("pass_fused", fused)
    try:
        for n, k, pad in [(200, 16, 0), (611, 19, 3), (1025, 2, 1)]:
            seed = 31 + n + k + seg
            L = inputs.spd_factor(n, seed, ld=n + pad).numpy()
            V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(n * k)).numpy()
            sig = inputs.sigma_vector(k, seed).numpy()
            st, info, g = run(L, V, sig)
            ost, _, o = ref(L, V, sig)
            assert st == ost == 0
            err = colscaled_err(g, o)
            assert err <= TOL_F64, (n, k, seg, kb, d, err)
            L32, V32 = L.astype(np.float32), V.astype(np.float32)
            st, info, g32 = run(L32, V32, sig, dtype=torch.float32)
            o32 = np.array(L32, copy=True)
            assert oracle.modify_mixed32(o32, np.ascontiguousarray(V32), sig, n=n, group=kb)[0] == 0
            o64 = np.array(L32, dtype=np.float64, copy=True)
            assert oracle.modify_b(o64, np.ascontiguousarray(V32, dtype=np.float64), sig, n=n)[0] == 0
            dm, e_gpu, e_emu = colscaled_err(g32, o32, n=n), colscaled_err(g32, o64, n=n), colscaled_err(o32, o64, n=n)
            print("seg=%d kb=%d d=%d n=%d k=%d: f64 %.2e; mixed |gpu-emu| %.2e (bound %.2e), gpu %.2e emu %.2e"
                  % (seg, kb, d, n, k, err, dm, tol_mixed(n, k), e_gpu, e_emu))
            assert st == 0 and dm <= tol_mixed(n, k)
            assert accuracy_as_serial(e_gpu, e_emu)
    finally:
        chm.config_set("pass_seg", 0)
        chm.config_set("pass_kb", 0)
        chm.config_set("pass_d", 0)
        chm.config_set("pass_fused", 1)


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (31, 1), (32, 16), (64, 1), (95, 4), (1025, 2), (2049, 33)])
def test_ragged_shapes_with_sentinels(n, k):
    ld = n + 5
    seed = 900 + n
    L = inputs.spd_factor(n, seed, ld=ld).numpy()
    lower = np.triu(np.ones((n, ld), dtype=bool), 1)
    L[lower] = np.nan
    V = inputs.update_block(n, k, seed, scale=0.4 / np.sqrt(n * k)).numpy()
    sig = inputs.sigma_vector(k, seed).numpy()
    st, info, g = run(L, V, sig)
    ost, _, o = ref(L, V, sig)
    assert st == ost == 0
    assert np.all(np.isnan(g[lower]))
    assert colscaled_err(np.where(lower, 0, g), np.where(lower, 0, o)) <= TOL_F64


def test_update_then_downdate_stressed():
    """Downdate by 0.9 U after the update by U: the remaining matrix is
    A + 0.19 U U^T, with cancellation in every Compute."""
    n, k = 1500, 16
    L = inputs.spd_factor(n, 5).numpy()
    U = inputs.update_block(n, k, 5).numpy()
    st, _, g1 = run(L, U, 1)
    _, _, o1 = ref(L, U, 1)
    assert st == 0 and colscaled_err(g1, o1) <= TOL_F64
    st, _, g2 = run(g1, 0.9 * U, -1)
    _, _, o2 = ref(o1, 0.9 * U, -1)
    assert st == 0 and colscaled_err(g2, o2) <= TOL_F64


@pytest.mark.parametrize("kb", [1, 16])
def test_first_failing_row(kb):
    chm.config_set("pass_kb", kb)
    try:
        n = 300
        V = np.zeros((3, n))
        V[0, 200] = 0.5
        V[2, 130] = 1.5   # 1 - 2.25 < 0 at row 130 in the third vector
        st, info, _ = run(np.eye(n), V, [1, 1, -1])
        ost, oinfo, _ = ref(np.eye(n), V, [1, 1, -1])
        assert ost == oracle.ERR_NOT_PD and oinfo == 130
        assert st == chm.CHM_ERR_NOT_PD and info == 130
        st, info, _ = run(np.eye(n, dtype=np.float32), V.astype(np.float32), [1, 1, -1], dtype=torch.float32)
        assert st == chm.CHM_ERR_NOT_PD and info == 130
        # a non-positive diagonal on entry
        L = np.eye(n)
        L[77, 77] = -1.0
        V = np.full((1, n), 1e-3)
        st, info, _ = run(L, V, 1)
        assert st == chm.CHM_ERR_NOT_PD and info == 77
    finally:
        chm.config_set("pass_kb", 0)


@pytest.mark.parametrize("k", [1, 4])
def test_full_factor_n32768(k):
    """The whole factor of order 32768 against the oracle on every row."""
    n = 32768
    seed = inputs.config_seed(2)
    Ld = inputs.spd_factor(n, seed, device="cuda")
    V = inputs.update_block(n, k, seed + k, device="cuda")
    L0 = Ld.cpu().numpy()
    assert chm.modify(Ld, V, 1) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    g = Ld.cpu().numpy()
    del Ld
    torch.cuda.empty_cache()
    st, _ = oracle.modify_b(L0, V.cpu().numpy(), 1)
    assert st == 0
    err = colscaled_err(g, L0)
    print("n=32768 k=%d full-factor column-scaled error %.3g" % (k, err))
    assert err <= TOL_F64
