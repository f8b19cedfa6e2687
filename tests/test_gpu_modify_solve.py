"""GPU parity of chm_modify_solve: L <- L~ (the rank-k modification) and
B <- (L~^T L~)^{-1} B, against the oracle's CholeskyModifyB followed by its
forward and back substitution with the oracle's L~ (Sec. 1: the factor is
kept up to date to solve with the modified matrix).

On the pass kernels the forward half rides in the last pass: the
substitution carries B's columns beside V's and a recurrence task applies
the pass's rotations to them (the bordered factor's extra column is
L~^{-T} B).  In float the last pass carries up to 8 - (its vectors) of them
and the others take a substitution of their own with the new factor; in
double it carries as many as fill its kernels' unused vector columns and
the others take chm_solve.  The cases below cover right-hand sides carried
that way, those that take the other route (more than the last pass has room
for, a last pass of 8 vectors, passes not fused), both at once, the
wave-kernel form (modification then chm_solve), ragged orders, padded
leading dimensions and mixed signs, in both precisions.

Tolerances.  The factor: the column-scaled 1e-11 of the other float64
parity tests.  The solution: per right-hand side max |x_gpu - x_oracle| <=
1e-12 max |x_oracle|, as chm_solve's tests (the same exact quantity in
another rounding order on factors with condition number about 5).  Mixed
precision: the factor against the emulation with the pass's group of
vectors within tol_mixed; the solution against the oracle's double solve
with the GPU's own float factor (promoted), which isolates the float
forward half: a forward substitution and a recurrence of (k + 1) n float
operations per entry, within 32 u sqrt(n (k + 1)) of max |x| (u = 2^-24;
the first-order bound 4 sqrt(m) u of tol_mixed's derivation, times the
factor's condition number, about 2.2, and a margin of 4 for the
substitution's error).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, U_F32, colscaled_err, tol_mixed

pytestmark = pytest.mark.gpu

TOL_X = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    yield
    for key in ("path", "pass_kb", "pass_seg"):
        chm.config_set(key, 0)
    chm.config_set("pass_fused", 1)


def rhs(n, nrhs, seed, ldb):
    g = torch.Generator().manual_seed(seed)
    B = torch.full((nrhs, ldb), 7.0, dtype=torch.float64)
    B[:, :n] = torch.randn((nrhs, n), generator=g, dtype=torch.float64)
    return B


def rel_err(got, ref, n):
    g, r = np.asarray(got)[:, :n], np.asarray(ref)[:, :n]
    return max(float(np.abs(g[i] - r[i]).max() / max(np.abs(r[i]).max(), 1e-300)) for i in range(r.shape[0]))


def run(L0, V, B0, sig, n):
    Ld, Vd, Bd = L0.cuda(), V.cuda(), B0.cuda()
    info = torch.full((2,), 99, dtype=torch.int64, device="cuda")
    assert chm.modify_solve(Ld, Vd, Bd, sig, n=n, d_info=info) == chm.CHM_OK
    assert chm.status_sync() == (chm.CHM_OK, -1)
    assert info.tolist() == [chm.CHM_OK, -1]
    return Ld.cpu(), Bd.cpu()


# (n, k, nrhs, pad, path, vectors per pass, fused); in double a pass's
# kernels take the next power of two of its vectors, and the right-hand
# sides fill the columns left over
CASES = [
    (300, 3, 1, 1, chm.PATH_AUTO, 0, 1),     # the wave kernel, then chm_solve
    (100, 1, 1, 0, chm.PATH_PASS, 0, 1),     # one pass of 1: chm_solve after it
    (257, 3, 2, 2, chm.PATH_PASS, 4, 1),     # a last pass of 3: 1 carried, 1 by chm_solve
    (900, 5, 3, 1, chm.PATH_PASS, 8, 1),     # a last pass of 5: all 3 carried
    (600, 7, 3, 2, chm.PATH_PASS, 8, 1),     # a last pass of 7: 1 carried, 2 by chm_solve
    (2049, 11, 2, 1, chm.PATH_PASS, 4, 1),   # passes of 4, 4 and 3, ragged: 1 carried
    (1000, 5, 4, 0, chm.PATH_PASS, 4, 1),    # passes of 4 and 1: none carried
    (1000, 8, 3, 0, chm.PATH_PASS, 8, 1),    # a last pass of 8: none carried
    (500, 3, 2, 0, chm.PATH_PASS, 4, 0),     # passes not fused: none carried
    (64, 2, 40, 0, chm.PATH_PASS, 2, 1),     # many right-hand sides, none carried
]


@pytest.mark.parametrize("n,k,nrhs,pad,path,kb,fused", CASES)
def test_modify_solve_matches_oracle_f64(n, k, nrhs, pad, path, kb, fused):
    chm.config_set("path", path)
    chm.config_set("pass_kb", kb)
    chm.config_set("pass_fused", fused)
    try:
        seed = 1300 + n + k + nrhs
        L0 = inputs.spd_factor(n, seed, ld=n + pad)
        V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(n))
        sig = inputs.sigma_vector(k, seed).tolist()
        B0 = rhs(n, nrhs, seed, n + pad)
        ref_L = L0.numpy().copy()
        assert oracle.modify_b(ref_L, V.numpy(), sig, n=n)[0] == oracle.OK
        ref_X = B0.numpy().copy()
        assert oracle.solve(ref_L, ref_X, n=n)[0] == oracle.OK
        got_L, got_X = run(L0, V, B0, sig, n)
        e_l = colscaled_err(got_L.numpy(), ref_L, n=n)
        e_x = rel_err(got_X.numpy(), ref_X, n)
        print("n=%d k=%d nrhs=%d path=%d kb=%d fused=%d: factor %.2e, solution %.2e" % (n, k, nrhs, path, kb, fused, e_l, e_x))
        assert e_l <= TOL_F64
        assert e_x <= TOL_X
        assert np.all(got_X.numpy()[:, n:] == 7.0)      # padding rows of B untouched
        assert np.array_equal(got_L.numpy()[:, n:], L0.numpy()[:, n:])
    finally:
        chm.config_set("path", 0)
        chm.config_set("pass_kb", 0)
        chm.config_set("pass_fused", 1)


@pytest.mark.parametrize("n,k,nrhs,kb,fused", [
    (700, 3, 2, 8, 1),      # both carried
    (1500, 6, 5, 4, 1),     # passes of 4 and 2; 5 carried
    (1000, 8, 3, 8, 1),     # a last pass of 8: all 3 in a pass of their own
    (700, 2, 20, 4, 1),     # 6 carried, 14 in a pass of their own
    (64, 2, 40, 2, 1),      # 6 carried, then passes of 16, 16 and 2
    (500, 3, 2, 4, 0),      # passes not fused: a pass of their own
    (257, 1, 1, 1, 1),      # ragged order, one vector, one right-hand side
])
def test_modify_solve_mixed_precision(n, k, nrhs, kb, fused):
    chm.config_set("path", chm.PATH_PASS)
    chm.config_set("pass_kb", kb)
    chm.config_set("pass_fused", fused)
    try:
        seed = 1700 + n + k
        L64 = inputs.spd_factor(n, seed)
        V64 = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(n))
        sig = inputs.sigma_vector(k, seed).tolist()
        L0, V = L64.float(), V64.float()
        B0 = rhs(n, nrhs, seed, n).float()
        got_L, got_X = run(L0, V, B0, sig, n)
        # the factor: the emulation with the pass's group of vectors
        emu = L0.numpy().copy()
        assert oracle.modify_mixed32(emu, V.numpy(), sig, n=n, group=min(k, kb))[0] == oracle.OK
        e_l = colscaled_err(got_L.numpy(), emu, n=n)
        # the solution: the oracle's double solve with the GPU's own factor
        ref_X = B0.double().numpy().copy()
        assert oracle.solve(got_L.double().numpy(), ref_X, n=n)[0] == oracle.OK
        e_x = rel_err(got_X.double().numpy(), ref_X, n)
        bound = 32 * U_F32 * np.sqrt(n * (k + 1))
        print("mixed n=%d k=%d nrhs=%d: factor %.2e (bound %.2e), solution %.2e (bound %.2e)"
              % (n, k, nrhs, e_l, tol_mixed(n, k), e_x, bound))
        assert e_l <= tol_mixed(n, k)
        assert e_x <= bound
    finally:
        chm.config_set("path", 0)
        chm.config_set("pass_kb", 0)
        chm.config_set("pass_fused", 1)


def test_modify_solve_full_size_f64():
    """n = 32768, rank-1 update, one right-hand side, the library's own
    choice (the pass kernels): the whole factor and solution against the
    oracle."""
    n, k, nrhs = 32768, 1, 1
    seed = inputs.config_seed(2)
    Ld = inputs.spd_factor(n, seed, device="cuda")
    L0 = Ld.cpu()
    V = inputs.update_block(n, k, seed + 1)
    B0 = rhs(n, nrhs, seed, n)
    assert chm.path_for(n, k, chm.CHM_F64) == chm.PATH_PASS
    Vd, Bd = V.cuda(), B0.cuda()
    assert chm.modify_solve(Ld, Vd, Bd, 1) == chm.CHM_OK
    assert chm.status_sync() == (chm.CHM_OK, -1)
    ref_L = L0.numpy().copy()
    assert oracle.modify_b(ref_L, V.numpy(), [1])[0] == oracle.OK
    ref_X = B0.numpy().copy()
    assert oracle.solve(ref_L, ref_X)[0] == oracle.OK
    e_l = colscaled_err(Ld.cpu().numpy(), ref_L)
    e_x = rel_err(Bd.cpu().numpy(), ref_X, n)
    print("n=32768: factor %.2e, solution %.2e" % (e_l, e_x))
    assert e_l <= TOL_F64
    assert e_x <= TOL_X


def test_modify_solve_full_size_mixed():
    """n = 32768 in float storage, rank-1 update, one right-hand side carried
    by the pass (the library's own choice): the solution against the
    oracle's double solve with the GPU's own factor, and the factor's
    leading rows against the emulation."""
    n, k, nrhs, m_rows = 32768, 1, 1, 48
    seed = inputs.config_seed(2)
    Ld = inputs.spd_factor(n, seed, device="cuda").float()
    L0 = Ld.cpu()
    V = inputs.update_block(n, k, seed + 1).float()
    B0 = rhs(n, nrhs, seed, n).float()
    assert chm.path_for(n, k, chm.CHM_F32_MIXED) == chm.PATH_PASS
    Vd, Bd = V.cuda(), B0.cuda()
    assert chm.modify_solve(Ld, Vd, Bd, 1) == chm.CHM_OK
    assert chm.status_sync() == (chm.CHM_OK, -1)
    got_L = Ld.cpu()
    ref_X = B0.double().numpy().copy()
    assert oracle.solve(got_L.double().numpy(), ref_X)[0] == oracle.OK
    e_x = rel_err(Bd.cpu().double().numpy(), ref_X, n)
    # rows i < m_rows of every column (storage entries [j, i]) depend only on those rows
    emu = L0.numpy().copy()
    assert oracle.modify_mixed32(emu, V.numpy(), [1], m_rows=m_rows, group=1)[0] == oracle.OK
    g = got_L[:, :m_rows].double().numpy()
    r = emu[:, :m_rows].astype(np.float64)
    mask = np.arange(m_rows)[None, :] <= np.arange(n)[:, None]
    scale = np.maximum(np.abs(r), np.max(np.where(mask, np.abs(r), 0.0), axis=1, keepdims=True))
    e_l = float(np.where(mask, np.abs(g - r) / np.where(scale == 0, 1.0, scale), 0.0).max())
    bound = 32 * U_F32 * np.sqrt(n * (k + 1))
    print("mixed n=32768: leading rows %.2e (bound %.2e), solution %.2e (bound %.2e)"
          % (e_l, tol_mixed(m_rows, k), e_x, bound))
    assert e_l <= tol_mixed(m_rows, k)
    assert e_x <= bound
