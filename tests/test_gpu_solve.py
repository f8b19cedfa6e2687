"""GPU parity of chm_solve, B <- (L^T L)^{-1} B, against the oracle's
forward and back substitution (Sec. 1: the factor is kept to solve with).

Tolerance (float64): per right-hand side, max |x_gpu - x_oracle| <=
1e-12 * max |x_oracle|.  Both sides compute the same exact quantity with
different rounding orders (the GPU applies each 32 x 32 diagonal block
through its explicit inverse and sums tiles in another order); on these
factors (A = B^T B / n + I, condition number about 5) the difference is a
few units of 1e-15.  Mixed precision: the GPU computes in double from the
float inputs and rounds once, so it must match the oracle run on the
promoted inputs, rounded to float, within 1e-6 relative.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)


def rhs(n, nrhs, seed, ldb=None):
    ldb = n if ldb is None else ldb
    g = torch.Generator().manual_seed(seed)
    B = torch.full((nrhs, ldb), 7.0, dtype=torch.float64)
    B[:, :n] = torch.randn((nrhs, n), generator=g, dtype=torch.float64)
    return B


def oracle_solve(L, B, n):
    X = B.numpy().copy()
    st, info = oracle.solve(L.numpy(), X, n=n)
    assert st == 0
    return X


def rel_err(got, ref, n):
    g, r = np.asarray(got)[:, :n], np.asarray(ref)[:, :n]
    return max(float(np.abs(g[i] - r[i]).max() / max(np.abs(r[i]).max(), 1e-300)) for i in range(r.shape[0]))


@pytest.mark.parametrize("n,nrhs,pad", [(1, 1, 0), (2, 2, 1), (31, 1, 0), (32, 3, 0), (33, 1, 2),
                                        (64, 4, 0), (100, 5, 3), (257, 1, 0), (1000, 2, 0), (2049, 9, 1)])
def test_solve_matches_oracle(n, nrhs, pad):
    seed = 800 + n + nrhs
    L = inputs.spd_factor(n, seed, ld=n + pad)
    B = rhs(n, nrhs, seed, ldb=n + pad)
    ref = oracle_solve(L, B, n)
    Ld, Bd = L.cuda(), B.cuda()
    L0 = Ld.clone()
    assert chm.solve(Ld, Bd) == chm.CHM_OK
    assert chm.status_sync() == (chm.CHM_OK, -1)
    got = Bd.cpu().numpy()
    assert rel_err(got, ref, n) <= TOL, (n, nrhs)
    assert np.all(got[:, n:] == 7.0)             # padding rows of B untouched
    assert torch.equal(Ld, L0)                   # L is read only


def test_solve_is_deterministic_and_repeatable():
    n, nrhs = 1500, 5
    L = inputs.spd_factor(n, 3).cuda()
    B = rhs(n, nrhs, 3).cuda()
    outs = []
    for _ in range(3):
        X = B.clone()
        assert chm.solve(L, X) == chm.CHM_OK
        outs.append(X)
    assert chm.status_sync()[0] == chm.CHM_OK
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    # the columns are independent: one right-hand side alone gives the same bits
    for r in (0, 4):
        X = B[r:r + 1].clone()
        assert chm.solve(L, X) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        assert torch.allclose(X[0], outs[0][r], rtol=1e-14, atol=0)


def test_solve_mixed_precision():
    n, nrhs = 777, 3
    L = inputs.spd_factor(n, 9).float()
    B = rhs(n, nrhs, 9).float()
    ref = oracle_solve(L.double(), B.double(), n).astype(np.float32)
    Ld, Bd = L.cuda(), B.cuda()
    assert chm.solve(Ld, Bd) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    assert rel_err(Bd.cpu().numpy(), ref, n) <= 1e-6


@pytest.mark.parametrize("sigma", [1, -1])
def test_modify_then_solve_on_one_stream(sigma):
    """A modification and a solve enqueued back to back solve with the
    modified matrix: (L~^T L~) x = b with L~^T L~ = L^T L + sigma V V^T."""
    n, k, nrhs = 900, 16, 2
    L = inputs.spd_factor(n, 21)
    V = inputs.update_block(n, k, 21, scale=0.5 / np.sqrt(n * k))
    B = rhs(n, nrhs, 21)
    ref_L = L.numpy().copy()
    assert oracle.modify_b(ref_L, V.numpy(), sigma)[0] == 0
    X = B.numpy().copy()
    assert oracle.solve(ref_L, X)[0] == 0
    Ld, Vd, Bd = L.cuda(), V.cuda(), B.cuda()
    assert chm.modify(Ld, Vd, sigma) == chm.CHM_OK
    assert chm.solve(Ld, Bd) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    assert rel_err(Bd.cpu().numpy(), X, n) <= 1e-11
    # the residual against the modified matrix itself
    U = torch.triu(Ld.T)
    A = U.T @ U
    res = (A @ Bd.T - B.cuda().T).abs().max() / (A.abs().max() * Bd.abs().max())
    assert float(res) <= 1e-13


def test_solve_not_a_factor_reports_row():
    n = 100
    L = inputs.spd_factor(n, 2)
    L[70, 70] = 0.0          # zero diagonal: not a Cholesky factor
    Ld, Bd = L.cuda(), rhs(n, 1, 2).cuda()
    assert chm.solve(Ld, Bd) == chm.CHM_OK
    assert chm.status_sync() == (chm.CHM_ERR_NOT_PD, 70)
    # the next call on the stream starts clean
    L[70, 70] = 1.0
    assert chm.solve(L.cuda(), rhs(n, 1, 2).cuda()) == chm.CHM_OK
    assert chm.status_sync() == (chm.CHM_OK, -1)


def test_solve_host_resident():
    n, nrhs = 600, 2
    L = inputs.spd_factor(n, 31)
    B = rhs(n, nrhs, 31)
    Bd = B.cuda()
    assert chm.solve(L.cuda(), Bd) == chm.CHM_OK
    Lh = torch.empty(L.shape, dtype=L.dtype, pin_memory=True)
    Lh.copy_(L)
    Bh = torch.empty(B.shape, dtype=B.dtype, pin_memory=True)
    Bh.copy_(B)
    assert chm.solve(Lh, Bh) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    assert torch.equal(Bh, Bd.cpu())
    # pageable host memory is rejected before any work
    st = chm.chm_solve(L.data_ptr(), n, n, Bd.data_ptr(), n, nrhs, chm.CHM_F64,
                       torch.cuda.current_stream().cuda_stream)
    assert st == chm.CHM_ERR_ARG


def test_solve_large_residual():
    """n = 16384: checked by its residual A x - b with A = L^T L applied as
    two triangular products on the GPU (torch), relative to |A| |x|."""
    n = 16384
    L = inputs.random_factor(n, 5, device="cuda")
    B = rhs(n, 1, 5).cuda()
    X = B.clone()
    assert chm.solve(L, X) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    U = torch.triu(L.T)
    r = U.T @ (U @ X[0]) - B[0]
    den = (U.abs().T @ (U.abs() @ X[0].abs())).max()
    assert float(r.abs().max() / den) <= 2e-13
