"""The identity chm_modify_solve's forward half rests on, checked with the
CPU oracle (no GPU).

Border A = F^T F with right-hand sides B: the upper Cholesky factor of
[[A, B], [B^T, B^T A^{-1} B + I]] is [[F, Y], [0, I]] with Y = F^{-T} B.
Modifying the bordered matrix by V padded with zero rows (Algorithm 1 on
the bordered factor) leaves, in the border's columns, L~^{-T} B, where L~
is the modification of F alone: the bordered matrix plus [V; 0] diag(sigma)
[V; 0]^T has A~ = A + V diag(sigma) V^T in its leading block and B beside
it, so its factor's border column is L~^{-T} B.  The GPU applies the pass's
rotations to Y exactly so, with carries that start at zero.  Here the
oracle's CholeskyModifyB runs on the bordered factor, and the leading block
must equal the oracle's modification of F bit for bit (the leading columns
never see the border), the border the forward substitution with L~^T.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1011_1173_gb300 import inputs
from tests.common import cm_from_upper, upper_from_cm


def _forward_solve_upper_t(U, B):
    """X with U^T X = B for upper triangular U (plain column sweep)."""
    n = U.shape[0]
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(n):
        X[i] = (X[i] - U[:i, i] @ X[:i]) / U[i, i]
    return X


@pytest.mark.parametrize("n,k,m", [(1, 1, 1), (7, 2, 3), (40, 3, 2), (97, 5, 4)])
def test_bordered_factor_carries_the_forward_solve(n, k, m):
    seed = 5150 + n + k + m
    F = upper_from_cm(inputs.spd_factor(n, seed).numpy())
    V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(n)).numpy()  # (k, n)
    sig = inputs.sigma_vector(k, seed).tolist()
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, m))
    # the bordered factor [[F, Y], [0, I]] and V with zero rows below n
    Y = _forward_solve_upper_t(F, B)
    Faug = np.zeros((n + m, n + m))
    Faug[:n, :n] = F
    Faug[:n, n:] = Y
    Faug[n:, n:] = np.eye(m)
    Vaug = np.zeros((k, n + m))
    Vaug[:, :n] = V
    # the oracle on the bordered factor and on F alone
    La = cm_from_upper(Faug)
    assert oracle.modify_b(La, Vaug, sig)[0] == oracle.OK
    Lf = cm_from_upper(F)
    assert oracle.modify_b(Lf, V, sig)[0] == oracle.OK
    Ua, Uf = upper_from_cm(La), upper_from_cm(Lf)
    assert np.array_equal(Ua[:n, :n], Uf)  # the leading columns never see the border
    X = _forward_solve_upper_t(Uf, B)       # L~^{-T} B
    err = np.max(np.abs(Ua[:n, n:] - X)) / max(np.max(np.abs(X)), 1e-300)
    assert err <= 1e-12, err
    # a planted mistake: the border rotated with carries that start at V's
    # entries of the first border row instead of zero
    Vbad = np.array(Vaug, copy=True)
    Vbad[:, n] = V[:, 0]
    Lb = cm_from_upper(Faug)
    st, _ = oracle.modify_b(Lb, Vbad, sig)
    if st == oracle.OK:
        bad = np.max(np.abs(upper_from_cm(Lb)[:n, n:] - X)) / max(np.max(np.abs(X)), 1e-300)
        assert bad > 1e-6
