"""The kernels' restatements of Algorithm 1 (no GPU): the exact identities
the pass kernels and the wave kernel compute, written out in numpy in
float64 and checked against the CPU oracle's CholeskyModifyB.

For a block of kb vectors V (signs sigma) applied to the factor F:
  P = F^{-T} V;  for row r the prefix Gram H_r = Sigma + sum_{i<r} p_i p_i^T,
  H_r = L D L^T (L unit lower), z = L^{-1} p_r, |D_q| = sigma_q D_q,
  Dc_q = 1 + sum_{q'<=q} sigma_q' z_q'^2 / |D_q'|,
  a_q = sigma_q z_q,  b_q = z_q / (|D_q| Dc_q),  e = Dc_kb^{-1/2};
then down column j, with carries u_q starting at V_jq, each entry
  S = F_rj;  S <- S + a_q u_q;  u_q <- u_q - b_q S  (q = 1 .. kb);  L~_rj = S e_r,
and the diagonal L~_jj = F_jj Dc_kb(j)^{1/2}.  A sweep that starts at row R
rebuilds its carries from the substitution's partial residual:
  u = |D_R|^{-1} L_R^{-1} w(R),  w_j(R) = V_j - sum_{i<R} F_ij p_i.
These are the readings the pass kernels rest on; the GPU parity tests check
the kernels against the oracle, these check the identities themselves.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1011_1173_gb300 import inputs
from tests.common import cm_from_upper, colscaled_err, upper_from_cm


def _ldl(H):
    """H = L D L^T with L unit lower triangular (no pivoting)."""
    k = H.shape[0]
    L = np.eye(k)
    D = np.zeros(k)
    for j in range(k):
        D[j] = H[j, j] - np.sum(L[j, :j] ** 2 * D[:j])
        for i in range(j + 1, k):
            L[i, j] = (H[i, j] - np.sum(L[i, :j] * L[j, :j] * D[:j])) / D[j]
    return L, D


def _pass_coefficients(F, V, sigma):
    """P, and per row its (a, b), e and Dc_kb, and the LDL^T of H_r."""
    n, kb = V.shape
    sig = np.asarray(sigma, dtype=np.float64)
    P = np.linalg.solve(F.T, V)  # F^T P = V
    a = np.zeros((n, kb))
    b = np.zeros((n, kb))
    e = np.zeros(n)
    dc = np.zeros(n)
    ldl = []
    H = np.diag(sig)
    for r in range(n):
        L, D = _ldl(H)
        ldl.append((L, D))
        z = np.linalg.solve(L, P[r])
        absd = sig * D
        assert np.all(absd > 0)
        c = 1.0 + np.cumsum(sig * z * z / absd)
        a[r] = sig * z
        b[r] = z / (absd * c)
        e[r] = c[-1] ** -0.5
        dc[r] = c[-1]
        H = H + np.outer(P[r], P[r])
    return P, a, b, e, dc, ldl


def _sweep(F, V, a, b, e, dc, start=None):
    """The scaled two-FMA sweep of every column; `start` = (R, carries at R
    for every column) begins each column at row R instead of row 0."""
    n, kb = V.shape
    Lt = np.zeros_like(F)
    for j in range(n):
        r0 = 0
        u = V[j].copy()
        if start is not None and start[0] <= j:
            r0, U = start
            u = U[j].copy()
        for r in range(r0, j):
            S = F[r, j]
            for q in range(kb):
                S = S + a[r, q] * u[q]
                u[q] = u[q] - b[r, q] * S
            Lt[r, j] = S * e[r]
        Lt[j, j] = F[j, j] * np.sqrt(dc[j])
    return Lt


def _carries_at(F, V, a, b, R):
    """The carries of every column entering row R, by the sequential sweep."""
    n, kb = V.shape
    U = np.zeros((n, kb))
    for j in range(n):
        u = V[j].copy()
        for r in range(min(R, j)):
            S = F[r, j]
            for q in range(kb):
                S = S + a[r, q] * u[q]
                u[q] = u[q] - b[r, q] * S
        U[j] = u
    return U


def _problem(n, kb, seed):
    F = upper_from_cm(inputs.spd_factor(n, seed).numpy())
    V = inputs.update_block(n, kb, seed, scale=0.5 / np.sqrt(n)).numpy().T  # (n, kb)
    sigma = inputs.sigma_vector(kb, seed).tolist()
    return F, V, sigma


@pytest.mark.parametrize("n,kb", [(1, 1), (5, 2), (33, 3), (64, 1), (70, 5)])
def test_restated_pass_equals_modify_b(n, kb):
    F, V, sigma = _problem(n, kb, 880 + n + kb)
    _, a, b, e, dc, _ = _pass_coefficients(F, V, sigma)
    got = _sweep(F, V, a, b, e, dc)
    ref = cm_from_upper(F)
    assert oracle.modify_b(ref, np.ascontiguousarray(V.T), sigma)[0] == oracle.OK
    err = colscaled_err(cm_from_upper(got), ref)
    assert err <= 1e-12, err


@pytest.mark.parametrize("n,kb,R", [(33, 3, 8), (64, 2, 32), (70, 5, 40)])
def test_segment_restart_from_partial_residual(n, kb, R):
    F, V, sigma = _problem(n, kb, 990 + n + kb + R)
    P, a, b, e, dc, ldl = _pass_coefficients(F, V, sigma)
    seq = _carries_at(F, V, a, b, R)
    # u = |D_R|^{-1} L_R^{-1} w(R), w_j(R) = V_j - sum_{i<R} F_ij p_i
    L, D = ldl[R]
    absd = np.asarray(sigma) * D
    W = V - F[:R, :].T @ P[:R]
    rebuilt = np.linalg.solve(L, W.T).T / absd
    cols = np.arange(n) >= R  # columns whose sweep reaches row R
    scale = np.max(np.abs(seq[cols]))
    assert np.max(np.abs(rebuilt[cols] - seq[cols])) <= 1e-12 * scale
    # and a sweep restarted there from the rebuilt carries gives the same
    # rows R .. of the factor
    full = _sweep(F, V, a, b, e, dc)
    restarted = _sweep(F, V, a, b, e, dc, start=(R, rebuilt))
    rows = np.arange(n)[:, None] >= R
    d = np.max(np.abs(np.where(rows, restarted - full, 0.0)))
    assert d <= 1e-12 * np.max(np.abs(full)), d


def test_restatement_rejects_a_dropped_prefix():
    """A plausible mistake: coefficients from Sigma alone (the prefix Gram's
    earlier rows dropped) no longer reproduce Algorithm 1."""
    n, kb = 40, 3
    F, V, sigma = _problem(n, kb, 4242)
    P, a, b, e, dc, _ = _pass_coefficients(F, V, sigma)
    sig = np.asarray(sigma, dtype=np.float64)
    a2, b2, e2, dc2 = a.copy(), b.copy(), e.copy(), dc.copy()
    for r in range(n):
        z = P[r]
        c = 1.0 + np.cumsum(sig * z * z)
        a2[r] = sig * z
        b2[r] = z / c
        e2[r] = c[-1] ** -0.5
        dc2[r] = c[-1]
    ref = cm_from_upper(F)
    assert oracle.modify_b(ref, np.ascontiguousarray(V.T), sigma)[0] == oracle.OK
    assert colscaled_err(cm_from_upper(_sweep(F, V, a2, b2, e2, dc2)), ref) > 1e-6


def test_wave_restatement_with_row_scales_equals_modify_b():
    """The wave kernel's restatement (no GPU): per vector (wave) v with sign
    sigma, p = F^{-T} v for the current factor, T_0 = 1,
    T_{i+1} = T_i + sigma p_i^2, and, with the off-diagonal of row i held
    as S_i. = L_i. / e_i, each entry S <- S + a_i u, u <- u - b_i S with
    a_i = sigma p_i / e_i, b_i = p_i e_i / T_{i+1} (u the column's carry
    divided by sqrt(T_i), starting at v_j), the diagonal multiplied by
    c_i = sqrt(T_{i+1} / T_i) and the row scale divided by it; the true
    values e_i S_ij once after the last wave.  Checked against
    CholeskyModifyB for several waves with mixed signs."""
    n, k = 45, 4
    F, V, sigma = _problem(n, k, 3131)
    S = np.triu(F, 1).copy()   # e = 1 to start
    diag = np.diag(F).copy()
    e = np.ones(n)
    for q in range(k):
        sg = float(sigma[q])
        Fcur = np.diag(diag) + e[:, None] * S
        p = np.linalg.solve(Fcur.T, V[:, q])
        T = np.concatenate(([1.0], 1.0 + np.cumsum(sg * p * p)))
        u = V[:, q].copy()
        for i in range(n):
            a = sg * p[i] / e[i]
            b = p[i] * e[i] / T[i + 1]
            for j in range(i + 1, n):
                S[i, j] = S[i, j] + a * u[j]
                u[j] = u[j] - b * S[i, j]
            c = np.sqrt(T[i + 1] / T[i])
            diag[i] *= c
            e[i] /= c
    got = np.diag(diag) + e[:, None] * S
    ref = cm_from_upper(F)
    assert oracle.modify_b(ref, np.ascontiguousarray(V.T), sigma)[0] == oracle.OK
    err = colscaled_err(cm_from_upper(got), ref)
    assert err <= 1e-12, err
