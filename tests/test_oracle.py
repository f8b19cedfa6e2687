"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: hand-derived
closed forms, a 60-digit brute-force Cholesky of the modified matrix, textbook
special cases, invariants of the exact result, and the bit-level identities
that follow from the algorithm's dependency structure.  The mutant tests plant
plausible mistakes in the numpy restatement and show that the pins reject
them.
"""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

import oracle
from oracle.bruteforce import modified_factor_decimal
from oracle.hyperbolic_np import NotPositiveDefinite, modify_b_np, modify_mixed32_np
from paper_1011_1173_gb300 import inputs
from oracle import from_cm, to_cm
from tests.common import (colscaled_err, cm_from_upper, load_hand_examples, modified_matrix,
                          upper_from_cm)


def _problem(n, k, seed, ld=None):
    L = inputs.spd_factor(n, seed, ld=ld).numpy()
    V = inputs.update_block(n, k, seed).numpy()
    return L, V


def _run_b(L_cm, V_cm, sigma, **kw):
    L = np.array(L_cm, copy=True)
    st, info = oracle.modify_b(L, np.ascontiguousarray(V_cm), sigma, **kw)
    return st, info, L


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("case", load_hand_examples(), ids=lambda c: c["name"])
def test_hand_examples(case):
    L_cm = cm_from_upper(case["L"])
    V_cm = np.ascontiguousarray(case["V"].T)
    st, info, out = _run_b(L_cm, V_cm, case["sigma"])
    assert st == oracle.OK
    got = upper_from_cm(out)
    np.testing.assert_allclose(got, case["expected"], rtol=0, atol=4e-15 * np.abs(case["expected"]).max())


def test_n1_sequential_square_roots():
    rng = np.random.default_rng(3)
    for _ in range(20):
        l = rng.uniform(0.5, 3.0)
        v = rng.normal(size=5) * 0.3
        sig = rng.choice([-1, 1], size=5).astype(np.int8)
        st, info, out = _run_b(np.array([[l]]), v[:, None].copy(), sig)
        assert st == 0
        ref = l
        for p in range(5):
            ref = np.sqrt(ref * ref + sig[p] * v[p] * v[p])
        assert out[0, 0] == pytest.approx(ref, rel=2e-16, abs=0)


def test_zero_update_is_identity_bitwise():
    L, _ = _problem(37, 3, 11, ld=41)
    V = np.zeros((3, 37))
    for sig in (1, -1):
        st, info, out = _run_b(L, V, sig)
        assert st == 0
        assert np.array_equal(out, L)


def test_identity_first_unit_vector():
    n = 9
    for a, sig in ((0.75, 1), (0.75, -1), (3.0, 1)):
        V = np.zeros((1, n))
        V[0, 0] = a
        st, info, out = _run_b(np.eye(n), V, sig)
        assert st == 0
        exp = np.eye(n)
        exp[0, 0] = np.sqrt(1 + sig * a * a)
        np.testing.assert_allclose(upper_from_cm(out), exp, rtol=1e-16, atol=0)


def test_diagonal_factor_diagonal_update():
    # L = D, V = diag(a) (k = n): every column touches one row only, so the
    # result is diag(sqrt(d^2 + sigma a^2)) and the off-diagonal stays zero.
    rng = np.random.default_rng(5)
    n = 12
    d = rng.uniform(1.0, 2.0, n)
    a = rng.uniform(0.0, 0.9, n)
    for sig in (1, -1):
        st, info, out = _run_b(np.diag(d), np.diag(a), sig)
        assert st == 0
        exp = np.diag(np.sqrt(d * d + sig * a * a))
        np.testing.assert_allclose(upper_from_cm(out), exp, rtol=2e-16, atol=0)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (3, 2), (7, 1), (7, 3), (16, 2), (24, 6)])
def test_decimal_bruteforce(n, k):
    rng = np.random.default_rng(100 + 7 * n + k)
    B = rng.standard_normal((n, n))
    U = np.linalg.cholesky(B.T @ B / n + np.eye(n)).T
    V = 0.5 * rng.standard_normal((n, k)) / np.sqrt(n * k)
    for sig in (np.ones(k, np.int8), -np.ones(k, np.int8),
                rng.choice([-1, 1], size=k).astype(np.int8)):
        exact = modified_factor_decimal(U, V, sig)
        assert exact is not None
        st, info, out = _run_b(cm_from_upper(U), np.ascontiguousarray(V.T), sig)
        assert st == 0
        assert colscaled_err(out, cm_from_upper(exact)) <= 2e-14


@pytest.mark.parametrize("n,k", [(200, 1), (200, 8), (333, 5)])
def test_numpy_cholesky_of_modified_matrix(n, k):
    L, V = _problem(n, k, 21 + n + k)
    U = upper_from_cm(L)
    for sig in (1, -1):
        st, info, out = _run_b(L, V, sig)
        assert st == 0
        ref = np.linalg.cholesky(modified_matrix(U, V.T, [sig] * k)).T
        assert colscaled_err(out, cm_from_upper(ref)) <= 1e-12


def test_paper_uniform_generator_max_abs_error():
    # The paper's experiment (Sec. 5): U[0,1] B and V, A = B^T B + I
    # (+ V V^T for the downdate); error max_ij |At - Lt^T Lt|.
    n, k = 150, 16
    for down in (False, True):
        G, V, A = inputs.paper_uniform_problem(n, k, 9, down)
        L = G.numpy().copy()
        st, info = oracle.modify_b(L, V.numpy(), -1 if down else 1)
        assert st == 0
        U = upper_from_cm(L)
        Vn = V.numpy().T
        At = A.numpy() + (-1 if down else 1) * Vn @ Vn.T
        err = np.abs(At - U.T @ U).max()
        assert err <= 1e-12 * np.abs(At).max()


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("n,k", [(100, 4), (500, 16)])
def test_residual_invariant(n, k):
    L, V = _problem(n, k, 33 + n)
    U = upper_from_cm(L)
    for sig in (1, -1):
        st, info, out = _run_b(L, V, sig)
        assert st == 0
        Ut = upper_from_cm(out)
        At = modified_matrix(U, V.T, [sig] * k)
        res = np.linalg.norm(Ut.T @ Ut - At) / np.linalg.norm(At)
        assert res <= 1e-13


def test_update_then_downdate_roundtrip():
    n, k = 300, 4
    L, V = _problem(n, k, 44)
    st, info, up = _run_b(L, V, 1)
    assert st == 0
    st, info, back = _run_b(up, V, -1)
    assert st == 0
    assert colscaled_err(back, L) <= 1e-11


def test_rank_k_equals_k_rank1_bitwise():
    n, k = 64, 7
    L, V = _problem(n, k, 55)
    sig = inputs.sigma_vector(k, 55).numpy()
    # keep it positive definite: downdates smaller
    Vs = V.copy()
    Vs[sig < 0] *= 0.5
    st, info, full = _run_b(L, Vs, sig)
    assert st == 0
    seq = L.copy()
    for p in range(k):
        st, info = oracle.modify_b(seq, np.ascontiguousarray(Vs[p:p + 1]), sig[p:p + 1])
        assert st == 0
    assert np.array_equal(full, seq)


def test_modify_a_equals_modify_b_bitwise():
    n, k = 80, 5
    L, V = _problem(n, k, 66, ld=83)
    sig = np.array([1, -1, 1, 1, -1], np.int8)
    V[sig < 0] *= 0.5
    st, info, outb = _run_b(L, V, sig)
    outa = L.copy()
    st2, info2 = oracle.modify_a(outa, V, sig)
    assert st == st2 == 0
    assert np.array_equal(outa, outb)


def test_c_equals_numpy_restatement_bitwise():
    n, k = 40, 3
    L, V = _problem(n, k, 77)
    sig = np.array([1, -1, 1], np.int8)
    V[1] *= 0.5
    st, info, out = _run_b(L, V, sig)
    ref = modify_b_np(upper_from_cm(L), V.T, sig.astype(np.float64))
    assert np.array_equal(upper_from_cm(out), ref)


def test_truncated_rows_match_full_run():
    n, k, m = 90, 4, 37
    L, V = _problem(n, k, 88)
    st, info, full = _run_b(L, V, 1)
    st2, info2, part = _run_b(L, V, 1, m_rows=m)
    assert st == st2 == 0
    # rows < m of L are entries i < m of every column j
    assert np.array_equal(full[:, :m], part[:, :m])


def test_padding_and_lower_triangle_untouched():
    n, ld, k = 30, 35, 2
    L, V = _problem(n, k, 99, ld=ld)
    sentinel = L.copy()
    lower = np.triu(np.ones((n, ld), dtype=bool), 1)  # row j, entries i > j (incl. padding)
    sentinel[lower] = np.nan
    st, info, out = _run_b(sentinel, V, 1)
    assert st == 0
    assert np.all(np.isnan(out[lower]))


# ---------------------------------------------------------------- failures

def test_not_positive_definite_detected():
    n = 6
    V = np.zeros((1, n))
    V[0, 0] = 2.0
    st, info, _ = _run_b(np.eye(n), V, -1)
    assert st == oracle.ERR_NOT_PD and info == 0
    V = np.zeros((1, n))
    V[0, 3] = 1.0
    st, info, _ = _run_b(np.eye(n), V, -1)  # 1 - 1 = 0 at row 3
    assert st == oracle.ERR_NOT_PD and info == 3
    L = np.eye(n)
    L[4, 4] = -1.0
    st, info, _ = _run_b(L, np.zeros((1, n)), 1)
    assert st == oracle.ERR_NOT_PD and info == 4
    with pytest.raises(NotPositiveDefinite):
        modify_b_np(np.eye(3), np.array([[0.0], [0.0], [1.5]]), -1)


def test_argument_errors():
    L = np.eye(4)
    V = np.zeros((1, 4))
    assert oracle.modify_b(L, V, [2])[0] == oracle.ERR_ARG
    assert oracle.modify_b(L, V, 1, n=5)[0] == oracle.ERR_ARG  # ld < n
    assert oracle.modify_b(L, V, 1, n=0)[0] == oracle.OK


# ---------------------------------------------------------------- mutants

MUTANTS = ["old_l_in_v", "sign_apply", "no_div_c", "c_swapped", "s_from_w", "compute_first",
           "no_v_update"]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_pins_reject_planted_mistakes(mutant):
    rng = np.random.default_rng(7)
    n, k = 8, 2
    B = rng.standard_normal((n, n))
    U = np.linalg.cholesky(B.T @ B / n + np.eye(n)).T
    V = rng.standard_normal((n, k)) / np.sqrt(n)
    sig = np.array([1, -1], np.int8)
    exact = modified_factor_decimal(U, V, sig)
    good = modify_b_np(U, V, sig.astype(np.float64))
    assert colscaled_err(cm_from_upper(good), cm_from_upper(exact)) <= 2e-14
    try:
        bad = modify_b_np(U, V, sig.astype(np.float64), mutant=mutant)
    except NotPositiveDefinite:
        return  # rejected: a PD problem reported as not PD
    assert colscaled_err(cm_from_upper(bad), cm_from_upper(exact)) > 1e-6


# ---------------------------------------------------------------- mixed precision

def test_mixed32_zero_update_and_closed_forms():
    L, _ = _problem(20, 1, 5)
    Lf = L.astype(np.float32)
    out = Lf.copy()
    st, info = oracle.modify_mixed32(out, np.zeros((2, 20), np.float32), 1)
    assert st == 0 and np.array_equal(out, Lf)
    # n = 1: the diagonal is carried in double across the group and rounded
    # once (sqrt(9 + 16 - 4 + 1) = sqrt(22)); in groups of one vector it is
    # rounded after each step
    out = np.array([[3.0]], np.float32)
    st, info = oracle.modify_mixed32(out, np.array([[4.0], [2.0], [1.0]], np.float32),
                                     [1, -1, 1])
    assert st == 0 and out[0, 0] == np.float32(np.sqrt(22.0))
    out = np.array([[3.0]], np.float32)
    st, info = oracle.modify_mixed32(out, np.array([[4.0], [2.0], [1.0]], np.float32),
                                     [1, -1, 1], group=1)
    ref = np.float32(3.0)
    for v, s in ((4.0, 1), (2.0, -1), (1.0, 1)):
        ref = np.float32(np.sqrt(np.float64(ref) ** 2 + s * v * v))
    assert st == 0 and out[0, 0] == ref
    # L = I, V = a e1
    n = 5
    V = np.zeros((1, n), np.float32)
    V[0, 0] = 0.5
    out = np.eye(n, dtype=np.float32)
    st, info = oracle.modify_mixed32(out, V, -1)
    exp = np.eye(n, dtype=np.float32)
    exp[0, 0] = np.float32(np.sqrt(0.75))
    assert st == 0 and np.array_equal(out, exp)


@pytest.mark.parametrize("n,k", [(12, 3), (24, 2)])
def test_mixed32_against_exact(n, k):
    rng = np.random.default_rng(n * 31 + k)
    B = rng.standard_normal((n, n))
    U = np.linalg.cholesky(B.T @ B / n + np.eye(n)).T.astype(np.float32).astype(np.float64)
    V = (rng.standard_normal((n, k)) / np.sqrt(n)).astype(np.float32).astype(np.float64)
    for sig in (1, -1):
        exact = modified_factor_decimal(U, V, [sig] * k)
        out = cm_from_upper(U).astype(np.float32)
        st, info = oracle.modify_mixed32(out, np.ascontiguousarray(V.T).astype(np.float32), sig)
        assert st == 0
        e = colscaled_err(out, cm_from_upper(exact))
        assert 1e-9 < e <= 2e-6  # float rounding is visible, and bounded


def test_mixed32_tracks_float64_oracle():
    n, k = 400, 8
    L, V = _problem(n, k, 123)
    L32 = L.astype(np.float32)
    V32 = V.astype(np.float32)
    out32 = L32.copy()
    st, info = oracle.modify_mixed32(out32, V32, 1)
    out64 = L32.astype(np.float64)
    st2, info2 = oracle.modify_b(out64, V32.astype(np.float64), 1)
    assert st == st2 == 0
    assert colscaled_err(out32, out64) <= 2e-5


def test_torch_generator_shapes():
    L = inputs.spd_factor(10, 1, ld=12)
    assert L.shape == (10, 12) and L.dtype == torch.float64
    assert torch.all(L[:, 10:] == 0)
    assert torch.all(torch.triu(L[:, :10], 1) == 0)  # strictly lower part of L is zero
    assert torch.all(torch.diagonal(L[:, :10]) > 0)


# ---------------------------------------------------------------- solve with the factor

def _exact_solve(U, B):
    """X with (U^T U) X = B in exact rational arithmetic (Gauss-Jordan on the
    normal matrix, independent of triangular substitution)."""
    from fractions import Fraction
    n = U.shape[0]
    Uf = [[Fraction(int(U[i, j])) for j in range(n)] for i in range(n)]
    A = [[sum(Uf[m][i] * Uf[m][j] for m in range(n)) for j in range(n)] for i in range(n)]
    M = [A[i] + [Fraction(int(v)) for v in B[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return np.array([[float(v) for v in row[n:]] for row in M])


@pytest.mark.parametrize("n,nrhs", [(1, 1), (2, 3), (5, 2), (9, 4), (12, 1)])
def test_solve_exact_rational(n, nrhs):
    rng = np.random.default_rng(500 + n)
    U = np.triu(rng.integers(-3, 4, (n, n))).astype(np.float64)
    U[np.diag_indices(n)] = rng.integers(1, 5, n)
    B = rng.integers(-5, 6, (n, nrhs)).astype(np.float64)
    exact = _exact_solve(U, B)
    X = np.array(B.T, order="C", copy=True)  # B.T may be a view for nrhs == 1
    st, info = oracle.solve(cm_from_upper(U), X)
    assert st == 0 and info == -1
    for r in range(nrhs):
        scale = max(1.0, np.abs(exact[:, r]).max())
        assert np.abs(X[r] - exact[:, r]).max() <= 1e-12 * scale


def test_solve_closed_forms():
    n = 17
    d = np.linspace(0.5, 3.0, n)
    B = np.arange(2 * n, dtype=np.float64).reshape(2, n) - 7.0
    X = B.copy()
    assert oracle.solve(cm_from_upper(np.diag(d)), X)[0] == 0
    np.testing.assert_allclose(X, B / d ** 2, rtol=1e-15)
    X = B.copy()
    assert oracle.solve(cm_from_upper(np.eye(n)), X)[0] == 0
    assert np.array_equal(X, B)
    X = np.array([[6.0]])
    assert oracle.solve(np.array([[2.0]]), X)[0] == 0
    assert X[0, 0] == 1.5


@pytest.mark.parametrize("n,nrhs", [(64, 1), (300, 3)])
def test_solve_residual_and_library(n, nrhs):
    L = inputs.spd_factor(n, 40 + n).numpy()
    U = upper_from_cm(L)
    A = U.T @ U
    B = np.random.default_rng(n).standard_normal((n, nrhs))
    X = np.array(B.T, order="C", copy=True)  # B.T may be a view for nrhs == 1
    assert oracle.solve(L, X)[0] == 0
    res = np.abs(A @ X.T - B).max() / (np.abs(A).max() * np.abs(X).max())
    assert res <= 1e-14
    ref = np.linalg.solve(A, B)
    assert np.abs(X.T - ref).max() <= 1e-11 * np.abs(ref).max()
    # solving with L first (the transposed order) gives another answer
    wrong = np.linalg.solve(U @ U.T, B)
    assert np.abs(X.T - wrong).max() > 1e-3 * np.abs(ref).max()


def test_solve_errors_and_padding():
    n = 6
    U = np.eye(n)
    U[3, 3] = 0.0
    B = np.ones((1, n))
    st, info = oracle.solve(cm_from_upper(U), B)
    assert st == oracle.ERR_NOT_PD and info == 3
    assert np.array_equal(B, np.ones((1, n)))
    # leading dimensions beyond n: padding left alone
    L = inputs.spd_factor(10, 3, ld=13).numpy()
    Bp = np.full((2, 12), 9.0)
    Bp[:, :10] = np.random.default_rng(1).standard_normal((2, 10))
    st, _ = oracle.solve(L, Bp, n=10)
    assert st == 0 and np.all(Bp[:, 10:] == 9.0)


# ---------------------------------------------------------------- mixed precision: the reading

def load_mixed_examples():
    import json
    from fractions import Fraction
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed_examples.json")) as f:
        data = json.load(f)

    def ev(x):
        num, _, den = x.partition("/")
        val = Fraction(eval(num, {"__builtins__": {}}))
        if den:
            val /= Fraction(eval(den, {"__builtins__": {}}))
        return np.float32(float(val))

    return [dict(c, L=np.array([[ev(x) for x in r] for r in c["L"]], np.float32),
                 V=np.array([[ev(x) for x in r] for r in c["V"]], np.float32),
                 expected=np.array([[ev(x) for x in r] for r in c["expected"]], np.float32))
            for c in data["cases"]]


MIXED_CASES = load_mixed_examples()


@pytest.mark.parametrize("case", MIXED_CASES, ids=[c["name"] for c in MIXED_CASES])
def test_mixed32_hand_derived_bits(case):
    """The emulation (C and its numpy restatement) reproduces the hand-derived
    float32 results bit for bit."""
    out = to_cm(case["L"])
    st, _ = oracle.modify_mixed32(out, np.ascontiguousarray(case["V"].T), case["sigma"], group=case["group"])
    assert st == 0
    assert np.array_equal(from_cm(out), case["expected"])
    got = modify_mixed32_np(case["L"], case["V"], case["sigma"], group=case["group"])
    assert np.array_equal(np.triu(got), case["expected"])


@pytest.mark.parametrize("mutant", ["cs_unrounded", "diag_per_vector", "apply_in_double"])
def test_mixed32_pins_reject_planted_mistakes(mutant):
    """Each planted deviation from the reading changes some hand-derived bits."""
    changed = False
    for case in MIXED_CASES:
        bad = modify_mixed32_np(case["L"], case["V"], case["sigma"], group=case["group"], mutant=mutant)
        changed = changed or not np.array_equal(np.triu(bad), case["expected"])
    assert changed, mutant


@pytest.mark.parametrize("n,k,group", [(7, 3, None), (40, 5, 2), (33, 4, 1), (65, 6, 4)])
def test_mixed32_c_equals_numpy_restatement(n, k, group):
    rng = np.random.default_rng(n * 3 + k)
    B = rng.standard_normal((n, n))
    U = np.linalg.cholesky(B.T @ B / n + np.eye(n)).T.astype(np.float32)
    V = (rng.standard_normal((n, k)) / np.sqrt(n)).astype(np.float32)
    sig = np.where(rng.random(k) < 0.5, 1, -1).astype(np.int8)
    sig[0] = 1
    V[:, sig < 0] *= np.float32(0.3)
    out = to_cm(U)
    st, _ = oracle.modify_mixed32(out, np.ascontiguousarray(V.T), sig, group=group)
    assert st == 0
    assert np.array_equal(from_cm(out), np.triu(modify_mixed32_np(U, V, sig, group=group)))


def test_mixed32_groups_change_only_diagonal_rounding():
    """Groups of the same vectors differ by float rounding only, and a single
    vector per group gives the same result for any group size."""
    rng = np.random.default_rng(3)
    n, k = 50, 6
    B = rng.standard_normal((n, n))
    U = np.linalg.cholesky(B.T @ B / n + np.eye(n)).T.astype(np.float32)
    V = (rng.standard_normal((n, k)) / np.sqrt(n)).astype(np.float32)
    outs = []
    for g in (1, 2, 6):
        out = to_cm(U)
        assert oracle.modify_mixed32(out, np.ascontiguousarray(V.T), 1, group=g)[0] == 0
        outs.append(out)
    assert colscaled_err(outs[0], outs[2]) < 1e-5
    one = to_cm(U)
    two = to_cm(U)
    oracle.modify_mixed32(one, np.ascontiguousarray(V[:, :1].T), 1, group=1)
    oracle.modify_mixed32(two, np.ascontiguousarray(V[:, :1].T), 1, group=16)
    assert np.array_equal(one, two)


def test_mixed32_first_failing_row_across_groups():
    """A later group's failure above an earlier group's is the one reported
    (the smallest failing row, as CholeskyModifyB over all vectors)."""
    n = 20
    V = np.zeros((2, n), np.float32)
    V[0, 15] = 2.0   # group 1 fails at row 15
    V[1, 4] = 2.0    # group 2 fails at row 4
    out = np.eye(n, dtype=np.float32)
    st, info = oracle.modify_mixed32(out, V, -1, group=1)
    assert st == oracle.ERR_NOT_PD and info == 4
    o64 = np.eye(n)
    st, info = oracle.modify_b(o64, V.astype(np.float64), -1)
    assert st == oracle.ERR_NOT_PD and info == 4
