"""The bounds-checked build (libchm_check.so, the same sources compiled with
-DCHM_CHECK) on small ragged shapes: every global index the kernels form is
checked against the arrays the call declares (the upper triangle of L, the
leading n rows of V and B) and every workspace region against its
allocation.  Valid calls must pass every check (status CHM_OK), give the
oracle's result and the same result as the unchecked library; with the
"check_cut" test setting the checks treat the factor as narrower than it is,
so that accesses to real, valid memory are reported as CHM_ERR_BOUNDS and
skipped, the launch ends without a fault, and the next call is clean.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, colscaled_err, tol_mixed

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 0), (33, 3, 1), (100, 17, 5), (257, 2, 0), (300, 16, 7)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    yield
    for lib in (False, True):
        if lib:
            with chm.checked_library():
                chm.config_set("path", chm.PATH_AUTO)
                chm.config_set("check_cut", 0)
        else:
            chm.config_set("path", chm.PATH_AUTO)


def problem(n, k, pad, seed, dtype):
    L = inputs.spd_factor(n, seed, ld=n + pad).to(dtype)
    V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(max(1, n * k))).to(dtype)
    sig = inputs.sigma_vector(k, seed).tolist()
    return L, V, sig


def run(L, V, sig, n):
    Ld, Vd = L.cuda(), V.cuda()
    assert chm.modify(Ld, Vd, sig, n=n) == chm.CHM_OK
    st, info = chm.status_sync()
    return st, info, Ld.cpu()


@pytest.mark.parametrize("path", [chm.PATH_WAVE, chm.PATH_PASS])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_checked_build_passes_every_check_and_matches(path, dtype):
    for n, k, pad in SHAPES:
        seed = 4400 + n + k
        L, V, sig = problem(n, k, pad, seed, dtype)
        chm.config_set("path", path)
        st, info, plain = run(L, V, sig, n)
        assert st == chm.CHM_OK, (n, k, st, info)
        with chm.checked_library():
            assert chm.config_get("checked") == 1
            chm.config_set("path", path)
            st, info, got = run(L, V, sig, n)
        assert st == chm.CHM_OK, (n, k, path, st, info)
        diff = colscaled_err(got.numpy(), plain.numpy(), n=n)
        assert torch.equal(got[:, n:], L[:, n:]), "padding written"
        if dtype == torch.float64:
            ref = L.numpy().copy()
            assert oracle.modify_b(ref, V.numpy(), sig, n=n)[0] == 0
            err = colscaled_err(got.numpy(), ref, n=n)
            print("n=%d k=%d path=%d f64: checked vs oracle %.2e, vs unchecked %.2e" % (n, k, path, err, diff))
            assert err <= TOL_F64
            assert diff <= TOL_F64
        else:
            print("n=%d k=%d path=%d f32: checked vs unchecked %.2e" % (n, k, path, diff))
            assert diff <= tol_mixed(n, k)


def test_checked_solve_and_batch():
    n, k, pad = 200, 4, 3
    L, V, sig = problem(n, k, pad, 91, torch.float64)
    B = torch.randn(3, n + 1, dtype=torch.float64, generator=torch.Generator().manual_seed(5))
    refB = B.numpy().copy()
    assert oracle.solve(L.numpy(), refB, n=n)[0] == 0
    with chm.checked_library():
        Ld, Bd = L.cuda(), B.cuda()
        assert chm.solve(Ld, Bd, n=n) == chm.CHM_OK
        st, info = chm.status_sync()
        assert st == chm.CHM_OK, (st, info)
        got = Bd.cpu().numpy()
        assert np.max(np.abs(got[:, :n] - refB[:, :n]) / np.maximum(1.0, np.abs(refB[:, :n]))) <= 1e-12
        # a batch of ragged factors through the checked wave kernel
        specs = [(64, 2, 1), (130, 5, 0), (33, 1, 2)]
        Ls = [problem(m, kk, p, 700 + m, torch.float64) for m, kk, p in specs]
        plan = chm.BatchPlan([m for m, _, _ in specs], [m + p for m, _, p in specs], [kk for _, kk, _ in specs])
        dev = [x[0].cuda() for x in Ls]
        assert plan.execute(dev, [x[1].cuda() for x in Ls]) == chm.CHM_OK
        assert plan.status()[0] == chm.CHM_OK
        plan.close()
    for (m, kk, p), (L0, V0, _), d in zip(specs, Ls, dev):
        ref = L0.numpy().copy()
        assert oracle.modify_b(ref, V0.numpy(), [1] * kk, n=m)[0] == 0
        assert colscaled_err(d.cpu().numpy(), ref, n=m) <= TOL_F64


@pytest.mark.parametrize("path", [chm.PATH_WAVE, chm.PATH_PASS])
def test_checks_report_accesses_outside_the_declared_extent(path):
    """check_cut = 1: the checks take the last column off the factor's
    declared extent, so the kernels' accesses to it (real memory, inside the
    tensor) are reported: CHM_ERR_BOUNDS, info = the offset of an element of
    that column, the access skipped, and the launch ends (no wait is left to
    time out).  The next call, with the setting cleared, is clean."""
    n, k, pad = 100, 3, 2
    L, V, sig = problem(n, k, pad, 17, torch.float64)
    ld = n + pad
    with chm.checked_library():
        chm.config_set("path", path)
        chm.config_set("check_cut", 1)
        try:
            st, info, _ = run(L, V, sig, n)
        finally:
            chm.config_set("check_cut", 0)
        assert st == chm.CHM_ERR_BOUNDS, (st, info)
        # the smallest offset reported lies in the last column (j = n - 1)
        assert (n - 1) * ld <= info < n * ld, info
        st, info, got = run(L, V, sig, n)
        assert st == chm.CHM_OK, (st, info)
    ref = L.numpy().copy()
    assert oracle.modify_b(ref, V.numpy(), sig, n=n)[0] == 0
    assert colscaled_err(got.numpy(), ref, n=n) <= TOL_F64
