"""The reciprocal and reciprocal square root the kernels use in double
precision, against CUDA's correctly rounded 1.0/x and 1.0/sqrt(x).

The kernels refine the hardware's flush-to-zero approximations by one
third-order Newton-Raphson step and fall back to IEEE division and square
root outside [2^-1020, 2^1020].  Bound checked here: at most 1 ulp from the
correctly rounded value (1/x: CUDA's IEEE quotient; 1/sqrt(x): rounded once
from 50-digit decimal arithmetic) for every normal and subnormal input, with
no input flushed to zero.
"""
from __future__ import annotations

import ctypes
import decimal

import numpy as np
import pytest
import torch

from paper_1011_1173_gb300 import chm

pytestmark = pytest.mark.gpu


def ulp_distance(a, b):
    """|a - b| in units in the last place, by the ordering of the IEEE bit patterns."""
    ia = np.asarray(a, dtype=np.float64).view(np.int64)
    ib = np.asarray(b, dtype=np.float64).view(np.int64)
    # map sign-magnitude to a monotone integer line
    ia = np.where(ia < 0, np.int64(-0x8000000000000000) - ia, ia)
    ib = np.where(ib < 0, np.int64(-0x8000000000000000) - ib, ib)
    return np.abs(ia - ib)


def inputs():
    rng = np.random.default_rng(20101104)
    xs = []
    # every binade of the normal range, eight random mantissas each
    for e in range(-1022, 1024):
        xs.append(np.ldexp(1.0 + rng.random(8), e))
        xs.append(np.array([np.ldexp(1.0, e), np.nextafter(np.ldexp(1.0, e), np.inf)]))
    # subnormals (the flush-to-zero seed would treat these as 0)
    xs.append(np.array([5e-324, 1e-320, 2.5e-310, np.nextafter(2.2250738585072014e-308, 0)]))
    xs.append(np.ldexp(rng.random(64) + 0.01, -1030))
    # both sides of the fallback boundaries
    for e in (-1020, 1020):
        b = np.ldexp(1.0, e)
        xs.append(np.array([np.nextafter(b, 0), b, np.nextafter(b, np.inf)]))
    x = np.concatenate(xs)
    return x[x > 0]


def rsqrt_correctly_rounded(x):
    """1/sqrt(x) rounded once to the nearest double (50-digit decimal arithmetic
    on the exact value of each double, then one correctly rounded conversion)."""
    ctx = decimal.Context(prec=50)
    return np.array([float(ctx.divide(1, ctx.sqrt(decimal.Decimal(float(v))))) for v in x])


def run(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(4 * x.size, dtype=np.float64)
    st = chm.chm_selftest_reciprocals(x.ctypes.data_as(ctypes.c_void_p), x.size,
                                      out.ctypes.data_as(ctypes.c_void_p))
    assert st == chm.CHM_OK
    return out.reshape(-1, 4)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)


def test_reciprocal_within_one_ulp_of_ieee():
    x = inputs()
    o = run(x)
    # CUDA's quotient is the IEEE one (the host computes the same); 1/x of
    # the smallest subnormals overflows to infinity, and must do so here too
    with np.errstate(over="ignore", divide="ignore"):
        ieee = 1.0 / x
    assert np.array_equal(o[:, 2], ieee)
    assert np.array_equal(np.isinf(o[:, 0]), np.isinf(ieee))
    fin = np.isfinite(ieee)
    d = ulp_distance(o[fin, 0], ieee[fin])
    print("rcp: max ulp %d over %d inputs" % (d.max(), x.size))
    assert d.max() <= 1
    # negative inputs mirror
    on = run(-x[::7])
    assert np.max(ulp_distance(on[:, 0], on[:, 2])) <= 1


def test_reciprocal_sqrt_within_one_ulp_of_ieee():
    x = inputs()
    o = run(x)
    # CUDA's 1.0 / sqrt(x) is two IEEE operations, as on the host
    assert np.array_equal(o[:, 3], 1.0 / np.sqrt(x))
    assert np.all(np.isfinite(o[:, 1]))
    d = ulp_distance(o[:, 1], rsqrt_correctly_rounded(x))
    print("rsqrt: max ulp %d over %d inputs" % (d.max(), x.size))
    assert d.max() <= 1


def test_no_input_is_flushed():
    # subnormal inputs whose reciprocals are finite (a flushed input would give inf)
    tiny = np.array([6e-309, 1e-308, 2.0e-308])
    o = run(tiny)
    assert np.all(o[:, 0] > 0) and np.all(np.isfinite(o[:, 0]))
    assert np.array_equal(ulp_distance(o[:, 0], 1.0 / tiny) <= 1, np.ones(3, bool))
    # every subnormal has a finite reciprocal square root
    tiny = np.array([5e-324, 1e-310, 2.0e-308])
    o = run(tiny)
    assert np.all(o[:, 1] > 0) and np.all(np.isfinite(o[:, 1]))
    assert np.max(ulp_distance(o[:, 1], rsqrt_correctly_rounded(tiny))) <= 1
