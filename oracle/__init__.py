"""CPU oracle for the rank-k Cholesky up/downdate (Walder 2010).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product library
never loads it, and it shares no code with the CUDA path.

Two implementations of the same serial algorithm (Algorithm 1):

* ``chm_oracle.c`` (plain C, double, ``-ffp-contract=off``), wrapped here by
  ``modify_b`` / ``modify_a`` / ``modify_mixed32``;
* ``hyperbolic_np.py``, a numpy restatement of ``CholeskyModifyB`` that is
  bit-identical to the C routine (numpy rounds every elementwise operation
  separately, as the C build does).

``solve`` (``orc_solve`` in the C file) solves with a factor, the use the
factor is kept for (Sec. 1): forward substitution with L^T, then back
substitution with L.

Layout convention for every function: ``L`` is an (n, n) array holding the
column-major upper-triangular factor, i.e. a C-contiguous array whose ROW j is
column j of L (so ``L_cm[j, i]`` is L_ij).  Helpers ``to_cm``/``from_cm``
convert between a mathematical upper-triangular matrix and that layout.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

OK = 0
ERR_ARG = -1
ERR_NOT_PD = -2

_lib = None


def build(force: bool = False) -> str:
    """Compile chm_oracle.c into a shared library (plain gcc, no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, vp = ctypes.c_int64, ctypes.c_void_p
        lib.orc_modify_b.argtypes = [vp, i64, i64, vp, i64, i64, vp, i64, ctypes.POINTER(i64)]
        lib.orc_modify_b.restype = ctypes.c_int
        lib.orc_modify_mixed32.argtypes = [vp, i64, i64, vp, i64, i64, vp, i64, i64, ctypes.POINTER(i64)]
        lib.orc_modify_mixed32.restype = ctypes.c_int
        lib.orc_modify_a.argtypes = [vp, i64, i64, vp, i64, i64, vp, ctypes.POINTER(i64)]
        lib.orc_modify_a.restype = ctypes.c_int
        lib.orc_solve.argtypes = [vp, i64, i64, vp, i64, i64, ctypes.POINTER(i64)]
        lib.orc_solve.restype = ctypes.c_int
        _lib = lib
    return _lib


def _sig_array(sigma, k):
    if np.isscalar(sigma):
        sig = np.full(k, int(sigma), dtype=np.int8)
    else:
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.int8))
    if sig.shape != (k,):
        raise ValueError("sigma must be a scalar or have one entry per column of V")
    return sig


def _prep(L_cm, V_cm, dtype):
    """L_cm: (n, ld) array, row j = column j of L (first n entries used).
    V_cm: (k, ldv) array, row p = column p of V."""
    L_cm = np.asarray(L_cm)
    V_cm = np.asarray(V_cm)
    if L_cm.dtype != dtype or V_cm.dtype != dtype:
        raise TypeError("expected %s arrays" % np.dtype(dtype).name)
    if not (L_cm.flags.c_contiguous and V_cm.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous")
    if L_cm.ndim != 2 or V_cm.ndim != 2:
        raise ValueError("L_cm must be (n, ld) and V_cm must be (k, ldv)")
    return L_cm, V_cm


def modify_b(L_cm, V_cm, sigma, n=None, m_rows=None):
    """CholeskyModifyB, rank k, in place on ``L_cm`` (float64).

    ``L_cm`` is (n, ld) with row j holding column j of L; ``V_cm`` is (k, ldv)
    with row p holding column p of V.  Returns (status, info)."""
    L_cm, V_cm = _prep(L_cm, V_cm, np.float64)
    n = L_cm.shape[0] if n is None else n
    k = V_cm.shape[0]
    sig = _sig_array(sigma, k)
    info = ctypes.c_int64(-1)
    st = _load().orc_modify_b(L_cm.ctypes.data, n, L_cm.shape[1], V_cm.ctypes.data,
                              V_cm.shape[1], k, sig.ctypes.data,
                              -1 if m_rows is None else m_rows, ctypes.byref(info))
    return st, info.value


def modify_a(L_cm, V_cm, sigma, n=None):
    """CholeskyModifyA (Compute after the inner loop), rank k, in place."""
    L_cm, V_cm = _prep(L_cm, V_cm, np.float64)
    n = L_cm.shape[0] if n is None else n
    k = V_cm.shape[0]
    sig = _sig_array(sigma, k)
    info = ctypes.c_int64(-1)
    st = _load().orc_modify_a(L_cm.ctypes.data, n, L_cm.shape[1], V_cm.ctypes.data,
                              V_cm.shape[1], k, sig.ctypes.data, ctypes.byref(info))
    return st, info.value


def modify_mixed32(L_cm, V_cm, sigma, n=None, m_rows=None, group=None):
    """Mixed precision: float32 storage and Apply, float64 Compute.

    ``group`` is the number of consecutive vectors whose new diagonals are
    carried in double before being rounded to float (one launch or pass of
    the GPU path); None means all k vectors in one group."""
    L_cm, V_cm = _prep(L_cm, V_cm, np.float32)
    n = L_cm.shape[0] if n is None else n
    k = V_cm.shape[0]
    sig = _sig_array(sigma, k)
    info = ctypes.c_int64(-1)
    st = _load().orc_modify_mixed32(L_cm.ctypes.data, n, L_cm.shape[1], V_cm.ctypes.data,
                                    V_cm.shape[1], k, sig.ctypes.data,
                                    -1 if m_rows is None else m_rows,
                                    0 if group is None else int(group), ctypes.byref(info))
    return st, info.value


def solve(L_cm, B_cm, n=None):
    """X = (L^T L)^{-1} B in place on ``B_cm`` (float64): forward substitution
    with L^T, then back substitution with L (``orc_solve``).

    ``L_cm`` is (n, ld) with row j holding column j of L; ``B_cm`` is
    (nrhs, ldb) with row r holding column r of B.  Returns (status, info)."""
    L_cm, B_cm = _prep(L_cm, B_cm, np.float64)
    n = L_cm.shape[0] if n is None else n
    info = ctypes.c_int64(-1)
    st = _load().orc_solve(L_cm.ctypes.data, n, L_cm.shape[1], B_cm.ctypes.data, B_cm.shape[1],
                           B_cm.shape[0], ctypes.byref(info))
    return st, info.value


def to_cm(U):
    """Mathematical upper-triangular matrix -> column-major storage (row j = column j)."""
    return np.array(np.asarray(U).T, order="C", copy=True)


def from_cm(L_cm, n=None):
    """Column-major storage -> mathematical upper-triangular matrix (lower part zeroed)."""
    L_cm = np.asarray(L_cm)
    n = L_cm.shape[0] if n is None else n
    return np.triu(L_cm[:n, :n].T)
