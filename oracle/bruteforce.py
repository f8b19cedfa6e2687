"""Brute-force references that pin the oracle (tiny sizes only).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The modified factor has a plain definition (Sec. 1): the unique upper
triangular Lt with positive diagonal such that Lt^T Lt = L^T L + V S V^T,
S = diag(sigma).  ``modified_factor_decimal`` forms that matrix from the
binary64 inputs with 60 significant decimal digits (every product of two
doubles is exact at that precision and the few sums lose nothing visible at
double precision) and factors it by the textbook Cholesky recurrence in the
same arithmetic, so its result is the exact answer to far below double
rounding.
"""
from __future__ import annotations

from decimal import Decimal, getcontext, localcontext

import numpy as np


def _dec(x):
    return Decimal(float(x))  # exact binary64 -> decimal conversion


def modified_matrix_decimal(U, V, sigma, prec=60):
    """A_t = U^T U + V diag(sigma) V^T in ``prec``-digit decimal arithmetic."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    n, k = V.shape
    sig = np.broadcast_to(np.asarray(sigma), (k,))
    with localcontext() as ctx:
        ctx.prec = prec
        Ud = [[_dec(U[i, j]) if i <= j else Decimal(0) for j in range(n)] for i in range(n)]
        Vd = [[_dec(V[i, p]) for p in range(k)] for i in range(n)]
        A = [[Decimal(0)] * n for _ in range(n)]
        for a in range(n):
            for b in range(a, n):
                acc = Decimal(0)
                for r in range(min(a, b) + 1):
                    acc += Ud[r][a] * Ud[r][b]
                for p in range(k):
                    acc += int(sig[p]) * Vd[a][p] * Vd[b][p]
                A[a][b] = acc
                A[b][a] = acc
    return A


def cholesky_upper_decimal(A, prec=60):
    """Textbook Cholesky A = R^T R in decimal; returns R as float64 (None if not PD)."""
    n = len(A)
    with localcontext() as ctx:
        ctx.prec = prec
        R = [[Decimal(0)] * n for _ in range(n)]
        for i in range(n):
            d = A[i][i] - sum((R[r][i] * R[r][i] for r in range(i)), Decimal(0))
            if d <= 0:
                return None
            R[i][i] = d.sqrt()
            for j in range(i + 1, n):
                e = A[i][j] - sum((R[r][i] * R[r][j] for r in range(i)), Decimal(0))
                R[i][j] = e / R[i][i]
    return np.array([[float(R[i][j]) for j in range(n)] for i in range(n)])


def modified_factor_decimal(U, V, sigma, prec=60):
    return cholesky_upper_decimal(modified_matrix_decimal(U, V, sigma, prec), prec)
