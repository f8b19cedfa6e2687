"""numpy restatement of CholeskyModifyB (Algorithm 1), rank k.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Works on the mathematical upper-triangular matrix ``U`` (U[i, j] = L_ij for
i <= j).  For each row i and each column p of V in ascending order it runs
Compute on (L_ii, V_i^p) and then Apply on row i to the right of the
diagonal, vectorised over j; every elementwise operation is rounded on its
own, so the result equals the C oracle bit for bit.

``mutant`` plants one plausible mistake so that the tests can show their pins
catch it.  It is used only by the tests; ``None`` is the algorithm itself.
Mutants:
  "old_l_in_v"    V_j update uses the OLD L_ij instead of the new one
  "sign_apply"    L_ij update uses -sigma instead of +sigma
  "no_div_c"      L_ij update forgets the division by c
  "c_swapped"     c = L_ii / w instead of w / L_ii
  "s_from_w"      s = V_i / w instead of V_i / L_ii
  "compute_first" CholeskyModifyA as printed: the column's Compute happens
                  before the rows above it have rotated V_i
  "no_v_update"   V_j is never rotated (the carry of V between rows dropped)

``modify_mixed32_np`` restates the mixed-precision emulation
(``orc_modify_mixed32``: float storage and Apply, double Compute, the new
diagonal carried in double across a group of vectors) with numpy float32
arithmetic, equal to the C routine bit for bit.  Its mutants:
  "cs_unrounded"     Apply uses c and s in double (each result still
                     rounded to float)
  "diag_per_vector"  the new diagonal is rounded to float after every
                     vector instead of once per group
  "apply_in_double"  Apply in double, rounded to float once per step
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefinite(Exception):
    def __init__(self, row):
        super().__init__("modified matrix not positive definite at row %d" % row)
        self.row = row


def modify_b_np(U, V, sigma, mutant=None):
    """Return the modified upper-triangular factor (float64 copies)."""
    U = np.array(U, dtype=np.float64, copy=True)
    V = np.array(V, dtype=np.float64, copy=True)
    if V.ndim == 1:
        V = V[:, None]
    n, k = V.shape
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (k,)).copy()
    if mutant == "compute_first":
        return _modify_a_printed(U, V, sig)
    for i in range(n):
        for p in range(k):
            v = V[:, p]
            l = U[i, i]
            if not (l > 0.0 and np.isfinite(l)):
                raise NotPositiveDefinite(i)
            t = l * l + sig[p] * v[i] * v[i]
            if not (t > 0.0 and np.isfinite(t)):
                raise NotPositiveDefinite(i)
            w = np.sqrt(t)
            c = w / l
            s = v[i] / l
            if mutant == "c_swapped":
                c = l / w
            if mutant == "s_from_w":
                s = v[i] / w
            U[i, i] = w
            row = U[i, i + 1:]
            vj = v[i + 1:]
            sg = -sig[p] if mutant == "sign_apply" else sig[p]
            if mutant == "no_div_c":
                new = row + sg * s * vj
            else:
                new = (row + sg * s * vj) / c
            if mutant == "old_l_in_v":
                vnew = c * vj - s * row
            else:
                vnew = c * vj - s * new
            U[i, i + 1:] = new
            if mutant != "no_v_update":
                v[i + 1:] = vnew
    return U


def _modify_a_printed(U, V, sig):
    """CholeskyModifyA with Compute placed before the inner loop, as printed."""
    n, k = V.shape
    cs = np.zeros((n, k, 2))
    for i in range(n):
        vi = V[i, :].copy()
        for p in range(k):
            l = U[i, i]
            t = l * l + sig[p] * vi[p] * vi[p]
            if not (t > 0.0):
                raise NotPositiveDefinite(i)
            w = np.sqrt(t)
            cs[i, p] = (w / l, vi[p] / l)
            U[i, i] = w
        for j in range(i):
            for p in range(k):
                c, s = cs[j, p]
                new = (U[j, i] + sig[p] * s * vi[p]) / c
                vi[p] = c * vi[p] - s * new
                U[j, i] = new
    return U


def modify_mixed32_np(U, V, sigma, group=None, mutant=None):
    """Mixed-precision emulation on the upper-triangular float32 matrix ``U``
    (float32 copies in, float32 out); ``group`` vectors per group (None: all)."""
    f32 = np.float32
    U = np.array(U, dtype=f32, copy=True)
    V = np.array(V, dtype=f32, copy=True)
    if V.ndim == 1:
        V = V[:, None]
    n, k = V.shape
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (k,)).copy()
    g = k if group is None or group <= 0 or group > k else int(group)
    for g0 in range(0, k, g):
        for i in range(n):
            lii = np.float64(U[i, i])
            for p in range(g0, min(k, g0 + g)):
                v = V[:, p]
                if not (lii > 0.0 and np.isfinite(lii)):
                    raise NotPositiveDefinite(i)
                t = lii * lii + sig[p] * np.float64(v[i]) * np.float64(v[i])
                if not (t > 0.0 and np.isfinite(t)):
                    raise NotPositiveDefinite(i)
                w = np.sqrt(t)
                c = w / lii
                s = np.float64(v[i]) / lii
                lii = w
                if mutant == "diag_per_vector":
                    lii = np.float64(f32(lii))
                row = U[i, i + 1:]
                vj = v[i + 1:]
                if mutant == "cs_unrounded":
                    new = ((row + (sig[p] * s * vj.astype(np.float64)).astype(f32)).astype(np.float64) / c).astype(f32)
                    vnew = ((c * vj.astype(np.float64)).astype(f32) - (s * new.astype(np.float64)).astype(f32)).astype(f32)
                elif mutant == "apply_in_double":
                    r64, v64 = row.astype(np.float64), vj.astype(np.float64)
                    n64 = (r64 + sig[p] * s * v64) / c
                    new = n64.astype(f32)
                    vnew = (c * v64 - s * n64).astype(f32)
                else:
                    cf, sf, sg = f32(c), f32(s), f32(sig[p])
                    prod = (sg * sf) * vj
                    new = (row + prod) / cf
                    vnew = cf * vj - sf * new
                U[i, i + 1:] = new
                v[i + 1:] = vnew
            U[i, i] = f32(lii)
    return U
