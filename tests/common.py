"""Shared test helpers (no method arithmetic here)."""
from __future__ import annotations

import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Parity tolerance for the float64 path, elementwise and column-scaled:
#   |g_ij - o_ij| <= TOL_F64 * max(|o_ij|, max_r |o_rj|)
TOL_F64 = 1e-11

# Mixed precision (float storage and Apply, double Compute).  The GPU path
# and the oracle's emulation evaluate the same rotations in float with
# different operation orders, so they agree to float rounding, not bit for
# bit.  Bound used, column-scaled: an entry in row i is the end of a chain
# of at most m = (i + 1) k rotations; each adds at most 4 float roundings
# (the two products and sums of Apply, and the coefficient's own rounding),
# relative u = 2^-24 each; treating them as independent (the standard
# first-order model of rounding, under which such errors grow as sqrt(m) u)
# each evaluation is within 4 sqrt(m) u of the exact result, and the two
# within 8 sqrt(m) u of each other.
U_F32 = 2.0 ** -24


def tol_mixed(rows, k):
    """Column-scaled bound on |GPU - emulation| for a float modification of
    `rows` rows by k vectors (see above)."""
    return 8.0 * U_F32 * math.sqrt(max(1, rows) * max(1, k))


def accuracy_as_serial(e_gpu, e_serial):
    """The paper's accuracy claim (Sec. 5: the GPU's error and the serial
    CPU code's are always very similar), as a test: the GPU path's error
    against the float64 oracle is at most twice that of the serial algorithm
    in the same precision split, plus four float ulps."""
    return e_gpu <= 2.0 * e_serial + 4.0 * U_F32


def colscaled_err(got_cm, ref_cm, n=None, chunk=2048):
    """Max over the upper triangle of |got - ref| / max(|ref_ij|, max_r |ref_rj|).

    Both arrays use the (n, ld) storage of the C ABI: row j is column j of L.
    Works through the storage rows in chunks, so that a factor of order 32768
    needs no full-size temporaries."""
    n = np.asarray(ref_cm).shape[0] if n is None else n
    worst = 0.0
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        g = np.asarray(got_cm[j0:j1, :n], dtype=np.float64)
        r = np.asarray(ref_cm[j0:j1, :n], dtype=np.float64)
        mask = np.arange(n)[None, :] <= np.arange(j0, j1)[:, None]  # row j, entries i <= j
        colmax = np.max(np.where(mask, np.abs(r), 0.0), axis=1, keepdims=True)
        scale = np.maximum(np.abs(r), colmax)
        scale = np.where(scale == 0, 1.0, scale)
        err = np.where(mask, np.abs(g - r) / scale, 0.0)
        worst = max(worst, float(err.max()))
    return worst


def elementwise_rel_err(got_cm, ref_cm, n=None, floor=1e-300, chunk=2048):
    """Max over the upper triangle of |got - ref| / max(|ref_ij|, floor): the
    plain elementwise relative error (entries below `floor` in magnitude are
    compared absolutely against it)."""
    n = np.asarray(ref_cm).shape[0] if n is None else n
    worst = 0.0
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        g = np.asarray(got_cm[j0:j1, :n], dtype=np.float64)
        r = np.asarray(ref_cm[j0:j1, :n], dtype=np.float64)
        mask = np.arange(n)[None, :] <= np.arange(j0, j1)[:, None]
        err = np.where(mask, np.abs(g - r) / np.maximum(np.abs(r), floor), 0.0)
        worst = max(worst, float(err.max()))
    return worst


def upper_from_cm(L_cm, n=None):
    L_cm = np.asarray(L_cm)
    n = L_cm.shape[0] if n is None else n
    return np.triu(L_cm[:n, :n].T)


def cm_from_upper(U, ld=None):
    U = np.asarray(U, dtype=np.float64)
    n = U.shape[0]
    ld = n if ld is None else ld
    out = np.zeros((n, ld))
    out[:, :n] = np.triu(U).T
    return out


def modified_matrix(U, V, sigma):
    """L^T L + V diag(sigma) V^T in float64 (numpy BLAS)."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (V.shape[1],))
    return U.T @ U + (V * sig) @ V.T


def load_hand_examples():
    with open(os.path.join(GOLDEN, "hand_examples.json")) as f:
        data = json.load(f)

    def ev(s):
        return float(eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt}))

    out = []
    for c in data["cases"]:
        out.append({
            "name": c["name"],
            "L": np.array([[ev(x) for x in row] for row in c["L"]]),
            "V": np.array([[ev(x) for x in row] for row in c["V"]]),
            "sigma": np.array(c["sigma"], dtype=np.int8),
            "expected": np.array([[ev(x) for x in row] for row in c["expected"]]),
        })
    return out
