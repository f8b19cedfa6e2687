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


def colscaled_err(got_cm, ref_cm, n=None):
    """Max over the upper triangle of |got - ref| / max(|ref_ij|, max_r |ref_rj|).

    Both arrays use the (n, ld) storage of the C ABI: row j is column j of L."""
    got = np.asarray(got_cm, dtype=np.float64)
    ref = np.asarray(ref_cm, dtype=np.float64)
    n = ref.shape[0] if n is None else n
    g = got[:n, :n]
    r = ref[:n, :n]
    mask = np.tril(np.ones((n, n), dtype=bool))  # row j, entries i <= j
    colmax = np.max(np.where(mask, np.abs(r), 0.0), axis=1, keepdims=True)
    scale = np.maximum(np.abs(r), colmax)
    scale = np.where(scale == 0, 1.0, scale)
    err = np.where(mask, np.abs(g - r) / scale, 0.0)
    return float(err.max()) if n else 0.0


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
