"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5).

This module draws random matrices and factors them; it holds none of the
up/downdate arithmetic, and both the CUDA path and the CPU oracle take their
inputs from it.

Storage convention (shared with the C ABI): an upper-triangular factor L of
order n with leading dimension ``ld`` is a C-contiguous tensor of shape
(n, ld) whose ROW j holds COLUMN j of L, i.e. ``L_cm[j, i] == L[i, j]`` and the
column-major element L[i + j*ld] of the C ABI.  Entries with i > j (the
strictly lower part of L) and the padding i >= n are zero unless a caller
fills them.  V (n x k) is stored the same way: a (k, ldv) tensor whose row p
is column p of V.

Workload recipe: B ~ N(0, 1) of order n, A = B^T B / n + I, L the upper
Cholesky factor of A, V ~ N(0, 1/n).  The paper's own experiment (Sec. 5)
uses B and V with i.i.d. U[0, 1] entries and A = B^T B + I (plus V V^T for the
downdate test); ``paper_uniform_problem`` draws that variant.
"""
from __future__ import annotations

import torch

SEED_BASE = 20101104


def config_seed(index: int) -> int:
    """Seed for workload configuration ``index``."""
    return SEED_BASE + int(index)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def spd_factor(n: int, seed: int, ld: int | None = None, device="cpu",
               dtype=torch.float64, factor_dtype=None) -> torch.Tensor:
    """Upper Cholesky factor of A = B^T B / n + I, B ~ N(0, 1), in (n, ld) storage.

    ``factor_dtype`` is the precision in which B, A and the factorisation are
    formed (default: float64 for n <= 8192, float32 above, where forming A in
    float64 would dominate the run on a part with a slow FP64 pipe).  The
    returned factor is whatever that factorisation gives, cast to ``dtype``:
    a valid upper-triangular factor with positive diagonal, which is all the
    method needs (A is then L^T L by definition)."""
    ld = n if ld is None else int(ld)
    if ld < max(1, n):
        raise ValueError("ld must be >= max(1, n)")
    if factor_dtype is None:
        factor_dtype = torch.float64 if n <= 8192 else torch.float32
    out = torch.zeros((n, ld), dtype=dtype, device=device)
    if n == 0:
        return out
    g = _gen(seed, device)
    B = torch.randn((n, n), generator=g, dtype=factor_dtype, device=device)
    A = B.T @ B
    del B
    A.div_(n)
    A.diagonal().add_(1.0)
    # torch's lower factor G (A = G G^T) in row-major order has exactly the
    # memory image of the column-major upper factor L = G^T.  Orders up to
    # 8192 are factored on the host (LAPACK), larger ones on the device, or
    # on the host when the device factorisation is unavailable (torch loads
    # its device linear-algebra library lazily, and a profiler's process
    # environment can keep it from loading).
    if n <= 8192:
        G = torch.linalg.cholesky(A.cpu())
    else:
        try:
            G = torch.linalg.cholesky(A)
        except RuntimeError:
            if A.device.type == "cpu":
                raise
            G = torch.linalg.cholesky(A.cpu())
    del A
    out[:, :n].copy_(G)
    return out


def update_block(n: int, k: int, seed: int, ldv: int | None = None, device="cpu",
                 dtype=torch.float64, scale: float | None = None) -> torch.Tensor:
    """V ~ N(0, 1/n) (or N(0, scale^2)) in (k, ldv) storage."""
    ldv = n if ldv is None else int(ldv)
    if ldv < max(1, n):
        raise ValueError("ldv must be >= max(1, n)")
    out = torch.zeros((k, ldv), dtype=dtype, device=device)
    if n == 0 or k == 0:
        return out
    g = _gen(seed + 7919, device)
    s = (1.0 / n) ** 0.5 if scale is None else float(scale)
    out[:, :n].copy_(torch.randn((k, n), generator=g, dtype=torch.float64, device=device) * s)
    return out


def paper_uniform_problem(n: int, k: int, seed: int, downdate: bool, device="cpu"):
    """The paper's experiment (Sec. 5): B, V with i.i.d. U[0, 1] entries,
    A = B^T B + I for the update test and A = B^T B + I + V V^T for the
    downdate test; returns (L_cm, V_cm, A) in float64."""
    g = _gen(seed, device)
    B = torch.rand((n, n), generator=g, dtype=torch.float64, device=device)
    V = torch.rand((n, k), generator=g, dtype=torch.float64, device=device)
    A = B.T @ B + torch.eye(n, dtype=torch.float64, device=device)
    if downdate:
        A = A + V @ V.T
    G = torch.linalg.cholesky(A)
    return G.contiguous(), V.T.contiguous(), A


def sigma_vector(k: int, seed: int, p_update: float = 0.5) -> torch.Tensor:
    """Random per-column signs (+1 update, -1 downdate) as int8."""
    g = _gen(seed + 104729, "cpu")
    r = torch.rand((k,), generator=g)
    return torch.where(r < p_update, 1, -1).to(torch.int8)


def random_factor(n: int, seed: int, ld: int | None = None, device="cpu",
                  dtype=torch.float64) -> torch.Tensor:
    """A cheap upper-triangular factor for workloads that need many of them
    (batched and served runs): diagonal 1 + U[0, 1), strictly upper entries
    N(0, 1/n), in (n, ld) storage.  Any upper-triangular matrix with positive
    diagonal is the Cholesky factor of A = L^T L, so this is a valid input of
    the method; its conditioning is close to that of ``spd_factor``'s."""
    ld = n if ld is None else int(ld)
    if ld < max(1, n):
        raise ValueError("ld must be >= max(1, n)")
    out = torch.zeros((n, ld), dtype=dtype, device=device)
    if n == 0:
        return out
    g = _gen(seed, device)
    # row j of the storage is column j of L: its entries i <= j are the lower
    # triangle (with the diagonal) of the (n, n) storage block
    R = torch.randn((n, n), generator=g, dtype=dtype, device=device).mul_(n ** -0.5).tril_(-1)
    R.diagonal().copy_(1.0 + torch.rand((n,), generator=g, dtype=dtype, device=device))
    out[:, :n].copy_(R)
    return out
