"""The seeded input generators: the storage convention of the C ABI (row j
of an (n, ld) tensor is column j of the upper factor, zeros below the
diagonal and in the padding) and the workload recipe (A = B^T B / n + I with
B ~ N(0, 1), V ~ N(0, 1/n), the cheap random factors of the batched and
served runs, the signs).  CPU only."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1011_1173_gb300 import inputs


def test_spd_factor_is_the_upper_factor_of_the_recipe():
    n, ld, seed = 60, 64, 123
    Lcm = inputs.spd_factor(n, seed, ld=ld).numpy()
    assert Lcm.shape == (n, ld)
    assert np.all(Lcm[:, n:] == 0)                       # padding
    assert np.all(np.triu(Lcm[:, :n], 1) == 0)           # storage row j holds entries i <= j of column j
    assert np.all(np.diag(Lcm[:, :n]) > 0)
    g = torch.Generator().manual_seed(seed)
    B = torch.randn((n, n), generator=g, dtype=torch.float64).numpy()
    A = B.T @ B / n + np.eye(n)
    # L^T L with L[i, j] = Lcm[j, i]: (L^T L)[a, b] = sum_i Lcm[a, i] Lcm[b, i]
    np.testing.assert_allclose(Lcm[:, :n] @ Lcm[:, :n].T, A, rtol=0, atol=1e-12 * np.abs(A).max())


def test_update_block_scale_and_layout():
    n, k, seed = 400, 5, 9
    V = inputs.update_block(n, k, seed, ldv=410).numpy()
    assert V.shape == (k, 410) and np.all(V[:, n:] == 0)
    g = torch.Generator().manual_seed(seed + 7919)
    ref = (torch.randn((k, n), generator=g, dtype=torch.float64) * (1.0 / n) ** 0.5).numpy()
    np.testing.assert_array_equal(V[:, :n], ref)
    assert inputs.update_block(n, k, seed, scale=0.5).numpy()[:, :n] == pytest.approx(ref * 0.5 * n ** 0.5)


def test_random_factor_is_a_valid_factor():
    n = 77
    Lcm = inputs.random_factor(n, 5, ld=80).numpy()
    assert np.all(Lcm[:, n:] == 0) and np.all(np.triu(Lcm[:, :n], 1) == 0)
    d = np.diag(Lcm[:, :n])
    assert np.all((d >= 1.0) & (d < 2.0))


def test_seeds_and_signs():
    assert inputs.config_seed(0) == 20101104 and inputs.config_seed(3) == 20101107
    s = inputs.sigma_vector(1000, 4).numpy()
    assert set(np.unique(s).tolist()) <= {-1, 1} and 0.4 < (s == 1).mean() < 0.6
    assert np.array_equal(s, inputs.sigma_vector(1000, 4).numpy())


def test_empty_shapes():
    assert inputs.spd_factor(0, 1, ld=1).shape == (0, 1)
    assert inputs.update_block(10, 0, 1).shape == (0, 10)
    with pytest.raises(ValueError):
        inputs.spd_factor(5, 1, ld=4)
