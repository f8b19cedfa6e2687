"""The no-allocation entry point, chm_modify_noalloc.

Some callers cannot allocate device memory (under an allocator that owns
all device memory, or from budgeted real-time threads where cudaMalloc can
block, fail or synchronise the device).  chm_modify_noalloc serves them from a fixed device array; these
tests call it through the C ABI and check its factor against chm_modify_ex's
on two calls in a row.  This file is collected last so that a run stopping
at the first failure has already run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, colscaled_err, tol_mixed


def _call(fn, L, V, sigma, d_info=None):
    k = V.shape[0]
    sig = (ctypes.c_int8 * k)(*[int(s) for s in sigma])
    return fn(L.data_ptr(), L.shape[0], L.shape[1], V.data_ptr(), V.shape[1], k,
              ctypes.cast(sig, ctypes.c_void_p), 1, chm.dtype_code(L),
              torch.cuda.current_stream().cuda_stream,
              None if d_info is None else d_info.data_ptr())


def test_noalloc_rejects_too_large_without_work():
    # the size and argument checks come before any CUDA call, so this needs no GPU
    info = 16  # an aligned address that is never dereferenced
    st = chm.chm_modify_noalloc(8, 8193, 8193, 8, 8193, 1, None, 1, chm.CHM_F64, None, info)
    assert st == chm.CHM_ERR_BUDGET
    st = chm.chm_modify_noalloc(8, 10, 9, 8, 10, 1, None, 1, chm.CHM_F64, None, info)
    assert st == chm.CHM_ERR_ARG


def test_noalloc_requires_status_pointer_without_work():
    # its status word is in the shared array, which chm_status_sync does not
    # read: without d_info a failed modification could not be seen
    st = chm.chm_modify_noalloc(8, 10, 10, 8, 10, 1, None, 1, chm.CHM_F64, None, None)
    assert st == chm.CHM_ERR_ARG
    # nothing to do: no status is needed
    assert chm.chm_modify_noalloc(8, 10, 10, 8, 10, 0, None, 1, chm.CHM_F64, None, None) == chm.CHM_OK


@pytest.mark.gpu
@pytest.mark.parametrize("n,k,dtype", [(1500, 16, torch.float64), (4100, 40, torch.float64),
                                       (700, 9, torch.float32),
                                       # the documented limit: the array holds few vectors per
                                       # launch at this order, so k is split over many launches
                                       (8192, 64, torch.float64)])
def test_noalloc_matches_allocating_path_twice(n, k, dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    seed = 4242 + n + k
    L0 = inputs.spd_factor(n, seed, ld=n + 3).to("cuda", dtype)
    V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(n * k)).to("cuda", dtype)
    sig = inputs.sigma_vector(k, seed).tolist()
    tol = TOL_F64 if dtype == torch.float64 else tol_mixed(n, k)
    ref = L0.clone()
    got = L0.clone()
    info = torch.full((2,), 99, dtype=torch.int64, device="cuda")
    for _ in range(2):  # two calls in a row, each continuing from the last
        assert _call(chm.chm_modify_ex, ref, V, sig) == chm.CHM_OK
        assert _call(chm.chm_modify_noalloc, got, V, sig, info) == chm.CHM_OK
        torch.cuda.synchronize()
        assert info.tolist() == [chm.CHM_OK, -1]
        assert chm.status_sync()[0] == chm.CHM_OK
        assert colscaled_err(got.cpu().numpy(), ref.cpu().numpy()) <= tol
