"""Factors resident in page-locked host memory.

The paper keeps only O(n) panels of L on the device and streams the rest
from host memory (abstract, Sec. 4 and Sec. 5), so the factor's size is
bounded by host memory.  Here the kernel reads and writes L in place in
page-locked host memory across the CPU-GPU link; the device holds only the
O(n k) workspace.  The arithmetic is the same as for a device-resident
factor on the same path (the wave kernel or the pass kernels), so results
must be bit-identical to it, and within the float64 tolerance of the
oracle.  Under the automatic rule a host factor of order >= 64 modified by
k >= 2 vectors takes the pass kernels (three crossings of the link per pass
of up to 16 vectors, against two per vector for the wave kernel).
Pageable host memory is rejected on the host.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, colscaled_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)
    yield
    chm.config_set("path", chm.PATH_AUTO)
    chm.config_set("pass_kb", 0)


def pinned(t):
    out = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    out.copy_(t)
    return out


def problem(n, k, pad, dtype, seed):
    L = inputs.spd_factor(n, seed, ld=n + pad).to(dtype)
    V = inputs.update_block(n, k, seed, scale=0.5 / np.sqrt(max(1, n * k))).to(dtype)
    return L, V


@pytest.mark.parametrize("n,k,pad,dtype", [(1, 1, 0, torch.float64), (33, 5, 3, torch.float64),
                                           (257, 16, 0, torch.float64), (1000, 3, 1, torch.float64),
                                           (300, 16, 0, torch.float32), (1025, 40, 2, torch.float32)])
def test_host_resident_matches_device_resident(n, k, pad, dtype):
    seed = 9100 + n + k
    L, V = problem(n, k, pad, dtype, seed)
    sig = inputs.sigma_vector(k, seed).tolist()
    ref = None
    if dtype == torch.float64:
        ref = L.numpy().copy()
        assert oracle.modify_b(ref, V.numpy(), sig)[0] == 0
    by_path = {}
    # a factor in host memory takes 16 vectors per pass by default (each pass
    # crosses the CPU-GPU link); the device factor is given the same here, so
    # that the two run the same passes
    chm.config_set("pass_kb", 16)
    for path in (chm.PATH_WAVE, chm.PATH_PASS):
        chm.config_set("path", path)
        dev_L = L.cuda()
        assert chm.modify(dev_L, V.cuda(), sig) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        host_L, host_V = pinned(L), pinned(V)
        assert chm.modify(host_L, host_V, sig) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        assert torch.equal(host_L, dev_L.cpu()), (n, k, path)
        assert torch.equal(host_V, V)  # V is read only
        if ref is not None:
            assert colscaled_err(host_L.numpy(), ref) <= TOL_F64
        by_path[path] = host_L
    # the automatic rule: a host factor of order >= 64 with k >= 2 on the pass
    # kernels, with 16 vectors per pass
    chm.config_set("path", chm.PATH_AUTO)
    chm.config_set("pass_kb", 0)
    host_L = pinned(L)
    assert chm.modify(host_L, pinned(V), sig) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    assert torch.equal(host_L, by_path[chm.PATH_PASS if n >= 64 and k >= 2 else chm.PATH_WAVE]), (n, k)


def test_mixed_residency_and_noalloc():
    """One operand on the host and the other on the device, and the
    no-allocation entry point (the wave kernel) with a host factor; every
    call on the wave kernel so that the results are bit-identical."""
    n, k = 700, 9
    L, V = problem(n, k, 0, torch.float64, 77)
    chm.config_set("path", chm.PATH_WAVE)
    ref = L.cuda()
    assert chm.modify(ref, V.cuda(), 1) == chm.CHM_OK
    # L on the host, V on the device, and the reverse
    a = pinned(L)
    assert chm.modify(a, V.cuda(), 1) == chm.CHM_OK
    b = L.cuda()
    assert chm.modify(b, pinned(V), 1) == chm.CHM_OK
    assert chm.status_sync()[0] == chm.CHM_OK
    assert torch.equal(a, ref.cpu()) and torch.equal(b, ref)
    # the no-allocation entry point with a host-resident factor
    c = pinned(L)
    info = torch.full((2,), 99, dtype=torch.int64, device="cuda")
    st = chm.chm_modify_noalloc(c.data_ptr(), n, n, V.cuda().data_ptr(), n, k, None, 1, chm.CHM_F64,
                                torch.cuda.current_stream().cuda_stream, info.data_ptr())
    assert st == chm.CHM_OK
    torch.cuda.synchronize()
    assert info.tolist() == [0, -1]
    assert torch.equal(c, ref.cpu())
    chm.config_set("path", chm.PATH_AUTO)


def test_batch_with_host_resident_factors():
    specs = [(64, 2), (300, 16), (1000, 1), (45, 7)]
    Ls, Vs = [], []
    for i, (n, k) in enumerate(specs):
        L, V = problem(n, k, 0, torch.float64, 300 + i)
        Ls.append(L)
        Vs.append(V)
    ns, ks = [n for n, _ in specs], [k for _, k in specs]
    dev = [L.cuda() for L in Ls]
    host = [pinned(L) for L in Ls]
    plan = chm.BatchPlan(ns, ns, ks, [1, -1, 1, -1])
    assert plan.execute(dev, [V.cuda() for V in Vs]) == chm.CHM_OK
    assert plan.execute(host, [pinned(V) for V in Vs]) == chm.CHM_OK
    assert plan.status()[0] == chm.CHM_OK
    plan.close()
    for d, h in zip(dev, host):
        assert torch.equal(d.cpu(), h)


def test_pageable_host_memory_is_rejected_before_any_work():
    n, k = 100, 2
    L, V = problem(n, k, 0, torch.float64, 5)
    keep = L.clone()
    stream = torch.cuda.current_stream().cuda_stream
    # pageable L, device V
    Vd = V.cuda()
    st = chm.chm_modify_ex(L.data_ptr(), n, n, Vd.data_ptr(), n, k, None, 1, chm.CHM_F64, stream, None)
    assert st == chm.CHM_ERR_ARG
    # device L, pageable V
    Ld = L.cuda()
    st = chm.chm_update(Ld.data_ptr(), n, n, V.data_ptr(), k, chm.CHM_F64, stream)
    assert st == chm.CHM_ERR_ARG
    info = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = chm.chm_modify_noalloc(L.data_ptr(), n, n, Vd.data_ptr(), n, k, None, 1, chm.CHM_F64, stream,
                                info.data_ptr())
    assert st == chm.CHM_ERR_ARG
    plan = chm.BatchPlan([n], [n], [k])
    assert plan.execute([L], [Vd]) == chm.CHM_ERR_ARG
    plan.close()
    assert chm.status_sync()[0] == chm.CHM_OK
    assert torch.equal(L, keep) and torch.equal(Ld.cpu(), keep)


def test_device_memory_is_the_workspace_only():
    """With L on the host, the device memory a modification adds is the
    workspace chm_workspace_bytes reports (O(n k)), not the n^2 factor."""
    n, k = 6000, 4
    L, V = problem(n, k, 0, torch.float64, 11)
    host_L, dev_V = pinned(L), V.cuda()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(s):
        assert chm.modify(host_L, dev_V, 1, stream=s) == chm.CHM_OK
    assert chm.status_sync(s)[0] == chm.CHM_OK
    used = free0 - torch.cuda.mem_get_info()[0]
    ws = chm.workspace_bytes(n, k)
    factor = 8 * n * n
    assert ws < factor / 10
    # the driver rounds allocations to its own granularity (2 MiB pages)
    assert used <= ws + (16 << 20), (used, ws, factor)
    assert used < factor / 10
