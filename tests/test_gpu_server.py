"""GPU tests of the serving loop (chm_server_*): resident factors, requests
admitted against a budget, continuous batching over several launch slots.
Each factor's final value must be bit-identical to applying its requests
alone, in submission order, with chm_modify_ex; launches must overlap; the
budget must be enforced; a failed downdate must invalidate only its factor."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle
from paper_1011_1173_gb300 import chm, inputs
from tests.common import TOL_F64, colscaled_err

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chm.load(build_if_missing=True)
    torch.cuda.set_device(0)


def request_stream(ns, count, seed, kmax=8):
    """(fid, V (k, n) float64 CPU tensor, sign): 70 % updates with a fresh V,
    30 % downdates of the factor's most recent update still applied."""
    rng = np.random.default_rng(seed)
    history = {f: [] for f in range(len(ns))}
    out = []
    for r in range(count):
        f = int(min(len(ns) - 1, rng.zipf(1.3) - 1))
        if rng.random() < 0.3 and history[f]:
            V = history[f].pop()
            out.append((f, V, -1))
        else:
            n = ns[f]
            k = int(rng.integers(1, kmax + 1))
            V = torch.as_tensor(rng.standard_normal((k, n)) * (0.3 / np.sqrt(n)))
            history[f].append(V)
            out.append((f, V, 1))
    return out


def test_server_mix_equals_alone():
    ns = [40, 64, 100, 150, 200, 257, 300, 333, 500, 700]
    L0 = [inputs.spd_factor(n, 900 + i) for i, n in enumerate(ns)]
    srv = chm.Server(4 * GB, chm.CHM_F64, max_inflight=2)
    fids = [srv.add_factor(L.cuda() if i % 2 else L) for i, L in enumerate(L0)]
    assert fids == list(range(len(ns)))
    reqs = request_stream(ns, 60, 1234)
    rng = np.random.default_rng(5)
    ids = []
    for j, (f, V, s) in enumerate(reqs):
        src = V.cuda().contiguous() if j % 3 == 0 else V.contiguous()
        ids.append(srv.submit(f, src, s))
        if rng.random() < 0.2:
            time.sleep(0.0005)  # arrivals while launches are in flight
    assert srv.drain(60.0) == chm.CHM_OK
    done = srv.poll()
    assert sorted(d[0] for d in done) == sorted(ids)
    assert all(d[1] == chm.CHM_OK for d in done)
    assert all(d[2] > 0.0 for d in done)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["outstanding"] == 0 and st["launches"] >= 1
    for f, n in enumerate(ns):
        got = torch.empty((n, n), dtype=torch.float64, device="cuda")
        assert srv.get_factor(f, got) == chm.CHM_OK
        alone = L0[f].cuda().clone()
        seq = [(V, s) for (g, V, s) in reqs if g == f]
        for V, s in seq:
            assert chm.modify(alone, V.cuda().contiguous(), s) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        assert torch.equal(got, alone), f
        if f in (0, 5) and seq:
            ref = L0[f].numpy().copy()
            for V, s in seq:
                oracle.modify_b(ref, V.numpy(), s)
            assert colscaled_err(got.cpu().numpy(), ref) <= 10 * TOL_F64
    srv.close()


def test_server_launches_overlap():
    n, k = 1000, 16
    srv = chm.Server(8 * GB, chm.CHM_F64, max_inflight=2)
    fids = [srv.add_factor(inputs.spd_factor(n, 50 + i).cuda()) for i in range(24)]
    V = inputs.update_block(n, k, 3).cuda()
    for f in fids[:12]:
        srv.submit(f, V, 1)
    for f in fids[12:]:
        srv.submit(f, V, 1)
    for f in fids:
        srv.submit(f, V, -1)
    assert srv.drain(60.0) == chm.CHM_OK
    st = srv.stats()
    assert st["completed"] == 48
    assert st["max_concurrent"] >= 2, st
    assert all(d[1] == chm.CHM_OK for d in srv.poll())
    srv.close()


def test_server_budget_is_enforced():
    with pytest.raises(chm.ChmError) as e:
        chm.Server(300 << 20, chm.CHM_F64, max_inflight=2)   # below the slots' scratch
    assert e.value.status == chm.CHM_ERR_BUDGET
    srv = chm.Server(600 << 20, chm.CHM_F64, max_inflight=2)  # 512 MiB scratch, 88 MiB for data
    with pytest.raises(chm.ChmError) as e:
        srv.add_factor(inputs.spd_factor(4000, 1).cuda())     # 128 MB
    assert e.value.status == chm.CHM_ERR_BUDGET
    f = srv.add_factor(inputs.spd_factor(2000, 2).cuda())      # 32 MB
    g = srv.add_factor(inputs.spd_factor(2000, 3).cuda())      # 32 MB
    with pytest.raises(chm.ChmError) as e:
        srv.add_factor(inputs.spd_factor(2000, 4).cuda())
    assert e.value.status == chm.CHM_ERR_BUDGET
    V = inputs.update_block(2000, 64, 5).cuda()                # 1 MB each
    rid = srv.submit(f, V, 1)
    assert rid >= 1
    with pytest.raises(chm.ChmError) as e:
        srv.submit(g, torch.zeros((65, 2000), dtype=torch.float64, device="cuda"), 1)  # k > 64
    assert e.value.status == chm.CHM_ERR_ARG
    assert srv.drain(30.0) == chm.CHM_OK
    srv.close()


def test_server_failed_downdate_invalidates_only_its_factor():
    n = 40
    srv = chm.Server(2 * GB, chm.CHM_F64, max_inflight=2)
    bad = srv.add_factor(torch.eye(n, dtype=torch.float64))
    good_L = inputs.spd_factor(64, 9)
    good = srv.add_factor(good_L)
    v = torch.zeros((1, n), dtype=torch.float64)
    v[0, 0] = 2.0
    r1 = srv.submit(bad, v, -1)
    Vg = inputs.update_block(64, 3, 9)
    r2 = srv.submit(good, Vg, 1)
    assert srv.drain(30.0) == chm.CHM_OK
    r3 = srv.submit(bad, v, 1)  # after the failure: refused with CHM_ERR_STATE
    assert srv.drain(30.0) == chm.CHM_OK
    res = {i: s for i, s, _ in srv.poll()}
    assert res[r1] == chm.CHM_ERR_NOT_PD
    assert res[r2] == chm.CHM_OK
    assert res[r3] == chm.CHM_ERR_STATE
    out = torch.empty((64, 64), dtype=torch.float64)
    assert srv.get_factor(good, out) == chm.CHM_OK
    ref = good_L.numpy().copy()
    oracle.modify_b(ref, Vg.numpy(), 1)
    assert colscaled_err(out.numpy(), ref) <= TOL_F64
    assert srv.get_factor(bad, torch.empty((n, n), dtype=torch.float64)) == chm.CHM_ERR_NOT_PD
    srv.close()
