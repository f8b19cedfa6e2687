"""GPU tests of the batch API (chm_batch_*): many independent factors in one
launch.  Each factor's result must match the CPU oracle within the float64
tolerance and be bit-identical to the same factor modified alone through
chm_modify_ex (the arithmetic of a factor does not depend on what else runs
in the launch)."""
from __future__ import annotations

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


# (n, k, sign, ld padding): ragged tails, single-block factors, a factor of
# order 1 and factors with padded leading dimension.
SPECS = [(1, 1, 1, 0), (31, 3, -1, 0), (33, 5, 1, 2), (64, 1, -1, 0), (100, 16, 1, 0), (257, 7, -1, 5),
         (300, 3, 1, 0), (129, 16, -1, 31), (45, 2, 1, 0), (512, 1, 1, 0), (96, 33, -1, 0), (200, 64, 1, 1)]


def make_factor(i, n, k, pad, dtype=torch.float64):
    seed = 7000 + 17 * i
    L = inputs.spd_factor(n, seed, ld=n + pad)
    # small enough that every downdate stays positive definite (A >= I)
    V = inputs.update_block(n, k, seed, scale=0.2 / np.sqrt(max(1, n * k)))
    return L.to(dtype), V.to(dtype)


def run_batch(specs, dtype=torch.float64, tune=False):
    Ls, Vs = [], []
    for i, (n, k, s, pad) in enumerate(specs):
        L, V = make_factor(i, n, k, pad, dtype)
        Ls.append(L.cuda().contiguous())
        Vs.append(V.cuda().contiguous())
    plan = chm.BatchPlan([n for n, _, _, _ in specs], [L.shape[1] for L in Ls], [k for _, k, _, _ in specs],
                         [s for _, _, s, _ in specs], chm.CHM_F64 if dtype == torch.float64 else chm.CHM_F32_MIXED)
    if tune:
        assert plan.autotune() == chm.CHM_OK
    L0 = [L.clone() for L in Ls]
    assert plan.execute(Ls, Vs) == chm.CHM_OK
    st, infos = plan.status()
    plan.close()
    return st, infos, L0, Ls, Vs


def test_batch_matches_oracle_and_solo_calls():
    st, infos, L0, Ls, Vs = run_batch(SPECS)
    assert st == chm.CHM_OK
    assert all(i == (0, -1) for i in infos)
    for (n, k, s, pad), l0, l, v in zip(SPECS, L0, Ls, Vs):
        # oracle
        ref = l0.cpu().numpy().copy()
        ost, _ = oracle.modify_b(ref, v.cpu().numpy(), s)
        assert ost == 0
        got = l.cpu().numpy()
        assert colscaled_err(got[:, :n], ref[:, :n]) <= TOL_F64, (n, k, s)
        # padding untouched
        assert np.array_equal(got[:, n:], l0.cpu().numpy()[:, n:])
        # the same factor alone
        solo = l0.clone()
        assert chm.modify(solo, v, s) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        assert torch.equal(solo, l), (n, k, s)


def test_batch_mixed_precision_matches_solo_calls():
    specs = SPECS[:8]
    st, infos, L0, Ls, Vs = run_batch(specs, dtype=torch.float32)
    assert st == chm.CHM_OK
    for (n, k, s, pad), l0, l, v in zip(specs, L0, Ls, Vs):
        solo = l0.clone()
        assert chm.modify(solo, v, s) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        assert torch.equal(solo, l), (n, k, s)


def test_batch_update_then_downdate_and_replay():
    specs = [(n, k, 1, pad) for n, k, _, pad in SPECS]
    Ls, Vs = [], []
    for i, (n, k, s, pad) in enumerate(specs):
        L, V = make_factor(i, n, k, pad)
        Ls.append(L.cuda().contiguous())
        Vs.append(V.cuda().contiguous())
    L0 = [L.clone() for L in Ls]
    ns, lds, ks = [n for n, _, _, _ in specs], [L.shape[1] for L in Ls], [k for _, k, _, _ in specs]
    up = chm.BatchPlan(ns, lds, ks, [1] * len(specs))
    down = chm.BatchPlan(ns, lds, ks, [-1] * len(specs))
    # several executions of each plan (graph replays, both staging buffers)
    for _ in range(3):
        assert up.execute(Ls, Vs) == chm.CHM_OK
        assert down.execute(Ls, Vs) == chm.CHM_OK
    assert up.status()[0] == chm.CHM_OK and down.status()[0] == chm.CHM_OK
    for (n, k, _, _), l0, l in zip(specs, L0, Ls):
        assert colscaled_err(l.cpu().numpy()[:, :n], l0.cpu().numpy()[:, :n]) <= 10 * TOL_F64, (n, k)
    up.close()
    down.close()


def test_batch_not_pd_is_reported_per_factor():
    n = 40
    specs = [(64, 2, 1, 0), (n, 1, -1, 0), (100, 3, -1, 0)]
    Ls, Vs = [], []
    for i, (nn, k, s, pad) in enumerate(specs):
        L, V = make_factor(i, nn, k, pad)
        Ls.append(L.cuda().contiguous())
        Vs.append(V.cuda().contiguous())
    # factor 1: L = I, v = 2 e_0, downdate -> 1 - 4 < 0 at row 0
    Ls[1] = torch.eye(n, dtype=torch.float64, device="cuda").contiguous()
    v = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    v[0, 0] = 2.0
    Vs[1] = v
    L0 = [L.clone() for L in Ls]
    plan = chm.BatchPlan([s[0] for s in specs], [L.shape[1] for L in Ls], [s[1] for s in specs],
                         [s[2] for s in specs])
    assert plan.execute(Ls, Vs) == chm.CHM_OK
    st, infos = plan.status()
    plan.close()
    assert st == chm.CHM_ERR_NOT_PD
    assert infos[1] == (chm.CHM_ERR_NOT_PD, 0)
    assert infos[0] == (0, -1) and infos[2] == (0, -1)
    for idx in (0, 2):
        nn, k, s, _ = specs[idx]
        ref = L0[idx].cpu().numpy().copy()
        oracle.modify_b(ref, Vs[idx].cpu().numpy(), s)
        assert colscaled_err(Ls[idx].cpu().numpy(), ref) <= TOL_F64


def test_batch_noop_entries_and_empty_plan():
    specs = [(0, 3, 1, 0), (50, 0, 1, 0), (70, 2, -1, 0)]
    Ls = [torch.zeros((0, 1), dtype=torch.float64, device="cuda"),
          inputs.spd_factor(50, 3).cuda(), make_factor(2, 70, 2, 0)[0].cuda()]
    Vs = [torch.zeros((3, 1), dtype=torch.float64, device="cuda"),
          torch.zeros((0, 50), dtype=torch.float64, device="cuda"), make_factor(2, 70, 2, 0)[1].cuda()]
    L0 = [L.clone() for L in Ls]
    plan = chm.BatchPlan([0, 50, 70], [1, 50, 70], [3, 0, 2], [1, 1, -1])
    assert plan.execute(Ls, Vs) == chm.CHM_OK
    st, infos = plan.status()
    plan.close()
    assert st == chm.CHM_OK and infos == [(0, -1)] * 3
    assert torch.equal(Ls[1], L0[1])
    ref = L0[2].cpu().numpy().copy()
    oracle.modify_b(ref, Vs[2].cpu().numpy(), -1)
    assert colscaled_err(Ls[2].cpu().numpy(), ref) <= TOL_F64
    empty = chm.BatchPlan([], [], [], None)
    assert empty.execute([], []) == chm.CHM_OK
    assert empty.status()[0] == chm.CHM_OK
    empty.close()


def test_batch_autotune_keeps_results():
    st, infos, L0, Ls, Vs = run_batch(SPECS[:6], tune=True)
    assert st == chm.CHM_OK
    for (n, k, s, pad), l0, l, v in zip(SPECS[:6], L0, Ls, Vs):
        solo = l0.clone()
        assert chm.modify(solo, v, s) == chm.CHM_OK
        assert torch.equal(solo, l)


def test_batch_rejects_bad_arguments():
    with pytest.raises(chm.ChmError):
        chm.BatchPlan([10], [5], [1])          # ld < n
    with pytest.raises(chm.ChmError):
        chm.BatchPlan([10], [10], [65])        # k above the per-factor limit
    with pytest.raises(chm.ChmError):
        chm.BatchPlan([10], [10], [1], [0])    # sign not +-1
    plan = chm.BatchPlan([10], [10], [1])
    assert plan.execute([None], [None]) == chm.CHM_ERR_ARG
    plan.close()


def test_batch_many_groups_many_factors_match_solo_calls():
    """Many factors under the default many-group configuration, several
    executions: every factor's final pass (the last wave's scales) must run
    in full before the launch ends."""
    rng = np.random.default_rng(77)
    count = 128
    ns = np.exp(rng.uniform(np.log(64), np.log(2048), count)).astype(int).tolist()
    ks = rng.choice([1, 4, 16], count).tolist()
    sg = rng.choice([1, -1], count).tolist()
    Ls = [inputs.random_factor(n, 500 + i, device="cuda") for i, n in enumerate(ns)]
    Vs = [inputs.update_block(n, k, 500 + i, device="cuda", scale=0.2 / np.sqrt(n * k))
          for i, (n, k) in enumerate(zip(ns, ks))]
    L0 = [L.clone() for L in Ls]
    fwd = chm.BatchPlan(ns, ns, ks, sg)
    inv = chm.BatchPlan(ns, ns, ks, [-s for s in sg])
    for r in range(3):
        assert fwd.execute(Ls, Vs) == chm.CHM_OK
        assert inv.execute(Ls, Vs) == chm.CHM_OK
    assert fwd.execute(Ls, Vs) == chm.CHM_OK
    assert fwd.status()[0] == chm.CHM_OK and inv.status()[0] == chm.CHM_OK
    fwd.close()
    inv.close()
    for i in range(count):
        solo = L0[i].clone()
        for r in range(3):
            assert chm.modify(solo, Vs[i], sg[i]) == chm.CHM_OK
            assert chm.modify(solo, Vs[i], -sg[i]) == chm.CHM_OK
        assert chm.modify(solo, Vs[i], sg[i]) == chm.CHM_OK
        assert torch.equal(solo, Ls[i]), (i, ns[i], ks[i])
    assert chm.status_sync()[0] == chm.CHM_OK
