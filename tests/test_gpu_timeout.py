"""Failure detection without a GPU fault: a launch in which one rotation
panel is never released (a flag that nothing sets, through the library's
test hook) must end by its bounded waits with CHM_ERR_TIMEOUT, and the next
launch in the same process must run normally and give the oracle's result.

Runs in a child process so that the short wait limit (CHM_TIMEOUT_NS) and
the one-shot hook (CHM_TEST_SKIP_PUBLISH) are read from its environment."""
from __future__ import annotations

import os
import subprocess
import sys
import textwrap

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys, time
    sys.path.insert(0, %r)
    import numpy as np, torch
    import oracle
    from paper_1011_1173_gb300 import chm, inputs
    from tests.common import TOL_F64, colscaled_err
    chm.load(build_if_missing=True)
    n, k = 512, 2
    L0 = inputs.spd_factor(n, 77)
    V = inputs.update_block(n, k, 77)
    # 1. panel of block 3 never released: the launch must end by timeout
    L = L0.cuda()
    t0 = time.time()
    d_info = torch.full((2,), 99, dtype=torch.int64, device="cuda")
    assert chm.modify(L, V.cuda(), 1, d_info=d_info) == chm.CHM_OK
    st, info = chm.status_sync()
    dt = time.time() - t0
    print("timeout run: status", st, "info", info, "seconds %%.3f" %% dt, "per-call", d_info.tolist())
    assert st == chm.CHM_ERR_TIMEOUT, st
    assert int(d_info[0]) == chm.CHM_ERR_TIMEOUT   # the call's own word says so too
    assert dt < 30.0
    # 2. the next launch is normal and correct
    L = L0.cuda()
    assert chm.modify(L, V.cuda(), 1) == chm.CHM_OK
    st, info = chm.status_sync()
    assert st == chm.CHM_OK, (st, info)
    ref = L0.numpy().copy()
    assert oracle.modify_b(ref, V.numpy(), 1)[0] == 0
    err = colscaled_err(L.cpu().numpy(), ref)
    print("recovery run: error %%.3e" %% err)
    assert err <= TOL_F64
    print("OK")
""" % ROOT)


def test_unreleased_panel_times_out_and_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ)
    env["CHM_TIMEOUT_NS"] = str(200_000_000)  # 0.2 s per wait
    env["CHM_TEST_SKIP_PUBLISH"] = "3"
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    sys.stdout.write(r.stdout)
    sys.stderr.write(r.stderr[-2000:])
    assert r.returncode == 0
    assert "OK" in r.stdout
