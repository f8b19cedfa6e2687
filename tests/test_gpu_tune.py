"""The autotuner (chm_tune) on the GPU: it picks a configuration for a
shape, stores it in the tuning cache, the cached configuration decides the
path of every shape in the same (dtype, n bucket, k bucket), and the
modification it runs still matches the oracle."""
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
    assert chm.chm_tune_clear() == chm.CHM_OK
    yield
    chm.chm_tune_clear()


@pytest.mark.parametrize("n,k,dtype", [(2000, 3, chm.CHM_F64), (3000, 16, chm.CHM_F32_MIXED)])
def test_tune_picks_and_caches_a_configuration(n, k, dtype):
    r = chm.tune(n, k, dtype)
    print("tuned n=%d k=%d dtype=%d: %s" % (n, k, dtype, r))
    assert r["path"] in ("wave", "pass")
    assert 1 <= r["vectors_per_pass"] <= 16 and 2 <= r["lookahead"] <= 10 and r["segment_blocks"] >= 0
    assert 0 < r["ms"] <= r["default_ms"] * 1.0001   # the default is one of the candidates
    want = chm.PATH_PASS if r["path"] == "pass" else chm.PATH_WAVE
    assert chm.path_for(n, k, dtype) == want
    # another shape of the same bucket takes the cached configuration, and the result is right
    m, kk = n + n // 4, k - 1 if k > 2 else k
    assert chm.path_for(m, kk, dtype) == want
    if dtype == chm.CHM_F64:
        L = inputs.spd_factor(m, 61).numpy()
        V = inputs.update_block(m, kk, 61).numpy()
        ref = L.copy()
        assert oracle.modify_b(ref, V, 1)[0] == 0
        Ld = torch.as_tensor(L).cuda()
        assert chm.modify(Ld, torch.as_tensor(V).cuda(), 1) == chm.CHM_OK
        assert chm.status_sync()[0] == chm.CHM_OK
        assert colscaled_err(Ld.cpu().numpy(), ref) <= TOL_F64


def test_cache_file_written_by_the_tuner_reloads(tmp_path):
    chm.chm_tune_clear()
    r = chm.tune(1000, 2, chm.CHM_F64)
    f = tmp_path / "cache.txt"
    assert chm.chm_tune_save(str(f)) == chm.CHM_OK
    lines = f.read_text().splitlines()
    assert lines[0] == "chm-tune 1" and len(lines) == 2
    fields = [int(x) for x in lines[1].split()]
    assert fields[:3] == [chm.CHM_F64, 9, 1]
    assert fields[3] == (chm.PATH_PASS if r["path"] == "pass" else chm.PATH_WAVE)
    chm.chm_tune_clear()
    assert chm.chm_tune_load(str(f)) == chm.CHM_OK
    assert chm.path_for(1000, 2, chm.CHM_F64) == fields[3]
