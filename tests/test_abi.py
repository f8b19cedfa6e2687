"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

from paper_1011_1173_gb300 import build as chm_build
from paper_1011_1173_gb300 import chm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_ \*]*?)\b(chm_[A-Za-z0-9_]+)\s*\(", text):
            names.append(m.group(2))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    chm_build.build()
    return ctypes.CDLL(chm_build.LIB)


def test_header_declares_core_calls():
    names = declared_functions()
    for required in ("chm_update", "chm_downdate", "chm_modify_ex", "chm_status_sync"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    for n in declared_functions():
        assert hasattr(chm, n), "binding lacks %s" % n


def test_host_only_calls_without_gpu():
    assert chm.chm_version() >= 100
    assert "NOT_PD" in chm.chm_status_string(chm.CHM_ERR_NOT_PD)


def test_argument_errors_return_synchronously_without_gpu():
    E = chm.CHM_ERR_ARG
    assert chm.chm_update(None, -1, 1, None, 1, chm.CHM_F64, None) == E
    assert chm.chm_update(None, 4, 3, None, 1, chm.CHM_F64, None) == E       # ld < n
    assert chm.chm_update(None, 4, 4, None, 1, 7, None) == E                 # bad dtype
    assert chm.chm_update(None, 4, 4, None, 1, chm.CHM_F64, None) == E       # NULL L
    assert chm.chm_modify_ex(8, 4, 4, 8, 4, 1, None, 0, chm.CHM_F64, None, None) == E  # sign 0
    assert chm.chm_update(12, 4, 4, 16, 1, chm.CHM_F64, None) == E           # misaligned L
    # n == 0 or k == 0 with no per-call info word: nothing to do, no CUDA call
    assert chm.chm_update(None, 0, 1, None, 3, chm.CHM_F64, None) == chm.CHM_OK
    assert chm.chm_update(8, 5, 5, None, 0, chm.CHM_F64, None) == chm.CHM_OK


def test_batch_argument_errors_without_gpu():
    E = chm.CHM_ERR_ARG
    i64 = ctypes.c_int64
    plan = ctypes.c_void_p()
    n, ld, k = (i64 * 2)(10, 20), (i64 * 2)(10, 19), (i64 * 2)(1, 2)       # ld[1] < n[1]
    vp = lambda a: ctypes.cast(a, ctypes.c_void_p)
    assert chm.chm_batch_plan_create(2, vp(n), vp(ld), vp(k), None, chm.CHM_F64, ctypes.byref(plan)) == E
    ld2, k2 = (i64 * 2)(10, 20), (i64 * 2)(1, 65)                            # k above 64
    assert chm.chm_batch_plan_create(2, vp(n), vp(ld2), vp(k2), None, chm.CHM_F64, ctypes.byref(plan)) == E
    sig = (ctypes.c_int8 * 2)(1, 0)                                          # sign not +-1
    assert chm.chm_batch_plan_create(2, vp(n), vp(ld2), vp(k), vp(sig), chm.CHM_F64, ctypes.byref(plan)) == E
    assert chm.chm_batch_plan_create(-1, None, None, None, None, chm.CHM_F64, ctypes.byref(plan)) == E
    assert chm.chm_batch_plan_create(1, vp(n), vp(ld2), vp(k), None, 9, ctypes.byref(plan)) == E  # dtype
    assert chm.chm_batch_plan_create(1, vp(n), vp(ld2), vp(k), None, chm.CHM_F64, None) == E      # no out
    assert not plan.value
    assert chm.chm_batch_execute(None, None, None, None) == E
    assert chm.chm_batch_status(None, None) == E
    assert chm.chm_batch_plan_destroy(None) == E


def test_server_argument_errors_without_gpu():
    E = chm.CHM_ERR_ARG
    srv = ctypes.c_void_p()
    assert chm.chm_server_create(1 << 30, 9, 2, ctypes.byref(srv)) == E   # bad dtype
    assert chm.chm_server_create(1 << 30, chm.CHM_F64, 2, None) == E        # no out
    assert not srv.value
    assert chm.chm_server_add_factor(None, None, 4, 4, None) == E
    assert chm.chm_server_submit(None, 0, None, 1, 1, None) == E
    got = ctypes.c_int()
    assert chm.chm_server_poll(None, None, None, None, 0, ctypes.byref(got)) == E
    assert chm.chm_server_drain(None, 1.0) == E
    assert chm.chm_server_get_factor(None, 0, None, 1) == E
    assert chm.chm_server_stats(None, None) == E
    assert chm.chm_server_destroy(None) == E


def test_workspace_bytes_grow_as_n_times_k():
    """Host-only sizing: the device workspace of a single-factor modification
    is O(n min(k, 64)), far below the n^2 factor (so a factor kept in host
    memory needs only this much device memory)."""
    ws = chm.workspace_bytes
    n = 1 << 16
    chm.config_set("path", chm.PATH_WAVE)
    try:
        assert ws(0, 5) == 0 and ws(n, 0) == 0
        assert 1.95 <= ws(2 * n, 8) / ws(n, 8) <= 2.05
        assert 1.9 <= ws(n, 16) / ws(n, 8) <= 2.05
        assert ws(n, 100) == ws(n, 64)
        assert ws(n, 16) < 8 * n * n / 40
        assert ws(n, 16, chm.CHM_F32_MIXED) == ws(n, 16)
        for bad in ((-1, 1), (1, -1), (1 << 27, 1)):
            with pytest.raises(chm.ChmError):
                ws(*bad)
        with pytest.raises(chm.ChmError):
            ws(10, 1, 9)
    finally:
        chm.config_set("path", chm.PATH_AUTO)


def test_pass_workspace_is_linear_in_n_and_independent_of_k():
    """The pass kernels' workspace is sized for one pass of up to 16
    vectors: O(n), the same for every k."""
    ws = chm.workspace_bytes
    n = 1 << 15
    chm.config_set("path", chm.PATH_PASS)
    try:
        assert ws(n, 1) == ws(n, 16) == ws(n, 100)
        assert 1.95 <= ws(2 * n, 8) / ws(n, 8) <= 2.05
        assert ws(n, 16) < 8 * n * n / 40
        assert ws(n, 4, chm.CHM_F32_MIXED) < ws(n, 4)
        assert ws(0, 3) == 0
    finally:
        chm.config_set("path", chm.PATH_AUTO)


def test_path_settings_and_automatic_rule():
    """Host-only: the settings interface and the size rule that picks the
    pass kernels (float: upper triangle >= 32 MB; double: >= 256 MB and k <= 8)
    and the default vectors per pass (8 in float, 4 in double)."""
    F32, F64 = chm.CHM_F32_MIXED, chm.CHM_F64
    assert chm.config_get("path") == chm.PATH_AUTO
    assert chm.path_for(2048, 4, F32) == chm.PATH_WAVE
    assert chm.path_for(4096, 4, F32) == chm.PATH_PASS
    assert chm.path_for(32768, 64, F32) == chm.PATH_PASS
    assert chm.path_for(5000, 16, F64) == chm.PATH_WAVE
    assert chm.path_for(8192, 1, F64) == chm.PATH_PASS
    assert chm.path_for(32768, 8, F64) == chm.PATH_PASS
    assert chm.path_for(32768, 9, F64) == chm.PATH_WAVE
    for p in (chm.PATH_WAVE, chm.PATH_PASS):
        chm.config_set("path", p)
        assert chm.path_for(100, 1, F64) == p and chm.path_for(40000, 1, F32) == p
    chm.config_set("path", chm.PATH_AUTO)
    chm.config_set("pass_kb", 5)
    assert chm.config_get("pass_kb") == 5
    assert chm.config_get("pass_kb_f32") == 5 and chm.config_get("pass_kb_f64") == 5
    chm.config_set("pass_kb", 0)
    assert chm.config_get("pass_kb") == 0
    assert chm.config_get("pass_kb_f32") == 8 and chm.config_get("pass_kb_f64") == 4
    chm.config_set("pass_d", 9)
    assert chm.config_get("pass_d_f32") == 9 and chm.config_get("pass_d_f64") == 6
    chm.config_set("pass_d", 0)
    assert chm.config_get("pass_d_f32") == 10 and chm.config_get("pass_d_f64") == 3
    for key, val in (("path", 3), ("pass_kb", 17), ("pass_kb", -1), ("nope", 1)):
        assert chm.chm_config_set(key, val) == chm.CHM_ERR_ARG


def test_solve_argument_errors_without_gpu():
    E = chm.CHM_ERR_ARG
    assert chm.chm_solve(8, -1, 1, 8, 1, 1, chm.CHM_F64, None) == E          # n < 0
    assert chm.chm_solve(8, 4, 3, 8, 4, 1, chm.CHM_F64, None) == E           # ld < n
    assert chm.chm_solve(8, 4, 4, 8, 3, 1, chm.CHM_F64, None) == E           # ldb < n
    assert chm.chm_solve(8, 4, 4, 8, 4, -1, chm.CHM_F64, None) == E          # nrhs < 0
    assert chm.chm_solve(8, 4, 4, 8, 4, 1, 5, None) == E                     # dtype
    assert chm.chm_solve(None, 4, 4, 8, 4, 1, chm.CHM_F64, None) == E        # NULL L
    assert chm.chm_solve(8, 4, 4, None, 4, 1, chm.CHM_F64, None) == E        # NULL B
    assert chm.chm_solve(12, 4, 4, 8, 4, 1, chm.CHM_F64, None) == E          # misaligned L
    assert chm.chm_solve(8, 4, 4, 6, 4, 1, chm.CHM_F32_MIXED, None) == E     # misaligned B
    # nothing to do: no CUDA call
    assert chm.chm_solve(None, 0, 1, None, 1, 3, chm.CHM_F64, None) == chm.CHM_OK
    assert chm.chm_solve(8, 5, 5, None, 5, 0, chm.CHM_F64, None) == chm.CHM_OK


def test_modify_solve_argument_errors_without_gpu():
    E = chm.CHM_ERR_ARG
    F64 = chm.CHM_F64
    ms = chm.chm_modify_solve
    # (L, n, ld, V, ldv, k, sigma, sign, B, ldb, nrhs, dtype, stream, d_info)
    assert ms(8, -1, 1, 8, 1, 1, None, 1, 8, 1, 1, F64, None, None) == E      # n < 0
    assert ms(8, 4, 3, 8, 4, 1, None, 1, 8, 4, 1, F64, None, None) == E       # ld < n
    assert ms(8, 4, 4, 8, 4, 1, None, 0, 8, 4, 1, F64, None, None) == E       # sign 0
    assert ms(8, 4, 4, 8, 4, 1, None, 1, 8, 3, 1, F64, None, None) == E       # ldb < n
    assert ms(8, 4, 4, 8, 4, 1, None, 1, 8, 4, -1, F64, None, None) == E      # nrhs < 0
    assert ms(8, 4, 4, 8, 4, 1, None, 1, None, 4, 1, F64, None, None) == E    # NULL B
    assert ms(8, 4, 4, 8, 4, 1, None, 1, 12, 4, 1, F64, None, None) == E      # misaligned B
    assert ms(8, 4, 4, 8, 4, 1, None, 1, 8, 4, 1, 3, None, None) == E         # dtype
    # nothing to do: no CUDA call
    assert ms(None, 0, 1, None, 1, 2, None, 1, None, 1, 2, F64, None, None) == chm.CHM_OK
    assert ms(8, 5, 5, None, 5, 0, None, 1, 8, 5, 0, F64, None, None) == chm.CHM_OK


def test_checked_build_exports_the_same_symbols_and_reports_itself():
    """The bounds-checked variant (-DCHM_CHECK) is built beside the library,
    exports every declared symbol, and answers the "checked" and
    "check_cut" settings that only it accepts."""
    chm_build.build()
    plain = ctypes.CDLL(chm_build.LIB)
    missing = [n for n in declared_functions() if not hasattr(ctypes.CDLL(chm_build.LIB_CHECK), n)]
    assert not missing, missing
    v = ctypes.c_int64(-1)
    plain.chm_config_get.argtypes = [ctypes.c_char_p, ctypes.c_void_p]
    plain.chm_config_set.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    assert plain.chm_config_get(b"checked", ctypes.byref(v)) == 0 and v.value == 0
    assert plain.chm_config_set(b"check_cut", 1) == chm.CHM_ERR_ARG
    with chm.checked_library(build_if_missing=False):
        assert chm.config_get("checked") == 1
        assert chm.chm_config_set(b"check_cut", -1) == chm.CHM_ERR_ARG
        assert chm.chm_config_set(b"check_cut", 2) == chm.CHM_OK
        assert chm.config_get("check_cut") == 2
        assert chm.chm_config_set(b"check_cut", 0) == chm.CHM_OK
        assert "BOUNDS" in chm.chm_status_string(chm.CHM_ERR_BOUNDS)
    assert chm.config_get("checked") == 0


def test_tuning_cache_file_round_trip_and_lookup(tmp_path):
    """chm_tune_load / chm_tune_save / chm_tune_clear without a GPU: a loaded
    entry decides the path of its (dtype, floor(log2 n), ceil(log2 k))
    bucket, an explicit "path" setting still wins, a malformed file changes
    nothing, and a saved cache reads back to the same entries."""
    assert chm.chm_tune_clear() == chm.CHM_OK
    # float32 n in [2048, 4096), k in (4, 8]: the built-in rule takes the wave kernel (8 MB < 32 MB)
    assert chm.path_for(3000, 6, chm.CHM_F32_MIXED) == chm.PATH_WAVE
    f = tmp_path / "tune.txt"
    f.write_text("chm-tune 1\n%d 11 3 2 4 6 32 123456\n" % chm.CHM_F32_MIXED)
    assert chm.chm_tune_load(str(f)) == chm.CHM_OK
    assert chm.path_for(3000, 6, chm.CHM_F32_MIXED) == chm.PATH_PASS
    assert chm.path_for(2048, 5, chm.CHM_F32_MIXED) == chm.PATH_PASS
    assert chm.path_for(2047, 6, chm.CHM_F32_MIXED) == chm.PATH_WAVE   # the n bucket below
    assert chm.path_for(3000, 9, chm.CHM_F32_MIXED) == chm.PATH_WAVE   # next k bucket
    assert chm.path_for(3000, 6, chm.CHM_F64) == chm.PATH_WAVE         # other dtype
    chm.config_set("path", chm.PATH_WAVE)
    try:
        assert chm.path_for(3000, 6, chm.CHM_F32_MIXED) == chm.PATH_WAVE
    finally:
        chm.config_set("path", chm.PATH_AUTO)
    out = tmp_path / "saved.txt"
    assert chm.chm_tune_save(str(out)) == chm.CHM_OK
    assert out.read_text() == "chm-tune 1\n%d 11 3 2 4 6 32 123456\n" % chm.CHM_F32_MIXED
    for bad in ("chm-tune 2\n", "chm-tune 1\n1 11 3 2 4 6 32\n", "chm-tune 1\n1 11 3 3 4 6 32 1\n",
                "chm-tune 1\n1 11 3 2 17 6 32 1\n", "chm-tune 1\n7 11 3 2 4 6 32 1\n"):
        f.write_text(bad)
        assert chm.chm_tune_load(str(f)) == chm.CHM_ERR_ARG, bad
    assert chm.path_for(3000, 6, chm.CHM_F32_MIXED) == chm.PATH_PASS   # unchanged
    assert chm.chm_tune_load(str(tmp_path / "missing.txt")) == chm.CHM_ERR_ARG
    assert chm.chm_tune(0, 1, chm.CHM_F64, None) == chm.CHM_ERR_ARG
    assert chm.chm_tune(10, 0, chm.CHM_F64, None) == chm.CHM_ERR_ARG
    assert chm.chm_tune(10, 1, 5, None) == chm.CHM_ERR_ARG
    assert chm.chm_tune_clear() == chm.CHM_OK
    assert chm.path_for(3000, 6, chm.CHM_F32_MIXED) == chm.PATH_WAVE


def test_fused_pass_setting():
    assert chm.config_get("pass_fused") == 1
    assert chm.chm_config_set(b"pass_fused", 2) == chm.CHM_ERR_ARG
    chm.config_set("pass_fused", 0)
    try:
        assert chm.config_get("pass_fused") == 0
    finally:
        chm.config_set("pass_fused", 1)
