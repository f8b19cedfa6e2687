"""Python binding of the C ABI in ``include/chm.h`` (argument marshalling only).

Every function here forwards to the CUDA library ``libchm.so``; none of them
computes anything.  The library is loaded on first use and there is no
fallback: if it has not been built, or cannot be loaded, the call raises.

Tensor helpers take torch tensors in the storage convention of the C ABI:
an order-n upper factor is a C-contiguous (n, ld) tensor whose row j is
column j of L, and V is a C-contiguous (k, ldv) tensor whose row p is column
p of V (see ``inputs.py``).
"""
from __future__ import annotations

import contextlib
import ctypes
import os

import torch

from . import build as _build

CHM_F64 = 0
CHM_F32_MIXED = 1

CHM_OK = 0
CHM_ERR_ARG = -1
CHM_ERR_NOT_PD = -2
CHM_ERR_TIMEOUT = -3
CHM_ERR_CUDA = -4
CHM_ERR_NOMEM = -5
CHM_ERR_BUDGET = -6
CHM_ERR_STATE = -7
CHM_ERR_BOUNDS = -8

_lib = None
_lib_checked = None
_use_checked = False


class ChmError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s%s" % (what + ": " if what else "", chm_status_string(status)))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libchm.so (optionally building it first).  Raises if unavailable.
    Inside ``with checked_library():`` this is the bounds-checked build."""
    global _lib, _lib_checked
    if _use_checked:
        if _lib_checked is None:
            _lib_checked = _open(_build.LIB_CHECK, build_if_missing)
        return _lib_checked
    if _lib is None:
        _lib = _open(_build.LIB, build_if_missing)
    return _lib


@contextlib.contextmanager
def checked_library(build_if_missing: bool = True):
    """Route every call of this module made inside the block to
    libchm_check.so, the library built with -DCHM_CHECK (every global index
    of the kernels checked; an index outside the arguments' arrays reports
    CHM_ERR_BOUNDS instead of being accessed)."""
    global _use_checked
    prev = _use_checked
    _use_checked = True
    try:
        load(build_if_missing)
        yield _lib_checked
    finally:
        _use_checked = prev


def _open(path, build_if_missing):
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("%s is not built (run paper_1011_1173_gb300.build.build())" % os.path.basename(path))
        _build.build()
    lib = ctypes.CDLL(path)
    i64, vp, i32 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    sig = {
        "chm_update": ([vp, i64, i64, vp, i64, i32, vp], i32),
        "chm_downdate": ([vp, i64, i64, vp, i64, i32, vp], i32),
        "chm_modify_ex": ([vp, i64, i64, vp, i64, i64, vp, i32, i32, vp, vp], i32),
        "chm_modify_noalloc": ([vp, i64, i64, vp, i64, i64, vp, i32, i32, vp, vp], i32),
        "chm_modify_solve": ([vp, i64, i64, vp, i64, i64, vp, i32, vp, i64, i64, i32, vp, vp], i32),
        "chm_status_sync": ([vp, vp], i32),
        "chm_status_string": ([i32], ctypes.c_char_p),
        "chm_version": ([], i32),
        "chm_trace_dump": ([ctypes.c_char_p], i32),
        "chm_batch_plan_create": ([i32, vp, vp, vp, vp, i32, vp], i32),
        "chm_batch_autotune": ([vp, vp], i32),
        "chm_batch_config": ([vp, vp, vp, vp], i32),
        "chm_batch_execute": ([vp, vp, vp, vp], i32),
        "chm_batch_status": ([vp, vp], i32),
        "chm_batch_plan_destroy": ([vp], i32),
        "chm_server_create": ([ctypes.c_size_t, i32, i32, vp], i32),
        "chm_server_add_factor": ([vp, vp, i64, i64, vp], i32),
        "chm_server_submit": ([vp, i64, vp, i64, i32, vp], i32),
        "chm_server_poll": ([vp, vp, vp, vp, i32, vp], i32),
        "chm_server_drain": ([vp, ctypes.c_double], i32),
        "chm_server_get_factor": ([vp, i64, vp, i64], i32),
        "chm_server_stats": ([vp, vp], i32),
        "chm_server_destroy": ([vp], i32),
        "chm_microbench": ([i32, vp, i32], i32),
        "chm_selftest_reciprocals": ([vp, i64, vp], i32),
        "chm_config_set": ([ctypes.c_char_p, i64], i32),
        "chm_config_get": ([ctypes.c_char_p, vp], i32),
        "chm_path_for": ([i64, i64, i32, vp], i32),
        "chm_workspace_bytes": ([i64, i64, i32, vp], i32),
        "chm_solve": ([vp, i64, i64, vp, i64, i64, i32, vp], i32),
        "chm_tune": ([i64, i64, i32, vp], i32),
        "chm_tune_clear": ([], i32),
        "chm_tune_save": ([ctypes.c_char_p], i32),
        "chm_tune_load": ([ctypes.c_char_p], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- raw C ABI

def chm_update(L, n, ld, V, k, dtype, stream):
    return load().chm_update(L, n, ld, V, k, dtype, stream)


def chm_downdate(L, n, ld, V, k, dtype, stream):
    return load().chm_downdate(L, n, ld, V, k, dtype, stream)


def chm_modify_ex(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info):
    return load().chm_modify_ex(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info)


def chm_modify_noalloc(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info):
    return load().chm_modify_noalloc(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info)


def chm_status_sync(stream, info):
    return load().chm_status_sync(stream, info)


def chm_status_string(status) -> str:
    return load().chm_status_string(int(status)).decode()


def chm_version() -> int:
    return load().chm_version()


def chm_trace_dump(path) -> int:
    return load().chm_trace_dump(path.encode() if isinstance(path, str) else path)


def chm_batch_plan_create(count, n, ld, k, sigma, dtype, plan_out):
    return load().chm_batch_plan_create(count, n, ld, k, sigma, dtype, plan_out)


def chm_batch_autotune(plan, stream):
    return load().chm_batch_autotune(plan, stream)


def chm_batch_config(plan, groups, ctas, largest_first):
    return load().chm_batch_config(plan, groups, ctas, largest_first)


def chm_batch_execute(plan, L, V, stream):
    return load().chm_batch_execute(plan, L, V, stream)


def chm_batch_status(plan, info):
    return load().chm_batch_status(plan, info)


def chm_batch_plan_destroy(plan):
    return load().chm_batch_plan_destroy(plan)


def chm_server_create(budget, dtype, max_inflight, srv_out):
    return load().chm_server_create(budget, dtype, max_inflight, srv_out)


def chm_server_add_factor(srv, L, n, ld, fid_out):
    return load().chm_server_add_factor(srv, L, n, ld, fid_out)


def chm_server_submit(srv, fid, V, k, sigma, req_out):
    return load().chm_server_submit(srv, fid, V, k, sigma, req_out)


def chm_server_poll(srv, ids, status, latency, max_count, got):
    return load().chm_server_poll(srv, ids, status, latency, max_count, got)


def chm_server_drain(srv, timeout_s):
    return load().chm_server_drain(srv, timeout_s)


def chm_server_get_factor(srv, fid, out, ld):
    return load().chm_server_get_factor(srv, fid, out, ld)


def chm_server_stats(srv, out):
    return load().chm_server_stats(srv, out)


def chm_server_destroy(srv):
    return load().chm_server_destroy(srv)


def chm_microbench(which, out, nout):
    return load().chm_microbench(which, out, nout)


def chm_config_set(key, value):
    return load().chm_config_set(key.encode() if isinstance(key, str) else key, int(value))


def chm_config_get(key, value):
    return load().chm_config_get(key.encode() if isinstance(key, str) else key, value)


def chm_path_for(n, k, dtype, path):
    return load().chm_path_for(n, k, dtype, path)


PATH_AUTO, PATH_WAVE, PATH_PASS = 0, 1, 2


def config_set(key, value):
    check(chm_config_set(key, value), "chm_config_set(%s)" % key)


def config_get(key) -> int:
    v = ctypes.c_int64()
    check(chm_config_get(key, ctypes.byref(v)), "chm_config_get(%s)" % key)
    return int(v.value)


def path_for(n, k, dtype=CHM_F64) -> int:
    p = ctypes.c_int()
    check(chm_path_for(int(n), int(k), int(dtype), ctypes.byref(p)), "chm_path_for")
    return int(p.value)


def chm_selftest_reciprocals(x, count, out):
    return load().chm_selftest_reciprocals(x, count, out)


def chm_tune(n, k, dtype, result):
    return load().chm_tune(n, k, dtype, result)


def chm_tune_clear():
    return load().chm_tune_clear()


def chm_tune_save(path):
    return load().chm_tune_save(path.encode() if isinstance(path, str) else path)


def chm_tune_load(path):
    return load().chm_tune_load(path.encode() if isinstance(path, str) else path)


def tune(n, k, dtype=CHM_F64) -> dict:
    """Autotune single-factor modifications of this shape (chm_tune); the
    choice enters the library's tuning cache.  Returns the chosen
    configuration and the tuned and default times per modification (ms)."""
    r = (ctypes.c_int64 * 6)()
    check(chm_tune(int(n), int(k), int(dtype), ctypes.cast(r, ctypes.c_void_p)), "chm_tune")
    return {"path": "pass" if r[0] == PATH_PASS else "wave", "vectors_per_pass": int(r[1]), "lookahead": int(r[2]),
            "segment_blocks": int(r[3]), "ms": r[4] / 1e6, "default_ms": r[5] / 1e6}


def chm_solve(L, n, ld, B, ldb, nrhs, dtype, stream):
    return load().chm_solve(L, n, ld, B, ldb, nrhs, dtype, stream)


def chm_modify_solve(L, n, ld, V, ldv, k, sigma, sign, B, ldb, nrhs, dtype, stream, d_info):
    return load().chm_modify_solve(L, n, ld, V, ldv, k, sigma, sign, B, ldb, nrhs, dtype, stream, d_info)


def chm_workspace_bytes(n, k, dtype, out):
    return load().chm_workspace_bytes(n, k, dtype, out)


def workspace_bytes(n, k, dtype=CHM_F64) -> int:
    """Device bytes a single-factor modification of order n by k vectors holds."""
    out = ctypes.c_size_t()
    check(chm_workspace_bytes(int(n), int(k), int(dtype), ctypes.byref(out)), "chm_workspace_bytes")
    return int(out.value)


MICROBENCH = {"fp64_rate": 0, "fp32_rate": 1, "fp64_warp": 2, "shfl_split": 3, "hbm_copy": 4,
              "flag_round_trip": 5, "fp64_lanes": 6}


def microbench(name):
    """Run one microbenchmark (chm_microbench); returns its two numbers."""
    out = (ctypes.c_double * 2)()
    check(chm_microbench(MICROBENCH[name], ctypes.cast(out, ctypes.c_void_p), 2), "chm_microbench")
    return float(out[0]), float(out[1])


# ---------------------------------------------------------------- tensor helpers

def dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return CHM_F64
    if t.dtype == torch.float32:
        return CHM_F32_MIXED
    raise TypeError("L and V must be float64 or float32")


def _check_layout(L: torch.Tensor, V: torch.Tensor, n):
    if not all(t.is_cuda or t.is_pinned() for t in (L, V)):
        raise ValueError("L and V must be CUDA tensors or page-locked host tensors")
    if L.dtype != V.dtype:
        raise TypeError("L and V must have the same dtype")
    if L.dim() != 2 or V.dim() != 2 or not L.is_contiguous() or not V.is_contiguous():
        raise ValueError("L must be a contiguous (n, ld) tensor and V a contiguous (k, ldv) tensor")
    n = L.shape[0] if n is None else int(n)
    return n


def modify(L: torch.Tensor, V: torch.Tensor, sigma=1, n=None, stream=None, d_info=None) -> int:
    """Enqueue L <- modified factor (chm_modify_ex); returns the call's status.

    ``sigma`` is +1, -1, or a sequence of k signs."""
    n = _check_layout(L, V, n)
    k = V.shape[0]
    if isinstance(sigma, int):
        sig_ptr, sign = None, int(sigma)
        keep = None
    else:
        keep = (ctypes.c_int8 * k)(*[int(s) for s in sigma])
        sig_ptr, sign = ctypes.cast(keep, ctypes.c_void_p), 1
    info_ptr = None if d_info is None else d_info.data_ptr()
    return chm_modify_ex(L.data_ptr(), n, L.shape[1], V.data_ptr(), V.shape[1], k, sig_ptr, sign,
                         dtype_code(L), _stream_handle(stream), info_ptr)


def update(L, V, n=None, stream=None) -> int:
    n = _check_layout(L, V, n)
    if V.shape[1] != n:
        return modify(L, V, 1, n=n, stream=stream)
    return chm_update(L.data_ptr(), n, L.shape[1], V.data_ptr(), V.shape[0], dtype_code(L),
                      _stream_handle(stream))


def downdate(L, V, n=None, stream=None) -> int:
    n = _check_layout(L, V, n)
    if V.shape[1] != n:
        return modify(L, V, -1, n=n, stream=stream)
    return chm_downdate(L.data_ptr(), n, L.shape[1], V.data_ptr(), V.shape[0], dtype_code(L),
                        _stream_handle(stream))


def solve(L: torch.Tensor, B: torch.Tensor, n=None, stream=None) -> int:
    """Enqueue B <- (L^T L)^{-1} B (chm_solve); returns the call's status.

    ``L`` is the (n, ld) factor storage and ``B`` a contiguous (nrhs, ldb)
    tensor whose row r is right-hand side r."""
    n = _check_layout(L, B, n)
    return chm_solve(L.data_ptr(), n, L.shape[1], B.data_ptr(), B.shape[1], B.shape[0], dtype_code(L),
                     _stream_handle(stream))


def modify_solve(L: torch.Tensor, V: torch.Tensor, B: torch.Tensor, sigma=1, n=None, stream=None,
                 d_info=None) -> int:
    """Enqueue L <- modified factor and B <- (L~^T L~)^{-1} B
    (chm_modify_solve); returns the call's status.

    ``V`` and ``B`` are contiguous (k, ldv) and (nrhs, ldb) tensors (row r =
    vector or right-hand side r); ``sigma`` is +1, -1, or k signs."""
    n = _check_layout(L, V, n)
    _check_layout(L, B, n)
    k = V.shape[0]
    if isinstance(sigma, int):
        sig_ptr, sign = None, int(sigma)
        keep = None
    else:
        keep = (ctypes.c_int8 * k)(*[int(s) for s in sigma])
        sig_ptr, sign = ctypes.cast(keep, ctypes.c_void_p), 1
    info_ptr = None if d_info is None else d_info.data_ptr()
    return chm_modify_solve(L.data_ptr(), n, L.shape[1], V.data_ptr(), V.shape[1], k, sig_ptr, sign,
                            B.data_ptr(), B.shape[1], B.shape[0], dtype_code(L), _stream_handle(stream), info_ptr)


def status_sync(stream=None):
    """Synchronise the stream and return (status, info) of its status word."""
    info = (ctypes.c_int64 * 2)()
    st = chm_status_sync(_stream_handle(stream), ctypes.cast(info, ctypes.c_void_p))
    return st, int(info[1])


def check(status, what=""):
    if status != CHM_OK:
        raise ChmError(status, what)


class BatchPlan:
    """A batch plan (chm_batch_*): shapes fixed at creation, factors given per execution.

    ``ns``, ``lds``, ``ks``: per-factor order, leading dimension and vector
    count; ``signs``: per-factor +1/-1 (or None for all updates)."""

    def __init__(self, ns, lds, ks, signs=None, dtype=CHM_F64):
        self.count = len(ns)
        arr = ctypes.c_int64 * max(1, self.count)
        self._n = arr(*[int(x) for x in ns])
        self._ld = arr(*[int(x) for x in lds])
        self._k = arr(*[int(x) for x in ks])
        self._sig = None if signs is None else (ctypes.c_int8 * max(1, self.count))(*[int(s) for s in signs])
        h = ctypes.c_void_p()
        st = chm_batch_plan_create(self.count, ctypes.cast(self._n, ctypes.c_void_p),
                                   ctypes.cast(self._ld, ctypes.c_void_p), ctypes.cast(self._k, ctypes.c_void_p),
                                   None if self._sig is None else ctypes.cast(self._sig, ctypes.c_void_p),
                                   int(dtype), ctypes.byref(h))
        check(st, "chm_batch_plan_create")
        self.handle = h

    def autotune(self, stream=None) -> int:
        return chm_batch_autotune(self.handle, _stream_handle(stream))

    def config(self):
        g, c, l = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(chm_batch_config(self.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(l)))
        return g.value, c.value, l.value

    def execute(self, Ls, Vs, stream=None) -> int:
        """Ls, Vs: sequences of CUDA tensors (or raw device addresses) in factor order."""
        ptr = ctypes.c_void_p * max(1, self.count)
        addr = lambda t: t if isinstance(t, int) else (0 if t is None else t.data_ptr())
        self._Lp = ptr(*[addr(t) for t in Ls])
        self._Vp = ptr(*[addr(t) for t in Vs])
        return chm_batch_execute(self.handle, ctypes.cast(self._Lp, ctypes.c_void_p),
                                 ctypes.cast(self._Vp, ctypes.c_void_p), _stream_handle(stream))

    def status(self):
        """(first non-OK status, [(status, row)] per factor)."""
        info = (ctypes.c_int64 * max(2, 2 * self.count))()
        st = chm_batch_status(self.handle, ctypes.cast(info, ctypes.c_void_p))
        return st, [(int(info[2 * i]), int(info[2 * i + 1])) for i in range(self.count)]

    def close(self):
        if getattr(self, "handle", None):
            chm_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop (chm_server_*): resident factors, queued requests, continuous batching."""

    def __init__(self, budget_bytes, dtype=CHM_F64, max_inflight=2):
        h = ctypes.c_void_p()
        check(chm_server_create(int(budget_bytes), int(dtype), int(max_inflight), ctypes.byref(h)),
              "chm_server_create")
        self.handle = h
        self.dtype = dtype

    def add_factor(self, L: torch.Tensor, n=None) -> int:
        """L: (n, ld) tensor in the C-ABI storage convention (host or device)."""
        n = L.shape[0] if n is None else int(n)
        fid = ctypes.c_int64()
        st = chm_server_add_factor(self.handle, L.data_ptr(), n, L.shape[1], ctypes.byref(fid))
        if st != CHM_OK:
            raise ChmError(st, "chm_server_add_factor")
        return fid.value

    def submit(self, fid, V: torch.Tensor, sigma=1) -> int:
        """V: contiguous (k, n) tensor (host or device).  Returns the request id or raises.

        The server copies V on its own stream before returning, so a device V
        is first made complete on the current stream (the one that wrote it)."""
        if V.is_cuda:
            torch.cuda.current_stream(V.device).synchronize()
        rid = ctypes.c_int64()
        st = chm_server_submit(self.handle, int(fid), V.data_ptr(), V.shape[0], int(sigma), ctypes.byref(rid))
        if st != CHM_OK:
            raise ChmError(st, "chm_server_submit")
        return rid.value

    def poll(self, max_count=4096):
        ids = (ctypes.c_int64 * max_count)()
        sts = (ctypes.c_int * max_count)()
        lat = (ctypes.c_double * max_count)()
        got = ctypes.c_int()
        check(chm_server_poll(self.handle, ctypes.cast(ids, ctypes.c_void_p), ctypes.cast(sts, ctypes.c_void_p),
                              ctypes.cast(lat, ctypes.c_void_p), max_count, ctypes.byref(got)), "chm_server_poll")
        return [(int(ids[i]), int(sts[i]), float(lat[i])) for i in range(got.value)]

    def drain(self, timeout_s=60.0) -> int:
        return chm_server_drain(self.handle, float(timeout_s))

    def get_factor(self, fid, out: torch.Tensor) -> int:
        return chm_server_get_factor(self.handle, int(fid), out.data_ptr(), out.shape[1])

    def stats(self):
        out = (ctypes.c_int64 * 6)()
        check(chm_server_stats(self.handle, ctypes.cast(out, ctypes.c_void_p)), "chm_server_stats")
        keys = ("launches", "requests_launched", "completed", "max_concurrent", "bytes_held", "outstanding")
        return dict(zip(keys, [int(x) for x in out]))

    def close(self):
        if getattr(self, "handle", None):
            chm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
