"""Python binding of the fz C ABI (``include/fz.h``): argument marshalling only.

Every step of the path -- counting table, memo build, unranking, enumeration
-- runs in the CUDA kernels of ``libfz.so`` (built in-tree by
``paper_2407_20474_gb300._build.build()``).  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises ``FzError``.

Device buffers are passed as torch CUDA tensors (or raw integer device
addresses); streams default to torch's current stream when torch is present.
Tuples are int32, row-major, in descending lexicographic order.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfz.so")

FZ_MAX_D = 16
FZ_AUTO = -1

FZ_OK = 0
FZ_EINVAL = -1
FZ_EOVERFLOW = -2
FZ_ENOSPC = -3
FZ_ENOMEM = -4
FZ_EAGAIN = -5
FZ_ETIMEOUT = -6
FZ_ECUDA = -7
FZ_ENOTFOUND = -8
FZ_EINTERNAL = -9
FZ_ECANCELED = -10

# Every symbol include/fz.h declares (checked by the CPU tests).
EXPORTS = (
    "fz_version", "fz_last_error_string", "fz_status_string", "fz_kernel_launches",
    "fz_write_probe", "fz_selftest_bounded_wait",
    "fz_count", "fz_count_upto", "fz_count_upto_noalloc", "fz_count_table",
    "fz_memo_rows", "fz_build_memo_into", "fz_build_memo_schedule", "fz_build_memo",
    "fz_memo_info",
    "fz_memo_release",
    "fz_autotune", "fz_autotune_report", "fz_plan_create", "fz_plan_info", "fz_plan_set_enum_ctas_per_sm",
    "fz_plan_rebuild",
    "fz_plan_enumerate",
    "fz_plan_unrank", "fz_plan_sync", "fz_plan_destroy",
    "fz_enumerate", "fz_enumerate_host", "fz_enumerate_host_chunks",
    "fz_batch_create", "fz_batch_info", "fz_batch_layout", "fz_batch_rebuild",
    "fz_batch_set_enum_ctas_per_sm",
    "fz_batch_enumerate", "fz_batch_sync", "fz_batch_destroy", "fz_enumerate_batch",
    "fz_plan_batch", "fz_batch_autotune", "fz_batch_policy", "fz_batch_policy_reset",
    "fz_serve_create", "fz_serve_register", "fz_serve_submit", "fz_serve_poll",
    "fz_serve_wait", "fz_serve_copy", "fz_serve_release", "fz_serve_stats", "fz_serve_destroy",
    "fz_serve_submit_gens", "fz_serve_cancel", "fz_serve_replay",
)


class FzError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (status_string(status), message))
        self.status = status


class fz_opts_t(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("top", ctypes.c_int32),
                ("slice_rows", ctypes.c_int32), ("flags", ctypes.c_int32)]


class fz_tune_entry_t(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("slice_rows", ctypes.c_int32),
                ("run_order", ctypes.c_int32), ("screened_out", ctypes.c_int32),
                ("memo_rows", ctypes.c_uint64), ("build_ms", ctypes.c_double),
                ("enum_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class fz_plan_info_t(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("d", ctypes.c_int32), ("n", ctypes.c_int32),
                ("k", ctypes.c_int32), ("top", ctypes.c_int32),
                ("memo_rows", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("slice_rows", ctypes.c_int32), ("run_order", ctypes.c_int32)]


class fz_memo_info_t(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("top", ctypes.c_int32), ("rows", ctypes.c_uint64),
                ("offsets_dev", ctypes.c_void_p), ("rows_dev", ctypes.c_void_p)]


class fz_instance_t(ctypes.Structure):
    _fields_ = [("g", ctypes.POINTER(ctypes.c_int32)), ("d", ctypes.c_int32),
                ("n", ctypes.c_int32)]


class fz_batch_tune_entry_t(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("run_order", ctypes.c_int32),
                ("instances", ctypes.c_int32), ("memos", ctypes.c_int32),
                ("cap_rows", ctypes.c_double), ("rows", ctypes.c_uint64),
                ("memo_rows", ctypes.c_uint64), ("build_ms", ctypes.c_double),
                ("enum_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class fz_batch_info_t(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("memos", ctypes.c_int32),
                ("total_rows", ctypes.c_uint64), ("total_words", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("work_items", ctypes.c_uint64),
                ("run_order", ctypes.c_int32), ("run_memos", ctypes.c_int32),
                ("coop_memos", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fz_serve_cfg_t(ctypes.Structure):
    _fields_ = [("memory_bytes", ctypes.c_uint64), ("max_in_flight", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class fz_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("d", ctypes.c_int32), ("count", ctypes.c_uint64),
                ("rows_dev", ctypes.c_void_p), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class fz_serve_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64),
                ("bytes_budget", ctypes.c_uint64), ("sets", ctypes.c_int32),
                ("last_error", ctypes.c_int32)]


FZ_SERVE_PER_REQUEST = 1

FZ_SERVE_DONE = 0
FZ_SERVE_QUEUED = 1
FZ_SERVE_RUNNING = 2

_lib = None
_P = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_U64P = ctypes.POINTER(ctypes.c_uint64)

_SIGS = {
    "fz_version": (ctypes.c_int, []),
    "fz_last_error_string": (ctypes.c_char_p, []),
    "fz_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fz_kernel_launches": (ctypes.c_uint64, []),
    "fz_write_probe": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "fz_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_int), _P]),
    "fz_count": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, _U64P, _P]),
    "fz_count_upto": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, _U64P, _P]),
    "fz_count_table": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, _P, _P]),
    "fz_count_upto_noalloc": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, _P, _P]),
    "fz_memo_rows": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, _U64P, _P]),
    "fz_build_memo_into": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, _P, _P,
                                          ctypes.c_uint64, _U64P, _P]),
    "fz_build_memo_schedule": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32, ctypes.c_int,
                                              _P, _P, ctypes.c_uint64, _U64P, _P]),
    "fz_build_memo": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                     ctypes.POINTER(_P), _P]),
    "fz_memo_info": (ctypes.c_int, [_P, ctypes.POINTER(fz_memo_info_t)]),
    "fz_memo_release": (ctypes.c_int, [_P]),
    "fz_plan_create": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                      ctypes.POINTER(fz_opts_t), ctypes.POINTER(_P), _P]),
    "fz_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(fz_plan_info_t)]),
    "fz_autotune": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                   ctypes.POINTER(fz_opts_t), ctypes.POINTER(ctypes.c_double), _P]),
    "fz_autotune_report": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                          ctypes.POINTER(fz_tune_entry_t), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(fz_opts_t),
                                          ctypes.POINTER(ctypes.c_double), _P]),
    "fz_plan_rebuild": (ctypes.c_int, [_P, _P]),
    "fz_plan_set_enum_ctas_per_sm": (ctypes.c_int, [_P, ctypes.c_int32]),
    "fz_plan_enumerate": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, _P,
                                         ctypes.c_uint64, _U64P, _P]),
    "fz_plan_unrank": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P, _P]),
    "fz_plan_sync": (ctypes.c_int, [_P, _P]),
    "fz_plan_destroy": (ctypes.c_int, [_P]),
    "fz_enumerate": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                    ctypes.POINTER(fz_opts_t), ctypes.c_uint64,
                                    ctypes.c_uint64, _P, ctypes.c_uint64, _U64P, _P]),
    "fz_enumerate_host": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                         ctypes.POINTER(fz_opts_t), ctypes.c_uint64,
                                         ctypes.c_uint64, _P, ctypes.c_uint64, _U64P, _P]),
    "fz_enumerate_host_chunks": (ctypes.c_int, [_I32P, ctypes.c_int, ctypes.c_int32,
                                                ctypes.POINTER(fz_opts_t), ctypes.c_uint64,
                                                ctypes.c_uint64, _P, ctypes.c_uint64,
                                                ctypes.c_uint64, _U64P, _P]),
    "fz_batch_create": (ctypes.c_int, [ctypes.POINTER(fz_instance_t), ctypes.c_int,
                                       ctypes.POINTER(fz_opts_t), ctypes.POINTER(_P), _P]),
    "fz_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(fz_batch_info_t)]),
    "fz_batch_layout": (ctypes.c_int, [_P, _U64P, _U64P, _I32P, _I32P]),
    "fz_batch_rebuild": (ctypes.c_int, [_P, _P]),
    "fz_batch_set_enum_ctas_per_sm": (ctypes.c_int, [_P, ctypes.c_int32]),
    "fz_batch_enumerate": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P]),
    "fz_batch_sync": (ctypes.c_int, [_P, _P]),
    "fz_batch_destroy": (ctypes.c_int, [_P]),
    "fz_batch_autotune": (ctypes.c_int, [ctypes.POINTER(fz_instance_t), ctypes.c_int,
                                         ctypes.POINTER(fz_batch_tune_entry_t), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), _P]),
    "fz_batch_policy": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "fz_batch_policy_reset": (ctypes.c_int, []),
    "fz_plan_batch": (ctypes.c_int, [ctypes.POINTER(fz_instance_t), ctypes.c_int,
                                     ctypes.POINTER(fz_opts_t), _U64P, _U64P, _U64P, _P]),
    "fz_enumerate_batch": (ctypes.c_int, [ctypes.POINTER(fz_instance_t), ctypes.c_int,
                                          ctypes.POINTER(fz_opts_t), _U64P, _P,
                                          ctypes.c_uint64, _U64P, _P]),
    "fz_serve_create": (ctypes.c_int, [ctypes.POINTER(fz_serve_cfg_t), ctypes.POINTER(_P)]),
    "fz_serve_register": (ctypes.c_int, [_P, _I32P, ctypes.c_int, ctypes.c_int32, _I32P]),
    "fz_serve_submit": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _U64P]),
    "fz_serve_submit_gens": (ctypes.c_int, [_P, _I32P, ctypes.c_int, ctypes.c_int32, _U64P]),
    "fz_serve_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "fz_serve_replay": (ctypes.c_int, [_P, _I32P, _I32P, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_double), _U64P,
                                       ctypes.POINTER(ctypes.c_double)]),
    "fz_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(fz_result_t)]),
    "fz_serve_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.POINTER(fz_result_t)]),
    "fz_serve_copy": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_uint64, _P]),
    "fz_serve_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "fz_serve_stats": (ctypes.c_int, [_P, ctypes.POINTER(fz_serve_stats_t)]),
    "fz_serve_destroy": (ctypes.c_int, [_P]),
}


def lib():
    """The loaded ``libfz.so`` (raises FzError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FzError(FZ_ECUDA, "libfz.so not built (run __graft_entry__.build())")
        try:
            L = ctypes.CDLL(LIB_PATH)
        except OSError as e:
            raise FzError(FZ_ECUDA, "cannot load libfz.so: %s" % e)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


_STATUS_NAMES = {FZ_OK: "FZ_OK", FZ_EINVAL: "FZ_EINVAL", FZ_EOVERFLOW: "FZ_EOVERFLOW",
                 FZ_ENOSPC: "FZ_ENOSPC", FZ_ENOMEM: "FZ_ENOMEM", FZ_EAGAIN: "FZ_EAGAIN",
                 FZ_ETIMEOUT: "FZ_ETIMEOUT", FZ_ECUDA: "FZ_ECUDA",
                 FZ_ENOTFOUND: "FZ_ENOTFOUND", FZ_EINTERNAL: "FZ_EINTERNAL",
                 FZ_ECANCELED: "FZ_ECANCELED"}


def status_string(status: int) -> str:
    """Name of a status code (from the library when it is loaded)."""
    if _lib is None:  # never load the library just to name an error
        return _STATUS_NAMES.get(int(status), "FZ_STATUS_%d" % status)
    return _lib.fz_status_string(int(status)).decode()


def _check(rc: int):
    if rc != FZ_OK:
        msg = lib().fz_last_error_string().decode(errors="replace")
        raise FzError(rc, msg)


def _gens(g: Sequence[int]):
    arr = (ctypes.c_int32 * len(g))(*[int(x) for x in g])
    return arr, len(g)


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _devbuf(x, itemsize: int, need: int, what: str) -> Optional[int]:
    """Device address of ``x`` after checking, for a torch tensor, that it is
    a contiguous CUDA tensor of ``itemsize``-byte elements holding at least
    ``need`` of them (the C side writes ``need`` elements through the raw
    pointer and cannot check).  Raw integer addresses are passed through:
    their size is the caller's responsibility."""
    if x is None or not hasattr(x, "data_ptr"):
        return _ptr(x)
    if need > 0:
        if not getattr(x, "is_cuda", False):
            raise FzError(FZ_EINVAL, "%s: expected a CUDA tensor" % what)
        if x.element_size() != itemsize:
            raise FzError(FZ_EINVAL, "%s: expected %d-byte elements, got %d"
                          % (what, itemsize, x.element_size()))
        if not x.is_contiguous():
            raise FzError(FZ_EINVAL, "%s: tensor must be contiguous" % what)
        if x.numel() < need:
            raise FzError(FZ_EINVAL, "%s: %d elements, %d needed" % (what, x.numel(), need))
    return x.data_ptr()


def _opts(k=FZ_AUTO, top=FZ_AUTO, slice_rows=0):
    return fz_opts_t(int(k), int(top), int(slice_rows), 0)


# ---------------------------------------------------------------- counting
def fz_version() -> int:
    return int(lib().fz_version())


def fz_kernel_launches() -> int:
    """Kernels the library has enqueued in this process (tracing counter)."""
    return int(lib().fz_kernel_launches())


def fz_selftest_bounded_wait(limit_ms: int = 20, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status the device reported
    (FZ_ETIMEOUT when waits give up as designed)."""
    st = ctypes.c_int(0)
    _check(lib().fz_selftest_bounded_wait(int(limit_ms), ctypes.byref(st), _stream(stream)))
    return int(st.value)


def fz_write_probe(out, stream=None):
    """Write out[w] = w over a 16-byte aligned int32 CUDA tensor (measurement
    utility: the write-only ceiling for distinct data)."""
    _check(lib().fz_write_probe(ctypes.c_void_p(out.data_ptr()), int(out.numel()),
                                _stream(stream)))


def fz_count(g: Sequence[int], n: int, stream=None) -> int:
    """|Z(n, g)| (device counting table)."""
    ga, d = _gens(g)
    out = ctypes.c_uint64(0)
    _check(lib().fz_count(ga, d, int(n), ctypes.byref(out), _stream(stream)))
    return int(out.value)


def fz_count_upto(g: Sequence[int], n_max: int, stream=None) -> np.ndarray:
    """|Z(r, g)| for r = 0..n_max (uint64; saturated entries are 2^64 - 1)."""
    ga, d = _gens(g)
    out = np.zeros(int(n_max) + 1, dtype=np.uint64)
    _check(lib().fz_count_upto(ga, d, int(n_max),
                               out.ctypes.data_as(_U64P), _stream(stream)))
    return out


FZ_NOALLOC_MAX_N = 262143


def fz_count_upto_noalloc(g: Sequence[int], n_max: int, counts, stream=None) -> None:
    """|Z(r, g)|, r = 0..n_max, into device uint64 ``counts`` without any
    device allocation (for callers that cannot call cudaMalloc).  Scratch is
    a fixed array inside the library shared by all calls, so n_max is at most
    FZ_NOALLOC_MAX_N and overlapping calls race.  Asynchronous."""
    ga, d = _gens(g)
    ptr = _devbuf(counts, 8, int(n_max) + 1, "counts")
    _check(lib().fz_count_upto_noalloc(ga, d, int(n_max), ptr, _stream(stream)))


def fz_count_table(g: Sequence[int], n: int, table, stream=None) -> None:
    """Fill a device uint64 buffer of (d+1)*(n+1) entries with the count table."""
    ga, d = _gens(g)
    ptr = _devbuf(table, 8, (d + 1) * (int(n) + 1), "table")
    _check(lib().fz_count_table(ga, d, int(n), ptr, _stream(stream)))


# -------------------------------------------------------------------- memo
def fz_memo_rows(tail: Sequence[int], top: int, stream=None) -> int:
    ga, k = _gens(tail)
    out = ctypes.c_uint64(0)
    _check(lib().fz_memo_rows(ga, k, int(top), ctypes.byref(out), _stream(stream)))
    return int(out.value)


def fz_build_memo_into(tail: Sequence[int], top: int, offsets, rows, rows_capacity: int,
                       stream=None) -> int:
    """Build Memo[r] = Z(r, tail), r < top, into caller device buffers
    (offsets: top+1 uint64; rows: rows_capacity*k int32).  Returns the rows."""
    ga, k = _gens(tail)
    need = ctypes.c_uint64(0)
    po = _devbuf(offsets, 8, int(top) + 1, "offsets")
    pr = _devbuf(rows, 4, int(rows_capacity) * k, "rows")
    _check(lib().fz_build_memo_into(ga, k, int(top), po, pr,
                                    int(rows_capacity), ctypes.byref(need), _stream(stream)))
    return int(need.value)


FZ_MEMO_BATCHED, FZ_MEMO_PER_BATCH, FZ_MEMO_PER_COPY = 0, 1, 2


def fz_build_memo_schedule(tail: Sequence[int], top: int, schedule: int, offsets, rows,
                           rows_capacity: int, stream=None) -> int:
    """fz_build_memo_into with an explicit launch schedule (FZ_MEMO_*)."""
    ga, k = _gens(tail)
    need = ctypes.c_uint64(0)
    po = _devbuf(offsets, 8, int(top) + 1, "offsets")
    pr = _devbuf(rows, 4, int(rows_capacity) * k, "rows")
    _check(lib().fz_build_memo_schedule(ga, k, int(top), int(schedule), po,
                                        pr, int(rows_capacity), ctypes.byref(need),
                                        _stream(stream)))
    return int(need.value)


class Memo:
    """Library-owned memo (fz_build_memo / fz_memo_release)."""

    def __init__(self, tail: Sequence[int], top: int, stream=None):
        ga, k = _gens(tail)
        h = _P()
        _check(lib().fz_build_memo(ga, k, int(top), ctypes.byref(h), _stream(stream)))
        self._h = h
        info = fz_memo_info_t()
        _check(lib().fz_memo_info(h, ctypes.byref(info)))
        self.k, self.top, self.rows = info.k, info.top, int(info.rows)
        self.offsets_dev, self.rows_dev = info.offsets_dev, info.rows_dev

    def close(self):
        if getattr(self, "_h", None):
            lib().fz_memo_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fz_build_memo(tail: Sequence[int], top: int, stream=None) -> Memo:
    return Memo(tail, top, stream)


# ------------------------------------------------------------------- plans
def fz_autotune(g: Sequence[int], n: int, stream=None):
    """Measured best (k, slice_rows) for Z(n, g); remembered for later
    FZ_AUTO plans of the same (g, n).  Returns (k, slice_rows, est_ms)."""
    ga, d = _gens(g)
    o = fz_opts_t(0, 0, 0, 0)
    ms = ctypes.c_double(0.0)
    _check(lib().fz_autotune(ga, d, int(n), ctypes.byref(o), ctypes.byref(ms),
                             _stream(stream)))
    return int(o.k), int(o.slice_rows), float(ms.value)


def fz_autotune_report(g: Sequence[int], n: int, stream=None):
    """fz_autotune plus every timed candidate: ((k, slice_rows, ms),
    [dict(k, slice_rows, run_order, screened_out, memo_rows, build_ms, enum_ms,
    total_ms)])."""
    ga, d = _gens(g)
    cap = 64
    arr = (fz_tune_entry_t * cap)()
    got = ctypes.c_int(0)
    o = fz_opts_t(0, 0, 0, 0)
    ms = ctypes.c_double(0.0)
    _check(lib().fz_autotune_report(ga, d, int(n), arr, cap, ctypes.byref(got), ctypes.byref(o),
                                    ctypes.byref(ms), _stream(stream)))
    entries = [dict(k=int(e.k), slice_rows=int(e.slice_rows), run_order=int(e.run_order),
                    screened_out=int(e.screened_out),
                    memo_rows=int(e.memo_rows), build_ms=float(e.build_ms),
                    enum_ms=float(e.enum_ms), total_ms=float(e.total_ms))
               for e in arr[:got.value]]
    return (int(o.k), int(o.slice_rows), float(ms.value)), entries


class Plan:
    """One instance Z(n, g) with its count table and memo resident on the device."""

    def __init__(self, g: Sequence[int], n: int, k: int = FZ_AUTO, top: int = FZ_AUTO,
                 slice_rows: int = 0, stream=None):
        ga, d = _gens(g)
        h = _P()
        o = _opts(k, top, slice_rows)
        _check(lib().fz_plan_create(ga, d, int(n), ctypes.byref(o), ctypes.byref(h),
                                    _stream(stream)))
        self._h = h
        self.g = tuple(int(x) for x in g)
        self.n = int(n)
        info = fz_plan_info_t()
        _check(lib().fz_plan_info(h, ctypes.byref(info)))
        self.count = int(info.count)
        self.d, self.k, self.top = int(info.d), int(info.k), int(info.top)
        self.memo_rows = int(info.memo_rows)
        self.device_bytes = int(info.device_bytes)
        self.slice_rows = int(info.slice_rows)
        self.run_order = bool(info.run_order)

    def rebuild(self, stream=None):
        _check(lib().fz_plan_rebuild(self._h, _stream(stream)))

    def set_enum_ctas_per_sm(self, ctas: int):
        """Cap the enumeration kernel's blocks per SM (0 = no cap)."""
        _check(lib().fz_plan_set_enum_ctas_per_sm(self._h, int(ctas)))

    def enumerate(self, out, rank_begin: int = 0, rank_end: Optional[int] = None,
                  capacity_rows: Optional[int] = None, stream=None) -> int:
        """Asynchronously write ranks [rank_begin, rank_end) into ``out``."""
        end = (1 << 64) - 1 if rank_end is None else int(rank_end)
        if capacity_rows is None:
            capacity_rows = (out.numel() // self.d) if hasattr(out, "numel") else 0
        w = ctypes.c_uint64(0)
        if hasattr(out, "element_size") and out.element_size() != 4:
            raise FzError(FZ_EINVAL, "out: expected int32 elements")
        _check(lib().fz_plan_enumerate(self._h, int(rank_begin), end, _ptr(out),
                                       int(capacity_rows), ctypes.byref(w), _stream(stream)))
        return int(w.value)

    def unrank(self, ranks, out, stream=None):
        """Asynchronously write the tuples of device uint64 ``ranks`` into ``out``."""
        m = ranks.numel() if hasattr(ranks, "numel") else len(ranks)
        pr = _devbuf(ranks, 8, int(m), "ranks")
        po = _devbuf(out, 4, int(m) * self.d, "out")
        _check(lib().fz_plan_unrank(self._h, pr, int(m), po, _stream(stream)))

    def sync(self, stream=None):
        _check(lib().fz_plan_sync(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().fz_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fz_plan_create(g, n, k=FZ_AUTO, top=FZ_AUTO, slice_rows=0, stream=None) -> Plan:
    return Plan(g, n, k, top, slice_rows, stream)


# --------------------------------------------------------------- one-shot
def fz_enumerate(g: Sequence[int], n: int, out, rank_begin: int = 0,
                 rank_end: Optional[int] = None, k: int = FZ_AUTO, top: int = FZ_AUTO,
                 slice_rows: int = 0, capacity_rows: Optional[int] = None,
                 stream=None) -> int:
    """Rows of ranks [rank_begin, rank_end) into device buffer ``out``; returns rows."""
    ga, d = _gens(g)
    o = _opts(k, top, slice_rows)
    end = (1 << 64) - 1 if rank_end is None else int(rank_end)
    if capacity_rows is None:
        capacity_rows = (out.numel() // d) if hasattr(out, "numel") else 0
    w = ctypes.c_uint64(0)
    if hasattr(out, "element_size") and out.element_size() != 4:
        raise FzError(FZ_EINVAL, "out: expected int32 elements")
    _check(lib().fz_enumerate(ga, d, int(n), ctypes.byref(o), int(rank_begin), end,
                              _ptr(out), int(capacity_rows), ctypes.byref(w),
                              _stream(stream)))
    return int(w.value)


def fz_enumerate_host(g: Sequence[int], n: int, out, rank_begin: int = 0,
                      rank_end: Optional[int] = None, k: int = FZ_AUTO, top: int = FZ_AUTO,
                      slice_rows: int = 0, chunk_rows: int = 0, stream=None) -> int:
    """As fz_enumerate into host memory ``out`` (numpy int32 array or pinned
    torch CPU tensor, at least rows*d entries).  Pageable output is streamed
    in chunks of ``chunk_rows`` rows (0 = the library's default)."""
    ga, d = _gens(g)
    o = _opts(k, top, slice_rows)
    end = (1 << 64) - 1 if rank_end is None else int(rank_end)
    if isinstance(out, np.ndarray):
        assert out.dtype == np.int32 and out.flags.c_contiguous
        ptr, cap = out.ctypes.data, out.size // d
    else:
        ptr, cap = out.data_ptr(), out.numel() // d
    if hasattr(out, "element_size") and out.element_size() != 4:
        raise FzError(FZ_EINVAL, "out: expected int32 elements")
    w = ctypes.c_uint64(0)
    _check(lib().fz_enumerate_host_chunks(ga, d, int(n), ctypes.byref(o), int(rank_begin), end,
                                          ptr, int(cap), int(chunk_rows), ctypes.byref(w),
                                          _stream(stream)))
    return int(w.value)


# ----------------------------------------------------------------- batches
def _instances(instances):
    """(array of fz_instance_t, keep-alive list) for [(g, n), ...]."""
    keep = []
    arr = (fz_instance_t * len(instances))()
    for i, (g, n) in enumerate(instances):
        ga, d = _gens(g)
        keep.append(ga)
        arr[i].g = ctypes.cast(ga, ctypes.POINTER(ctypes.c_int32))
        arr[i].d = d
        arr[i].n = int(n)
    return arr, keep


class Batch:
    """Many instances [(g, n), ...] enumerated by one persistent launch."""

    def __init__(self, instances, k: int = FZ_AUTO, top: int = FZ_AUTO, stream=None):
        arr, keep = _instances(instances)
        h = _P()
        o = _opts(k, top, 0)
        _check(lib().fz_batch_create(arr, len(instances), ctypes.byref(o), ctypes.byref(h),
                                     _stream(stream)))
        self._h = h
        self.count = len(instances)
        info = fz_batch_info_t()
        _check(lib().fz_batch_info(h, ctypes.byref(info)))
        self.memos = int(info.memos)
        self.total_rows = int(info.total_rows)
        self.total_words = int(info.total_words)
        self.device_bytes = int(info.device_bytes)
        self.work_items = int(info.work_items)
        self.run_order = int(info.run_order)
        self.run_memos = int(info.run_memos)
        self.coop_memos = int(info.coop_memos)
        self.rows = np.zeros(self.count, dtype=np.uint64)
        self.word_offsets = np.zeros(self.count + 1, dtype=np.uint64)
        self.k = np.zeros(self.count, dtype=np.int32)
        self.top = np.zeros(self.count, dtype=np.int32)
        _check(lib().fz_batch_layout(h, self.rows.ctypes.data_as(_U64P),
                                     self.word_offsets.ctypes.data_as(_U64P),
                                     self.k.ctypes.data_as(_I32P), self.top.ctypes.data_as(_I32P)))

    def rebuild(self, stream=None):
        _check(lib().fz_batch_rebuild(self._h, _stream(stream)))

    def set_enum_ctas_per_sm(self, ctas: int):
        """Cap the enumeration kernel's blocks per SM (0 = no cap)."""
        _check(lib().fz_batch_set_enum_ctas_per_sm(self._h, int(ctas)))

    def enumerate(self, out, capacity_words: Optional[int] = None, stream=None):
        if capacity_words is None:
            capacity_words = out.numel() if hasattr(out, "numel") else 0
        _check(lib().fz_batch_enumerate(self._h, _ptr(out), int(capacity_words),
                                        _stream(stream)))

    def sync(self, stream=None):
        _check(lib().fz_batch_sync(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().fz_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fz_batch_autotune(instances, stream=None):
    """Measure the memo policy per tuple width on a sample of ``instances``
    ([(g, n), ...]); later batches on this device use it.  Returns the timed
    candidates as dicts and the chosen policy {d: (cap_rows, run_order)}."""
    arr, keep = _instances(instances)
    cap = 256
    ent = (fz_batch_tune_entry_t * cap)()
    got = ctypes.c_int(0)
    _check(lib().fz_batch_autotune(arr, len(instances), ent, cap, ctypes.byref(got),
                                   _stream(stream)))
    rows = [dict(d=int(e.d), run_order=int(e.run_order), instances=int(e.instances),
                 memos=int(e.memos), cap_rows=float(e.cap_rows), rows=int(e.rows),
                 memo_rows=int(e.memo_rows), build_ms=float(e.build_ms),
                 enum_ms=float(e.enum_ms), total_ms=float(e.total_ms))
            for e in ent[:got.value]]
    chosen = {}
    for d in sorted({len(g) for g, _ in instances}):
        chosen[d] = fz_batch_policy(d)
    return rows, chosen


def fz_batch_policy(d: int):
    """(cap_rows, run_order) of the batch memo policy for width d."""
    c = ctypes.c_double(0.0)
    r = ctypes.c_int32(0)
    _check(lib().fz_batch_policy(int(d), ctypes.byref(c), ctypes.byref(r)))
    return float(c.value), bool(r.value)


def fz_batch_policy_reset():
    _check(lib().fz_batch_policy_reset())


def fz_plan_batch(instances, k: int = FZ_AUTO, top: int = FZ_AUTO, stream=None):
    """Exact layout of a batch before enumerating it: (word offsets, count + 1;
    rows per instance), the offsets fz_enumerate_batch will use."""
    arr, keep = _instances(instances)
    o = _opts(k, top, 0)
    offs = np.zeros(len(instances) + 1, dtype=np.uint64)
    rows = np.zeros(max(len(instances), 1), dtype=np.uint64)
    need = ctypes.c_uint64(0)
    _check(lib().fz_plan_batch(arr, len(instances), ctypes.byref(o),
                               offs.ctypes.data_as(_U64P), rows.ctypes.data_as(_U64P),
                               ctypes.byref(need), _stream(stream)))
    return offs, rows[:len(instances)]


def fz_enumerate_batch(instances, out, k: int = FZ_AUTO, top: int = FZ_AUTO,
                       capacity_words: Optional[int] = None, stream=None) -> np.ndarray:
    """One-shot batch; returns the word offsets (count + 1)."""
    arr, keep = _instances(instances)
    o = _opts(k, top, 0)
    offs = np.zeros(len(instances) + 1, dtype=np.uint64)
    need = ctypes.c_uint64(0)
    if capacity_words is None:
        capacity_words = out.numel() if hasattr(out, "numel") else 0
    _check(lib().fz_enumerate_batch(arr, len(instances), ctypes.byref(o),
                                    offs.ctypes.data_as(_U64P), _ptr(out), int(capacity_words),
                                    ctypes.byref(need), _stream(stream)))
    return offs


# ----------------------------------------------------------------- serving
class Server:
    """Request loop over resident generator sets (continuous batching)."""

    def __init__(self, memory_bytes: int = 0, max_in_flight: int = 64, streams: int = 8,
                 max_queue: int = 1 << 20, per_request: bool = False):
        """``per_request``: launch every request on its own (FZ_SERVE_PER_REQUEST)
        instead of the requests admitted together as one launch."""
        cfg = fz_serve_cfg_t(int(memory_bytes), int(max_in_flight), int(streams),
                             int(max_queue), FZ_SERVE_PER_REQUEST if per_request else 0)
        h = _P()
        _check(lib().fz_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def register(self, g: Sequence[int], n_max: int) -> int:
        ga, d = _gens(g)
        sid = ctypes.c_int32(0)
        _check(lib().fz_serve_register(self._h, ga, d, int(n_max), ctypes.byref(sid)))
        return int(sid.value)

    def submit(self, set_id: int, n: int) -> int:
        t = ctypes.c_uint64(0)
        _check(lib().fz_serve_submit(self._h, int(set_id), int(n), ctypes.byref(t)))
        return int(t.value)

    def submit_gens(self, g: Sequence[int], n: int) -> int:
        """Queue Z(n, g) by its generators (registers the set on first use)."""
        ga, d = _gens(g)
        t = ctypes.c_uint64(0)
        _check(lib().fz_serve_submit_gens(self._h, ga, d, int(n), ctypes.byref(t)))
        return int(t.value)

    def replay(self, set_ids, ns, arrivals_s):
        """Replay a request stream from native threads (fz_serve_replay):
        request i of set set_ids[i] and element ns[i] is submitted at
        arrivals_s[i] s.  Returns (latency seconds, rows, span seconds)."""
        sid = np.ascontiguousarray(np.asarray(set_ids, dtype=np.int32))
        nn = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
        at = np.ascontiguousarray(np.asarray(arrivals_s, dtype=np.float64))
        m = int(sid.size)
        if nn.size != m or at.size != m:
            raise FzError(FZ_EINVAL, "replay: arrays of different lengths")
        lat = np.zeros(m, dtype=np.float64)
        rows = np.zeros(m, dtype=np.uint64)
        span = ctypes.c_double(0.0)
        _check(lib().fz_serve_replay(self._h, sid.ctypes.data_as(_I32P), nn.ctypes.data_as(_I32P),
                                     at.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m,
                                     lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     rows.ctypes.data_as(_U64P), ctypes.byref(span)))
        return lat, rows, float(span.value)

    def cancel(self, ticket: int):
        """Cancel a queued request (FzError FZ_EAGAIN if it is already running)."""
        _check(lib().fz_serve_cancel(self._h, int(ticket)))

    def poll(self, ticket: int) -> fz_result_t:
        r = fz_result_t()
        _check(lib().fz_serve_poll(self._h, int(ticket), ctypes.byref(r)))
        return r

    def wait(self, ticket: int, timeout_ms: int = -1) -> fz_result_t:
        r = fz_result_t()
        _check(lib().fz_serve_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(r)))
        return r

    def copy(self, ticket: int, dst, capacity_words: Optional[int] = None, stream=None):
        """Copy a finished result into ``dst`` (torch tensor, host or device)."""
        if capacity_words is None:
            capacity_words = dst.numel() if hasattr(dst, "numel") else 0
        _check(lib().fz_serve_copy(self._h, int(ticket), _ptr(dst), int(capacity_words),
                                   _stream(stream)))

    def release(self, ticket: int):
        _check(lib().fz_serve_release(self._h, int(ticket)))

    def stats(self) -> fz_serve_stats_t:
        st = fz_serve_stats_t()
        _check(lib().fz_serve_stats(self._h, ctypes.byref(st)))
        return st

    def close(self):
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            _check(lib().fz_serve_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
