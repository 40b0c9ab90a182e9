"""ctypes loader for libtsqr.so (argument marshalling only).

The CUDA library must have been built in-tree (``python -m paper_0912_2572_gb300.build``
or ``__graft_entry__.build()``). There is no fallback: if the shared library is
missing, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsqr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tsqr.h")

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_vp = ctypes.c_void_p
_dp = ctypes.c_void_p  # device pointers travel as plain addresses

class BatchItem(ctypes.Structure):
    """Mirror of tsqr_batch_item (include/tsqr.h)."""
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int32), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("k", ctypes.c_int32),
                ("R", ctypes.c_void_p), ("ldr", ctypes.c_int64), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64),
                ("prec", ctypes.c_int32)]


SIGNATURES = {
    "tsqr_factor": (_i32, [_dp, _i64, _i32, _i64, _i32, _i32, _i32, _i32, _vp,
                           ctypes.POINTER(_vp), _dp, _i64]),
    "tsqr_factor_qt": (_i32, [_dp, _i64, _i32, _i64, _dp, _i64, _i32, _i32, _i32, _i32, _i32, _vp,
                              ctypes.POINTER(_vp), _dp, _i64]),
    "tsqr_caqr": (_i32, [_dp, _i64, _i32, _i64, _i32, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp), _dp, _i64]),
    "tsqr_apply_qt": (_i32, [_vp, _dp, _i64, _i32, _vp]),
    "tsqr_apply_q": (_i32, [_vp, _dp, _i64, _i32, _vp]),
    "tsqr_form_q": (_i32, [_vp, _dp, _i64, _vp]),
    "tsqr_orthonormalize": (_i32, [_dp, _i64, _i32, _i64, _dp, _i64, _dp, _i64, _i32, _i32, _i32, _i32, _vp]),
    "tsqr_lstsq": (_i32, [_dp, _i64, _i32, _i64, _dp, _i64, _i32, _dp, _i64, _i32, _i32, _i32, _i32,
                          _i32, _vp, ctypes.POINTER(ctypes.c_double)]),
    "tsqr_solve_r": (_i32, [_vp, _dp, _i64, _i32, _dp, _i64, _dp, _vp]),
    "tsqr_lstsq_static": (_i32, [_dp, _i64, _i32, _i64, _dp, _i64, _i32, _dp, _i64, _vp]),
    "tsqr_batch_solve": (_i32, [ctypes.POINTER(BatchItem), _i32, _i32, _i32, _vp, ctypes.POINTER(_i32),
                                 ctypes.POINTER(ctypes.c_double)]),
    "tsqr_batch_autotune": (_i32, [ctypes.POINTER(BatchItem), _i32, _i32, _vp, ctypes.POINTER(_i32),
                                    ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float)]),
    "tsqr_factor_autotune": (_i32, [_dp, _i64, _i32, _i64, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                     ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float)]),
    "tsqr_free": (_i32, [_vp]),
    "tsqr_error_word": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "tsqr_qr_solve_host": (_i32, [_vp, _i64, _i32, _i64, _vp, _i64, _i32, _vp, _i64, _vp, _i64, _vp, _i64, _vp,
                                  _i32, _i32, _i32, _vp, _vp, _vp]),
    "tsqr_debug_fail_allocations": (_i32, [_i32]),
    "tsqr_set_mixed_wy_min_n": (_i32, [_i32]),
    "tsqr_set_apply_tile_pairs": (_i32, [_i32]),
    "tsqr_batch_describe": (_i32, [ctypes.POINTER(BatchItem), _i32, _i32, _i32, _i32, _i64, _i64, _i64,
                                   ctypes.POINTER(_i64), ctypes.POINTER(_i64), _i64]),
    "tsqr_plan_clusters": (_i32, [_i64, _i32, _i32, _i32, _i32, _i32, _i64, _i64, _i64, ctypes.POINTER(_i64),
                                  ctypes.POINTER(_i32), _i64, ctypes.POINTER(_i32), _i64]),
    "tsqr_probe_fp64_peak": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "tsqr_probe_dmma_peak": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "tsqr_batch_plan_create": (_i32, [ctypes.POINTER(BatchItem), _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    "tsqr_batch_plan_run": (_i32, [_vp, _vp]),
    "tsqr_batch_plan_results": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)]),
    "tsqr_batch_plan_destroy": (_i32, [_vp]),
    "tsqr_server_create": (_i32, [_i64, _i32, _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    "tsqr_server_create_resident": (_i32, [_i64, _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    "tsqr_debug_resident_ring_entries": (_i32, [_i64]),
    "tsqr_server_submit": (_i32, [_vp, ctypes.POINTER(BatchItem), ctypes.POINTER(_i64)]),
    "tsqr_server_poll": (_i32, [_vp, _i32, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "tsqr_server_drain": (_i32, [_vp]),
    "tsqr_server_stats": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "tsqr_server_destroy": (_i32, [_vp]),
    "tsqr_profile_start": (_i32, []),
    "tsqr_profile_stop": (_i32, [_i64, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(_i64)]),
    "tsqr_factors_info": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "tsqr_plan_describe": (_i32, [_i64, _i32, _i32, _i32, _i32, _i32, _i32, _i64, _i64, _i64,
                                  ctypes.POINTER(_i64), ctypes.POINTER(_i64), _i64,
                                  ctypes.POINTER(_i64), _i64]),
    "tsqr_strerror": (ctypes.c_char_p, [_i32]),
    "tsqr_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class TSQRError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


def load() -> ctypes.CDLL:
    """Load libtsqr.so and attach the C signatures. Raises if it was not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_0912_2572_gb300.build` (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def load_checked() -> ctypes.CDLL:
    """Load the bounds-checked build libtsqr_check.so (its own handle, its own device error
    word) with the same signatures; built by ``build.build(check=True)``."""
    path = os.path.join(HERE, "libtsqr_check.so")
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_0912_2572_gb300.build --check`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is not None:
            fn.restype = res
            fn.argtypes = args
    return lib


def check(status: int, where: str) -> None:
    if status != 0:
        lib = load()
        detail = lib.tsqr_last_error().decode() or lib.tsqr_strerror(status).decode()
        raise TSQRError(status, where, detail)


def declared_functions() -> list[str]:
    """Names of every function the public header declares."""
    import re
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsqr_[a-z_0-9]+)\s*\(", text)))
