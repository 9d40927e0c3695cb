"""ctypes binding of libscaletrack.so (argument marshalling only).

Every computation happens in the CUDA library; this module declares the C
signatures of include/scaletrack.h and loads the in-tree build.  Loading
fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

ST_OK, ST_ERR_INVALID_ARG, ST_ERR_OOM, ST_ERR_CUDA, ST_ERR_STATE, ST_ERR_TIMEOUT, ST_ERR_NONFINITE, \
    ST_ERR_OVERFLOW = range(8)
STATUS_NAMES = ["ST_OK", "ST_ERR_INVALID_ARG", "ST_ERR_OOM", "ST_ERR_CUDA", "ST_ERR_STATE", "ST_ERR_TIMEOUT",
                "ST_ERR_NONFINITE", "ST_ERR_OVERFLOW"]
ST_FP64, ST_MIXED_F32, ST_MIXED_BF16V = 0, 1, 2
ST_DTYPE_F32, ST_DTYPE_F64 = 0, 1
PRECISIONS = {"fp64": ST_FP64, "mixed_f32": ST_MIXED_F32, "mixed_bf16": ST_MIXED_BF16V}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class StError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


# name -> (restype, argtypes); mirrors include/scaletrack.h
_P = C.POINTER
_vp, _i, _i64, _d, _u64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
SIGNATURES = {
    "st_create_grid": (_i, [_i, _i, _i, _d, _d, _d, _i, _i, _P(Allocator), _vp, _P(_vp)]),
    "st_destroy": (None, [_vp]),
    "st_last_error": (C.c_char_p, [_vp]),
    "st_set_stream": (_i, [_vp, _vp]),
    "st_synchronize": (_i, [_vp]),
    "st_set_fluid_async": (_i, [_vp, _vp, _i]),
    "st_get_sources_async": (_i, [_vp, _vp, _i]),
    "st_set_params": (_i, [_vp, _d, _d, _P(_d), _d, _d, _i]),
    "st_set_physics": (_i, [_vp, _i, _i, _i, _i, _d]),
    "st_timers_enable": (_i, [_vp, _i]),
    "st_probe_fma": (_i, [_vp, _P(_d), _P(_d)]),
    "st_timers_read": (_i, [_vp, _P(_d), _P(_i64), _i]),
    "st_set_fluid": (_i, [_vp, _vp, _i, _i]),
    "st_reserve": (_i, [_vp, _i64]),
    "st_add_particles": (_i, [_vp, _i64, _vp, _vp, _vp, _vp, _i]),
    "st_num_particles": (_i, [_vp, _P(_i64)]),
    "st_step": (_i, [_vp, _i, _d]),
    "st_get_sources": (_i, [_vp, _vp, _i, _i]),
    "st_get_sources_fixed": (_i, [_vp, _vp, _P(_i), _i]),
    "st_reorder": (_i, [_vp]),
    "st_get_particles": (_i, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i]),
    "st_get_cells": (_i, [_vp, _i64, _i64, _vp, _i]),
    "st_get_cell_counts": (_i, [_vp, _vp, _i]),
    "st_invariants": (_i, [_vp, _P(_d)]),
    "st_kernel_launches": (_i, [_vp, _P(_i64)]),
    "st_clear_particles": (_i, [_vp]),
    "st_adjoint_forward": (_i, [_vp, _i, _d, _i]),
    "st_adjoint_backward": (_i, [_vp, _vp, _i, _vp, _P(_d), _vp, _i]),
    "st_sort_keys_static": (_i, [_vp, _i64, _i, _vp, _vp, _vp]),
    "st_sort_keys_static_status": (_i, [_vp]),
    "st_chunks_create": (_i, [_vp, _i64]),
    "st_chunks_add": (_i, [_vp, _i64, _vp, _vp, _vp, _i]),
    "st_chunks_step": (_i, [_vp, _i, _d, _P(_d)]),
    "st_chunks_get": (_i, [_vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "st_chunks_count": (_i, [_vp, _P(_i64), _P(_i64)]),
    "st_set_microphysics": (_i, [_vp, _i, _d, _d, _d, _d, _d, _d, _d]),
    "st_set_thermo": (_i, [_vp, _vp, _vp, _i, _i]),
    "st_set_temperatures": (_i, [_vp, _i64, _i64, _vp, _i]),
    "st_get_temperatures": (_i, [_vp, _i64, _i64, _vp, _i]),
    "st_get_micro_sources": (_i, [_vp, _vp, _i, _i]),
    "st_micro_invariants": (_i, [_vp, _P(_d)]),
    "st_gen_particles": (_i, [_vp, _u64, _i64, _i64, _P(_d), _d, _vp, _i, _vp, _vp, _vp, _vp]),
    "st_chunk_bounds": (_i, [_vp, _vp, _i]),
    "st_couple_params": (_i, [_vp, _d, _d, _i, _i, _i]),
    "st_couple_run": (_i, [_vp, _i, _d]),
    "st_get_fluid": (_i, [_vp, _vp, _i]),
    "st_get_pending_sources": (_i, [_vp, _vp, _i]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libscaletrack.so from the package's _build folder."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise ImportError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, handle, where: str):
    if status != ST_OK:
        msg = ""
        if handle:
            m = load().st_last_error(handle)
            msg = m.decode() if m else ""
        raise StError(status, where, msg)
