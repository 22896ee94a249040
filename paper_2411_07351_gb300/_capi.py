"""ctypes binding of libfht.so: the entry points of ``include/fht.h`` under the
same names, argument marshalling only.

Loading fails loudly (``RuntimeError``) when the library has not been built:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfht.so")

FHT_OK, FHT_ERR_INVALID, FHT_ERR_NOMEM, FHT_ERR_CUDA, FHT_ERR_TIMEOUT, FHT_ERR_BUSY, \
    FHT_ERR_UNSUPPORTED, FHT_ERR_DEVICE = range(8)
FHT_U8_I32, FHT_I32_I32, FHT_F32_F32, FHT_F64_F64 = range(4)
FHT_Q0, FHT_Q1, FHT_Q2, FHT_Q3, FHT_QALL = 1, 2, 4, 8, 15
FHT_CYCLIC, FHT_EXTENDED = 0, 1
FHT_SPLIT_T, FHT_SPLIT_S = 0, 1
FHT_TABLE_QUADS, FHT_TABLE_FUSED, FHT_TABLE_OPS, FHT_TABLE_ROWS, FHT_TABLE_PASS_BEGIN, FHT_TABLE_BAND_ITEMS, \
    FHT_TABLE_SPINE_ROWS, FHT_TABLE_SPINE_TERMS, FHT_TABLE_SPINE_BEGIN, FHT_TABLE_ADJ_ROWS, FHT_TABLE_ADJ_TERMS, \
    FHT_TABLE_ADJ_BEGIN, FHT_TABLE_ADJ_PTR, FHT_TABLE_ADJ_OPS = range(14)


class fht_tuning_t(ctypes.Structure):
    _fields_ = [("fused_rows", ctypes.c_int32), ("tile_cols", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("with_adjoint", ctypes.c_int32), ("rounding", ctypes.c_int32),
                ("spine_chunk", ctypes.c_int32), ("generic_cols", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fht_plan_info_t(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("rows", ctypes.c_int32 * 4), ("cols", ctypes.c_int32 * 4),
                ("out_offset", ctypes.c_int64 * 4), ("out_elems", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t), ("adjoint_workspace_bytes", ctypes.c_size_t),
                ("adds", ctypes.c_int64),
                ("model_bytes", ctypes.c_int64), ("ideal_bytes", ctypes.c_int64),
                ("fused_rows", ctypes.c_int32), ("tile_cols", ctypes.c_int32),
                ("upper_passes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fht_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("in_pitch", ctypes.c_int64),
                ("d_out", ctypes.c_void_p), ("d_ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t),
                ("tag", ctypes.c_uint64), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


FHT_JOB_WITHHOLD_DEPENDENCY = 1

# name -> (restype, argtypes); mirrors include/fht.h
_vp, _i32, _u32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "fht_plan": (ctypes.c_int, [ctypes.POINTER(_vp), _i32, _i32, ctypes.c_int, _u32, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.POINTER(fht_tuning_t)]),
    "fht_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(fht_plan_info_t)]),
    "fht_forward": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _sz, _vp]),
    "fht_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _sz, _vp]),
    "fht_plan_table": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                                      ctypes.POINTER(_i32)]),
    "fht_plan_check": (ctypes.c_int, [_vp]),
    "fht_plan_launches": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "fht_plan_launch_info": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "fht_forward_timed": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _sz, _vp, ctypes.POINTER(_vp), _i32]),
    "fht_forward_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "fht_noalloc_status": (ctypes.c_int, [ctypes.c_int, _vp]),
    "fht_plan_destroy": (ctypes.c_int, [_vp]),
    "fht_builder_create": (ctypes.c_int, [ctypes.POINTER(_vp), _i32]),
    "fht_builder_submit": (ctypes.c_int, [_vp, ctypes.c_uint64, _i32, _i32, ctypes.c_int, _u32, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(fht_tuning_t)]),
    "fht_builder_poll": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_vp),
                                        ctypes.POINTER(ctypes.c_int), _i32, ctypes.POINTER(_i32)]),
    "fht_builder_pending": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "fht_builder_destroy": (ctypes.c_int, [_vp]),
    "fht_pattern_errors": (ctypes.c_int, [_i32, _i32, ctypes.c_int, _vp, _vp]),
    "fht_queue_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i32, _i64]),
    "fht_queue_set_wait_limit": (ctypes.c_int, [_vp, _i64]),
    "fht_submit": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(fht_job), _vp]),
    "fht_queue_poll": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), _i32, ctypes.POINTER(_i32)]),
    "fht_queue_status": (ctypes.c_int, [_vp, _vp]),
    "fht_queue_ready": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "fht_queue_reset_status": (ctypes.c_int, [_vp, _vp]),
    "fht_queue_destroy": (ctypes.c_int, [_vp]),
    "fht_pipe_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, _i32, _i32]),
    "fht_pipe_submit": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
    "fht_pipe_sync": (ctypes.c_int, [_vp]),
    "fht_pipe_destroy": (ctypes.c_int, [_vp]),
    "fht_ws_status": (ctypes.c_int, [_vp, _vp]),
    "fht_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fht_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfht.so (build it first with ``paper_2411_07351_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfht.so is not built ({path}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FHTError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        self.status = status
        msg = lib.fht_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.fht_status_string(status).decode()}: {msg}")


def check(status: int, where: str):
    if status != FHT_OK:
        raise FHTError(status, where)
