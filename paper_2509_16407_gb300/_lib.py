"""ctypes declarations of the C ABI in include/warpspeed.h (no logic here).

The shared library is built in-tree by ``paper_2509_16407_gb300.build``.
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwarpspeed.so")

vp, u64, u32, i32, u8p = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
st = ctypes.c_int  # ws_status


class WsConfig(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_uint64), ("scheme", ctypes.c_int32), ("metadata", ctypes.c_int32),
                ("bucket_slots", ctypes.c_int32), ("tile", ctypes.c_int32), ("max_probe", ctypes.c_uint32),
                ("spin_limit", ctypes.c_uint32), ("device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class WsInfo(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint64), ("buckets", ctypes.c_uint64), ("bucket_slots", ctypes.c_uint64),
                ("tile", ctypes.c_uint64), ("max_probe", ctypes.c_uint64), ("seed1", ctypes.c_uint64),
                ("seed2", ctypes.c_uint64), ("bytes", ctypes.c_uint64), ("scheme", ctypes.c_int32),
                ("metadata", ctypes.c_int32), ("device", ctypes.c_int32), ("never_erased", ctypes.c_int32),
                ("front_buckets", ctypes.c_uint64)]


class WsBatchItem(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("kind", ctypes.c_int32), ("op", ctypes.c_int32),
                ("phase", ctypes.c_int32), ("reserved", ctypes.c_int32), ("keys", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("vals_out", ctypes.c_void_p), ("status_out", ctypes.c_void_p),
                ("n", ctypes.c_uint64)]


class WsServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("max_batch_ops", ctypes.c_uint64),
                ("max_batch_reqs", ctypes.c_uint32), ("plain", ctypes.c_int32), ("hbm_headroom", ctypes.c_double),
                ("grow_at", ctypes.c_double)]


class WsRequest(ctypes.Structure):
    _fields_ = [("table", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("ops", ctypes.c_void_p),
                ("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("vals_out", ctypes.c_void_p),
                ("status_out", ctypes.c_void_p), ("n", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class WsCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("status", ctypes.c_int32),
                ("table", ctypes.c_uint32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "ws_table_create": (st, [u64, i32, i32, ctypes.POINTER(vp)]),
    "ws_table_create_ex": (st, [ctypes.POINTER(WsConfig), ctypes.POINTER(vp)]),
    "ws_destroy": (st, [vp]),
    "ws_table_info_get": (st, [vp, ctypes.POINTER(WsInfo)]),
    "ws_clear": (st, [vp, vp]),
    "ws_set_tile": (st, [vp, i32]),
    "ws_set_spin_limit": (st, [vp, u32]),
    "ws_set_option": (st, [vp, i32, ctypes.c_int64]),
    "ws_insert": (st, [vp, vp, vp, u64, vp]),
    "ws_insert_ex": (st, [vp, vp, vp, u64, vp, vp]),
    "ws_upsert": (st, [vp, vp, vp, u64, i32, vp]),
    "ws_upsert_ex": (st, [vp, vp, vp, u64, i32, vp, vp]),
    "ws_query": (st, [vp, vp, vp, u64, vp]),
    "ws_query_ex": (st, [vp, vp, vp, vp, u64, vp]),
    "ws_erase": (st, [vp, vp, vp, u64, vp]),
    "ws_erase_ex": (st, [vp, vp, vp, vp, u64, vp]),
    "ws_mixed": (st, [vp, vp, vp, vp, vp, vp, u64, vp]),
    "ws_probe_cost": (st, [vp, vp, vp, vp, u64, vp]),
    "ws_count": (st, [vp, ctypes.POINTER(ctypes.c_uint64)]),
    "ws_last_error": (st, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                           ctypes.POINTER(ctypes.c_uint64)]),
    "ws_num_buckets": (st, [vp, ctypes.POINTER(ctypes.c_uint64)]),
    "ws_primary_bucket": (st, [vp, vp, vp, u64, vp]),
    "ws_rehash": (st, [vp, vp, vp, vp]),
    "ws_dump": (st, [vp, vp, vp]),
    "ws_debug_fill_locks": (st, [vp, i32, vp]),
    "ws_batch_plan_create": (st, [ctypes.POINTER(WsBatchItem), u64, ctypes.POINTER(vp)]),
    "ws_batch_plan_launch": (st, [vp, vp]),
    "ws_batch_plan_info": (st, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64)]),
    "ws_batch_plan_destroy": (st, [vp]),
    "ws_batch_run_noalloc": (st, [ctypes.POINTER(WsBatchItem), u64, vp]),
    "ws_server_create": (st, [ctypes.POINTER(WsServerConfig), ctypes.POINTER(vp)]),
    "ws_server_add_table": (st, [vp, u64, i32, i32, i32, ctypes.POINTER(ctypes.c_uint32)]),
    "ws_server_submit": (st, [vp, ctypes.POINTER(WsRequest), ctypes.POINTER(ctypes.c_uint64)]),
    "ws_server_poll": (st, [vp, ctypes.POINTER(WsCompletion), u64, ctypes.POINTER(ctypes.c_uint64), i32]),
    "ws_server_drain": (st, [vp]),
    "ws_server_pause": (st, [vp, i32]),
    "ws_server_table": (st, [vp, ctypes.c_uint32, ctypes.POINTER(vp)]),
    "ws_server_stats": (st, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "ws_server_destroy": (st, [vp]),
    "ws_read_bandwidth": (st, [u64, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_double)]),
    "ws_cuda_error_string": (ctypes.c_char_p, []),
    "ws_status_string": (ctypes.c_char_p, [i32]),
    "ws_version": (u32, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libwarpspeed.so and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L
