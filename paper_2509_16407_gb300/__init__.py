"""GB300-native batched concurrent hash tables (WarpSpeed, arXiv 2509.16407).

Thin Python binding over the C ABI of ``include/warpspeed.h``: argument
marshalling only; every step of an operation runs in the CUDA library.
Batch arguments may be CUDA tensors (the fast path), CPU tensors or numpy
arrays (the library stages them through device buffers).  Keys and values are
64-bit (``torch.int64`` / ``torch.uint64`` / ``numpy.uint64``: the bits are
what counts); per-op status arrays are ``uint8``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

__all__ = ["Table", "WsError", "SCHEMES", "UPSERT_OPS", "MISS", "FOUND", "INSERTED", "FAIL_FULL",
           "FAIL_BADKEY", "FAIL_TIMEOUT", "MX_QUERY", "MX_INSERT", "MX_ADD", "MX_MAX", "MX_REPLACE",
           "MX_ERASE", "lib", "BatchPlan", "BK_INSERT", "BK_UPSERT", "BK_QUERY", "BK_ERASE", "Server"]

SCHEMES = {"double": 0, "p2": 1, "iceberg": 2}
UPSERT_OPS = {"add": 0, "max": 1, "replace": 2, "insert": 3}
MISS, FOUND, INSERTED, FAIL_FULL, FAIL_BADKEY, FAIL_TIMEOUT = range(6)
MX_QUERY, MX_INSERT, MX_ADD, MX_MAX, MX_REPLACE, MX_ERASE = range(6)
BK_INSERT, BK_UPSERT, BK_QUERY, BK_ERASE = range(4)


def lib():
    return _lib.load()


class WsError(RuntimeError):
    def __init__(self, rc: int, what: str):
        L = lib()
        msg = L.ws_status_string(rc).decode()
        if rc == 6:
            msg += ": " + L.ws_cuda_error_string().decode()
        super().__init__(f"{what}: {msg} (status {rc})")
        self.status = rc


def _check(rc: int, what: str):
    if rc != 0:
        raise WsError(rc, what)


def _torch():
    import torch
    return torch


def _is_tensor(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, itemsize=None):
    if x is None:
        return None
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError("batch tensors must be contiguous")
        if itemsize and x.element_size() != itemsize:
            raise TypeError(f"expected {itemsize}-byte elements, got {x.dtype}")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("batch arrays must be C-contiguous")
        if itemsize and x.itemsize != itemsize:
            raise TypeError(f"expected {itemsize}-byte elements, got {x.dtype}")
        return x.ctypes.data
    raise TypeError(f"unsupported batch argument type {type(x)}")


def _numel(x):
    return x.numel() if _is_tensor(x) else x.size


def _empty_like(x, n, kind):
    """Output buffer on the same side as ``x``: kind 'u64' or 'u8'."""
    if _is_tensor(x):
        torch = _torch()
        if kind == "u8":
            dt = torch.uint8
        else:
            dt = x.dtype if x.element_size() == 8 else torch.int64
        return torch.empty(n, dtype=dt, device=x.device, pin_memory=(not x.is_cuda and x.is_pinned()))
    return np.empty(n, dtype=np.uint8 if kind == "u8" else np.uint64)


class Table:
    """A device-resident hash table (one GPU).

    scheme: "double" (DoubleHT), "p2" (P2HT) or "iceberg" (IcebergHT, metadata
    only); metadata: 16-bit fingerprints.
    bucket_slots / tile / max_probe / spin_limit: 0 selects the paper's default.
    """

    def __init__(self, capacity: int, scheme: str = "double", metadata: bool = False, bucket_slots: int = 0,
                 tile: int = 0, max_probe: int = 0, spin_limit: int = 0, device: int = -1):
        L = lib()
        cfg = _lib.WsConfig(int(capacity), SCHEMES[scheme], int(bool(metadata)), int(bucket_slots), int(tile),
                            int(max_probe), int(spin_limit), int(device), 0)
        h = ctypes.c_void_p()
        _check(L.ws_table_create_ex(ctypes.byref(cfg), ctypes.byref(h)), "ws_table_create_ex")
        self._h = h
        self.scheme, self.metadata = scheme, bool(metadata)
        self.device = self.info()["device"]

    # -- lifetime / introspection -------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = _lib.WsInfo()
        _check(lib().ws_table_info_get(self._h, ctypes.byref(inf)), "ws_table_info_get")
        return {n: int(getattr(inf, n)) for n, _ in inf._fields_}

    def _stream(self, stream):
        if stream is None:
            torch = _torch()
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
            return None
        if hasattr(stream, "cuda_stream"):
            return ctypes.c_void_p(stream.cuda_stream)
        return ctypes.c_void_p(int(stream))

    def set_tile(self, tile: int):
        _check(lib().ws_set_tile(self._h, int(tile)), "ws_set_tile")

    def set_spin_limit(self, spins: int):
        _check(lib().ws_set_spin_limit(self._h, int(spins)), "ws_set_spin_limit")

    def set_preload(self, on: bool):
        """The lane path with shared-memory bucket snapshots (on by default); off: tiles only."""
        _check(lib().ws_set_option(self._h, 1, int(bool(on))), "ws_set_option")

    def set_phased(self, on: bool):
        """Bulk-synchronous mode (weak cacheable loads, no locks; distinct keys only)."""
        _check(lib().ws_set_option(self._h, 2, int(bool(on))), "ws_set_option")

    def set_lane_waves(self, n: int):
        """Double hashing: buckets the lane path follows before the tiles (0 = default)."""
        _check(lib().ws_set_option(self._h, 3, int(n)), "ws_set_option")

    def set_stream(self, on):
        """Streaming lanes in single-table calls (True / 1, the default) or 32-op
        chunks (False / 0); 2 also streams plain two-choice queries and erases
        line by line instead of reading whole buckets."""
        _check(lib().ws_set_option(self._h, 4, int(on)), "ws_set_option")

    def set_stage_chunk(self, log2_ops: int):
        """Ops per chunk of the host-buffer staging pipeline, as a power of two (16..24)."""
        _check(lib().ws_set_option(self._h, 6, int(log2_ops)), "ws_set_option")

    def set_host_direct(self, mode: int):
        """Page-locked host buffers: 0 staged, 1 (default) inputs read in place, 2 results written in
        place too, 3 in place for inserts and erases and staged for the other calls."""
        _check(lib().ws_set_option(self._h, 5, int(mode)), "ws_set_option")

    def clear(self, stream=None):
        _check(lib().ws_clear(self._h, self._stream(stream)), "ws_clear")

    def count(self) -> int:
        v = ctypes.c_uint64()
        _check(lib().ws_count(self._h, ctypes.byref(v)), "ws_count")
        return int(v.value)

    def last_error(self) -> dict:
        f, t, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        rc = lib().ws_last_error(self._h, ctypes.byref(f), ctypes.byref(t), ctypes.byref(b))
        if rc == 6:
            raise WsError(rc, "ws_last_error")
        return {"status": rc, "full": int(f.value), "timeout": int(t.value), "badkey": int(b.value)}

    def num_buckets(self) -> int:
        v = ctypes.c_uint64()
        _check(lib().ws_num_buckets(self._h, ctypes.byref(v)), "ws_num_buckets")
        return int(v.value)

    # -- batch operations ------------------------------------------------------------
    def insert(self, keys, vals, return_status=False, stream=None):
        n = _numel(keys)
        stt = _empty_like(keys, n, "u8") if return_status else None
        _check(lib().ws_insert_ex(self._h, _ptr(keys, 8), _ptr(vals, 8), n, _ptr(stt), self._stream(stream)),
               "ws_insert_ex")
        return stt

    def upsert(self, keys, vals, op="add", return_status=False, stream=None):
        n = _numel(keys)
        stt = _empty_like(keys, n, "u8") if return_status else None
        code = UPSERT_OPS[op] if isinstance(op, str) else int(op)
        _check(lib().ws_upsert_ex(self._h, _ptr(keys, 8), _ptr(vals, 8), n, code, _ptr(stt),
                                  self._stream(stream)), "ws_upsert_ex")
        return stt

    def query(self, keys, return_status=False, out=None, stream=None):
        n = _numel(keys)
        vals = out if out is not None else _empty_like(keys, n, "u64")
        stt = _empty_like(keys, n, "u8") if return_status else None
        _check(lib().ws_query_ex(self._h, _ptr(keys, 8), _ptr(vals, 8), _ptr(stt), n, self._stream(stream)),
               "ws_query_ex")
        return (vals, stt) if return_status else vals

    def erase(self, keys, return_values=False, return_status=False, stream=None):
        n = _numel(keys)
        vals = _empty_like(keys, n, "u64") if return_values else None
        stt = _empty_like(keys, n, "u8") if return_status else None
        _check(lib().ws_erase_ex(self._h, _ptr(keys, 8), _ptr(vals, 8), _ptr(stt), n, self._stream(stream)),
               "ws_erase_ex")
        return vals, stt

    def mixed(self, ops, keys, vals=None, return_values=True, return_status=True, stream=None):
        n = _numel(keys)
        vo = _empty_like(keys, n, "u64") if return_values else None
        stt = _empty_like(keys, n, "u8") if return_status else None
        _check(lib().ws_mixed(self._h, _ptr(ops, 1), _ptr(keys, 8), _ptr(vals, 8), _ptr(vo, 8), _ptr(stt), n,
                              self._stream(stream)), "ws_mixed")
        return vo, stt

    def probe_cost(self, keys, stream=None):
        """Per-key (cache lines, DRAM sectors) a query touches now (no change)."""
        n = _numel(keys)
        out = _empty_like(keys, n, "u64")
        stt = _empty_like(keys, n, "u8")
        _check(lib().ws_probe_cost(self._h, _ptr(keys, 8), _ptr(out, 8), _ptr(stt), n, self._stream(stream)),
               "ws_probe_cost")
        return out, stt

    # -- hooks ------------------------------------------------------------------------
    def primary_bucket(self, keys, stream=None):
        n = _numel(keys)
        out = _empty_like(keys, n, "u64")
        _check(lib().ws_primary_bucket(self._h, _ptr(keys, 8), _ptr(out, 8), n, self._stream(stream)),
               "ws_primary_bucket")
        return out

    def rehash_into(self, dst: "Table", return_status=False, stream=None):
        """Insert every live pair of this table into ``dst`` (growth step)."""
        stt = None
        if return_status:
            torch = _torch()
            stt = torch.empty(self.info()["slots"], dtype=torch.uint8, device=f"cuda:{self.device}")
        _check(lib().ws_rehash(self._h, dst._h, _ptr(stt), self._stream(stream)), "ws_rehash")
        return stt

    def dump(self):
        """(slots u64[S, 2] as (key, value), tags u16[S] or None) on the host."""
        inf = self.info()
        S = inf["slots"]
        slots = np.empty((S, 2), dtype=np.uint64)
        tags = np.empty(S, dtype=np.uint16) if inf["metadata"] else None
        _check(lib().ws_dump(self._h, slots.ctypes.data, None if tags is None else tags.ctypes.data), "ws_dump")
        return slots, tags

    def debug_fill_locks(self, locked: bool, stream=None):
        _check(lib().ws_debug_fill_locks(self._h, int(bool(locked)), self._stream(stream)),
               "ws_debug_fill_locks")


class BatchPlan:
    """Many tables' op batches in one persistent launch per phase, captured
    into a CUDA graph.  ``items``: iterables of (table, kind, keys, vals,
    vals_out, status_out, phase[, op]) with CUDA tensors (or None)."""

    def __init__(self, items):
        arr = (_lib.WsBatchItem * len(items))()
        self._keep = []
        for i, it in enumerate(items):
            table, kind, keys, vals, vals_out, status_out, phase = it[:7]
            op = it[7] if len(it) > 7 else 0
            op = UPSERT_OPS[op] if isinstance(op, str) else int(op)
            self._keep.append((table, keys, vals, vals_out, status_out))
            arr[i] = _lib.WsBatchItem(table.handle.value if hasattr(table.handle, "value") else table.handle,
                                      int(kind), op, int(phase), 0, _ptr(keys, 8), _ptr(vals, 8),
                                      _ptr(vals_out, 8), _ptr(status_out), _numel(keys))
        h = ctypes.c_void_p()
        _check(lib().ws_batch_plan_create(arr, len(items), ctypes.byref(h)), "ws_batch_plan_create")
        self._h = h
        self._device = items[0][0].device

    def launch(self, stream=None):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream(self._device)
        _check(lib().ws_batch_plan_launch(self._h, ctypes.c_void_p(s.cuda_stream)), "ws_batch_plan_launch")

    def info(self):
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().ws_batch_plan_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "ws_batch_plan_info")
        return {"phases": a.value, "chunks": b.value, "fallback_items": c.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().ws_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over device-resident tables.

    Requests are mixed op batches on one table with host buffers (numpy
    arrays; pinned memory is fastest).  ``submit`` returns at once; outputs
    are filled in when ``poll`` / ``drain`` report the request complete.
    """

    def __init__(self, max_inflight=4, max_batch_ops=1 << 22, max_batch_reqs=256, plain=False,
                 hbm_headroom=0.05, grow_at=0.85, device=-1):
        cfg = _lib.WsServerConfig(int(device), int(max_inflight), int(max_batch_ops), int(max_batch_reqs),
                                  int(bool(plain)), float(hbm_headroom), float(grow_at))
        h = ctypes.c_void_p()
        _check(lib().ws_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ws_server_create")
        self._h = h
        self._live = {}
        self._done = {}

    def add_table(self, capacity, scheme="double", metadata=False, tile=0) -> int:
        i = ctypes.c_uint32()
        _check(lib().ws_server_add_table(self._h, int(capacity), SCHEMES[scheme], int(bool(metadata)), int(tile),
                                         ctypes.byref(i)), "ws_server_add_table")
        return int(i.value)

    def submit(self, table, ops, keys, vals=None, want_values=True, want_status=True, tag=0,
               vals_out=None, status_out=None) -> int:
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys = np.ascontiguousarray(keys).view(np.uint64)
        if vals is not None:
            vals = np.ascontiguousarray(vals).view(np.uint64)
        n = keys.size
        vo = vals_out if vals_out is not None else (np.empty(n, np.uint64) if want_values else None)
        so = status_out if status_out is not None else (np.empty(n, np.uint8) if want_status else None)
        req = _lib.WsRequest(int(table), 0, _ptr(ops), _ptr(keys), _ptr(vals), _ptr(vo), _ptr(so), n, int(tag))
        rid = ctypes.c_uint64()
        _check(lib().ws_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)), "ws_server_submit")
        self._live[int(rid.value)] = (ops, keys, vals, vo, so)
        return int(rid.value)

    def poll(self, max_n=4096, wait_ms=0):
        buf = (_lib.WsCompletion * max_n)()
        n = ctypes.c_uint64()
        _check(lib().ws_server_poll(self._h, buf, max_n, ctypes.byref(n), int(wait_ms)), "ws_server_poll")
        out = []
        for i in range(n.value):
            c = buf[i]
            ops, keys, vals, vo, so = self._live.pop(int(c.id))
            out.append({"id": int(c.id), "tag": int(c.tag), "t_submit": c.t_submit, "t_start": c.t_start,
                        "t_done": c.t_done, "status": int(c.status), "table": int(c.table), "vals": vo,
                        "st": so})
        return out

    def pause(self, paused=True):
        _check(lib().ws_server_pause(self._h, int(bool(paused))), "ws_server_pause")

    def drain(self):
        _check(lib().ws_server_drain(self._h), "ws_server_drain")
        res = []
        while True:
            got = self.poll()
            if not got:
                break
            res += got
        return res

    def table_handle(self, tid):
        h = ctypes.c_void_p()
        _check(lib().ws_server_table(self._h, int(tid), ctypes.byref(h)), "ws_server_table")
        return h

    def count(self, tid) -> int:
        v = ctypes.c_uint64()
        _check(lib().ws_count(self.table_handle(tid), ctypes.byref(v)), "ws_count")
        return int(v.value)

    def dump(self, tid):
        h = self.table_handle(tid)
        inf = _lib.WsInfo()
        _check(lib().ws_table_info_get(h, ctypes.byref(inf)), "ws_table_info_get")
        slots = np.empty((inf.slots, 2), dtype=np.uint64)
        tags = np.empty(inf.slots, dtype=np.uint16) if inf.metadata else None
        _check(lib().ws_dump(h, slots.ctypes.data, None if tags is None else tags.ctypes.data), "ws_dump")
        return slots, tags

    def stats(self):
        a, b, c, d = (ctypes.c_uint64() for _ in range(4))
        _check(lib().ws_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
               "ws_server_stats")
        return {"submitted": a.value, "completed": b.value, "launches": c.value, "grows": d.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().ws_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
