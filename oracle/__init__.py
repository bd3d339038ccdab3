"""CPU oracle for the batched hash-table path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The library (``paper_2509_16407_gb300``) never
imports it and shares no code with it.

The oracle is the plain map definition of the paper's API (WarpSpeed §5.1:
Upsert with a callback, Query, Erase) applied batch by batch with per-batch
phase semantics; see ``ws_oracle.cpp`` for the rules.  Its layout checker
re-derives legal placements from the written hash/probe specification.

Parity status: the map semantics are pinned (brute force, closed forms and
invariants in ``tests/test_oracle_pins.py``); the layout checker and the
probe-count recount are pinned by planted layouts with hand-counted results in
the same file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ws_oracle.cpp")
_LIB = os.path.join(_HERE, "libws_oracle.so")

# Documented status / op-code values of the library interface.
MISS, FOUND, INSERTED, FULL, BAD_KEY, TIMEOUT = 0, 1, 2, 3, 4, 5
UP_INSERT, UP_ADD, UP_MAX, UP_REPLACE = -1, 0, 1, 2
MX_QUERY, MX_INSERT, MX_ADD, MX_MAX, MX_REPLACE, MX_ERASE = 0, 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no CUDA involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Report(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "live", "tomb", "empty", "resv", "bad_bucket", "duplicates",
        "tag_mismatch", "early_exit", "empty_not_suffix")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.ora_new.restype = vp
        L.ora_free.argtypes = [vp]
        L.ora_count.argtypes = [vp]
        L.ora_count.restype = u64
        L.ora_clear.argtypes = [vp]
        L.ora_upsert.argtypes = [vp, vp, vp, u64, i32, vp]
        L.ora_insert.argtypes = [vp, vp, vp, u64, vp]
        L.ora_query.argtypes = [vp, vp, vp, vp, u64]
        L.ora_erase.argtypes = [vp, vp, vp, vp, u64]
        L.ora_mixed.argtypes = [vp, vp, vp, vp, vp, vp, u64]
        L.ora_items.argtypes = [vp, vp, vp]
        L.ora_load.argtypes = [vp, vp, vp, u64]
        L.ora_layout_check.argtypes = [vp, vp, u64, u64, i32, u64, u64, u64,
                                       ctypes.POINTER(_Report)]
        L.ora_layout_check.restype = i32
        L.ora_candidates_full.argtypes = [vp, vp, u64, u64, i32, u64, u64, u64, vp, u64, vp]
        L.ora_primary_bucket.argtypes = [vp, u64, u64, u64, vp]
        L.ora_iceberg_buckets.argtypes = [vp, u64, u64, u64, u64, vp]
        L.ora_probe_cost.argtypes = [vp, vp, u64, u64, i32, u64, u64, u64, u64, i32, vp, u64, vp, vp]
        L.ora_probe_cost.restype = i32
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


class OracleMap:
    """Single-threaded CPU map with the paper's API semantics."""

    def __init__(self):
        self._h = lib().ora_new()

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ora_free(self._h)
            self._h = None

    def count(self) -> int:
        return int(lib().ora_count(self._h))

    def clear(self):
        lib().ora_clear(self._h)

    def insert(self, keys, vals):
        k, v = _u64(keys), _u64(vals)
        st = np.empty(k.size, np.uint8)
        lib().ora_insert(self._h, _p(k), _p(v), k.size, _p(st))
        return st

    def upsert(self, keys, vals, op: int):
        k, v = _u64(keys), _u64(vals)
        st = np.empty(k.size, np.uint8)
        lib().ora_upsert(self._h, _p(k), _p(v), k.size, int(op), _p(st))
        return st

    def query(self, keys):
        k = _u64(keys)
        out = np.empty(k.size, np.uint64)
        st = np.empty(k.size, np.uint8)
        lib().ora_query(self._h, _p(k), _p(out), _p(st), k.size)
        return out, st

    def erase(self, keys):
        k = _u64(keys)
        out = np.empty(k.size, np.uint64)
        st = np.empty(k.size, np.uint8)
        lib().ora_erase(self._h, _p(k), _p(out), _p(st), k.size)
        return out, st

    def mixed(self, ops, keys, vals):
        o = np.ascontiguousarray(ops, dtype=np.uint8)
        k, v = _u64(keys), _u64(vals)
        out = np.empty(k.size, np.uint64)
        st = np.empty(k.size, np.uint8)
        lib().ora_mixed(self._h, _p(o), _p(k), _p(v), _p(out), _p(st), k.size)
        return out, st

    def items(self):
        n = self.count()
        k = np.empty(n, np.uint64)
        v = np.empty(n, np.uint64)
        lib().ora_items(self._h, _p(k), _p(v))
        return k, v

    def load(self, keys, vals):
        k, v = _u64(keys), _u64(vals)
        lib().ora_load(self._h, _p(k), _p(v), k.size)


def layout_check(slots, tags, nb, B, scheme, pmax, seed1, seed2) -> dict:
    """Structural check of a dumped table; ``slots`` is u64[2*S] (key, val)."""
    s = _u64(slots)
    t = None if tags is None else np.ascontiguousarray(tags, dtype=np.uint16)
    r = _Report()
    rc = lib().ora_layout_check(_p(s), _p(t), nb, B, scheme, pmax, seed1, seed2,
                                ctypes.byref(r))
    if rc != 0:
        raise ValueError("layout_check: bad geometry")
    return r.as_dict()


def candidates_full(slots, tags, nb, B, scheme, pmax, seed1, seed2, keys):
    s = _u64(slots)
    t = None if tags is None else np.ascontiguousarray(tags, dtype=np.uint16)
    k = _u64(keys)
    out = np.empty(k.size, np.uint8)
    lib().ora_candidates_full(_p(s), _p(t), nb, B, scheme, pmax, seed1, seed2,
                              _p(k), k.size, _p(out))
    return out.astype(bool)


def probe_cost(slots, tags, nb, B, scheme, pmax, seed1, seed2, tile, never_erased, keys):
    """Host recount of the probe count (cache lines, 32-byte sectors) a query
    of each key pays on a dumped table, and whether the key is present.
    Returns (lines u64[n], sectors u64[n], found bool[n])."""
    s = _u64(slots)
    t = None if tags is None else np.ascontiguousarray(tags, dtype=np.uint16)
    k = _u64(keys)
    cost = np.empty(k.size, np.uint64)
    found = np.empty(k.size, np.uint8)
    rc = lib().ora_probe_cost(_p(s), _p(t), nb, B, scheme, pmax, seed1, seed2, tile, int(bool(never_erased)),
                              _p(k), k.size, _p(cost), _p(found))
    if rc != 0:
        raise ValueError("probe_cost: bad geometry")
    return cost >> np.uint64(32), cost & np.uint64(0xFFFFFFFF), found.astype(bool)


def primary_bucket(keys, nb, seed1):
    k = _u64(keys)
    out = np.empty(k.size, np.uint64)
    lib().ora_primary_bucket(_p(k), k.size, nb, seed1, _p(out))
    return out


def iceberg_buckets(keys, nb, seed1, seed2):
    """(front, back_1, back_2) bucket of each key under the iceberg geometry."""
    k = _u64(keys)
    out = np.empty((k.size, 3), np.uint64)
    lib().ora_iceberg_buckets(_p(k), k.size, nb, seed1, seed2, _p(out))
    return out


def primary_bucket_of(scheme, keys, nb, seed1, seed2):
    """The bucket whose lock serialises inserters of a key: b_0, or the
    front-yard bucket for iceberg."""
    if scheme == 2:
        return iceberg_buckets(keys, nb, seed1, seed2)[:, 0].copy()
    return primary_bucket(keys, nb, seed1)
