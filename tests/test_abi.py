"""The C-ABI library builds, loads and exports every symbol the header
declares; host-side argument checks that need no GPU.  No GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "warpspeed.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ws_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2509_16407_gb300 import build as b
    b.build()
    from paper_2509_16407_gb300 import _lib
    return _lib.load()


def test_header_declares_core_api():
    names = _declared()
    for n in ("ws_table_create", "ws_insert", "ws_upsert", "ws_query", "ws_erase", "ws_count",
              "ws_destroy", "ws_mixed", "ws_last_error", "ws_dump", "ws_primary_bucket"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert missing == []


def test_binding_declares_every_header_symbol():
    from paper_2509_16407_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_host_side_checks_without_gpu(L):
    assert L.ws_version() == 0x000100
    h = ctypes.c_void_p()
    # invalid configurations are rejected before any CUDA call
    assert L.ws_table_create(0, 0, 0, ctypes.byref(h)) == 1
    assert L.ws_table_create(1 << 20, 7, 0, ctypes.byref(h)) == 1
    from paper_2509_16407_gb300 import _lib
    cfg = _lib.WsConfig(1 << 20, 0, 1, 8, 8, 0, 0, -1, 0)  # metadata needs 32-slot buckets
    assert L.ws_table_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg = _lib.WsConfig(1 << 20, 1, 0, 32, 12, 0, 0, -1, 0)  # tile 12
    assert L.ws_table_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == 1
    # null table handles
    assert L.ws_insert(None, None, None, 0, None) == 1
    assert L.ws_count(None, None) == 1
    assert L.ws_destroy(None) == 1
    assert L.ws_set_option(None, 5, 1) == 1  # WS_OPT_HOST_DIRECT on a null table
    assert L.ws_status_string(4) == b"an insert found no free slot"
