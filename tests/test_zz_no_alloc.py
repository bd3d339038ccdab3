"""ws_batch_run_noalloc: batched mode for callers that cannot allocate device
memory (a framework's caching allocator holds it all, memory reserved up
front, or a loop that cannot take cudaFree's device-wide synchronisation).
Its results must equal those of the allocating entry point (ws_batch_plan_*)
on the same items, bit for bit, on two calls in a row that reuse the
library's fixed scratch array, and the oracle's.  This file is collected last
on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

# table configurations: the first five run in the persistent kernel, the last
# one (16-slot buckets) as a separate kernel
CONFIGS = [("double", False, 8, 8), ("double", True, 32, 4), ("p2", False, 32, 8), ("p2", True, 32, 4),
           ("double", False, 8, 4), ("double", False, 16, 8)]


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


def _items(ws, tables, specs):
    """ctypes item array for (table index, kind, keys, vals, vals_out, status_out, phase, op)."""
    from paper_2509_16407_gb300 import _lib
    arr = (_lib.WsBatchItem * len(specs))()
    for i, (ti, kind, k, v, vo, so, ph, op) in enumerate(specs):
        arr[i] = _lib.WsBatchItem(tables[ti].handle.value, kind, op, ph, 0, k.data_ptr(),
                                  v.data_ptr() if v is not None else None,
                                  vo.data_ptr() if vo is not None else None,
                                  so.data_ptr() if so is not None else None, k.numel())
    return arr


def _outputs(specs):
    return [(x[4], x[5]) for x in specs]


def _make_specs(ws, round_no, n_tab):
    import torch
    specs_in, keep = [], []
    for i in range(n_tab):
        keys = W.distinct_keys(9000 + 31 * i, 1200)
        ins = keys[:900]
        q = np.concatenate([ins[::3], keys[900:]])
        kd, qd = dev(ins), dev(q)
        if round_no == 0:
            vd = dev(W.splitmix64(77 + i, ins.size))
            specs_in.append((i, ws.BK_INSERT, kd, vd, None, "st", 0, 0))
            specs_in.append((i, ws.BK_QUERY, qd, None, "v", "st", 1, 0))
        else:
            vd = dev(W.uniform_int(88 + i, ins.size, 1, 1000))
            er = dev(ins[::5])
            specs_in.append((i, ws.BK_UPSERT, kd, vd, None, "st", 0, ws.UPSERT_OPS["add"]))
            specs_in.append((i, ws.BK_ERASE, er, None, "v", "st", 1, 0))
            specs_in.append((i, ws.BK_QUERY, qd, None, "v", "st", 2, 0))
        keep.append((kd, vd, qd))
    return specs_in, keep


def _realise(specs_in):
    import torch
    out = []
    for (ti, kind, k, v, vo, so, ph, op) in specs_in:
        vo_t = torch.empty(k.numel(), dtype=torch.int64, device="cuda") if vo else None
        so_t = torch.full((k.numel(),), 255, dtype=torch.uint8, device="cuda") if so else None
        out.append((ti, kind, k, v, vo_t, so_t, ph, op))
    return out


def _oracle_check(oracle_mod, oms, specs):
    """Apply each table's items phase by phase to its oracle map and compare
    the no-alloc call's outputs (the items' keys are distinct per item)."""
    for (ti, kind, k, v, vo, so, ph, op) in sorted(specs, key=lambda x: (x[6], x[0])):
        om = oms[ti]
        keys = host(k)
        if kind == 0:
            wst, wv = om.insert(keys, host(v)), None
        elif kind == 1:
            wst, wv = om.upsert(keys, host(v), op), None
        elif kind == 2:
            wv, wst = om.query(keys)
        else:
            wv, wst = om.erase(keys)
        if so is not None:
            assert (host(so) == wst).all(), (ti, kind, ph)
        if vo is not None:
            assert (host(vo) == wv).all(), (ti, kind, ph)


def test_noalloc_matches_plan_on_two_calls(ws, oracle_mod):
    import torch
    L = ws.lib()
    n_tab = len(CONFIGS) * 2
    A = [ws.Table(1 << 12, *CONFIGS[i % len(CONFIGS)][:2], bucket_slots=CONFIGS[i % len(CONFIGS)][2],
                  tile=CONFIGS[i % len(CONFIGS)][3]) for i in range(n_tab)]
    B = [ws.Table(1 << 12, *CONFIGS[i % len(CONFIGS)][:2], bucket_slots=CONFIGS[i % len(CONFIGS)][2],
                  tile=CONFIGS[i % len(CONFIGS)][3]) for i in range(n_tab)]
    stream = torch.cuda.current_stream().cuda_stream
    oms = [oracle_mod.OracleMap() for _ in range(n_tab)]
    for round_no in range(2):  # two calls in a row, different item layouts
        specs_in, keep = _make_specs(ws, round_no, n_tab)
        sa, sb = _realise(specs_in), _realise(specs_in)
        rc = L.ws_batch_run_noalloc(_items(ws, A, sa), len(sa), ctypes.c_void_p(stream))
        assert rc == 0, L.ws_cuda_error_string()
        h = ctypes.c_void_p()
        assert L.ws_batch_plan_create(_items(ws, B, sb), len(sb), ctypes.byref(h)) == 0
        assert L.ws_batch_plan_launch(h, ctypes.c_void_p(stream)) == 0
        torch.cuda.synchronize()
        for (x, y) in zip(sa, sb):
            for ta, tb in ((x[4], y[4]), (x[5], y[5])):
                if ta is not None:
                    assert torch.equal(ta, tb), (round_no, x[0], x[1])
            if x[5] is not None:
                assert (host(x[5]) != 255).all()
        _oracle_check(oracle_mod, oms, sa)
        for ta, tb, om in zip(A, B, oms):
            assert ta.count() == tb.count() == om.count()
        assert L.ws_batch_plan_destroy(h) == 0


def test_noalloc_takes_no_device_memory(ws):
    """After a first call (which looks up the scratch array and loads the
    kernels), further calls leave the device's free memory unchanged."""
    import torch
    L = ws.lib()
    n_tab = len(CONFIGS)
    A = [ws.Table(1 << 12, *CONFIGS[i][:2], bucket_slots=CONFIGS[i][2], tile=CONFIGS[i][3]) for i in range(n_tab)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    specs_in, keep = _make_specs(ws, 0, n_tab)
    sa = _realise(specs_in)
    arr = _items(ws, A, sa)
    assert L.ws_batch_run_noalloc(arr, len(sa), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert L.ws_batch_run_noalloc(arr, len(sa), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_oversized_calls(ws):
    from paper_2509_16407_gb300 import _lib
    import torch
    L = ws.lib()
    t = ws.Table(1 << 10)
    k = dev(W.distinct_keys(1, 4))
    arr = (_lib.WsBatchItem * 1025)()
    for i in range(1025):
        arr[i] = _lib.WsBatchItem(t.handle.value, ws.BK_QUERY, 0, 0, 0, k.data_ptr(), None, k.data_ptr(), None, 4)
    assert L.ws_batch_run_noalloc(arr, 1025, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 1
    assert b"maximum of 1024" in L.ws_cuda_error_string()
    # 17 distinct phases (empty items are enough): rejected with its reason
    arr = (_lib.WsBatchItem * 17)()
    for i in range(17):
        arr[i] = _lib.WsBatchItem(t.handle.value, ws.BK_QUERY, 0, i, 0, k.data_ptr(), None, k.data_ptr(), None, 0)
    assert L.ws_batch_run_noalloc(arr, 17, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 1
    assert b"more than 16 distinct phases" in L.ws_cuda_error_string()
    # 16 are accepted
    assert L.ws_batch_run_noalloc(arr, 16, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
