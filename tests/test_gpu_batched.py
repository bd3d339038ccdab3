"""Batched mode: many tables of uneven sizes in one persistent launch per
phase, captured in a CUDA graph; per-table results must equal the oracle's
and the per-table launches'.  Needs a GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import check_layout, dev, host

pytestmark = pytest.mark.gpu

# (scheme, metadata, bucket_slots, tile): the first eight are in the compiled
# menu of the persistent kernel, the last two run as fallback kernels.
CONFIGS = [("double", False, 8, 4), ("double", False, 8, 8), ("double", True, 32, 4), ("double", True, 32, 8),
           ("p2", False, 32, 8), ("p2", False, 32, 32), ("p2", True, 32, 4), ("p2", True, 32, 8),
           ("double", False, 16, 8), ("p2", False, 8, 4)]


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


def _workload(n_tables, lo_cap, hi_cap, lo_ops, hi_ops, seed):
    caps = W.log_uniform_int(seed, n_tables, lo_cap, hi_cap)
    ops = W.log_uniform_int(seed + 1, n_tables, lo_ops, hi_ops)
    out = []
    for i in range(n_tables):
        n_ins = int(min(ops[i] // 2, int(0.85 * caps[i])))
        n_q = int(ops[i] - n_ins)
        keys = W.distinct_keys(seed * 7919 + i, n_ins + n_q // 2)
        ins, neg = keys[:n_ins], keys[n_ins:]
        pos = ins[W.splitmix64(seed + 31 * i, n_q - n_q // 2) % np.uint64(max(n_ins, 1))] if n_ins else \
            W.distinct_keys(seed + 99, n_q - n_q // 2, start=1 << 40)
        q = np.concatenate([pos, neg])
        out.append((int(caps[i]), ins, W.splitmix64(seed + 17 * i, n_ins), q))
    return out


def test_batched_plan_matches_oracle_and_plain_launches(ws, oracle_mod):
    import torch
    wl = _workload(40, 1 << 10, 1 << 16, 1 << 8, 1 << 14, 5)
    tables, plain, items, outs, refs = [], [], [], [], []
    for i, (cap, ins, vals, q) in enumerate(wl):
        sch, meta, B, T = CONFIGS[i % len(CONFIGS)]
        t = ws.Table(cap, sch, meta, bucket_slots=B, tile=T)
        u = ws.Table(cap, sch, meta, bucket_slots=B, tile=T)
        kd, vd, qd = dev(ins), dev(vals), dev(q)
        st_ins = torch.empty(ins.size, dtype=torch.uint8, device="cuda")
        qv = torch.empty(q.size, dtype=torch.int64, device="cuda")
        qs = torch.empty(q.size, dtype=torch.uint8, device="cuda")
        items.append((t, ws.BK_INSERT, kd, vd, None, st_ins, 0))
        items.append((t, ws.BK_QUERY, qd, None, qv, qs, 1))
        outs.append((st_ins, qv, qs))
        tables.append(t)
        plain.append((u, kd, vd, qd))
    plan = ws.BatchPlan(items)
    inf = plan.info()
    assert inf["phases"] == 2 and inf["fallback_items"] == 2 * sum(
        1 for i in range(len(wl)) if CONFIGS[i % len(CONFIGS)] in CONFIGS[8:])
    plan.launch()
    torch.cuda.synchronize()
    for i, (cap, ins, vals, q) in enumerate(wl):
        om = oracle_mod.OracleMap()
        wst = om.insert(ins, vals)
        wv, wq = om.query(q)
        st_ins, qv, qs = outs[i]
        full = host(st_ins) == ws.FAIL_FULL
        assert not full.any()
        assert (host(st_ins) == wst).all(), i
        assert (host(qv) == wv).all() and (host(qs) == wq).all(), i
        assert tables[i].count() == om.count()
        check_layout(oracle_mod, tables[i], om.count())
        # the same ops through per-table launches give the same results
        u, kd, vd, qd = plain[i]
        s2 = u.insert(kd, vd, return_status=True)
        v2, q2 = u.query(qd, return_status=True)
        assert (host(s2) == host(st_ins)).all() and (host(v2) == host(qv)).all() and (host(q2) == host(qs)).all()
    # a second launch replays the graph: inserts now find their keys, queries repeat
    plan.launch()
    torch.cuda.synchronize()
    for i, (cap, ins, vals, q) in enumerate(wl):
        st_ins, qv, qs = outs[i]
        assert (host(st_ins) == ws.FOUND).all()
        assert tables[i].count() == ins.size
    plan.close()


def test_batched_upsert_and_erase_phases(ws, oracle_mod):
    """Phase 0 upsert-add (with duplicates), phase 1 erase half + query the
    rest; the plan is rebuilt when a table it allowed the two-choice shortcut
    on gets erased."""
    import torch
    rng_tables = []
    items = []
    expect = []
    for i, (sch, meta, B, T) in enumerate(CONFIGS):
        t = ws.Table(1 << 12, sch, meta, bucket_slots=B, tile=T)
        base = W.distinct_keys(400 + i, 1500)
        keys = np.concatenate([base, base[:300]])
        vals = W.uniform_int(500 + i, keys.size, 1, 1000)
        er, qk = base[:700], base[700:]
        kd, vd, ed, qd = dev(keys), dev(vals), dev(er), dev(qk)
        ust = torch.empty(keys.size, dtype=torch.uint8, device="cuda")
        ev = torch.empty(er.size, dtype=torch.int64, device="cuda")
        es = torch.empty(er.size, dtype=torch.uint8, device="cuda")
        qv = torch.empty(qk.size, dtype=torch.int64, device="cuda")
        items += [(t, ws.BK_UPSERT, kd, vd, None, ust, 0, "add"), (t, ws.BK_ERASE, ed, None, ev, es, 1),
                  (t, ws.BK_QUERY, qd, None, qv, None, 1)]
        om = oracle_mod.OracleMap()
        wst = om.upsert(keys, vals, 0)
        wev, wes = om.erase(er)
        wqv, _ = om.query(qk)
        expect.append((t, keys, ust, wst, ev, es, wev, wes, qv, wqv, om.count()))
        rng_tables.append(t)
    plan = ws.BatchPlan(items)
    plan.launch()
    torch.cuda.synchronize()
    for (t, keys, ust, wst, ev, es, wev, wes, qv, wqv, cnt) in expect:
        g = host(ust)
        # per key: exactly one INSERTED; the rest FOUND (order inside a phase is free)
        ins_keys = keys[g == ws.INSERTED]
        assert np.unique(ins_keys).size == ins_keys.size == np.unique(keys).size
        assert ((g == ws.INSERTED) | (g == ws.FOUND)).all()
        assert (host(ev) == wev).all() and (host(es) == wes).all()
        assert (host(qv) == wqv).all()
        assert t.count() == cnt
        check_layout(oracle_mod, t, cnt)
    plan.close()
