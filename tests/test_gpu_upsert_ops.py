"""Upsert callbacks of §5.1 beyond add -- max and replace -- and the
insert-if-unique code, at batch scale, against the oracle: seeded batches of
present and absent keys on every design; 32 copies per key, contiguous and
shuffled (max exact; replace and insert leave one copy whose value is one of
the values supplied for that key); mixed batches that use every op code; and
the same callbacks through the batched plans and the serving loop.  Needs a
GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import DESIGNS, DESIGN_IDS, check_layout, dev, host

pytestmark = pytest.mark.gpu

UP = {"max": 1, "replace": 2}


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


def _state(t):
    slots, tags = t.dump()
    k = slots[:, 0]
    live = (k != 0) & (k < np.uint64((1 << 64) - 2))
    if tags is not None:
        live &= tags >= 2
    o = np.argsort(k[live])
    return k[live][o], slots[:, 1][live][o]


def _multiset(*cols):
    a = np.stack([np.asarray(c, np.uint64) for c in cols], 1)
    return a[np.lexsort(a.T[::-1])]


def _allowed_values(keys, vals):
    """key -> set of values supplied for it."""
    d = {}
    for k, v in zip(keys.tolist(), vals.tolist()):
        d.setdefault(k, set()).add(v)
    return d


@pytest.mark.parametrize("op", ["max", "replace"])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_upsert_distinct_keys_match_oracle(ws, oracle_mod, scheme, meta, op):
    """2^17 distinct keys, half present (0.6 load) and half absent."""
    S = 1 << 18
    t = ws.Table(S, scheme, meta)
    n0 = int(0.6 * S)
    both = W.distinct_keys(8800 + UP[op], n0 + (1 << 16))
    base, new = both[:n0], both[n0:]
    bvals = W.uniform_int(8801, n0, 1, 1 << 40)
    om = oracle_mod.OracleMap()
    assert (host(t.insert(dev(base), dev(bvals), return_status=True)) == om.insert(base, bvals)).all()
    keys = np.concatenate([base[W.permutation(8802, n0)[: 1 << 16]], new])
    keys = keys[W.permutation(8803, keys.size)]
    vals = W.uniform_int(8804, keys.size, 1, 1 << 40)
    st = host(t.upsert(dev(keys), dev(vals), op=op, return_status=True))
    assert (st == om.upsert(keys, vals, UP[op])).all()
    assert (st == ws.INSERTED).sum() == 1 << 16
    assert t.count() == om.count()
    gk, gv = _state(t)
    ok, ov = om.items()
    assert (gk == ok).all() and (gv == ov).all()
    check_layout(oracle_mod, t, om.count())
    assert t.last_error()["status"] == 0


@pytest.mark.parametrize("layout", ["contiguous", "shuffled"])
@pytest.mark.parametrize("op", ["max", "replace", "insert"])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_upsert_32_copies_per_key(ws, oracle_mod, scheme, meta, op, layout):
    """32 copies of each key in one batch, each with its own value; half the
    keys present before the batch."""
    n = 1 << 12
    base = W.distinct_keys(9100 + len(op), n)
    pre = base[: n // 2]
    pvals = W.uniform_int(9101, pre.size, 1, 1 << 40)
    t = ws.Table(1 << 15, scheme, meta)
    om = oracle_mod.OracleMap()
    t.insert(dev(pre), dev(pvals))
    om.insert(pre, pvals)
    keys = np.repeat(base, 32)
    if layout == "shuffled":
        keys = keys[W.permutation(9102, keys.size)]
    vals = W.uniform_int(9103, keys.size, 1, 1 << 40)
    code = {"max": 1, "replace": 2, "insert": 3}[op]
    st = host(t.upsert(dev(keys), dev(vals), op=op, return_status=True))
    wst = om.upsert(keys, vals, code if op != "insert" else -1)
    # statuses: per key, one INSERTED copy for absent keys, FOUND for the rest
    assert (_multiset(keys, st) == _multiset(keys, wst)).all()
    assert np.unique(keys[st == ws.INSERTED]).size == (st == ws.INSERTED).sum() == n - n // 2
    assert t.count() == om.count() == n
    gk, gv = _state(t)
    ok, ov = om.items()
    assert (gk == ok).all()
    if op == "max":
        assert (gv == ov).all()  # max is commutative: exact
    else:
        allowed = _allowed_values(keys, vals)
        prev = dict(zip(pre.tolist(), pvals.tolist()))
        for k, v in zip(gk.tolist(), gv.tolist()):
            if op == "insert" and k in prev:
                assert v == prev[k]  # insert-if-unique keeps the old value
            else:
                assert v in allowed[k]
        # the oracle took the last copy; any supplied copy is valid
        om.load(gk, gv)
    v, s = t.query(dev(base), return_status=True)
    wv, wsx = om.query(base)
    assert (host(v) == wv).all() and (host(s) == wsx).all()
    check_layout(oracle_mod, t, n)


@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_mixed_batches_with_every_code(ws, oracle_mod, scheme, meta):
    """Zipf mixed batches of query / insert / add / max / replace / erase;
    each key has one code per batch."""
    t = ws.Table(1 << 18, scheme, meta)
    om = oracle_mod.OracleMap()
    for b in range(4):
        ops, keys, vals = W.mixed_batch_codes(500 + b, n_ops=1 << 17, universe=1 << 15)
        before_v, before_s = om.query(keys)
        gv, gs = t.mixed(dev(ops), dev(keys), dev(vals))
        gv, gs = host(gv), host(gs)
        ov, os_ = om.mixed(ops, keys, vals)
        q = ops == W.MX_QUERY
        assert (gv[q] == ov[q]).all() and (gs[q] == os_[q]).all()
        for cls in (W.MX_ERASE, W.MX_ADD, W.MX_MAX, W.MX_REPLACE, W.MX_INSERT):
            m = ops == cls
            assert (_multiset(keys[m], gs[m], gv[m]) == _multiset(keys[m], os_[m], ov[m])).all(), cls
        assert t.count() == om.count()
        gk, gval = _state(t)
        okk, ovv = om.items()
        assert (gk == okk).all()
        # replace copies and insert copies of keys absent at batch start may
        # leave any of their supplied values; everything else is exact
        free = np.zeros(gk.size, bool)
        for cls in (W.MX_REPLACE, W.MX_INSERT):
            m = ops == cls
            if cls == W.MX_INSERT:
                m &= before_s == oracle_mod.MISS
            allowed = _allowed_values(keys[m], vals[m])
            idx = np.nonzero(np.isin(gk, keys[m]))[0]
            for i in idx.tolist():
                assert int(gval[i]) in allowed[int(gk[i])]
            free[idx] = True
        assert (gval[~free] == ovv[~free]).all()
        om.load(gk[free], gval[free])
    check_layout(oracle_mod, t, om.count())
    assert t.last_error()["status"] == 0


def test_batched_plan_max_and_replace(ws, oracle_mod):
    """Upsert max / replace items (with duplicates) through a batched plan on
    every compiled menu configuration and two fallback ones."""
    import torch
    configs = [("double", False, 8, 4), ("double", False, 8, 8), ("double", True, 32, 4), ("double", True, 32, 8),
               ("p2", False, 32, 8), ("p2", False, 32, 32), ("p2", True, 32, 4), ("p2", True, 32, 8),
               ("double", False, 16, 8), ("p2", False, 8, 4)]
    items, expect = [], []
    for i, (sch, meta, B, T) in enumerate(configs):
        for op in ("max", "replace"):
            t = ws.Table(1 << 12, sch, meta, bucket_slots=B, tile=T)
            base = W.distinct_keys(9300 + 2 * i + UP[op], 1500)
            pre, pv = base[:600], W.uniform_int(9400 + i, 600, 1, 1 << 40)
            t.insert(dev(pre), dev(pv))
            keys = np.concatenate([base, base[::5], base[::7]])
            keys = keys[W.permutation(9500 + i, keys.size)]
            vals = W.uniform_int(9600 + i + UP[op], keys.size, 1, 1 << 40)
            kd, vd = dev(keys), dev(vals)
            ust = torch.empty(keys.size, dtype=torch.uint8, device="cuda")
            items.append((t, ws.BK_UPSERT, kd, vd, None, ust, 0, op))
            om = oracle_mod.OracleMap()
            om.insert(pre, pv)
            wst = om.upsert(keys, vals, UP[op])
            expect.append((t, op, keys, vals, ust, wst, om, dict(zip(pre.tolist(), pv.tolist()))))
    plan = ws.BatchPlan(items)
    plan.launch()
    torch.cuda.synchronize()
    for (t, op, keys, vals, ust, wst, om, prev) in expect:
        assert (_multiset(keys, host(ust)) == _multiset(keys, wst)).all()
        assert t.count() == om.count()
        gk, gv = _state(t)
        ok, ov = om.items()
        assert (gk == ok).all()
        if op == "max":
            assert (gv == ov).all()
        else:
            counts = dict(zip(*np.unique(keys, return_counts=True)))
            allowed = _allowed_values(keys, vals)
            for k, v, w in zip(gk.tolist(), gv.tolist(), ov.tolist()):
                if counts[k] == 1:
                    assert v == w
                else:
                    assert v in allowed[k]
        check_layout(oracle_mod, t, om.count())
    plan.close()


def test_serving_requests_with_every_code(ws, oracle_mod):
    """Requests that use max and replace beside the other codes: continuous
    batching, plain per-request serving and the oracle agree request by
    request."""
    tables = [(1 << 12, "double", False, 8), (1 << 13, "double", True, 4), (1 << 13, "p2", False, 8),
              (1 << 13, "p2", True, 4), (1 << 13, "iceberg", True, 4)]
    universe = 2500
    sizes = W.log_uniform_int(77, 120, 1, 4096)
    tabs = (W.splitmix64(78, 120) % np.uint64(len(tables))).astype(int)
    reqs = []
    for i in range(120):
        ops, keys, vals = W.mixed_request_codes(9900 + i, int(sizes[i]), universe, int(tabs[i]) + 1)
        reqs.append((int(tabs[i]), ops, keys, vals))

    def serve(**kw):
        sv = ws.Server(**kw)
        ids = [sv.add_table(c, sch, m, tl) for (c, sch, m, tl) in tables]
        sv.pause()
        rid = [sv.submit(ids[t], ops, keys, vals) for (t, ops, keys, vals) in reqs]
        done = {c["id"]: c for c in sv.drain()}
        assert all(c["status"] == 0 for c in done.values())
        res = [(done[r]["vals"], done[r]["st"]) for r in rid]
        contents = []
        for i in ids:
            slots, tags = sv.dump(i)
            k = slots[:, 0]
            live = (k != 0) & (k < np.uint64((1 << 64) - 2))
            if tags is not None:
                live &= tags >= 2
            o = np.argsort(k[live])
            contents.append((k[live][o], slots[:, 1][live][o]))
        sv.close()
        return res, contents

    cont, cc = serve(max_inflight=4, max_batch_reqs=64, grow_at=0.5)
    plain, pc = serve(plain=True, grow_at=0.5)
    oms = [oracle_mod.OracleMap() for _ in tables]
    for i, (t, ops, keys, vals) in enumerate(reqs):
        ov, os_ = oms[t].mixed(ops, keys, vals)
        for res in (cont, plain):
            gv, gs = res[i]
            q = ops == W.MX_QUERY
            assert (gv[q] == ov[q]).all() and (gs[q] == os_[q]).all()
            for cls in (W.MX_ADD, W.MX_MAX, W.MX_REPLACE, W.MX_INSERT, W.MX_ERASE):
                m = ops == cls
                if m.any():
                    assert (_multiset(keys[m], gs[m], gv[m]) == _multiset(keys[m], os_[m], ov[m])).all()
    for ti in range(len(tables)):
        ok, ov = oms[ti].items()
        for contents in (cc, pc):
            assert (contents[ti][0] == ok).all() and (contents[ti][1] == ov).all()
