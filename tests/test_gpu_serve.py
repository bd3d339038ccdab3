"""Serving: a stream of mixed requests over several tables through the
continuous-batching server must give, request by request, what the same
requests give alone (per-table replay in arrival order), what plain
per-request serving gives, and what the oracle gives -- also when tables grow
on the way.  Needs a GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

# (capacity, scheme, metadata, tile); the first table is small so it must grow
TABLES = [(1 << 10, "double", False, 8), (1 << 13, "double", True, 4), (1 << 13, "p2", False, 8),
          (1 << 13, "p2", True, 4), (1 << 13, "double", False, 4), (1 << 12, "double", False, 16)]
UNIVERSE = 3000


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


def _requests(n_req, seed):
    sizes = W.log_uniform_int(seed, n_req, 1, 4096)
    tabs = (W.splitmix64(seed + 1, n_req) % np.uint64(len(TABLES))).astype(int)
    out = []
    for i in range(n_req):
        ops, keys, vals = W.mixed_request(seed * 100003 + i, int(sizes[i]), UNIVERSE, int(tabs[i]) + 1)
        out.append((int(tabs[i]), ops, keys, vals))
    return out


def _serve(ws, reqs, burst=False, **kw):
    sv = ws.Server(**kw)
    ids = [sv.add_table(c, sch, m, t) for (c, sch, m, t) in TABLES]
    if burst:
        sv.pause()  # queue everything first: launches must then batch requests
    rid = [sv.submit(ids[t], ops, keys, vals) for (t, ops, keys, vals) in reqs]
    done = {c["id"]: c for c in sv.drain()}
    assert len(done) == len(reqs) and all(c["status"] == 0 for c in done.values())
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
    stats = sv.stats()
    sv.close()
    return res, contents, stats


def _same(reqs, a, b):
    """Queries equal op by op; upsert and erase results equal as per-key multisets
    (which duplicate of a key inside one request got INSERTED / FOUND is free)."""
    for (t, ops, keys, vals), (va, sa), (vb, sb) in zip(reqs, a, b):
        q = ops == W.MX_QUERY
        assert (va[q] == vb[q]).all() and (sa[q] == sb[q]).all()
        for cls in (W.MX_ADD, W.MX_INSERT, W.MX_ERASE):
            m = ops == cls
            if m.any():
                x = np.stack([keys[m], sa[m].astype(np.uint64), va[m]], 1)
                y = np.stack([keys[m], sb[m].astype(np.uint64), vb[m]], 1)
                assert (x[np.lexsort(x.T[::-1])] == y[np.lexsort(y.T[::-1])]).all()


def test_serving_equals_solo_replay_plain_and_oracle(ws, oracle_mod):
    reqs = _requests(160, 5)
    cont, cont_contents, st = _serve(ws, reqs, burst=True, max_inflight=4, max_batch_reqs=64, grow_at=0.5)
    assert st["grows"] >= 1 and st["launches"] < len(reqs) // 2
    trickle, trickle_contents, _ = _serve(ws, reqs, max_inflight=4, grow_at=0.5)  # requests as they come
    plain, plain_contents, st_p = _serve(ws, reqs, burst=True, plain=True, grow_at=0.5)
    assert st_p["launches"] == len(reqs)
    _same(reqs, cont, plain)
    _same(reqs, cont, trickle)
    # solo replay: each table's requests alone, in arrival order, one ws_mixed call each
    solo = [None] * len(reqs)
    oracle_res = [None] * len(reqs)
    for ti, (c, sch, m, tile) in enumerate(TABLES):
        t = ws.Table(1 << 14, sch, m, tile=tile)
        om = oracle_mod.OracleMap()
        for i, (tt, ops, keys, vals) in enumerate(reqs):
            if tt != ti:
                continue
            gv, gs = t.mixed(dev(ops), dev(keys), dev(vals))
            solo[i] = (host(gv), host(gs))
            oracle_res[i] = om.mixed(ops, keys, vals)
        ok, ov = om.items()
        for contents in (cont_contents, plain_contents, trickle_contents):
            assert (contents[ti][0] == ok).all() and (contents[ti][1] == ov).all()
        t.close()
    _same(reqs, cont, solo)
    _same(reqs, cont, oracle_res)


def test_server_admission_rejects_what_memory_cannot_hold(ws):
    sv = ws.Server(max_inflight=1, hbm_headroom=0.05)
    with pytest.raises(ws.WsError) as e:
        sv.add_table(1 << 40)  # 16 TiB of slots: far beyond free device memory
    assert e.value.status == 3
    tid = sv.add_table(1 << 12)
    sv.submit(tid, np.array([W.MX_INSERT], np.uint8), np.array([42], np.uint64), np.array([7], np.uint64))
    assert sv.drain()[0]["st"][0] == ws.INSERTED
    assert sv.count(tid) == 1
    sv.close()
