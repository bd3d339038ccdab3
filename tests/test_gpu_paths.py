"""Every way a single-table call can be served gives the oracle's results:
streaming lanes (the default), 32-op chunks (WS_OPT_STREAM = 0), streaming
lanes also for plain two-choice queries and erases (WS_OPT_STREAM = 2, by
lines instead of whole buckets), a capped lane path (WS_OPT_LANE_WAVES), and
tiles only (WS_OPT_PRELOAD = 0), on every design and on two-choice tables with
16-slot buckets (lanes that read a bucket line by line).  Needs a GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import DESIGNS, DESIGN_IDS, check_layout, dev, host

pytestmark = pytest.mark.gpu

MODES = {"stream": dict(), "chunks": dict(stream=False), "lanes2": dict(lane_waves=2),
         "tiles": dict(preload=False), "stream_lines": dict(stream=2)}
CASES = [(s, m, 0) for s, m in DESIGNS] + [("p2", False, 16)]
CASE_IDS = DESIGN_IDS + ["P2HT-B16"]


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


def _table(ws, scheme, meta, B, mode):
    t = ws.Table(1 << 15, scheme, meta, bucket_slots=B)
    opts = MODES[mode]
    if "stream" in opts:
        t.set_stream(opts["stream"])
    if "lane_waves" in opts:
        t.set_lane_waves(opts["lane_waves"])
    if "preload" in opts:
        t.set_preload(opts["preload"])
    return t


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("scheme,meta,B", CASES, ids=CASE_IDS)
def test_paths_match_oracle(ws, oracle_mod, scheme, meta, B, mode):
    t = _table(ws, scheme, meta, B, mode)
    S = t.info()["slots"]
    n = int(0.75 * S)
    both = W.distinct_keys(777 + B, n + n // 2)
    keys, absent = both[:n], both[n:]
    vals = W.splitmix64(778, n)
    om = oracle_mod.OracleMap()
    st = host(t.insert(dev(keys), dev(vals), return_status=True))
    assert (st == om.insert(keys, vals)).all()
    q = np.concatenate([keys, absent])
    got, gst = t.query(dev(q), return_status=True)
    want, wst = om.query(q)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    # add to present keys and to some new ones
    ukeys = np.concatenate([keys[::3], absent[: n // 50]])
    uvals = W.uniform_int(779, ukeys.size, 1, 1000)
    ust = host(t.upsert(dev(ukeys), dev(uvals), op="add", return_status=True))
    assert (ust == om.upsert(ukeys, uvals, 0)).all()
    ek = keys[1::7]
    ev, es = t.erase(dev(ek), return_values=True, return_status=True)
    wv, wsx = om.erase(ek)
    assert (host(ev) == wv).all() and (host(es) == wsx).all()
    # a mixed batch with Zipf keys (key-disjoint classes)
    ops, mk, mv = W.mixed_batch(780, n_ops=1 << 14, universe=1 << 13)
    gv, gs = t.mixed(dev(ops), dev(mk), dev(mv))
    ov, os_ = om.mixed(ops, mk, mv)
    qm = ops == W.MX_QUERY
    assert (host(gv)[qm] == ov[qm]).all() and (host(gs)[qm] == os_[qm]).all()
    assert t.count() == om.count()
    got, gst = t.query(dev(q), return_status=True)
    want, wst = om.query(q)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    check_layout(oracle_mod, t, om.count())
    assert t.last_error()["status"] == 0
    t.close()
