"""Bulk-synchronous (phased) mode -- weak cacheable loads, no locks -- gives
the same map results as the concurrent mode on calls it is valid for
(distinct keys, no concurrent writers).  Needs a GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import DESIGNS, DESIGN_IDS, check_layout, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available()
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_phased_equals_concurrent(ws, oracle_mod, scheme, meta):
    S = 1 << 16
    n = int(0.85 * S)
    both = W.distinct_keys(3131, n + n // 2)
    keys, absent = both[:n], both[n:]
    vals = W.splitmix64(3232, n)
    om = oracle_mod.OracleMap()
    t = ws.Table(S, scheme, meta)
    t.set_phased(True)
    st = host(t.insert(dev(keys), dev(vals), return_status=True))
    assert (st == om.insert(keys, vals)).all()
    q = np.concatenate([keys, absent])
    want, wst = om.query(q)
    got, gst = t.query(dev(q), return_status=True)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    t.set_phased(False)
    got, gst = t.query(dev(q), return_status=True)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    assert t.count() == n
    check_layout(oracle_mod, t, n)
