"""Insert failures at high load, as the load sweep produces them: the table is
filled in 5% slices up to 0.95 load (0.5 ... 0.95, as in the paper's load
benchmark, §6.3), and every insert the table reports as FULL must have had its
whole candidate set taken (checked on the dumped table by the oracle's layout
routines); every other key must be present and the count exact.  At 2^22
slots for every design and tile; at 2^28 slots (the size of the bench's
tables) for the designs whose placement can fail.  Needs a GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import DESIGNS, DESIGN_IDS, check_layout, dev, host, layout_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2509_16407_gb300 import build as b
    b.build()
    import paper_2509_16407_gb300 as ws
    ws.lib()
    return ws


def _fill_by_slices(ws, t, S, keys):
    """Insert keys[: 0.95 S] in the sweep's slices; returns the failed keys."""
    failed = []
    have = 0
    for lf in (0.5, 0.7, 0.8, 0.9, 0.95):
        lo, hi = int((lf - 0.05) * S), int(lf * S)
        if lo > have:
            st = host(t.insert(keys[have:lo], keys[have:lo], return_status=True))
            failed.append(host(keys[have:lo])[st == ws.FAIL_FULL])
        st = host(t.insert(keys[lo:hi], keys[lo:hi], return_status=True))
        failed.append(host(keys[lo:hi])[st == ws.FAIL_FULL])
        have = hi
    return np.concatenate(failed)


@pytest.mark.parametrize("tile", [4, 8, 16, 32])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_full_reports_at_095_load_2p22(ws, oracle_mod, scheme, meta, tile):
    S = 1 << 22
    t = ws.Table(S, scheme, meta, tile=tile)
    keys = dev(W.distinct_keys(0xF00 + tile, int(0.95 * S)))
    failed = _fill_by_slices(ws, t, S, keys)
    if scheme == "double":
        assert failed.size == 0  # the probe cap of 80 buckets is never reached at 0.95
    assert failed.size < 0.02 * S
    r, L = check_layout(oracle_mod, t, keys.numel() - failed.size)
    if failed.size:
        assert oracle_mod.candidates_full(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"],
                                          L["seed1"], L["seed2"], failed).all()
        assert t.last_error()["full"] == failed.size
    assert t.count() == keys.numel() - failed.size
    # failed keys are absent, all others present
    v, s = t.query(keys, return_status=True)
    s = host(s)
    bad = np.isin(host(keys), failed)
    assert (s[bad] == ws.MISS).all() and (s[~bad] == ws.FOUND).all()
    t.close()


@pytest.mark.parametrize("scheme,meta", [("p2", False), ("p2", True), ("iceberg", True)],
                         ids=["P2HT", "P2HT(M)", "IcebergHT(M)"])
def test_full_reports_at_095_load_2p28(ws, oracle_mod, scheme, meta):
    import torch
    S = 1 << 28
    t = ws.Table(S, scheme, meta)
    n = int(0.95 * S)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    for off in range(0, n, 1 << 24):
        m = min(1 << 24, n - off)
        keys[off:off + m].copy_(torch.from_numpy(W.distinct_keys(0xF28, m, start=off).view(np.int64)))
    failed = _fill_by_slices(ws, t, S, keys)
    assert failed.size < 0.02 * S
    assert t.count() == n - failed.size
    assert t.last_error()["full"] == failed.size
    if failed.size:
        L = layout_of(t)
        assert oracle_mod.candidates_full(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"],
                                          L["seed1"], L["seed2"], failed).all()
        v, s = t.query(dev(failed), return_status=True)
        assert (host(s) == ws.MISS).all()
    t.close()
    del keys
    torch.cuda.empty_cache()
