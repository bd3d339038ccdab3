"""The probe-count instrumentation (§5 "probe count", Table 1) against a host
recount: for every design, at 0.5 and 0.9 load, on a table that has or has
not seen erases (tombstones), each key's (cache lines, sectors) from
``ws_probe_cost`` must equal the oracle's recount on the dumped table, bit
for bit, for present and absent keys.  These counts are the ``s`` of the
algorithmic bytes behind every roofline fraction the bench reports.  Needs a
GPU."""
import numpy as np
import pytest

import workloads as W
from tests._gpu import DESIGNS, DESIGN_IDS, check_layout, dev, host

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


def _recount(oracle_mod, t, L, keys):
    inf = t.info()
    return oracle_mod.probe_cost(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"], L["seed1"],
                                 L["seed2"], inf["tile"], inf["never_erased"], keys)


@pytest.mark.parametrize("erase_first", [False, True], ids=["fresh", "tombstones"])
@pytest.mark.parametrize("load", [0.5, 0.9])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_probe_cost_matches_host_recount(ws, oracle_mod, scheme, meta, load, erase_first):
    S = 1 << 16
    t = ws.Table(S, scheme, meta)
    n = int(load * S)
    both = W.distinct_keys(7100 + int(load * 100) + erase_first, n + n // 2 + n // 3)
    keys, absent, refill = both[:n], both[n:n + n // 2], both[n + n // 2:]
    t.insert(dev(keys), dev(keys))
    live = keys
    if erase_first:
        gone = keys[::3]
        t.erase(dev(gone))
        t.insert(dev(refill), dev(refill))  # claims reuse the tombstones
        live = np.concatenate([np.setdiff1d(keys, gone), refill])
        absent = np.concatenate([absent, gone[: gone.size // 2]])
    _, L = check_layout(oracle_mod, t)
    B = L["B"]
    probe = np.concatenate([live, absent, np.array([0, (1 << 64) - 1], np.uint64)])
    real = probe.size - 2
    tiles = (4, 8, 16, 32) if not meta else (4, 8)
    for tile in tiles:
        t.set_tile(tile)
        out, st = t.probe_cost(dev(probe))
        out, st = host(out), host(st)
        lines, sectors = out >> np.uint64(32), out & np.uint64(0xFFFFFFFF)
        w_lines, w_sectors, w_found = _recount(oracle_mod, t, L, probe[:real])
        assert (st[real:] == ws.FAIL_BADKEY).all() and (out[real:] == 0).all()
        assert (st[:real] == np.where(w_found, ws.FOUND, ws.MISS)).all(), tile
        bad = np.nonzero((lines[:real] != w_lines) | (sectors[:real] != w_sectors))[0]
        assert bad.size == 0, (tile, bad[:5], lines[bad[:5]], w_lines[bad[:5]], sectors[bad[:5]],
                               w_sectors[bad[:5]])
        # every key the table holds is found; absent keys never are
        assert int((st[:live.size] == ws.FOUND).sum()) == t.count()
        assert (st[live.size:real] == ws.MISS).all()
        # per-design sanity of the average: a plain 8-slot double-hashing
        # query reads at least one line, a metadata probe at least a tag line
        assert lines[:real].min() >= 1 and (meta or sectors[:real].min() >= min(tile, B) // 2)
    t.close()
