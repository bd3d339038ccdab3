"""Parity of the CUDA path against the CPU oracle (element by element on
seeded inputs), structural layout checks of the dumped tables, and the
paper's invariants.  Needs a GPU."""
import numpy as np
import pytest

import workloads as W
from tests import _golden
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


def _tiles_for(scheme, meta):
    return [4, 8, 16, 32]


# --------------------------------------------------------------------------
# worked examples
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_golden_api_semantics(ws, oracle_mod, scheme, meta):
    t = ws.Table(1 << 10, scheme, meta)

    class A:
        def upsert(self, k, v, op):
            st = t.upsert(dev(np.array(k, np.uint64)), dev(np.array(v, np.uint64)),
                          op=3 if op < 0 else op, return_status=True)
            return list(host(st)), None

        def query(self, k):
            v, s = t.query(dev(np.array(k, np.uint64)), return_status=True)
            return list(host(s)), list(host(v))

        def erase(self, k):
            v, s = t.erase(dev(np.array(k, np.uint64)), return_values=True, return_status=True)
            return list(host(s)), list(host(v))

        def count(self):
            return t.count()

    assert _golden.run_api_semantics(A()) == []
    check_layout(oracle_mod, t)


@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_golden_adversarial_fig2_single(ws, oracle_mod, scheme, meta):
    """Fig. 2 on one key pair whose primary buckets coincide."""
    t = ws.Table(1 << 10, scheme, meta)
    nb = t.num_buckets()
    cand = W.distinct_keys(77, 4096)
    inf = t.info()
    pb = host(t.primary_bucket(dev(cand)))
    assert (pb == oracle_mod.primary_bucket_of(inf["scheme"], cand, nb, inf["seed1"], inf["seed2"])).all()
    b = pb[0]
    X, Y = cand[0], cand[1:][pb[1:] == b][0]
    t.insert(dev(np.array([X], np.uint64)), dev(np.array([100], np.uint64)))
    out, st = t.mixed(dev(np.array([5, 1, 1], np.uint8)), dev(np.array([X, Y, Y], np.uint64)),
                      dev(np.array([0, 200, 201], np.uint64)))
    st, out = host(st), host(out)
    assert (int(st[0]), int(out[0])) == (1, 100)
    assert sorted(st[1:].tolist()) == [1, 2]
    assert t.count() == 1
    v, s = t.query(dev(np.array([Y, X], np.uint64)), return_status=True)
    assert host(s).tolist() == [1, 0] and int(host(v)[0]) in (200, 201)
    check_layout(oracle_mod, t, 1)


# --------------------------------------------------------------------------
# PR1: DoubleHT 2^20 slots, 8-slot buckets, tile 8, no metadata
# --------------------------------------------------------------------------
def test_pr1_parity(ws, oracle_mod):
    keys, vals, absent, eidx = W.pr1()
    K = keys.size
    t = ws.Table(1 << 20, "double", False)
    inf = t.info()
    assert (inf["buckets"], inf["bucket_slots"], inf["tile"], inf["slots"]) == (131072, 8, 8, 1 << 20)
    om = oracle_mod.OracleMap()
    st = host(t.insert(dev(keys), dev(vals), return_status=True))
    assert (st == om.insert(keys, vals)).all()
    assert t.count() == om.count() == K
    check_layout(oracle_mod, t, K)
    q = np.concatenate([keys, absent])
    got, gst = t.query(dev(q), return_status=True)
    want, wst = om.query(q)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    ek = keys[eidx]
    ev, es = t.erase(dev(ek), return_values=True, return_status=True)
    wv, wsx = om.erase(ek)
    assert (host(ev) == wv).all() and (host(es) == wsx).all()
    assert t.count() == om.count() == 471859
    got, gst = t.query(dev(q), return_status=True)
    want, wst = om.query(q)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    check_layout(oracle_mod, t, K - K // 2)
    assert t.last_error()["status"] == 0


# --------------------------------------------------------------------------
# Config-2 shape at a size the oracle finishes in seconds: every design,
# every tile, load factors 0.5 / 0.9 / 0.95
# --------------------------------------------------------------------------
def _map_state(t):
    slots, tags = t.dump()
    k = slots[:, 0]
    live = (k != 0) & (k < np.uint64((1 << 64) - 2))
    if tags is not None:
        live &= tags >= 2
    order = np.argsort(k[live])
    return k[live][order], slots[:, 1][live][order]


@pytest.mark.parametrize("load", [0.5, 0.9, 0.95])
@pytest.mark.parametrize("tile", [4, 8, 16, 32])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_config2_small(ws, oracle_mod, scheme, meta, tile, load):
    S = 1 << 17
    t = ws.Table(S, scheme, meta, tile=tile)
    assert t.info()["slots"] == S
    n = int(load * S)
    both = W.distinct_keys(1000 + tile, n + n // 2)
    keys, absent = both[:n], both[n:]
    vals = W.splitmix64(2000 + tile, n)
    om = oracle_mod.OracleMap()
    st = host(t.insert(dev(keys), dev(vals), return_status=True))
    ost = om.insert(keys, vals)
    full = st == ws.FAIL_FULL
    # two-choice placement depends on the interleaving: at 0.9 the sequential
    # order already fills some buckets, so a concurrent one can leave a key
    # with both buckets taken (iceberg: its front and both backyard buckets);
    # every such failure is validated below
    if scheme == "double" or load < 0.9:
        assert not full.any(), f"{full.sum()} inserts failed at load {load}"
    assert ((st == ost) | full).all()
    if full.any():
        # every reported failure must have had its whole candidate set taken
        r, L = check_layout(oracle_mod, t)
        cf = oracle_mod.candidates_full(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"],
                                        L["seed1"], L["seed2"], keys[full])
        assert cf.all()
        assert full.mean() < 0.02
        assert t.last_error()["full"] == int(full.sum())
        om.erase(keys[full])  # the expected map is the oracle's minus the validated failures
    assert t.count() == om.count()
    check_layout(oracle_mod, t, om.count())
    q = np.concatenate([keys, absent])
    got, gst = t.query(dev(q), return_status=True)
    want, wst = om.query(q)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    # upsert-add: a quarter of the keys (present or failed) plus some new keys
    ukeys = np.concatenate([keys[::4], absent[: n // 100]])
    uvals = W.uniform_int(3000 + tile, ukeys.size, 1, 1000)
    ust = host(t.upsert(dev(ukeys), dev(uvals), op="add", return_status=True))
    uost = om.upsert(ukeys, uvals, 0)
    ufull = ust == ws.FAIL_FULL
    if ufull.any():
        # the new keys take two-choice tables past 0.9 load: a key whose both
        # buckets are taken fails, and the layout must show both full
        assert scheme != "double" and load >= 0.9 and ufull.mean() < 0.02
        r, L = check_layout(oracle_mod, t)
        assert oracle_mod.candidates_full(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"],
                                          L["seed1"], L["seed2"], ukeys[ufull]).all()
        om.erase(ukeys[ufull])
    assert ((ust == uost) | ufull).all()
    # erase 10%, then query everything again
    ek = keys[1::10]
    ev, es = t.erase(dev(ek), return_values=True, return_status=True)
    wv, wsx = om.erase(ek)
    assert (host(ev) == wv).all() and (host(es) == wsx).all()
    got, gst = t.query(dev(q), return_status=True)
    want, wst = om.query(q)
    assert (host(got) == want).all() and (host(gst) == wst).all()
    # re-insert the erased keys over the tombstones
    st = host(t.insert(dev(ek), dev(vals[1::10]), return_status=True))
    ost = om.insert(ek, vals[1::10])
    rfull = st == ws.FAIL_FULL
    if rfull.any():
        om.erase(ek[rfull])
    assert ((st == ost) | rfull).all()
    gk, gv = _map_state(t)
    okk, ov = om.items()
    assert (gk == okk).all() and (gv == ov).all()
    check_layout(oracle_mod, t, om.count())


@pytest.mark.parametrize("scheme", ["double", "p2"])
@pytest.mark.parametrize("B", [8, 16])
def test_bucket_sizes(ws, oracle_mod, scheme, B):
    S = 1 << 16
    for tile in (4, 8, 16, 32):
        t = ws.Table(S, scheme, False, bucket_slots=B, tile=tile)
        n = int(0.85 * S)
        keys = W.distinct_keys(50 + B + tile, n)
        om = oracle_mod.OracleMap()
        st = host(t.insert(dev(keys), dev(keys), return_status=True))
        ok = st != ws.FAIL_FULL
        om.insert(keys[ok], keys[ok])
        got, gst = t.query(dev(keys), return_status=True)
        want, wst = om.query(keys)
        assert (host(got) == want).all() and (host(gst) == wst).all()
        assert (~ok).mean() < 0.02
        check_layout(oracle_mod, t, int(ok.sum()))
        t.close()


# --------------------------------------------------------------------------
# Config-3 shape: Zipf(0.99) mixed batches on metadata (and plain) tables
# --------------------------------------------------------------------------
def _multiset(keys, st, vals):
    a = np.stack([keys, st.astype(np.uint64), vals], 1)
    return a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_mixed_zipf_batches(ws, oracle_mod, scheme, meta):
    t = ws.Table(1 << 18, scheme, meta)
    om = oracle_mod.OracleMap()
    for b in range(4):
        ops, keys, vals = W.mixed_batch(100 + b, n_ops=1 << 17, universe=1 << 15)
        gv, gs = t.mixed(dev(ops), dev(keys), dev(vals))
        gv, gs = host(gv), host(gs)
        ov, os_ = om.mixed(ops, keys, vals)
        q = ops == W.MX_QUERY
        assert (gv[q] == ov[q]).all() and (gs[q] == os_[q]).all()
        for cls in (W.MX_ERASE, W.MX_ADD):
            m = ops == cls
            assert (_multiset(keys[m], gs[m], gv[m]) == _multiset(keys[m], os_[m], ov[m])).all()
        assert t.count() == om.count()
        gk, gvv = _map_state(t)
        okk, ovv = om.items()
        assert (gk == okk).all() and (gvv == ovv).all()
    check_layout(oracle_mod, t, om.count())


# --------------------------------------------------------------------------
# same-key race stress: 32 copies per key, contiguous and shuffled
# --------------------------------------------------------------------------
@pytest.mark.parametrize("layout", ["contiguous", "shuffled"])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_same_key_stress(ws, oracle_mod, scheme, meta, layout):
    n = 1 << 14
    base = W.distinct_keys(4242, n)
    keys = np.repeat(base, 32)
    if layout == "shuffled":
        keys = keys[W.permutation(17, keys.size)]
    t = ws.Table(1 << 16, scheme, meta)
    st = host(t.upsert(dev(keys), dev(np.ones(keys.size, np.uint64)), op="add", return_status=True))
    per_key_inserted = np.bincount(np.searchsorted(base, keys[st == ws.INSERTED]) if False else
                                   np.unique(keys[st == ws.INSERTED], return_counts=True)[1])
    assert (st == ws.INSERTED).sum() == n and (st == ws.FOUND).sum() == 31 * n
    assert np.unique(keys[st == ws.INSERTED]).size == n
    assert t.count() == n
    v, s = t.query(dev(base), return_status=True)
    assert (host(v) == 32).all() and (host(s) == ws.FOUND).all()
    check_layout(oracle_mod, t, n)
    # insert-if-unique copies keep the accumulated value
    st = host(t.insert(dev(keys), dev(np.arange(keys.size, dtype=np.uint64)), return_status=True))
    assert (st == ws.FOUND).all()
    assert (host(t.query(dev(base))) == 32).all()
    # 32 erase copies per key: exactly one succeeds
    ev, es = t.erase(dev(keys), return_values=True, return_status=True)
    es, ev = host(es), host(ev)
    assert (es == ws.FOUND).sum() == n and np.unique(keys[es == ws.FOUND]).size == n
    assert (ev[es == ws.FOUND] == 32).all() and (ev[es != ws.FOUND] == 0).all()
    assert t.count() == 0
    check_layout(oracle_mod, t, 0)
    # fresh same-key inserts into a table full of tombstones
    st = host(t.insert(dev(keys), dev(keys), return_status=True))
    assert (st == ws.INSERTED).sum() == n and t.count() == n
    check_layout(oracle_mod, t, n)
    del per_key_inserted


# --------------------------------------------------------------------------
# §4.1 adversarial benchmark: two keys per primary bucket in every bucket,
# Fig. 2 replayed in all buckets at once
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_adversarial_every_bucket(ws, oracle_mod, scheme, meta):
    t = ws.Table(1 << 13, scheme, meta)
    inf = t.info()
    nb = t.num_buckets()
    npb = inf["front_buckets"]  # buckets that are some key's primary bucket
    cand = W.distinct_keys(31337, 64 * nb)
    pb = host(t.primary_bucket(dev(cand)))
    assert (pb == oracle_mod.primary_bucket_of(inf["scheme"], cand, nb, inf["seed1"], inf["seed2"])).all()
    order = np.argsort(pb, kind="stable")
    spb, sk = pb[order], cand[order]
    first = np.searchsorted(spb, np.arange(npb))
    cnt = np.bincount(pb.astype(np.int64), minlength=npb)
    assert cnt.size == npb and (cnt >= 2).all()
    nb = npb
    X, Y = sk[first], sk[first + 1]
    for rnd in range(10):
        t.clear()
        assert (host(t.insert(dev(X), dev(np.full(nb, 100, np.uint64)), return_status=True)) == 2).all()
        ops = np.tile(np.array([5, 1, 1], np.uint8), nb)
        keys = np.stack([X, Y, Y], 1).reshape(-1)
        vals = np.stack([np.zeros(nb, np.uint64), np.full(nb, 200, np.uint64), np.full(nb, 201, np.uint64)],
                        1).reshape(-1)
        if rnd % 2:
            p = W.permutation(rnd, keys.size)
            ops, keys, vals = ops[p], keys[p], vals[p]
        gv, gs = t.mixed(dev(ops), dev(keys), dev(vals))
        gs = host(gs)
        assert (gs[ops == 5] == ws.FOUND).all()
        ins = ops == 1
        assert (gs[ins] == ws.INSERTED).sum() == nb and (gs[ins] == ws.FOUND).sum() == nb
        assert t.count() == nb
        r, _ = check_layout(oracle_mod, t, nb)
        v, s = t.query(dev(Y), return_status=True)
        assert (host(s) == ws.FOUND).all() and np.isin(host(v), [200, 201]).all()
        assert (host(t.query(dev(X), return_status=True)[1]) == ws.MISS).all()


# --------------------------------------------------------------------------
# failure paths, all injected from the host
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_full_reports_validated(ws, oracle_mod, scheme, meta):
    t = ws.Table(1 << 10, scheme, meta, max_probe=2)
    S = t.info()["slots"]
    keys = W.distinct_keys(55, 3 * S)
    st = host(t.insert(dev(keys), dev(keys), return_status=True))
    full = st == ws.FAIL_FULL
    assert full.any() and (st[~full] == ws.INSERTED).all()
    assert t.count() == int((~full).sum()) <= S
    r, L = check_layout(oracle_mod, t, int((~full).sum()))
    assert oracle_mod.candidates_full(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"],
                                      L["seed1"], L["seed2"], keys[full]).all()
    e = t.last_error()
    assert e["status"] == 4 and e["full"] == int(full.sum())
    # failed keys are absent; the rest read back
    v, s = t.query(dev(keys), return_status=True)
    assert (host(s)[full] == ws.MISS).all() and (host(v)[~full] == keys[~full]).all()


@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_lock_timeout_is_bounded(ws, oracle_mod, scheme, meta):
    """Every lock bit set from the host: absent-key inserts that need the lock
    (mixed batches; two-choice plain inserts) report TIMEOUT after spin_limit
    attempts instead of hanging; lock-free paths are unaffected."""
    t = ws.Table(1 << 12, scheme, meta, spin_limit=64)
    keys = W.distinct_keys(8, 1500)
    t.insert(dev(keys[:500]), dev(keys[:500]))
    t.debug_fill_locks(True)
    ops = np.full(500, W.MX_INSERT, np.uint8)
    _, st = t.mixed(dev(ops), dev(keys[500:1000]), dev(keys[500:1000]))
    assert (host(st) == ws.FAIL_TIMEOUT).all()
    # present keys need no lock (in-place update), queries are lock-free
    st = host(t.upsert(dev(keys[:500]), dev(np.ones(500, np.uint64)), op="add", return_status=True))
    assert (st == ws.FOUND).all()
    v, s = t.query(dev(keys[:1000]), return_status=True)
    assert (host(s)[:500] == ws.FOUND).all() and (host(s)[500:] == ws.MISS).all()
    assert (host(v)[:500] == keys[:500] + np.uint64(1)).all()
    # plain inserts: two-choice placement needs the lock, double hashing does not
    st = host(t.insert(dev(keys[1000:]), dev(keys[1000:]), return_status=True))
    want = ws.INSERTED if scheme == "double" else ws.FAIL_TIMEOUT  # two-choice and iceberg lock
    assert (st == want).all()
    e = t.last_error()
    assert e["status"] == 5 and e["timeout"] == 500 + (0 if scheme == "double" else 500)
    t.debug_fill_locks(False)
    rest = keys[500:] if scheme != "double" else keys[500:1000]
    assert (host(t.insert(dev(rest), dev(rest), return_status=True)) == ws.INSERTED).all()
    assert t.count() == 1500
    check_layout(oracle_mod, t, 1500)


def test_sentinel_keys_and_bad_codes(ws):
    t = ws.Table(1 << 10, "p2", True)
    S = (1 << 64) - 1
    bad = np.array([0, S, S - 1], np.uint64)
    assert (host(t.insert(dev(bad), dev(bad), return_status=True)) == ws.FAIL_BADKEY).all()
    assert (host(t.query(dev(bad), return_status=True)[1]) == ws.FAIL_BADKEY).all()
    assert (host(t.erase(dev(bad), return_status=True)[1]) == ws.FAIL_BADKEY).all()
    gv, gs = t.mixed(dev(np.array([9, 0], np.uint8)), dev(np.array([5, 5], np.uint64)),
                     dev(np.array([1, 1], np.uint64)))
    assert host(gs).tolist() == [ws.FAIL_BADKEY, ws.MISS]
    assert t.count() == 0
    e = t.last_error()
    assert e["status"] == 2 and e["badkey"] == 10


def test_empty_and_invalid_arguments(ws):
    import ctypes
    import torch
    t = ws.Table(1 << 10)
    L = ws.lib()
    z = torch.empty(0, dtype=torch.int64, device="cuda")
    assert L.ws_insert(t.handle, z.data_ptr(), z.data_ptr(), 0, None) == 0
    a = torch.zeros(16, dtype=torch.int64, device="cuda")
    assert L.ws_query(t.handle, a.data_ptr() + 4, a.data_ptr(), 4, None) == 1  # misaligned
    assert L.ws_upsert(t.handle, a.data_ptr(), None, 4, 0, None) == 1           # missing values
    assert L.ws_upsert(t.handle, a.data_ptr(), a.data_ptr(), 4, 9, None) == 1   # bad callback
    assert L.ws_set_tile(t.handle, 3) == 1
    assert t.count() == 0


# --------------------------------------------------------------------------
# host buffers: staged through the library's pipeline, more than one chunk
# --------------------------------------------------------------------------
def test_host_buffers_match_device_path(ws, oracle_mod):
    import torch
    n = (1 << 22) + 12345  # two staging chunks
    keys = W.distinct_keys(606, n)
    vals = W.splitmix64(607, n)
    ta = ws.Table(1 << 23, "double", False)
    tb = ws.Table(1 << 23, "double", False)
    sa = ta.insert(keys, vals, return_status=True)          # numpy (pageable)
    kb = torch.from_numpy(keys.view(np.int64)).pin_memory()
    vb = torch.from_numpy(vals.view(np.int64)).pin_memory()
    sb = tb.insert(kb, vb, return_status=True)               # pinned torch
    torch.cuda.synchronize()
    assert (sa == ws.INSERTED).all() and (sb.numpy() == ws.INSERTED).all()
    q = np.concatenate([keys[::3], W.distinct_keys(608, 1000)])
    va, qa = ta.query(q, return_status=True)
    torch.cuda.synchronize()
    vd, qd = tb.query(dev(q), return_status=True)
    assert (va == host(vd)).all() and (qa == host(qd)).all()
    om = oracle_mod.OracleMap()
    om.insert(keys, vals)
    want, wst = om.query(q)
    assert (va == want).all() and (qa == wst).all()
    assert ta.count() == tb.count() == n


# --------------------------------------------------------------------------
# growth: rehash a table's live pairs into a larger one (any design)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_rehash_into_larger_table(ws, oracle_mod, scheme, meta):
    src = ws.Table(1 << 14, scheme, meta)
    keys = W.distinct_keys(123, int(0.8 * (1 << 14)))
    vals = W.splitmix64(124, keys.size)
    om = oracle_mod.OracleMap()
    src.insert(dev(keys), dev(vals))
    om.insert(keys, vals)
    src.erase(dev(keys[::3]))
    om.erase(keys[::3])
    for dscheme, dmeta in DESIGNS:
        dst = ws.Table(1 << 16, dscheme, dmeta)
        st = host(src.rehash_into(dst, return_status=True))
        assert (st == ws.INSERTED).sum() == om.count() and ((st == ws.INSERTED) | (st == ws.MISS)).all()
        assert dst.count() == om.count()
        gk, gv = _map_state(dst)
        okk, ov = om.items()
        assert (gk == okk).all() and (gv == ov).all()
        check_layout(oracle_mod, dst, om.count())
        assert dst.last_error()["status"] == 0
        dst.close()


# --------------------------------------------------------------------------
# page-locked host buffers: staged (0), read in place (1), read and written
# in place (2), in place or staged by op kind (3) -- every mode gives the
# oracle's results; staging chunks of 2^16 ops, so the calls that stage
# run through several chunks and the four rotating buffers
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_host_direct_matches_oracle(ws, oracle_mod, scheme, meta, mode):
    import torch
    t = ws.Table(1 << 18, scheme, meta)
    t.set_host_direct(mode)
    t.set_stage_chunk(16)
    S = t.info()["slots"]
    n = int(0.8 * S)
    both = W.distinct_keys(909 + mode, n + n // 4)
    keys, absent = both[:n], both[n:]
    vals = W.splitmix64(910, n)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()
    om = oracle_mod.OracleMap()
    st = t.insert(pin(keys), pin(vals), return_status=True)
    torch.cuda.synchronize()
    assert (st.numpy() == om.insert(keys, vals)).all()
    q = np.concatenate([keys[::2], absent])
    out = torch.empty(q.size, dtype=torch.int64).pin_memory()
    _, qs = t.query(pin(q), out=out, return_status=True)
    torch.cuda.synchronize()
    want, wst = om.query(q)
    assert (out.numpy().view(np.uint64) == want).all() and (qs.numpy() == wst).all()
    ops, mk, mv = W.mixed_batch(911, n_ops=1 << 14, universe=1 << 13)
    gv, gs = t.mixed(torch.from_numpy(ops).pin_memory(), pin(mk), pin(mv))
    torch.cuda.synchronize()
    ov, os_ = om.mixed(ops, mk, mv)
    qm = ops == W.MX_QUERY
    assert (host(gv)[qm] == ov[qm]).all() and (host(gs)[qm] == os_[qm]).all()
    assert t.count() == om.count()
    check_layout(oracle_mod, t, om.count())
    t.close()


# --------------------------------------------------------------------------
# staging shared by the tables of a device: the staging copies of every
# table run on the device's two copy streams in call order; calls on every
# design's table, every buffer staged in 2^16-op chunks, the tables spread
# over two user streams and their calls interleaved without synchronising,
# give the oracle's results
# --------------------------------------------------------------------------
def test_staging_shared_across_tables_and_streams(ws, oracle_mod):
    import torch
    tabs = [ws.Table(1 << 20, scheme, meta) for scheme, meta in DESIGNS]
    for t in tabs:
        t.set_host_direct(0)
        t.set_stage_chunk(16)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()
    oms = [oracle_mod.OracleMap() for _ in tabs]
    n = 150000  # three chunks, the last one ragged
    pending = []
    for r in range(3):
        for i, t in enumerate(tabs):
            s = streams[i % 2]  # calls on one table stay on one stream
            keys = W.distinct_keys(7000 + 10 * i + r, n, start=r * n)
            vals = W.splitmix64(7100 + 10 * i + r, n)
            kb, vb = pin(keys), pin(vals)
            st = t.insert(kb, vb, return_status=True, stream=s)
            want_st = oms[i].insert(keys, vals)
            q = np.concatenate([keys[::2], W.distinct_keys(7200 + 10 * i + r, n // 4, start=10 * n)])
            qb = pin(q)
            out = torch.empty(q.size, dtype=torch.int64).pin_memory()
            _, qs = t.query(qb, out=out, return_status=True, stream=s)
            want_v, want_q = oms[i].query(q)
            pending.append((kb, vb, qb, st, want_st, out, qs, want_v, want_q))
    torch.cuda.synchronize()
    for kb, vb, qb, st, want_st, out, qs, want_v, want_q in pending:
        assert (st.numpy() == want_st).all()
        assert (out.numpy().view(np.uint64) == want_v).all() and (qs.numpy() == want_q).all()
    for t, om in zip(tabs, oms):
        assert t.count() == om.count()
        t.close()


# --------------------------------------------------------------------------
# work tickets: every single-table launch takes its work from a per-table
# ticket that the launch's last block returns to zero; back-to-back launches
# of sizes around a share (1 op ... a few shares, streaming and chunked
# kernels, every kind) must each see a fresh ticket
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,meta", DESIGNS, ids=DESIGN_IDS)
def test_back_to_back_launches_of_every_size(ws, oracle_mod, scheme, meta):
    t = ws.Table(1 << 16, scheme, meta)
    om = oracle_mod.OracleMap()
    keys = W.distinct_keys(5150, 30000)
    pos = 0
    sizes = [1, 2, 31, 32, 33, 255, 256, 257, 1000, 4097, 9000]
    for i, n in enumerate(sizes):
        k = keys[pos:pos + n]
        pos += n
        st = host(t.insert(dev(k), dev(k), return_status=True))
        assert (st == om.insert(k, k)).all(), n
        q = keys[max(0, pos - 2 * n):pos + n]
        v, s = t.query(dev(q), return_status=True)
        wv, wsx = om.query(q)
        assert (host(v) == wv).all() and (host(s) == wsx).all(), n
        u = k[: max(1, n // 2)]
        ust = host(t.upsert(dev(u), dev(np.ones(u.size, np.uint64)), op="add", return_status=True))
        assert (ust == om.upsert(u, np.ones(u.size, np.uint64), 0)).all(), n
        if i % 2:
            e = k[::3]
            ev, es = t.erase(dev(e), return_values=True, return_status=True)
            wv, wsx = om.erase(e)
            assert (host(ev) == wv).all() and (host(es) == wsx).all(), n
        assert t.count() == om.count(), n
    check_layout(oracle_mod, t, om.count())
