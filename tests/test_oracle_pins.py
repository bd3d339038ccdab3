"""Pins of the CPU oracle against things other than itself: a brute-force
linear list on tiny inputs, the paper's worked examples and invariants,
closed forms, and planted mistakes for the layout checker.  No GPU."""
import random

import numpy as np
import pytest

import workloads as W
from tests import _golden

MASK = (1 << 64) - 1
SENT = {0, MASK, MASK - 1}


# --------------------------------------------------------------------------
# brute force: a plain list of [key, value] pairs, ops applied in index order
# --------------------------------------------------------------------------
class BruteList:
    def __init__(self):
        self.items = []

    def _find(self, k):
        for i, (kk, _) in enumerate(self.items):
            if kk == k:
                return i
        return -1

    def upsert(self, k, v, op):
        if k in SENT:
            return 4, 0
        i = self._find(k)
        if i < 0:
            self.items.append([k, v])
            return 2, 0
        if op == 0:
            self.items[i][1] = (self.items[i][1] + v) & MASK
        elif op == 1:
            self.items[i][1] = max(self.items[i][1], v)
        elif op == 2:
            self.items[i][1] = v
        return 1, 0

    def query(self, k):
        if k in SENT:
            return 4, 0
        i = self._find(k)
        return (1, self.items[i][1]) if i >= 0 else (0, 0)

    def erase(self, k):
        if k in SENT:
            return 4, 0
        i = self._find(k)
        if i < 0:
            return 0, 0
        v = self.items[i][1]
        del self.items[i]
        return 1, v


def _oracle_batch(om, kind, keys, vals, op=None):
    if kind == "upsert":
        return list(om.upsert(keys, vals, op)), [0] * len(keys)
    if kind == "query":
        v, s = om.query(keys)
        return list(s), list(v)
    if kind == "erase":
        v, s = om.erase(keys)
        return list(s), list(v)
    raise ValueError(kind)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_single_class_batches(oracle_mod, seed):
    """Random batches of one op class over <= 24 distinct small keys (plus
    the sentinels): the oracle equals the brute-force list op by op."""
    rng = random.Random(seed)
    universe = [rng.getrandbits(64) for _ in range(24)] + [0, MASK, MASK - 1, 1, MASK - 2]
    om = oracle_mod.OracleMap()
    bl = BruteList()
    for _ in range(30):
        kind = rng.choice(["upsert", "upsert", "query", "erase"])
        n = rng.randint(0, 12)
        keys = [rng.choice(universe) for _ in range(n)]
        vals = [rng.choice([0, 1, 7, MASK, rng.getrandbits(64)]) for _ in range(n)]
        op = rng.choice([-1, 0, 1, 2])
        got_s, got_v = _oracle_batch(om, kind, np.array(keys, np.uint64),
                                     np.array(vals, np.uint64), op)
        for i, k in enumerate(keys):
            if kind == "upsert":
                ws, wv = bl.upsert(k, vals[i], op)
            elif kind == "query":
                ws, wv = bl.query(k)
            else:
                ws, wv = bl.erase(k)
            assert got_s[i] == ws, (kind, op, i, k)
            assert got_v[i] == wv, (kind, op, i, k)
        assert om.count() == len(bl.items)
    ok, ov = om.items()
    want = sorted((k, v) for k, v in bl.items)
    assert list(zip(ok.tolist(), ov.tolist())) == want


@pytest.mark.parametrize("seed", range(20))
def test_brute_force_mixed_disjoint(oracle_mod, seed):
    """Mixed batches whose query / erase / upsert classes use disjoint keys:
    the brute force applies them in plain index order (it knows nothing of
    the phase rule), so agreement pins the oracle's phase ordering."""
    rng = random.Random(1000 + seed)
    universe = [rng.getrandbits(64) | 1 for _ in range(48)]
    om = oracle_mod.OracleMap()
    bl = BruteList()
    for _ in range(20):
        pool = universe[:]
        rng.shuffle(pool)
        qk, ek, uk = pool[:16], pool[16:28], pool[28:]
        ops, keys, vals = [], [], []
        for _ in range(rng.randint(0, 40)):
            c = rng.random()
            if c < 0.35:
                ops.append(0); keys.append(rng.choice(qk)); vals.append(0)
            elif c < 0.5:
                ops.append(5); keys.append(rng.choice(ek)); vals.append(0)
            else:
                ops.append(rng.choice([1, 2, 3, 4])); keys.append(rng.choice(uk))
                vals.append(rng.getrandbits(64) if rng.random() < 0.5 else rng.randint(0, 9))
        o, k, v = (np.array(ops, np.uint8), np.array(keys, np.uint64), np.array(vals, np.uint64))
        out, st = om.mixed(o, k, v)
        for i in range(len(ops)):
            if ops[i] == 0:
                ws, wv = bl.query(keys[i])
            elif ops[i] == 5:
                ws, wv = bl.erase(keys[i])
            else:
                ws, wv = bl.upsert(keys[i], vals[i], {1: -1, 2: 0, 3: 1, 4: 2}[ops[i]])
            assert (int(st[i]), int(out[i])) == (ws, wv), (i, ops[i])
        assert om.count() == len(bl.items)


def test_golden_api_semantics(oracle_mod):
    om = oracle_mod.OracleMap()

    class Adapter:
        def upsert(self, k, v, op):
            return list(om.upsert(np.array(k, np.uint64), np.array(v, np.uint64), op)), None

        def query(self, k):
            v, s = om.query(np.array(k, np.uint64))
            return list(s), list(v)

        def erase(self, k):
            v, s = om.erase(np.array(k, np.uint64))
            return list(s), list(v)

        def count(self):
            return om.count()

    assert _golden.run_api_semantics(Adapter()) == []


def test_golden_adversarial_fig2(oracle_mod):
    """§4.1 Fig. 2: erase X and two inserts of Y in one batch -> one copy of Y."""
    om = oracle_mod.OracleMap()
    X, Y = 0x1234_5678_9ABC_DEF1, 0x0FED_CBA9_8765_4321
    om.insert(np.array([X], np.uint64), np.array([100], np.uint64))
    out, st = om.mixed(np.array([5, 1, 1], np.uint8), np.array([X, Y, Y], np.uint64),
                       np.array([0, 200, 201], np.uint64))
    assert (int(st[0]), int(out[0])) == (1, 100)
    assert sorted(st[1:].tolist()) == [1, 2]
    assert om.count() == 1
    v, s = om.query(np.array([Y, X], np.uint64))
    assert s.tolist() == [1, 0] and int(v[0]) in (200, 201) and int(v[1]) == 0


def test_pr1_closed_forms(oracle_mod):
    """PR1 (2^20 slots, 0.9 load): every inserted key reads back 3k, absent
    keys miss, erasing a random half leaves K - floor(K/2) keys."""
    keys, vals, absent, erase_idx = W.pr1()
    K = keys.size
    assert K == 943718
    assert np.unique(np.concatenate([keys, absent])).size == 2 * K
    om = oracle_mod.OracleMap()
    st = om.insert(keys, vals)
    assert (st == 2).all() and om.count() == K
    v, s = om.query(np.concatenate([keys, absent]))
    assert (s[:K] == 1).all() and (s[K:] == 0).all()
    with np.errstate(over="ignore"):
        assert (v[:K] == keys * np.uint64(3)).all()
    assert (v[K:] == 0).all()
    ev, es = om.erase(keys[erase_idx])
    assert (es == 1).all() and (ev == vals[erase_idx]).all()
    assert om.count() == K - K // 2 == 471859
    v, s = om.query(np.concatenate([keys, absent]))
    gone = np.zeros(K, bool)
    gone[erase_idx] = True
    assert (s[:K][gone] == 0).all() and (s[:K][~gone] == 1).all()
    assert (v[:K][~gone] == vals[~gone]).all() and (s[K:] == 0).all()


def test_same_key_accumulate_closed_form(oracle_mod):
    """32 copies of add(k, 1) in one batch give 32 (the §5.1 accumulate
    callback); 32 insert-if-unique copies give one INSERTED and 31 FOUND."""
    om = oracle_mod.OracleMap()
    keys = np.repeat(W.distinct_keys(5, 1000), 32)
    st = om.upsert(keys, np.ones(keys.size, np.uint64), 0)
    assert (st.reshape(-1, 32) == 2).sum(1).tolist() == [1] * 1000
    v, s = om.query(W.distinct_keys(5, 1000))
    assert (v == 32).all() and (s == 1).all()
    st = om.insert(keys, np.arange(keys.size, dtype=np.uint64))
    assert (st == 1).all()
    om2 = oracle_mod.OracleMap()
    st = om2.insert(keys, np.arange(keys.size, dtype=np.uint64))
    assert (st.reshape(-1, 32) == 2).sum(1).tolist() == [1] * 1000
    assert om2.count() == 1000


def test_wrapping_and_max_commutative(oracle_mod):
    om = oracle_mod.OracleMap()
    k = np.array([7, 7, 7], np.uint64)
    om.upsert(k, np.array([MASK, 1, 5], np.uint64), 0)
    v, _ = om.query(np.array([7], np.uint64))
    assert int(v[0]) == 5  # (2^64-1 + 1 + 5) mod 2^64
    for perm in ([3, 9, 1], [9, 1, 3], [1, 3, 9]):
        o = oracle_mod.OracleMap()
        o.upsert(np.full(3, 11, np.uint64), np.array(perm, np.uint64), 1)
        assert int(o.query(np.array([11], np.uint64))[0][0]) == 9


def test_invariants_random_batches(oracle_mod):
    """Every inserted key is found, absent keys never are, count equals the
    number of distinct live keys (paper invariants, §4.1 and §5.1)."""
    om = oracle_mod.OracleMap()
    live = {}
    for b in range(8):
        keys = W.distinct_keys(100 + b, 20000)
        keys = np.concatenate([keys, keys[:500]])  # duplicates inside a batch
        vals = W.splitmix64(200 + b, keys.size)
        st = om.insert(keys, vals)
        for k, v, s in zip(keys.tolist(), vals.tolist(), st.tolist()):
            if k not in live:
                assert s == 2
                live[k] = v
            else:
                assert s == 1
        er = np.array(list(live)[:: 7], np.uint64)
        _, es = om.erase(er)
        assert (es == 1).all()
        for k in er.tolist():
            del live[k]
        assert om.count() == len(live)
    q = np.array(list(live), np.uint64)
    v, s = om.query(q)
    assert (s == 1).all() and v.tolist() == [live[k] for k in q.tolist()]
    absent = W.distinct_keys(999, 5000)
    assert (om.query(absent)[1] == 0).all()


# --------------------------------------------------------------------------
# layout checker: planted mistakes must be caught, correct layouts pass
# --------------------------------------------------------------------------
def _fmix(x):
    x ^= x >> 33
    x = (x * 0xFF51AFD7ED558CCD) & MASK
    x ^= x >> 33
    x = (x * 0xC4CEB9FE1A85EC53) & MASK
    return x ^ (x >> 33)


S1, S2 = 0x243F6A8885A308D3, 0x13198A2E03707344


def _seq(k, nb, P):
    h1, h2 = _fmix(k ^ S1), _fmix(k ^ S2)
    return [(h1 + i * (h2 | 1)) % nb for i in range(P)]


def _tag(k):
    t = k & 0xFFFF
    return t + 2 if t < 2 else t


def _key_with_distinct_seq(nb, seed):
    rng = random.Random(seed)
    while True:
        k = rng.getrandbits(64)
        s = _seq(k, nb, 3)
        if len(set(s)) == 3:
            return k, s


@pytest.mark.parametrize("meta", [False, True])
def test_layout_checker_planted(oracle_mod, meta):
    nb, B, P = 16, 8, 80
    S = nb * B

    def fresh():
        return np.zeros(2 * S, np.uint64), (np.zeros(S, np.uint16) if meta else None)

    def put(slots, tags, b, j, k, v=1):
        slots[2 * (b * B + j)] = k
        slots[2 * (b * B + j) + 1] = v
        if tags is not None:
            tags[b * B + j] = _tag(k)

    chk = lambda s, t, scheme=0: oracle_mod.layout_check(s, t, nb, B, scheme, P, S1, S2)
    k, seq = _key_with_distinct_seq(nb, 1)
    s, t = fresh()
    r = chk(s, t)
    assert r["empty"] == S and sum(r[x] for x in ("bad_bucket", "duplicates", "tag_mismatch",
                                                 "early_exit", "empty_not_suffix")) == 0
    # correct placement in b_0
    s, t = fresh(); put(s, t, seq[0], 0, k)
    r = chk(s, t)
    assert r["live"] == 1 and r["bad_bucket"] == 0 and r["early_exit"] == 0
    # wrong bucket
    wrong = next(b for b in range(nb) if b not in _seq(k, nb, P))  if len(set(_seq(k, nb, P))) < nb else None
    if wrong is not None:
        s, t = fresh(); put(s, t, wrong, 0, k)
        assert chk(s, t)["bad_bucket"] == 1
    # duplicate copy
    s, t = fresh(); put(s, t, seq[0], 0, k); put(s, t, seq[0], 1, k)
    assert chk(s, t)["duplicates"] == 1
    # early exit: key in b_1 although b_0 still has an empty slot
    s, t = fresh(); put(s, t, seq[1], 0, k)
    assert chk(s, t)["early_exit"] == 1
    # ... but fine once b_0 is full
    rng = random.Random(7)
    j = 0
    while j < B:  # fillers whose own primary bucket is b_0, so they are legal
        f = rng.getrandbits(64)
        if f not in SENT and f != k and _seq(f, nb, 1)[0] == seq[0]:
            put(s, t, seq[0], j, f)
            j += 1
    r = chk(s, t)
    assert r["early_exit"] == 0 and r["live"] == B + 1
    # empty slots must form a suffix of the bucket
    s, t = fresh(); put(s, t, seq[0], 3, k)
    assert chk(s, t)["empty_not_suffix"] == 1
    # two-choice legality: b_0 or b_1 only
    h1, h2 = _fmix(k ^ S1) % nb, _fmix(k ^ S2) % nb
    b1 = h2 if h2 != h1 else (h1 + 1) % nb
    s, t = fresh(); put(s, t, b1, 0, k)
    assert chk(s, t, 1)["bad_bucket"] == 0
    other = next(b for b in range(nb) if b not in (h1, b1))
    s, t = fresh(); put(s, t, other, 0, k)
    assert chk(s, t, 1)["bad_bucket"] == 1
    if meta:
        s, t = fresh(); put(s, t, seq[0], 0, k)
        t[seq[0] * B] ^= 0x100
        assert chk(s, t)["tag_mismatch"] == 1
        s, t = fresh(); put(s, t, seq[0], 0, k)
        t[seq[0] * B] = 1  # tombstone tag over a live key
        assert chk(s, t)["tag_mismatch"] == 1


def test_candidates_full_planted(oracle_mod):
    nb, B = 8, 8
    k = 0x5555_AAAA_1234_0007
    h1, h2 = _fmix(k ^ S1) % nb, _fmix(k ^ S2) % nb
    b1 = h2 if h2 != h1 else (h1 + 1) % nb
    s = np.zeros(2 * nb * B, np.uint64)
    for b in (h1, b1):
        for j in range(B):
            s[2 * (b * B + j)] = 1000 + b * B + j
    assert oracle_mod.candidates_full(s, None, nb, B, 1, 80, S1, S2, [k]).tolist() == [True]
    s[2 * (b1 * B + 5)] = MASK  # a tombstone frees a slot
    assert oracle_mod.candidates_full(s, None, nb, B, 1, 80, S1, S2, [k]).tolist() == [False]


# --------------------------------------------------------------------------
# iceberg geometry (front yard / backyard): invariants and planted layouts
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nb", [4, 8, 64, 1024, 1 << 16])
def test_iceberg_geometry_invariants(oracle_mod, nb):
    keys = W.distinct_keys(11 + nb, 40 * nb if nb <= 1024 else 1 << 20)
    g = oracle_mod.iceberg_buckets(keys, nb, S1, S2).astype(np.int64)
    front, b1, b2 = g[:, 0], g[:, 1], g[:, 2]
    n_front = int(b1.min())
    # the front yard is a prefix, the backyard the rest; every bucket is used
    assert front.max() < n_front <= min(b1.min(), b2.min()) and max(b1.max(), b2.max()) == nb - 1
    assert np.unique(front).size == n_front and np.unique(np.concatenate([b1, b2])).size == nb - n_front
    # a backyard of about 17% of the buckets, at least two
    n_back = nb - n_front
    assert n_back >= 2 and (nb < 64 or 0.16 <= n_back / nb <= 0.18)
    assert (b1 != b2).all()
    if nb >= 64:  # uniform front and backyard choices (chi-square, generous bound)
        from scipy.stats import chisquare
        assert chisquare(np.bincount(front, minlength=n_front)).pvalue > 1e-6
        assert chisquare(np.bincount(b1 - n_front, minlength=n_back)).pvalue > 1e-6
        assert chisquare(np.bincount(b2 - n_front, minlength=n_back)).pvalue > 1e-6


def test_layout_checker_iceberg_planted(oracle_mod):
    nb, B = 16, 32
    S = nb * B
    geo = lambda ks: oracle_mod.iceberg_buckets(np.asarray(ks, np.uint64), nb, S1, S2).astype(np.int64)

    def fresh():
        return np.zeros(2 * S, np.uint64), np.zeros(S, np.uint16)

    def put(slots, tags, b, j, k, v=1):
        slots[2 * (b * B + j)] = k
        slots[2 * (b * B + j) + 1] = v
        tags[b * B + j] = _tag(k)

    chk = lambda s, t: oracle_mod.layout_check(s, t, nb, B, 2, 3, S1, S2)
    k = 0x0123_4567_89AB_CDEF
    f, c1, c2 = geo([k])[0]
    s, t = fresh(); put(s, t, f, 0, k)
    r = chk(s, t)
    assert r["live"] == 1 and r["bad_bucket"] == 0 and r["early_exit"] == 0
    other = next(b for b in range(nb) if b not in (f, c1, c2))
    s, t = fresh(); put(s, t, other, 0, k)
    assert chk(s, t)["bad_bucket"] == 1
    # backyard copy while the front bucket still has an EMPTY slot
    for c in (c1, c2):
        s, t = fresh(); put(s, t, c, 0, k)
        assert chk(s, t)["early_exit"] == 1 and chk(s, t)["bad_bucket"] == 0
    # legal once the front bucket is full (fillers whose own front is f)
    rng = random.Random(9)
    fillers = []
    while len(fillers) < B:
        x = rng.getrandbits(64)
        if x not in SENT and x != k and geo([x])[0][0] == f:
            fillers.append(x)
    for j, x in enumerate(fillers):
        put(s, t, f, j, x)
    r = chk(s, t)
    assert r["early_exit"] == 0 and r["live"] == B + 1 and r["bad_bucket"] == 0
    # a tombstone in the front does not make a backyard key illegal
    t[f * B + 7], s[2 * (f * B + 7)] = 1, MASK
    assert chk(s, t)["early_exit"] == 0
    # candidate set full only when all three buckets are
    s, t = fresh()
    for b in (f, c1, c2):
        for j in range(B):
            put(s, t, b, j, 7000 + b * B + j)
    full = lambda: oracle_mod.candidates_full(s, t, nb, B, 2, 3, S1, S2, [k]).tolist()
    assert full() == [True]
    t[c2 * B + 31] = 1  # a tombstone frees a slot of the second backyard bucket
    assert full() == [False]


# --------------------------------------------------------------------------
# probe-count recount (§5 "probe count", Table 1): hand-counted planted
# layouts.  Plain buckets cost T/2 sectors and one 128-byte line per step of
# a T-lane tile (T/B buckets side by side when T > B); fingerprint buckets
# cost a 64-byte tag line (2 sectors, 1 line) plus one sector and one line per
# candidate slot read.
# --------------------------------------------------------------------------
def _filler(rng, avoid, low16=None):
    while True:
        f = rng.getrandbits(64)
        if low16 is not None:
            f = (f & ~0xFFFF) | low16
        if f not in SENT and f not in avoid and (f & 0xFFFF) >= 2:
            return f


def test_probe_cost_planted_double_plain(oracle_mod):
    nb, B = 16, 8
    S = nb * B
    k, seq = _key_with_distinct_seq(nb, 3)
    rng = random.Random(5)

    def fresh():
        return np.zeros(2 * S, np.uint64)

    def fill(s, b, upto=B, skip=()):
        for j in range(upto):
            if j not in skip:
                s[2 * (b * B + j)] = _filler(rng, {k})

    def cost(s, tile, pmax=80, key=k):
        lines, sec, found = oracle_mod.probe_cost(s, None, nb, B, 0, pmax, S1, S2, tile, 1,
                                                  np.array([key], np.uint64))
        return int(lines[0]), int(sec[0]), bool(found[0])

    s = fresh()
    assert cost(s, 8) == (1, 4, False)          # b_0 empty: one line, then stop
    s[2 * (seq[0] * B + 3)] = k
    fill(s, seq[0], 3)
    assert cost(s, 8) == (1, 4, True)           # found in b_0
    assert cost(s, 4) == (1, 2, True)           # tile 4: slot 3 is in the first step
    s = fresh(); fill(s, seq[0], 5); s[2 * (seq[0] * B + 5)] = k
    assert cost(s, 4) == (2, 4, True)           # slot 5: second step of a 4-lane tile
    assert cost(s, 16) == (2, 8, True)          # 16 lanes read b_0 and b_1 side by side
    s = fresh(); fill(s, seq[0]); s[2 * (seq[1] * B)] = k
    assert cost(s, 8) == (2, 8, True)           # b_0 full, key in b_1
    assert cost(s, 16) == (2, 8, True)
    s = fresh(); fill(s, seq[0])
    assert cost(s, 8) == (2, 8, False)          # b_0 full, b_1 empty: a miss after two lines
    s = fresh(); fill(s, seq[0]); fill(s, seq[1]); s[2 * (seq[2] * B + 7)] = k; fill(s, seq[2], 7)
    assert cost(s, 8) == (3, 12, True)
    assert cost(s, 16) == (4, 16, True)         # second step of two buckets
    assert cost(s, 4) == (6, 12, True)          # two steps per bucket, key in the last one
    # tombstones do not end a scan
    s = fresh()
    for j in range(B):
        s[2 * (seq[0] * B + j)] = (1 << 64) - 1
    s[2 * (seq[1] * B)] = k
    assert cost(s, 8) == (2, 8, True)
    # the probe cap: every bucket full, key absent, pmax = 3
    s = fresh()
    for b in range(nb):
        fill(s, b)
    assert cost(s, 8, pmax=3) == (3, 12, False)
    assert cost(s, 16, pmax=3) == (3, 12, False)   # steps of 2 + 1 buckets
    assert cost(s, 8, pmax=80) == (nb, 4 * nb, False)  # clamped to nb
    assert cost(s, 8, key=0) == (0, 0, False)      # sentinel


def test_probe_cost_planted_two_choice_plain(oracle_mod):
    nb, B = 16, 32
    S = nb * B
    rng = random.Random(9)
    while True:
        k = rng.getrandbits(64)
        b0, b1 = _fmix(k ^ S1) % nb, _fmix(k ^ S2) % nb
        if b0 != b1:
            break

    def fresh():
        return np.zeros(2 * S, np.uint64)

    def fill(s, b, upto):
        for j in range(upto):
            s[2 * (b * B + j)] = _filler(rng, {k})

    def cost(s, never_erased, tile=8):
        lines, sec, found = oracle_mod.probe_cost(s, None, nb, B, 1, 2, S1, S2, tile, never_erased,
                                                  np.array([k], np.uint64))
        return int(lines[0]), int(sec[0]), bool(found[0])

    s = fresh(); fill(s, b0, 12)
    assert cost(s, 1) == (2, 8, False)      # 12 live < 24: the never-erased shortcut skips b_1
    assert cost(s, 0) == (3, 12, False)     # with erases behind it, b_1 is read too
    s = fresh(); fill(s, b0, 28)
    assert cost(s, 1) == (5, 20, False)     # 28 live: b_0 in four lines, then b_1's first
    s = fresh(); fill(s, b0, 32); fill(s, b1, 20); s[2 * (b1 * B + 20)] = k
    assert cost(s, 1) == (7, 28, True)      # b_0 whole, b_1 up to slot 20 (third line)
    assert cost(s, 1, tile=32) == (8, 32, True)   # a 32-lane tile reads a bucket (four lines) per step


def test_probe_cost_planted_metadata(oracle_mod):
    nb, B = 16, 32
    S = nb * B
    rng = random.Random(13)
    k, seq = _key_with_distinct_seq(nb, 21)

    def fresh():
        return np.zeros(2 * S, np.uint64), np.zeros(S, np.uint16)

    def put(s, t, b, j, key):
        s[2 * (b * B + j)] = key
        t[b * B + j] = _tag(key)

    def fill(s, t, b, upto, collide=()):
        for j in range(upto):
            f = _filler(rng, {k}, low16=(k & 0xFFFF) if j in collide else None)
            if j not in collide:
                while _tag(f) == _tag(k):
                    f = _filler(rng, {k})
            put(s, t, b, j, f)

    def cost(s, t, scheme, never_erased=1, P=80):
        lines, sec, found = oracle_mod.probe_cost(s, t, nb, B, scheme, P, S1, S2, 4, never_erased,
                                                  np.array([k], np.uint64))
        return int(lines[0]), int(sec[0]), bool(found[0])

    # double hashing: a tag collision in slot 2, the key in slot 5 of b_0
    s, t = fresh(); fill(s, t, seq[0], 5, collide=(2,)); put(s, t, seq[0], 5, k)
    assert cost(s, t, 0) == (3, 4, True)    # tag line + two candidates
    s, t = fresh(); fill(s, t, seq[0], 32)
    assert cost(s, t, 0) == (2, 4, False)   # full b_0 without a match, empty b_1: two tag lines
    s, t = fresh(); fill(s, t, seq[0], 32, collide=(7, 30))
    assert cost(s, t, 0) == (4, 6, False)   # two candidates read in vain
    # two choice: the shortcut on the tags' occupancy
    b0 = _fmix(k ^ S1) % nb
    s, t = fresh(); fill(s, t, b0, 10)
    assert cost(s, t, 1, 1, 2) == (1, 2, False)
    assert cost(s, t, 1, 0, 2) == (2, 4, False)
    s, t = fresh(); fill(s, t, b0, 24)
    assert cost(s, t, 1, 1, 2) == (2, 4, False)   # 24 live: not below 3/4, b_1 read
    # iceberg: a front bucket with an EMPTY slot ends the scan
    front = int(oracle_mod.iceberg_buckets(np.array([k], np.uint64), nb, S1, S2)[0, 0])
    s, t = fresh(); fill(s, t, front, 31)
    assert cost(s, t, 2) == (1, 2, False)
    s, t = fresh(); fill(s, t, front, 32)
    assert cost(s, t, 2) == (3, 6, False)         # full front: both backyard buckets
    t[front * B + 31] = 1                          # a tombstone is not EMPTY: still all three
    s[2 * (front * B + 31)] = (1 << 64) - 1
    assert cost(s, t, 2) == (3, 6, False)


def test_primary_bucket_is_h1(oracle_mod):
    keys = W.distinct_keys(3, 64)
    pb = oracle_mod.primary_bucket(keys, 1 << 10, S1)
    assert pb.tolist() == [_fmix(int(x) ^ S1) % (1 << 10) for x in keys]


# --------------------------------------------------------------------------
# input generators (shared by both sides) pinned to their published definitions
# --------------------------------------------------------------------------
def test_splitmix64_published_values():
    # Vigna's splitmix64.c seeded with 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, ...
    assert [int(x) for x in W.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in W.splitmix64(12345, 50)] == W.splitmix64_scalar(12345, 50)
    assert [int(x) for x in W.splitmix64(7, 10, start=5)] == W.splitmix64_scalar(7, 15)[5:]


def test_zipf_matches_exact_pmf():
    N, s, n = 20, 0.99, 400000
    r = W.zipf(11, n, N, s)
    assert r.min() >= 1 and r.max() <= N
    p = np.arange(1, N + 1, dtype=np.float64) ** -s
    p /= p.sum()
    obs = np.bincount(r, minlength=N + 1)[1:]
    chi2 = float(((obs - n * p) ** 2 / (n * p)).sum())
    assert chi2 < 60.0, chi2  # 19 dof: p < 1e-5 of exceeding by chance


def test_mixed_batch_classes_disjoint():
    ops, keys, vals = W.mixed_batch(3, n_ops=1 << 16, universe=1 << 12)
    assert ops.size == 1 << 16
    assert (ops == W.MX_ADD).sum() == 1 << 15
    cls = {}
    for o, k in zip(ops.tolist(), keys.tolist()):
        assert cls.setdefault(k, o) == o
    a = vals[ops == W.MX_ADD]
    assert a.min() >= 1 and a.max() <= 1000
