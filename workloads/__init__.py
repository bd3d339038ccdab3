"""Seeded synthetic inputs for the hash-table path (shared by tests and bench).

This module holds input generation only -- no hashing, probing or map
arithmetic of the method -- so that both the oracle side and the CUDA side of
a test draw the very same inputs from it.

Generators (each from its published definition):

* ``splitmix64`` -- Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators" (OOPSLA 2014), in the form of Vigna's reference ``splitmix64.c``:
  the state advances by the golden gamma 0x9e3779b97f4a7c15 and each output is
  the variant-13 finaliser of the new state.  The finaliser is a bijection of
  64-bit words, so one stream never repeats within 2^64 draws and distinct
  keys come for free.
* ``zipf`` -- rejection-inversion sampling of a Zipf(s) law on {1..N}
  (Hoermann & Derflinger, "Rejection-inversion to generate variates from
  monotone discrete distributions", ACM TOMACS 1996).

Keys 0, 2^64-1 and 2^64-2 are the table's reserved sentinels and are never
produced by the key generators here.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SENTINELS = (0, (1 << 64) - 1, (1 << 64) - 2)


def mix13(z: np.ndarray) -> np.ndarray:
    """splitmix64 output finaliser (variant 13) on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+n-1`` of the splitmix64 stream seeded by ``seed``.

    Output i (0-based) is mix13(seed + (i+1) * gamma) mod 2^64.
    """
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & ((1 << 64) - 1)) + idx * GOLDEN
    return mix13(state)


def splitmix64_scalar(seed: int, n: int):
    """Pure-Python big-int splitmix64 (used to pin the vectorised version)."""
    m = (1 << 64) - 1
    x = seed & m
    out = []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & m
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def _drop_sentinels(a: np.ndarray) -> np.ndarray:
    bad = (a == np.uint64(0)) | (a >= np.uint64((1 << 64) - 2))
    return a[~bad] if bad.any() else a


def distinct_keys(seed: int, n: int, start: int = 0) -> np.ndarray:
    """``n`` distinct non-sentinel uniform keys: the splitmix64 stream from
    position ``start`` with the (astronomically rare) sentinel outputs skipped.
    Distinct because the finaliser is a bijection of distinct states."""
    out = _drop_sentinels(splitmix64(seed, n, start))
    extra = start + n
    while out.size < n:
        more = _drop_sentinels(splitmix64(seed, n - out.size, extra))
        extra += n - out.size
        out = np.concatenate([out, more])
    return out[:n]


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the splitmix64 stream."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def permutation(seed: int, n: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1: the order of n distinct
    splitmix64 draws (no ties are possible)."""
    return np.argsort(splitmix64(seed, n), kind="stable")


def uniform_int(seed: int, n: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) by multiply-shift of the top
    32 bits (bias < 2^-22 for ranges below 1024)."""
    r = splitmix64(seed, n, start) >> np.uint64(32)
    span = np.uint64(hi - lo + 1)
    return (np.uint64(lo) + ((r * span) >> np.uint64(32))).astype(np.uint64)


# --------------------------------------------------------------------------
# Zipf(s) on {1..N} by rejection-inversion.
# H(x) = (x^(1-s) - 1)/(1-s) is an antiderivative of the hat x^-s; a uniform
# point of [H(N+1/2), H(3/2) - 1] is mapped back through H^-1, rounded to the
# nearest integer k, and accepted when it falls under the histogram of the
# exact mass k^-s (the squeeze k - x <= s_div accepts most draws at once).
# --------------------------------------------------------------------------
def _H(x, s):
    return np.log(x) if s == 1.0 else (np.power(x, 1.0 - s) - 1.0) / (1.0 - s)


def _Hinv(y, s):
    return np.exp(y) if s == 1.0 else np.power(1.0 + y * (1.0 - s), 1.0 / (1.0 - s))


def zipf(seed: int, n: int, N: int, s: float) -> np.ndarray:
    """``n`` Zipf(s) ranks in 1..N (int64), deterministic in ``seed``."""
    h_x1 = _H(1.5, s) - 1.0
    h_n = _H(N + 0.5, s)
    s_div = 2.0 - _Hinv(_H(2.5, s) - 2.0 ** (-s), s)
    out = np.empty(n, np.int64)
    filled = 0
    pos = 0
    while filled < n:
        m = max(1024, int((n - filled) * 1.15))
        u = uniform01(seed, m, pos)
        pos += m
        y = h_n + u * (h_x1 - h_n)
        x = _Hinv(y, s)
        k = np.clip(np.floor(x + 0.5), 1, N)
        ok = (k - x <= s_div) | (y >= _H(k + 0.5, s) - np.power(k, -s))
        acc = k[ok].astype(np.int64)
        take = min(acc.size, n - filled)
        out[filled:filled + take] = acc[:take]
        filled += take
    return out


def rank_to_key(ranks: np.ndarray, universe_seed: int = 0) -> np.ndarray:
    """Bijective map of ranks (1 <= rank < 2^40) to uniform-looking non-zero
    keys: the splitmix64 finaliser of rank + universe_seed * 2^40 (never 0, so
    the finaliser never returns 0)."""
    r = np.asarray(ranks, dtype=np.uint64)
    with np.errstate(over="ignore"):
        k = mix13(r + np.uint64(universe_seed) * np.uint64(1 << 40))
    if ((k == np.uint64(0)) | (k >= np.uint64((1 << 64) - 2))).any():
        raise ValueError("rank_to_key produced a sentinel; choose another universe seed")
    return k


# --------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------
def pr1(S: int = 1 << 20, load: float = 0.9, seed: int = 1, erase_seed: int = 2):
    """PR1: insert floor(load*S) keys of the seed stream with value 3k, query
    them plus as many absent keys (the continued stream), erase a random half.
    Returns (keys, vals, absent, erase_idx)."""
    K = int(load * S)
    both = distinct_keys(seed, 2 * K)
    keys, absent = both[:K], both[K:]
    with np.errstate(over="ignore"):
        vals = keys * np.uint64(3)
    perm = permutation(erase_seed, K)
    erase_idx = perm[: K // 2]
    return keys, vals, absent, erase_idx


# op codes of a mixed batch (documented interface values)
MX_QUERY, MX_INSERT, MX_ADD, MX_MAX, MX_REPLACE, MX_ERASE = 0, 1, 2, 3, 4, 5


def mixed_batch(batch_seed: int, n_ops: int = 1 << 24, universe: int = 1 << 26,
                s: float = 0.99, up_frac: float = 0.5, q_frac: float = 0.4,
                universe_seed: int = 0):
    """One mixed batch: Zipf(s) keys over ``universe`` ranks; each key's class
    (upsert-add / query / erase) is fixed per batch by a splitmix64 draw of
    key ^ batch_seed mod 10 (0-4 upsert, 5-8 query, 9 erase), which makes the
    three classes key-disjoint.  Draws are taken in order and kept while their
    class still has quota.  Upsert values are uniform in [1, 1000].
    Returns (ops u8, keys u64, vals u64)."""
    n_up = int(round(n_ops * up_frac))
    n_q = int(round(n_ops * q_frac))
    n_er = n_ops - n_up - n_q
    quota = {MX_ADD: n_up, MX_QUERY: n_q, MX_ERASE: n_er}
    ops_parts, key_parts = [], []
    pos_seed = batch_seed * 1000003 + 7
    round_no = 0
    while any(v > 0 for v in quota.values()):
        m = max(4096, int(sum(quota.values()) * 1.3))
        ranks = zipf(pos_seed + round_no, m, universe, s)
        round_no += 1
        keys = rank_to_key(ranks, universe_seed)
        cls = (mix13(keys ^ np.uint64(batch_seed & ((1 << 64) - 1))) % np.uint64(10)).astype(np.int64)
        op = np.where(cls <= 4, MX_ADD, np.where(cls <= 8, MX_QUERY, MX_ERASE)).astype(np.uint8)
        keep = np.zeros(m, bool)
        for code in (MX_ADD, MX_QUERY, MX_ERASE):
            idx = np.nonzero(op == code)[0][: quota[code]]
            keep[idx] = True
            quota[code] -= idx.size
        ops_parts.append(op[keep])
        key_parts.append(keys[keep])
    ops = np.concatenate(ops_parts)
    keys = np.concatenate(key_parts)
    vals = uniform_int(batch_seed + 0x51, ops.size, 1, 1000)
    vals[ops != MX_ADD] = 0
    return ops, keys, vals


def mixed_batch_codes(batch_seed: int, n_ops: int = 1 << 20, universe: int = 1 << 18, s: float = 0.99,
                      universe_seed: int = 0):
    """A mixed batch that uses every op code: Zipf(s) keys over ``universe``
    ranks; a key's code is fixed for the batch by a splitmix64 draw of
    key ^ batch_seed mod 20 (0-3 add, 4-5 max, 6-7 replace, 8-9 insert,
    10-17 query, 18-19 erase), so every key has one code per batch and the
    query / erase / upsert classes are key-disjoint.  Draws are taken in
    order (no quotas: the mix follows the Zipf mass of each class).  Values:
    add uniform in [1, 1000]; max, replace and insert uniform in [1, 2^40]
    per op, so duplicate replace / insert copies of one key carry different
    values.  Returns (ops u8, keys u64, vals u64)."""
    ranks = zipf(batch_seed * 1000003 + 11, n_ops, universe, s)
    keys = rank_to_key(ranks, universe_seed)
    c20 = (mix13(keys ^ np.uint64(batch_seed & ((1 << 64) - 1))) % np.uint64(20)).astype(np.int64)
    table = np.array([MX_ADD] * 4 + [MX_MAX] * 2 + [MX_REPLACE] * 2 + [MX_INSERT] * 2 + [MX_QUERY] * 8
                     + [MX_ERASE] * 2, np.uint8)
    ops = table[c20]
    vals = uniform_int(batch_seed + 0x61, n_ops, 1, (1 << 40))
    add = ops == MX_ADD
    vals[add] = uniform_int(batch_seed + 0x62, int(add.sum()), 1, 1000)
    vals[(ops == MX_QUERY) | (ops == MX_ERASE)] = 0
    return ops, keys, vals


def mixed_request_codes(seed: int, n: int, universe: int, universe_seed: int, s: float = 0.99):
    """A serving request that uses every op code, with results that do not
    depend on which concurrent copy of a key wins: a key's code is fixed per
    request by a splitmix64 draw of key ^ seed mod 20 (10 query, 4 add, 2
    max, 2 replace, 1 insert, 1 erase); every replace and insert copy of one
    key carries the same value (derived from the key and the request), max
    values are uniform in [1, 2^40] (max is commutative), add values in
    [1, 1000].  Returns (ops u8, keys u64, vals u64)."""
    ranks = zipf(seed * 7 + 3, n, universe, s)
    keys = rank_to_key(ranks, universe_seed)
    c20 = (mix13(keys ^ np.uint64(seed & ((1 << 64) - 1))) % np.uint64(20)).astype(np.int64)
    table = np.array([MX_QUERY] * 10 + [MX_ADD] * 4 + [MX_MAX] * 2 + [MX_REPLACE] * 2 + [MX_INSERT, MX_ERASE],
                     np.uint8)
    ops = table[c20]
    vals = uniform_int(seed + 0x91, n, 1, 1000)
    mx = ops == MX_MAX
    vals[mx] = uniform_int(seed + 0x92, int(mx.sum()), 1, 1 << 40)
    one = (ops == MX_REPLACE) | (ops == MX_INSERT)
    vals[one] = mix13(keys[one] ^ np.uint64((seed * 0x2545F491) & ((1 << 64) - 1))) % np.uint64(1 << 40) \
        + np.uint64(1)
    vals[(ops == MX_QUERY) | (ops == MX_ERASE)] = 0
    return ops, keys, vals


def log_uniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers whose log2 is uniform in [log2 lo, log2 hi] (rounded down)."""
    u = uniform01(seed, n)
    v = np.exp2(np.log2(lo) + u * (np.log2(hi) - np.log2(lo)))
    return np.clip(np.floor(v), lo, hi).astype(np.int64)


def mixed_request(seed: int, n: int, universe: int, universe_seed: int, s: float = 0.99,
                  fracs=(0.6, 0.3, 0.05, 0.05)):
    """One serving request of ``n`` ops on one table: Zipf(s) keys over the
    table's ``universe`` ranks (keys bijective in the rank and
    ``universe_seed``), op classes query / upsert-add / insert / erase with
    quotas ``fracs``.  A key's class is fixed for the request by a splitmix64
    draw of key ^ seed mod 20 (12 query, 6 add, 1 insert, 1 erase), so the
    classes are key-disjoint; draws are kept in order while their class has
    quota.  All inserts of one key carry the same value, so the result does
    not depend on which concurrent copy wins.  Returns (ops u8, keys u64,
    vals u64)."""
    quota = [int(round(n * f)) for f in fracs]
    quota[0] += n - sum(quota)
    codes = (MX_QUERY, MX_ADD, MX_INSERT, MX_ERASE)
    bounds = (12, 18, 19, 20)
    ops_parts, key_parts = [], []
    rnd = 0
    while sum(quota) > 0:
        m = max(64, int(sum(quota) * 1.5))
        ranks = zipf(seed * 7 + 1 + rnd * 1000003, m, universe, s)
        rnd += 1
        keys = rank_to_key(ranks, universe_seed)
        c20 = (mix13(keys ^ np.uint64(seed & ((1 << 64) - 1))) % np.uint64(20)).astype(np.int64)
        cls = np.searchsorted(np.array(bounds), c20, side="right")
        keep = np.zeros(m, bool)
        for ci in range(4):
            if quota[ci] <= 0:
                continue
            idx = np.nonzero(cls == ci)[0][: quota[ci]]
            keep[idx] = True
            quota[ci] -= idx.size
        ops_parts.append(np.array(codes, np.uint8)[cls[keep]])
        key_parts.append(keys[keep])
        if rnd == 200:  # a class whose keys carry almost no Zipf mass: its quota goes to queries
            quota[0] += sum(quota[1:])
            quota[1:] = [0, 0, 0]
    ops = np.concatenate(ops_parts)[:n]
    keys = np.concatenate(key_parts)[:n]
    vals = uniform_int(seed + 0x77, n, 1, 1000)
    # insert-if-unique copies of one key carry one value (derived from the
    # key): which copy wins is a race, the stored value is not
    ins = ops == MX_INSERT
    vals[ins] = mix13(keys[ins] ^ np.uint64(0x1D5)) % np.uint64(999) + np.uint64(1)
    return ops, keys, vals
