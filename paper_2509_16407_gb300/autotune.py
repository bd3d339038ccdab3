"""Autotuner: pick (scheme, metadata, bucket slots, tile) per table-size class.

The paper evaluates every (bucket, tile) combination and keeps the fastest
(§5).  This tuner does the same on the running GPU for each capacity class
(log2 of the slot count), timing each configuration of the persistent
kernel's compiled menu on the workload shape of batched mode: fill to the
target load, then as many queries, half present and half absent.  Tables of
one class are timed together in one batched launch, so small classes are
measured as they run in batched mode (many tables per launch), not as
launch-overhead-bound single calls.  Map results never depend on the choice.
"""
from __future__ import annotations

import json
import math

import numpy as np

MENU = [("double", False, 8, 4), ("double", False, 8, 8), ("double", True, 32, 4), ("double", True, 32, 8),
        ("p2", False, 32, 8), ("p2", False, 32, 32), ("p2", True, 32, 4), ("p2", True, 32, 8)]


def _keys(seed, n, device):
    import torch
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    z[(z == 0) | (z >= np.uint64((1 << 64) - 2))] = np.uint64(12345)
    return torch.from_numpy(z.view(np.int64)).to(device)


def time_config(cfg, log2_cap, load=0.85, total_slots=1 << 21, reps=3, device="cuda"):
    """Mean seconds per op of ``cfg`` on tables of 2^log2_cap slots."""
    import torch

    import paper_2509_16407_gb300 as ws
    scheme, meta, B, T = cfg
    cap = 1 << log2_cap
    n_tables = max(1, total_slots // cap)
    n_ins = int(load * cap)
    n_q = n_ins
    tables, items = [], []
    for i in range(n_tables):
        t = ws.Table(cap, scheme, meta, bucket_slots=B, tile=T)
        k = _keys(1000003 * log2_cap + i, n_ins + n_q // 2, device)
        ins, neg = k[:n_ins], k[n_ins:]
        q = torch.cat([ins[: n_q - n_q // 2], neg]).contiguous()
        out = torch.empty(q.numel(), dtype=torch.int64, device=device)
        items += [(t, ws.BK_INSERT, ins, ins, None, None, 0), (t, ws.BK_QUERY, q, None, out, None, 1)]
        tables.append(t)
    plan = ws.BatchPlan(items)
    best = math.inf
    for _ in range(reps + 1):
        for t in tables:
            t.clear()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.launch()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    plan.close()
    for t in tables:
        t.close()
    return best / (n_tables * (n_ins + n_q))


def tune(log2_caps=range(10, 23), load=0.85, menu=MENU, reps=3, device="cuda", log=None):
    """{log2_cap: config} of the fastest menu configuration per class, plus
    the measured ns/op of every configuration."""
    import torch
    choice, timings = {}, {}
    for lc in log2_caps:
        row = {}
        for cfg in menu:
            row[cfg] = time_config(cfg, lc, load=load, reps=reps, device=device) * 1e9
            torch.cuda.empty_cache()
        best = min(row, key=row.get)
        choice[lc] = best
        timings[lc] = {"/".join(map(str, k)): round(v, 3) for k, v in row.items()}
        if log:
            log(json.dumps({"log2_cap": lc, "best": "/".join(map(str, best)), "ns_per_op": timings[lc]}))
    return choice, timings


def config_for(capacity: int, choice: dict):
    """The tuned configuration for a table of ``capacity`` slots (nearest class)."""
    lc = max(1, int(round(math.log2(max(2, capacity)))))
    keys = sorted(choice)
    lc = min(keys, key=lambda k: abs(k - lc))
    return choice[lc]
