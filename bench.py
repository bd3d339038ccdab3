#!/usr/bin/env python
"""Benchmark of the batched hash-table path on GB300.

Default workload (one JSON line): four 2^28-slot tables -- DoubleHT,
DoubleHT(M), P2HT, P2HT(M), paper-default bucket and tile sizes -- each
prefilled to 0.85 load outside the timed region.  One step, per table:
  insert a 5% slice of new keys (0.85 -> 0.90 load), query 2^24 present keys,
  query 2^24 absent keys, upsert-add 2^24 present keys (values in [1, 1000]),
  erase the slice again (0.90 -> 0.85), read the live count.
``value`` = all ops of all tables / device time of K steps (Gops/s); ``e2e``
times the same steps through the C ABI with pinned host buffers (copies in).
Unless --no-extra, the line also carries the read-bandwidth probes, the same
step on 2^22-slot (L2-resident) tables, the batched leg (1024 tables, one
graph launch vs per-table launches), the serving leg (p50/p99 and Gops/s,
continuous batching vs per-request launches) and config 3's mixed Zipf
batches on 2^27-slot tables.

--impl reference: the CPU oracle (the map definition, single thread) on a
bounded sample of the same step; ``--sweep`` writes the load/tile sweep.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

DESIGNS = [("double", False, "DoubleHT"), ("double", True, "DoubleHT(M)"), ("p2", False, "P2HT"),
           ("p2", True, "P2HT(M)")]
# the front-yard / backyard table: not one of the four designs of the default
# line; selectable with --designs and part of the aging / phased comparisons
ICEBERG = ("iceberg", True, "IcebergHT(M)")
ALL_DESIGNS = DESIGNS + [ICEBERG]
METRIC = "Gops/s insert/query/upsert at 0.9 load; % of HBM roofline; serve p50/p99 latency"
UNIT = "Gops/s"
PHASES = ["insert", "query_pos", "query_neg", "upsert_add", "erase"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--log2-slots", type=int, default=28)
    p.add_argument("--load", type=float, default=0.9)
    p.add_argument("--nq", type=int, default=1 << 24, help="queries / upserts per phase")
    p.add_argument("--designs", default="all")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--sweep", default="", help="write the load/tile sweep as JSON lines to this file")
    p.add_argument("--sweep-log2-slots", default="28,22")
    p.add_argument("--aging-log2-slots", type=int, default=26)
    p.add_argument("--aging-iters", type=int, default=1000)
    p.add_argument("--workload", default="config2", choices=["config2", "batched", "serve", "aging", "phased", "mixed"],
                   help="config2 = the default line; batched = 1024 uneven tables in one graph launch")
    p.add_argument("--tables", type=int, default=1024)
    p.add_argument("--requests", type=int, default=600, help="serve: requests per run")
    p.add_argument("--host-direct", type=int, default=1, choices=[0, 1, 2, 3],
                   help="e2e: page-locked host buffers staged (0), inputs read in place (1, the library's "
                        "default), inputs and results in place (2), in place for inserts and erases and "
                        "staged otherwise (3)")
    p.add_argument("--no-extra", action="store_true",
                   help="default line only: skip the read-peak probes, the L2-resident leg, the short "
                        "batched and serving legs and the config-3 mixed-batch leg")
    p.add_argument("--serve-requests", type=int, default=240, help="requests of the default line's serving leg")
    p.add_argument("--tiles", default="auto", choices=["auto", "paper", "4", "8", "16", "32"],
                   help="auto: per design, the tile size with the fastest step (measured before timing); "
                        "paper: each design's tile from the paper; a number: that tile for every design")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def to_dev(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(dev, non_blocking=False)


def splitmix_torch(seed, n, start, dev):
    """The splitmix64 stream (positions start .. start+n-1) computed on the
    device in wrapping int64 arithmetic (same bits as workloads.splitmix64)."""
    import torch
    def s64(x):
        x &= (1 << 64) - 1
        return x - (1 << 64) if x >= 1 << 63 else x
    def srl(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)
    z = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=dev) * s64(0x9E3779B97F4A7C15) + s64(seed)
    z = (z ^ srl(z, 30)) * s64(0xBF58476D1CE4E5B9)
    z = (z ^ srl(z, 27)) * s64(0x94D049BB133111EB)
    z = z ^ srl(z, 31)
    if bool(((z == 0) | (z == -1) | (z == -2)).any()):
        raise RuntimeError("sentinel drawn from the key stream; pick another seed")
    return z


def gen_dev(seed, n, start, dev, chunk=1 << 24):
    """The splitmix64 key stream (positions start .. start+n-1) on the device."""
    import torch
    out = torch.empty(n, dtype=torch.int64, device=dev)
    for off in range(0, n, chunk):
        m = min(chunk, n - off)
        k = W.splitmix64(seed, m, start + off)
        if ((k == np.uint64(0)) | (k >= np.uint64((1 << 64) - 2))).any():
            raise RuntimeError("sentinel drawn from the key stream; pick another seed")
        out[off:off + m].copy_(torch.from_numpy(k.view(np.int64)))
    return out


def aggregate(ms, ops_per_rank, world, device=None):
    """Whole-job throughput under the multi-rank contract: every rank's time is
    reduced with MAX over ranks, ops are summed over ranks (weak scaling, each
    rank owns its own tables).  Returns (max_ms, Gops/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms), float(ops_per_rank)], dtype=torch.float64, device=device)
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = t[1:].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms, ops = float(mx.item()), float(tot.item())
    else:
        ops = float(ops_per_rank)
    return ms, ops / (ms * 1e-3) / 1e9


def peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def read_peaks(dev_index=0):
    """Memory rates of this GPU measured by the library's probe kernel
    (ws_read_bandwidth; CUDA events, best of five): sequential reads of an
    L2-resident buffer (the peak for tables that fit in L2) and of a 4 GiB
    buffer, and random 128-, 64- and 32-byte reads and 32- and 128-byte writes
    over 4 GiB, each at the in-flight depth (1-8 blocks per group of lanes)
    that runs fastest.  Random accesses per second are the bound of the hash
    table's probes: every probe step is one random line."""
    import ctypes
    import paper_2509_16407_gb300 as ws
    L = ws.lib()

    def rate(nbytes, pattern, passes, depths=(1, 2, 4, 8)):
        best, best_d = 0.0, None
        for d in depths:
            g = ctypes.c_double(0.0)
            if L.ws_read_bandwidth(nbytes, pattern, d, passes, dev_index, ctypes.byref(g)) == 0 and g.value > best:
                best, best_d = g.value, d
        return round(best, 1), best_d

    out = {}
    for name, nbytes, pattern, passes in (("l2_seq_32MiB", 32 << 20, 0, 200), ("l2_seq_64MiB", 64 << 20, 0, 100),
                                          ("hbm_seq_4GiB", 4 << 30, 0, 2)):
        out[name] = rate(nbytes, pattern, passes, depths=(1,))[0]
    out["l2_lines_64MiB"], _ = rate(64 << 20, 1, 50)
    for name, pattern, w in (("hbm_rand128", 1, 128), ("hbm_rand64", 2, 64), ("hbm_rand32", 3, 32),
                             ("hbm_wr32", 4, 32), ("hbm_wr128", 5, 128)):
        gbs, d = rate(4 << 30, pattern, 2)
        out[name + "_gbs"] = gbs
        out[name + "_gaccess_s"] = round(gbs / w, 2)
        out[name + "_depth"] = d
    l2 = [out[k] for k in ("l2_seq_32MiB", "l2_seq_64MiB") if out.get(k)]
    out["l2_peak_gbs"] = max(l2) if l2 else None
    out["how"] = ("ws_read_bandwidth: .cg 16-byte accesses, buffer touched once to warm, then `passes` sweeps "
                  "timed with CUDA events, best of 5; randN / wrN = random N-byte blocks read / written by N/16 "
                  "lanes together, best in-flight depth of 1, 2, 4, 8 blocks per group")
    return out


def kernel_source_hash():
    """Hash of the sources of the single-table kernels the default line runs
    (device header, kernel templates, instantiation units): recorded DRAM
    traffic is valid only for the kernels it was measured on."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2509_16407_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in ("ws_device.cuh", "ws_kernels.cuh") or (f.startswith("ws_inst_") and f.endswith(".cu")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of
    each design:phase kernel of the default workload, from the committed ncu
    summary (measured on 2^26-slot tables and scaled by the ops per launch,
    which grow 4x to 2^28; the tile changes them by under 2%); empty when the
    kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_config2.txt")
    out, src = {}, None
    try:
        with open(path) as f:
            for ln in f:
                ln = ln.split("#", 1)[0].split()
                if len(ln) == 2 and ln[0] == "source_hash":
                    src = ln[1]
                elif len(ln) == 2 and ln[0].count(":") == 1:  # design:phase bytes
                    out[ln[0]] = float(ln[1])
    except OSError:
        return {}
    return out if src == kernel_source_hash() else {}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def config2_workload(args, names):
    """The default line's workload, as both arms name it."""
    lq = int(np.log2(args.nq))
    return (f"2^{args.log2_slots}-slot tables at {args.load} load (0.85 -> {args.load} slice insert,"
            f" 2^{lq} positive + negative queries, 2^{lq} upsert-add, slice erase, count), designs {names}")


def bench_ours(args, rank, world, peak_override=None, access_peak=None):
    import torch
    import paper_2509_16407_gb300 as ws

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    S = 1 << args.log2_slots
    base_n = int(0.85 * S)
    top_n = int(args.load * S)
    slice_n = top_n - base_n
    nq = args.nq
    designs = DESIGNS if args.designs == "all" else [d for d in ALL_DESIGNS if d[2] in args.designs.split(",")]
    seed = 0x5EED + 7919 * rank

    # device-resident inputs (one key stream: base | slice | absent)
    keys_base = gen_dev(seed, base_n, 0, dev)
    keys_slice = gen_dev(seed, slice_n, base_n, dev)
    keys_neg = gen_dev(seed, nq, top_n, dev)
    vals_base = keys_base * 3
    vals_slice = keys_slice * 3
    pos_idx = torch.from_numpy((W.splitmix64(seed + 1, nq) % np.uint64(top_n)).astype(np.int64)).to(dev)
    allk = torch.cat([keys_base, keys_slice])
    keys_pos = allk[pos_idx].contiguous()
    del allk
    up_idx = torch.from_numpy((W.splitmix64(seed + 2, nq) % np.uint64(base_n)).astype(np.int64)).to(dev)
    keys_up = keys_base[up_idx].contiguous()
    vals_up = torch.from_numpy(W.uniform_int(seed + 3, nq, 1, 1000).view(np.int64)).to(dev)
    out_q = torch.empty(nq, dtype=torch.int64, device=dev)

    tables = []
    for scheme, meta, name in designs:
        t = ws.Table(S, scheme, meta)
        t.insert(keys_base, vals_base)
        torch.cuda.synchronize()
        assert t.count() == base_n, (name, t.count())
        assert t.last_error()["status"] == 0, name
        tables.append((name, t))

    stream = torch.cuda.current_stream(dev)

    def one_design_step(t):
        t.insert(keys_slice, vals_slice)
        t.query(keys_pos, out=out_q)
        t.query(keys_neg, out=out_q)
        t.upsert(keys_up, vals_up, op="add")
        t.erase(keys_slice)

    tuning = {}
    if args.tiles not in ("auto", "paper"):
        for name, t in tables:
            t.set_tile(int(args.tiles))
    if args.tiles == "auto":
        # the paper keeps each design's fastest (bucket, tile) combination;
        # here: the tile with the fastest step, measured once per design
        for name, t in tables:
            best = None
            for T in (4, 8, 16, 32):
                t.set_tile(T)
                one_design_step(t)  # warm
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                one_design_step(t)
                b.record(stream)
                torch.cuda.synchronize()
                ms_t = a.elapsed_time(b)
                tuning.setdefault(name, {})[T] = round(ms_t, 3)
                if best is None or ms_t < best[1]:
                    best = (T, ms_t)
            t.set_tile(best[0])
            assert t.count() == base_n

    def step(evs=None):
        for di, (name, t) in enumerate(tables):
            if evs is not None:
                evs[di][0].record(stream)
            t.insert(keys_slice, vals_slice)
            if evs is not None:
                evs[di][1].record(stream)
            t.query(keys_pos, out=out_q)
            if evs is not None:
                evs[di][2].record(stream)
            t.query(keys_neg, out=out_q)
            if evs is not None:
                evs[di][3].record(stream)
            t.upsert(keys_up, vals_up, op="add")
            if evs is not None:
                evs[di][4].record(stream)
            t.erase(keys_slice)
            if evs is not None:
                evs[di][5].record(stream)
        for name, t in tables:
            c = t.count()
            if c != base_n:
                raise RuntimeError(f"{name}: count {c} != {base_n} after a step")

    ops_per_table = 2 * slice_n + 3 * nq
    ops_per_step = ops_per_table * len(tables)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # probe costs (lines / sectors per op) measured on the live tables, untimed
    sample = 1 << 20
    costs = {}
    for name, t in tables:
        # counted with one cache line per probe step (T = 8, or B when smaller),
        # the method's own line count; a wider tile reads ahead speculatively
        t_run = t.info()["tile"]
        t.set_tile(min(8, t.info()["bucket_slots"]))
        c = {}
        cs, _ = t.probe_cost(keys_slice[:sample])  # insert scan cost at 0.85 load
        c["insert"] = cs
        t.insert(keys_slice, vals_slice)
        c["query_pos"], _ = t.probe_cost(keys_pos[:sample])
        c["query_neg"], _ = t.probe_cost(keys_neg[:sample])
        c["upsert_add"], _ = t.probe_cost(keys_up[:sample])
        c["erase"], _ = t.probe_cost(keys_slice[:sample])
        t.erase(keys_slice)
        t.set_tile(t_run)
        torch.cuda.synchronize()
        costs[name] = {}
        for ph, v in c.items():
            v = v.cpu().numpy().view(np.uint64)
            costs[name][ph] = {"sectors": float((v & np.uint64(0xFFFFFFFF)).mean()),
                               "lines": float((v >> np.uint64(32)).mean())}

    meta_of = {d[2]: d[1] for d in designs}

    def alg_bytes(name, ph):
        sec = costs[name][ph]["sectors"] * 32.0
        m = meta_of[name]
        if ph == "insert":      # scan + written slot sector (+ tag sector) + key, value in
            return sec + 32 + (32 if m else 0) + 16
        if ph in ("query_pos", "query_neg"):  # scan + key in, value out
            return sec + 16
        if ph == "upsert_add":  # scan + value sector write-back + key, value in
            return sec + 32 + 16
        return sec + 32 + (32 if m else 0) + 8  # erase: scan + slot (+ tag) write + key in

    def line_bytes(name, ph):
        """The same count with every line the probe touches charged 128 bytes:
        random DRAM reads on this part move whole 128-byte lines, so a 64-byte
        tag line or a 16-byte candidate slot costs as much as a full line."""
        return alg_bytes(name, ph) + (costs[name][ph]["lines"] * 128.0 - costs[name][ph]["sectors"] * 32.0)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in tables] for _ in range(args.steps)]
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms, value = aggregate(t0.elapsed_time(t1), ops_per_step * args.steps, world, dev)

    # per-phase times, achieved bandwidth and probe costs
    peak, peak_kind = peak_override if peak_override else peak_gbs()
    phase_ms = {name: {ph: 0.0 for ph in PHASES} for name, _ in tables}
    for k in range(args.steps):
        for di, (name, _) in enumerate(tables):
            for pi, ph in enumerate(PHASES):
                phase_ms[name][ph] += evs[k][di][pi].elapsed_time(evs[k][di][pi + 1])
    n_of = {"insert": slice_n, "query_pos": nq, "query_neg": nq, "upsert_add": nq, "erase": slice_n}
    breakdown = {}
    dom = None
    for name, _ in tables:
        breakdown[name] = {}
        for ph in PHASES:
            per_launch_ms = phase_ms[name][ph] / args.steps
            b = alg_bytes(name, ph)
            gbs = b * n_of[ph] / (per_launch_ms * 1e-3) / 1e9
            lb = line_bytes(name, ph)
            lgbs = lb * n_of[ph] / (per_launch_ms * 1e-3) / 1e9
            # random DRAM accesses per op: every line the probe reads, plus one
            # write-back per written sector (slot / value, and the tag with metadata)
            writes = {"insert": 2 if meta_of[name] else 1, "upsert_add": 1,
                      "erase": 2 if meta_of[name] else 1}.get(ph, 0)
            acc = costs[name][ph]["lines"] + writes
            gacc = acc * n_of[ph] / (per_launch_ms * 1e-3) / 1e9
            breakdown[name][ph] = {
                "gops": round(n_of[ph] / (per_launch_ms * 1e-3) / 1e9, 3),
                "ms": round(per_launch_ms, 4),
                "alg_bytes_per_op": round(b, 1),
                "lines_per_op": round(costs[name][ph]["lines"], 3),
                "sectors_per_op": round(costs[name][ph]["sectors"], 3),
                "achieved_gbs": round(gbs, 1),
                "frac_of_measured_hbm": round(gbs / peak, 4),
                "line_bytes_per_op": round(lb, 1),
                "frac_line_granularity": round(lgbs / peak, 4),
                "accesses_per_op": round(acc, 3),
                "gaccess_s": round(gacc, 2),
            }
            if access_peak:
                breakdown[name][ph]["frac_of_random_line_rate"] = round(gacc / access_peak, 4)
            if dom is None or per_launch_ms > dom[2]:
                dom = (name, ph, per_launch_ms, gbs, b * n_of[ph])
    kernel_names = {"insert": "batch_kernel<KIND_UPSERT, op=insert>", "query_pos": "batch_kernel<KIND_QUERY>",
                    "query_neg": "batch_kernel<KIND_QUERY>", "upsert_add": "batch_kernel<KIND_UPSERT, op=add>",
                    "erase": "batch_kernel<KIND_ERASE>"}
    tr = recorded_traffic()
    tile_of = {name: t.info()["tile"] for name, t in tables}
    # recorded DRAM traffic exists for the default workload only
    default_wl = args.log2_slots == 28 and args.nq == 1 << 24 and args.load == 0.9
    traffic = tr.get(f"{dom[0]}:{dom[1]}") if default_wl else None
    roofline = {"bound": "hbm", "achieved": round(dom[3], 1), "peak": peak, "unit": "GB/s",
                "frac": round(dom[3] / peak, 4), "traffic": traffic,
                "kernel": f"{dom[0]} {dom[1]}: {kernel_names[dom[1]]}",
                "alg_bytes_per_launch": int(dom[4]),
                "peak_kind": peak_kind if peak_override else f"{peak_kind} (burst copy)"}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = bench_e2e(args, tables, keys_slice, vals_slice, keys_pos, keys_neg, keys_up, vals_up, base_n,
                        ops_per_step, world, dev)

    launches = args.steps * len(tables) * len(PHASES)
    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {
            "workload": config2_workload(args, [d[2] for d in designs]),
            "slots": S, "load": args.load, "base_keys": base_n, "slice_keys": slice_n, "queries": nq,
            "ops_per_step": ops_per_step * world, "ops_per_step_per_gpu": ops_per_step,
            "tiles": {d[2]: t.info()["tile"] for d, (_, t) in zip(designs, tables)},
            "tile_choice": args.tiles, "tile_tuning_ms_per_step": tuning,
            "bucket_slots": {d[2]: t.info()["bucket_slots"] for d, (_, t) in zip(designs, tables)},
            "l2": (f"inputs larger than L2, no flush: each table ({S * 16 / 2**30:.2f} GiB of slots, "
                   f"{S * 16 / 129e6:.0f}x the 129 MB L2) is probed at random; query/upsert key arrays are "
                   f"{nq * 8 / 1e6:.0f} MB") if S * 16 > 129e6 else
                  (f"L2-resident tables, no flush: {S * 16 / 2**20:.0f} MiB of slots per table, which L2 holds "
                   f"while the table's phases run; query/upsert key arrays are {nq * 8 / 1e6:.0f} MB"),
            "parallelism": f"replicas x{world}",
        },
        "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "breakdown": breakdown,
    }
    return result


def bench_l2_leg(args, rank, world, peaks):
    """The default step on 2^22-slot tables (64 MiB of slots, each table
    L2-resident while its phases run) with the same 2^24 queries / upserts per
    phase; fractions against the measured L2 read peak instead of HBM, and
    random-line rates against the measured rate of random 128-byte L2 reads."""
    import copy
    import torch
    a = copy.copy(args)
    a.log2_slots, a.no_e2e = 22, True
    l2_peak = peaks["l2_peak_gbs"]
    lines = peaks.get("l2_lines_64MiB")
    r = bench_ours(a, rank, world, peak_override=(l2_peak, "measured L2 read, sequential (ws_read_bandwidth)"),
                   access_peak=lines / 128.0 if lines else None)
    torch.cuda.empty_cache()
    bd = {}
    for name, phases in r["breakdown"].items():
        bd[name] = {}
        for ph, d in phases.items():
            d = dict(d)
            d["frac_of_l2_peak"] = d.pop("frac_of_measured_hbm")
            d.pop("frac_line_granularity", None)
            d.pop("line_bytes_per_op", None)
            if "frac_of_random_line_rate" in d:
                d["frac_of_l2_random_line_rate"] = d.pop("frac_of_random_line_rate")
            bd[name][ph] = d
    roof = dict(r["roofline"], bound="l2")
    return {"workload": r["config"]["workload"], "value": r["value"], "unit": UNIT, "steps": r["steps"],
            "ms_per_step": r["ms_per_step"], "l2_peak_gbs": l2_peak, "l2_random_line_gbs": lines,
            "tiles": r["config"]["tiles"], "l2": r["config"]["l2"],
            "roofline": roof, "clocks": r["clocks"], "breakdown": bd}


def bench_e2e(args, tables, keys_slice, vals_slice, keys_pos, keys_neg, keys_up, vals_up, base_n, ops_per_step,
              world, dev):
    """Same steps through the C ABI with pinned host inputs and outputs."""
    import torch
    h = {n: x.cpu().pin_memory() for n, x in (("ks", keys_slice), ("vs", vals_slice), ("kp", keys_pos),
                                              ("kn", keys_neg), ("ku", keys_up), ("vu", vals_up))}
    out_host = torch.empty(keys_pos.numel(), dtype=torch.int64).pin_memory()
    stream = torch.cuda.current_stream(dev)
    for _, t in tables:
        t.set_host_direct(args.host_direct)

    def step():
        for name, t in tables:
            t.insert(h["ks"], h["vs"])
            t.query(h["kp"], out=out_host)
            t.query(h["kn"], out=out_host)
            t.upsert(h["ku"], h["vu"], op="add")
            t.erase(h["ks"])
        for name, t in tables:
            if t.count() != base_n:
                raise RuntimeError("e2e count mismatch")

    step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms, e2e_value = aggregate(a.elapsed_time(b), ops_per_step * args.steps, world, dev)
    n_t = len(tables)
    h2d = n_t * (keys_slice.numel() * 16 + keys_pos.numel() * 8 + keys_neg.numel() * 8 + keys_up.numel() * 16
                 + keys_slice.numel() * 8)
    d2h = n_t * (keys_pos.numel() * 8 + keys_neg.numel() * 8)
    return {"value": round(e2e_value, 4), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "host_buffers": ["staged through device chunks", "inputs read in place, results staged",
                             "read and written in place",
                             "inputs read in place by inserts and erases, staged for queries and upserts; "
                             "results staged"][args.host_direct]}


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_step_sample(log2_slots=22, load=0.9, nq=1 << 18, seed=0xC0FFEE, shard=0, n_shards=1):
    """One step of the same workload shape at 2^log2_slots slots, on the oracle.
    Returns (ops, runner, description); the runner times one step (prefill
    untimed).  With n_shards > 1 only the keys whose splitmix64 finaliser is
    shard mod n_shards take part (one map per shard)."""
    import oracle
    S = 1 << log2_slots
    base_n = int(0.85 * S)
    top_n = int(load * S)
    slice_n = top_n - base_n
    ks = W.distinct_keys(seed, top_n + nq)
    base, slc, neg = ks[:base_n], ks[base_n:top_n], ks[top_n:]
    with np.errstate(over="ignore"):
        vb, vs = base * np.uint64(3), slc * np.uint64(3)
    pos = ks[:top_n][W.splitmix64(seed + 1, nq) % np.uint64(top_n)]
    up = base[W.splitmix64(seed + 2, nq) % np.uint64(base_n)]
    vu = W.uniform_int(seed + 3, nq, 1, 1000)
    if n_shards > 1:
        mine = lambda k: (W.mix13(k) % np.uint64(n_shards)) == np.uint64(shard)
        mb, ms_, mp, mn, mu = mine(base), mine(slc), mine(pos), mine(neg), mine(up)
        base, vb, slc, vs, pos, neg, up, vu = base[mb], vb[mb], slc[ms_], vs[ms_], pos[mp], neg[mn], up[mu], vu[mu]
        base_n = base.size
    om = oracle.OracleMap()
    om.insert(base, vb)

    def run():
        t0 = time.perf_counter()
        om.insert(slc, vs)
        om.query(pos)
        om.query(neg)
        om.upsert(up, vu, 0)
        om.erase(slc)
        dt = time.perf_counter() - t0
        assert om.count() == base_n
        return dt

    n_ops = 2 * slc.size + pos.size + neg.size + up.size
    return n_ops, run, f"2^{log2_slots}-slot-equivalent map at 0.85->{load} load, {n_ops} ops/step"


def cpu_baseline(seconds=10.0):
    ops, run, desc = oracle_step_sample()
    done, spent = 0, 0.0
    while spent < seconds:
        spent += run()
        done += ops
    return {"value": round(done / spent / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{desc}; {done} ops in {spent:.1f} s (single-threaded std::unordered_map)"}


def _sharded_worker(args):
    shard, n_shards, seconds = args
    ops, run, _ = oracle_step_sample(shard=shard, n_shards=n_shards)
    done, spent = 0, 0.0
    while spent < seconds:
        spent += run()
        done += ops
    return done, spent


def cpu_baseline_sharded(seconds=10.0):
    """The oracle on every host core: keys sharded by hash, one map per
    process (spawn-started pool), throughput = all ops / the slowest shard."""
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_sharded_worker, [(r, n, seconds) for r in range(n)])
    # each shard ran for `seconds`; scale every shard's rate to a common span
    rate = sum(d / t for d, t in res)
    return {"value": round(rate / 1e9, 6), "unit": UNIT, "cores": n, "kind": "oracle, sharded by key hash",
            "sample": f"2^22-slot-equivalent workload split over {n} processes by splitmix64 finaliser of the key "
                      f"mod {n}; each shard ran about {seconds:.0f} s; sum of the shards' rates"}


def bench_reference(args, rank, world):
    if rank != 0:
        return None
    ops, run, desc = oracle_step_sample()
    for _ in range(args.warmup):
        run()
    spent = 0.0
    for _ in range(args.steps):
        spent += run()
    value = ops * args.steps / spent / 1e9
    return {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(spent / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": {"workload": config2_workload(args, [d[2] for d in DESIGNS]), "parallelism": "1 host thread",
                       "sample": "each step runs the same phases on one map of the oracle at 2^22 slots "
                                 f"(the workload's shape, scaled so the run ends in minutes): {desc}"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# batched mode (config 4): 1024 tables, capacities log-uniform 2^10..2^22,
# ops log-uniform 2^8..2^20 (inserts = min(n/2, 0.85 cap), the rest queries,
# half present / half absent); one persistent graph launch per step vs one
# insert + one query launch per table, identical results required.
# ---------------------------------------------------------------------------
def bench_batched(args, n_tables=None, reps=None, tune_reps=3):
    import torch
    import paper_2509_16407_gb300 as ws
    from paper_2509_16407_gb300 import autotune
    dev = torch.device("cuda", 0)
    n_t = n_tables or args.tables
    caps = W.log_uniform_int(41, n_t, 1 << 10, 1 << 22)
    nops = W.log_uniform_int(42, n_t, 1 << 8, 1 << 20)
    t_tune = time.time()
    choice, timings = autotune.tune(reps=tune_reps, log=lambda m: print(m, file=sys.stderr, flush=True))
    t_tune = time.time() - t_tune
    specs = []
    for i in range(n_t):
        cap, n = int(caps[i]), int(nops[i])
        n_ins = min(n // 2, int(0.85 * cap))
        n_q = n - n_ins
        k = W.distinct_keys(7_000_003 + i, n_ins + n_q // 2)
        ins, neg = k[:n_ins], k[n_ins:]
        pos = ins[W.splitmix64(88 + i, n_q - n_q // 2) % np.uint64(n_ins)]
        specs.append((cap, to_dev(ins, dev), to_dev(W.splitmix64(99 + i, n_ins), dev),
                      to_dev(np.concatenate([pos, neg]), dev)))
    total_ops = sum(int(nops[i]) for i in range(n_t))

    def make(tuned):
        tabs, outs = [], []
        for i, (cap, ki, vi, q) in enumerate(specs):
            if tuned:
                sch, meta, B, T = autotune.config_for(cap, choice)
                t = ws.Table(cap, sch, meta, bucket_slots=B, tile=T)
            else:
                t = ws.Table(cap, "double", False)
            outs.append((torch.empty(ki.numel(), dtype=torch.uint8, device=dev),
                         torch.empty(q.numel(), dtype=torch.int64, device=dev),
                         torch.empty(q.numel(), dtype=torch.uint8, device=dev)))
            tabs.append(t)
        return tabs, outs

    def run_plain(tabs, outs):
        for (cap, ki, vi, q), t, (si, qv, qs) in zip(specs, tabs, outs):
            lib = ws.lib()
            lib.ws_insert_ex(t.handle, ki.data_ptr(), vi.data_ptr(), ki.numel(), si.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
            lib.ws_query_ex(t.handle, q.data_ptr(), qv.data_ptr(), qs.data_ptr(), q.numel(),
                            torch.cuda.current_stream().cuda_stream)

    def timed(fn, tabs, reps):
        ts = []
        for _ in range(reps):
            for t in tabs:
                t.clear()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    tuned, tout = make(True)
    items = []
    for (cap, ki, vi, q), t, (si, qv, qs) in zip(specs, tuned, tout):
        items += [(t, ws.BK_INSERT, ki, vi, None, si, 0), (t, ws.BK_QUERY, q, None, qv, qs, 1)]
    plan = ws.BatchPlan(items)
    reps = reps or max(args.steps, 3)
    timed(plan.launch, tuned, args.warmup)
    ts_batched = timed(plan.launch, tuned, reps)
    res_b = [(si.clone(), qv.clone(), qs.clone()) for si, qv, qs in tout]
    timed(lambda: run_plain(tuned, tout), tuned, 1)
    ts_plain_tuned = timed(lambda: run_plain(tuned, tout), tuned, reps)
    same = all(torch.equal(a, b) for ra, rb in zip(res_b, tout) for a, b in zip(ra, rb))
    cfg_count = {}
    for t in tuned:
        inf = t.info()
        key = f"{'P2HT' if inf['scheme'] else 'DoubleHT'}{'(M)' if inf['metadata'] else ''}/B{inf['bucket_slots']}/T{inf['tile']}"
        cfg_count[key] = cfg_count.get(key, 0) + 1
    fallback = plan.info()["fallback_items"]
    plan.close()
    for t in tuned:
        t.close()
    torch.cuda.empty_cache()
    dflt, dout = make(False)
    timed(lambda: run_plain(dflt, dout), dflt, 1)
    ts_plain_default = timed(lambda: run_plain(dflt, dout), dflt, reps)
    same_default = all(torch.equal(a, b) for ra, rb in zip(res_b, dout) for a, b in zip(ra, rb))
    med = statistics.median
    return {
        "metric": "batched Gops/s (1024 tables, one graph launch) vs per-table launches", "unit": UNIT,
        "value": round(total_ops / (med(ts_batched) * 1e-3) / 1e9, 4), "higher_is_better": True,
        "plain_tuned_gops": round(total_ops / (med(ts_plain_tuned) * 1e-3) / 1e9, 4),
        "plain_default_gops": round(total_ops / (med(ts_plain_default) * 1e-3) / 1e9, 4),
        "ms": {"batched": round(med(ts_batched), 3), "plain_tuned": round(med(ts_plain_tuned), 3),
               "plain_default": round(med(ts_plain_default), 3)},
        "identical_results": {"batched_vs_plain_tuned": same, "batched_vs_plain_default": same_default},
        "total_ops": total_ops, "tables": n_t,
        "launches": {"batched": 1, "plain": 2 * n_t}, "configs": cfg_count, "fallback_items": fallback,
        "autotune_seconds": round(t_tune, 1),
        "autotune_choice": {str(k): "/".join(map(str, v)) for k, v in choice.items()},
        "config": {"workload": "config 4: capacities log-uniform 2^10-2^22, ops log-uniform 2^8-2^20, load 0.85",
                   "data": "synthetic"}}


# ---------------------------------------------------------------------------
# serving (config 5): 64 resident tables of 2^16..2^26 slots; requests of
# log-uniform 1..2^20 mixed ops (60% query, 30% upsert-add, 5% insert, 5%
# erase, Zipf(0.99) keys); saturated throughput, then Poisson arrivals at 50%
# and 90% of it; continuous batching vs plain per-request launches.
# ---------------------------------------------------------------------------
def bench_serve(args, n_req=None, reps=3):
    import torch
    import paper_2509_16407_gb300 as ws
    n_tab = 64
    caps = W.log_uniform_int(51, n_tab, 1 << 16, 1 << 26)
    n_req = n_req or args.requests
    sizes = W.log_uniform_int(52, n_req, 1, 1 << 20)
    tabs = (W.splitmix64(53, n_req) % np.uint64(n_tab)).astype(int)

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()

    reqs = []
    for i in range(n_req):
        t = int(tabs[i])
        ops, keys, vals = W.mixed_request(1000 + i, int(sizes[i]), max(1024, int(caps[t]) // 2), t + 1)
        reqs.append((t, pinned(ops), pinned(keys), pinned(vals)))
    total_ops = int(sizes.sum())
    mean_ops = total_ops / n_req

    def run(plain, arrivals=None):
        sv = ws.Server(plain=plain, max_inflight=4, max_batch_ops=1 << 22, grow_at=0.85)
        ids = [sv.add_table(int(c)) for c in caps]
        outs = [(pinned(np.empty(r[2].size, np.uint64)), pinned(np.empty(r[2].size, np.uint8))) for r in reqs]
        torch.cuda.synchronize()
        if arrivals is None:
            sv.pause()  # saturation: the whole burst is queued before the clock starts
        t0 = time.monotonic()
        rid = []
        for i, (t, ops, keys, vals) in enumerate(reqs):
            if arrivals is not None:
                target = t0 + arrivals[i]
                while time.monotonic() < target:
                    pass
            rid.append(sv.submit(ids[t], ops, keys, vals, vals_out=outs[i][0], status_out=outs[i][1]))
        if arrivals is None:
            t0 = time.monotonic()
        done = {c["id"]: c for c in sv.drain()}
        t_end = max(c["t_done"] for c in done.values())
        if arrivals is not None:
            lat = np.array([done[r]["t_done"] - (t0 + arrivals[i]) for i, r in enumerate(rid)])
        else:
            lat = np.array([done[r]["t_done"] - done[r]["t_submit"] for r in rid])
        st = sv.stats()
        counts = [sv.count(i) for i in ids]
        sv.close()
        torch.cuda.empty_cache()
        return {"gops": total_ops / (t_end - t0) / 1e9, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "launches": st["launches"], "grows": st["grows"],
                "seconds": t_end - t0}, outs, counts

    def median_run(plain, arrivals=None):
        # the median of `reps` runs by throughput (one process serves them all);
        # the spread is reported beside it
        rs = [run(plain, arrivals) for _ in range(reps)]
        rs.sort(key=lambda r: r[0]["gops"])
        med = rs[len(rs) // 2]
        med[0]["gops_runs"] = [round(r[0]["gops"], 4) for r in rs]
        return med

    run(False)  # warm-up, untimed: first-use costs (memory pool, module loading)
    sat_c, out_c, cnt_c = median_run(False)
    sat_p, out_p, cnt_p = median_run(True)
    same = cnt_c == cnt_p
    for (t, ops, keys, vals), (va, sa), (vb, sb) in zip(reqs, out_c, out_p):
        q = ops == W.MX_QUERY
        same &= bool((va[q] == vb[q]).all() and (sa[q] == sb[q]).all())
    res = {"saturated": {"continuous": sat_c, "plain": sat_p}}
    for load in (0.5, 0.9):
        lam = load * sat_c["gops"] * 1e9 / mean_ops  # requests per second
        gaps = -np.log(1.0 - W.uniform01(60 + int(load * 10), n_req)) / lam
        arrivals = np.cumsum(gaps) - gaps[0]
        c, _, _ = median_run(False, arrivals)
        p_, _, _ = median_run(True, arrivals)
        res[f"poisson_{int(load * 100)}pct"] = {"continuous": c, "plain": p_, "offered_gops": load * sat_c["gops"]}
    rnd = lambda d: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in d.items()}
    return {"metric": "serve p50/p99 latency and Gops/s, continuous batching vs plain per-request launches "
                      f"(median of {reps} runs per mode after a warm-up run)",
            "unit": UNIT, "value": round(sat_c["gops"], 4), "higher_is_better": True,
            "runs": {k: {kk: rnd(vv) if isinstance(vv, dict) else vv for kk, vv in v.items()} for k, v in res.items()},
            "identical_query_results_and_counts": same, "requests": n_req, "total_ops": total_ops,
            "config": {"workload": "config 5: 64 tables 2^16-2^26 slots, request sizes log-uniform 1-2^20, "
                                   "60/30/5/5 query/add/insert/erase, Zipf(0.99) keys, host (pinned) buffers",
                       "data": "synthetic"}}


# ---------------------------------------------------------------------------
# aging (paper §6.4): fill to 85%, then per iteration ONE mixed kernel that
# inserts 1% new keys, erases the oldest 1%, and queries 1% present and 1%
# absent keys; probe counts (ws_probe_cost) beside the paper's Table 1
# aging column.
# ---------------------------------------------------------------------------
TABLE1_AGING = {"IcebergHT(M)": (6.98, 2.2, 3.02, 6.22),
                "DoubleHT": (77.09, 1.61, 80.00, 4.57), "DoubleHT(M)": (23.52, 2.10, 19.39, 6.12),
                "P2HT": (11.02, 3.96, 8.01, 6.85), "P2HT(M)": (6.02, 2.42, 2.01, 6.4)}


def bench_aging(args):
    import torch
    import paper_2509_16407_gb300 as ws
    dev = torch.device("cuda", 0)
    S = 1 << args.aging_log2_slots
    m = S // 100
    fill = int(0.85 * S)
    iters = args.aging_iters
    pool = splitmix_torch(0xA61, fill + iters * m + m, 0, dev)
    negp = splitmix_torch(0xB62, iters * m, 0, dev)
    ops = torch.tensor([ws.MX_INSERT, ws.MX_ERASE, ws.MX_QUERY, ws.MX_QUERY], dtype=torch.uint8,
                       device=dev).repeat(m)
    out = {}
    for scheme, meta, name in ALL_DESIGNS:
        t = ws.Table(S, scheme, meta)
        t.insert(pool[:fill], pool[:fill] * 3)
        times, probes = [], {}
        for it in range(iters):
            ins = pool[fill + it * m: fill + (it + 1) * m]
            era = pool[it * m: (it + 1) * m]
            pos = pool[(it + 1) * m: (it + 2) * m]
            neg = negp[it * m: (it + 1) * m]
            if it % max(1, iters // 20) == 0 or it == iters - 1:
                costs = {}
                for ph, k in (("insert", ins), ("positive", pos), ("negative", neg), ("delete", era)):
                    c, _ = t.probe_cost(k[: 1 << 16])
                    costs[ph] = round(float((c.cpu().numpy().view(np.uint64) >> np.uint64(32)).mean()), 3)
                probes[it] = costs
            keys = torch.stack([ins, era, pos, neg], 1).reshape(-1).contiguous()
            vals = torch.stack([ins * 3, torch.zeros_like(ins), torch.zeros_like(ins), torch.zeros_like(ins)],
                               1).reshape(-1).contiguous()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            t.mixed(ops, keys, vals, return_values=False, return_status=False)
            b.record()
            times.append((a, b))
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in times])
        cnt = t.count()
        err = t.last_error()
        mean_probes = {ph: round(float(np.mean([c[ph] for c in probes.values()])), 3)
                       for ph in ("insert", "positive", "negative", "delete")}
        out[name] = {"gops_mean": round(4 * m / ms.mean() / 1e6, 3), "gops_first10": round(4 * m / ms[:10].mean() / 1e6, 3),
                     "gops_last10": round(4 * m / ms[-10:].mean() / 1e6, 3), "iter_ms_p50": round(float(np.median(ms)), 4),
                     "iter_ms_p99": round(float(np.percentile(ms, 99)), 4), "count_after": cnt, "count_expected": fill,
                     "failed_ops": err, "probe_lines": probes,
                     "probe_lines_mean_over_samples": mean_probes,
                     "paper_table1_aging_probes(ins,pos,neg,del)": TABLE1_AGING[name]}
        t.close()
        torch.cuda.empty_cache()
    return {"metric": "aging Gops/s (all ops of an iteration in one kernel) and probe lines per op", "unit": UNIT,
            "value": round(float(np.mean([v["gops_mean"] for v in out.values()])), 4), "higher_is_better": True,
            "designs": out, "config": {"workload": f"aging: 2^{args.aging_log2_slots} slots, fill 0.85, {iters} "
                                                    f"iterations of 1% insert / 1% erase oldest / 1% + 1% queries",
                                       "data": "synthetic"}}


# ---------------------------------------------------------------------------
# config 3: mixed Zipf(0.99) batches of 2^24 ops (50% upsert-add, 40% query,
# 10% erase, key-disjoint classes per batch) over a 2^26-rank universe on
# 2^27-slot tables; 16 batches, seed 3.  Batches are generated on the host
# cores in a spawn-started pool before any GPU work, then copied to the
# device; each batch is one mixed launch.
# ---------------------------------------------------------------------------
def _mixed_batch_job(args):
    seed, n_ops, universe = args
    return W.mixed_batch(seed, n_ops=n_ops, universe=universe)


def make_mixed_batches(n_batches=16, n_ops=1 << 24, universe=1 << 26, seed=3):
    import multiprocessing as mp
    jobs = [(seed * 100 + b, n_ops, universe) for b in range(n_batches)]
    procs = min(n_batches, max(1, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_mixed_batch_job, jobs)


def bench_mixed(args, batches):
    import torch
    import paper_2509_16407_gb300 as ws
    dev = torch.device("cuda", 0)
    S = 1 << 27
    dbs = [tuple(torch.from_numpy(np.ascontiguousarray(x).view(np.int64) if x.dtype == np.uint64 else x).to(dev)
                 for x in b) for b in batches]
    n_ops = sum(int(b[0].size) for b in batches)
    out = {}
    for scheme, meta, name in [DESIGNS[1], DESIGNS[3], DESIGNS[0], DESIGNS[2]]:
        t = ws.Table(S, scheme, meta)
        # warm-up on the first batch, then start from an empty table
        t.mixed(dbs[0][0], dbs[0][1], dbs[0][2])
        torch.cuda.synchronize()
        t.clear()
        evs = []
        for o, k, v in dbs:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            t.mixed(o, k, v)
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        err = t.last_error()
        out[name] = {"gops": round(n_ops / ms.sum() / 1e6, 3), "batch_ms_mean": round(float(ms.mean()), 3),
                     "batch_ms_first": round(float(ms[0]), 3), "batch_ms_last": round(float(ms[-1]), 3),
                     "live_keys_after": t.count(), "failed_ops": err}
        t.close()
        torch.cuda.empty_cache()
    return {"metric": "config 3 mixed Zipf batches, Gops/s per design (device-resident batches)", "unit": UNIT,
            "value": round(float(np.mean([out[d[2]]["gops"] for d in (DESIGNS[1], DESIGNS[3])])), 4),
            "higher_is_better": True, "designs": out,
            "config": {"workload": "config 3: 2^27-slot tables, 16 batches of 2^24 ops, Zipf(0.99) over 2^26 ranks, "
                                   "50% upsert-add / 40% query / 10% erase, key-disjoint classes per batch, seed 3; "
                                   "value = mean over the metadata designs", "data": "synthetic"}}


# ---------------------------------------------------------------------------
# cost of concurrency (paper §6.2, Table 1 right block): the same queries and
# inserts with the concurrent protocol and in bulk-synchronous (phased) mode
# -- weak cacheable loads, no locks -- on 2^28-slot tables at 0.9 load.
# ---------------------------------------------------------------------------
TABLE1_PHASED = {"DoubleHT": (3166, 3233), "DoubleHT(M)": (2624, 2624), "P2HT": (1471, 1471), "P2HT(M)": (2903, 2909),
                 "IcebergHT(M)": (2598, 2866)}


def bench_phased(args):
    import torch
    import paper_2509_16407_gb300 as ws
    dev = torch.device("cuda", 0)
    S = 1 << args.log2_slots
    base_n, top_n = int(0.85 * S), int(0.9 * S)
    nq = args.nq
    keys = splitmix_torch(0xD0D0, top_n + nq, 0, dev)
    vals = keys * 3
    slice_k, neg = keys[base_n:top_n], keys[top_n:]
    pos = keys[:top_n][torch.from_numpy((W.splitmix64(7, nq) % np.uint64(top_n)).astype(np.int64)).to(dev)]
    out_q = torch.empty(nq, dtype=torch.int64, device=dev)
    res = {}

    def tm(f, reps=3):
        best = 1e30
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    for scheme, meta, name in ALL_DESIGNS:
        t = ws.Table(S, scheme, meta)
        t.insert(keys[:base_n], vals[:base_n])
        r = {}
        for phased in (False, True):
            t.set_phased(phased)
            ins = tm(lambda: (t.insert(slice_k, vals[base_n:top_n]), t.erase(slice_k)), reps=2)
            t.set_phased(False)
            t.insert(slice_k, vals[base_n:top_n])
            t.set_phased(phased)
            qp = tm(lambda: t.query(pos, out=out_q))
            qn = tm(lambda: t.query(neg, out=out_q))
            t.set_phased(False)
            t.erase(slice_k)
            key = "phased" if phased else "concurrent"
            r[key] = {"query_gops": round(2 * nq / (qp + qn) / 1e6, 3), "query_pos_gops": round(nq / qp / 1e6, 3),
                      "query_neg_gops": round(nq / qn / 1e6, 3),
                      "insert_erase_pair_gops": round((top_n - base_n) / ins / 1e6, 3)}
        r["query_overhead_pct"] = round(100 * (1 - r["concurrent"]["query_gops"] / r["phased"]["query_gops"]), 2)
        r["paper_table1_concurrent_phased_mops(A40)"] = TABLE1_PHASED[name]
        res[name] = r
        t.close()
        torch.cuda.empty_cache()
    return {"metric": "query Gops/s, concurrent vs phased (bulk-synchronous) mode", "unit": UNIT,
            "value": round(float(np.mean([v["concurrent"]["query_gops"] for v in res.values()])), 4),
            "higher_is_better": True, "designs": res,
            "config": {"workload": f"2^{args.log2_slots} slots at 0.9 load, {nq} positive + {nq} negative queries, "
                                   "5% slice insert+erase", "data": "synthetic"}}


# ---------------------------------------------------------------------------
# load / tile sweep (config 2): one JSON line per (slots, design, tile, load)
# ---------------------------------------------------------------------------
def sweep(args):
    """Config 2's load / tile sweep: per (slots, design, tile, load) the 5%
    insert slice ending at that load, 2^24 positive and as many negative
    queries, their probe costs, and the fraction of the roofline:
    against the measured HBM copy peak for tables larger than L2, against the
    measured L2 read peak for the 2^22-slot tables."""
    import torch
    import paper_2509_16407_gb300 as ws
    dev = torch.device("cuda", 0)
    peak, _ = peak_gbs()
    peaks = read_peaks()
    out = open(args.sweep, "w")
    out.write(json.dumps({"read_peaks": peaks, "hbm_copy_peak_gbs": peak}) + "\n")
    loads = [0.5, 0.7, 0.8, 0.9, 0.95]
    for lg in [int(x) for x in args.sweep_log2_slots.split(",")]:
        S = 1 << lg
        nq = 1 << 24  # 2^24 positive and 2^24 negative queries at every size
        top = int(0.95 * S)
        keys = gen_dev(0xABC + lg, top + nq, 0, dev)
        vals = keys * 3
        neg = keys[top:]
        in_l2 = S * 16 < 100 * (1 << 20)
        den = peaks["l2_peak_gbs"] if in_l2 else peak
        for scheme, meta, name in ALL_DESIGNS:
            for tile in (4, 8, 16, 32):
                t = ws.Table(S, scheme, meta, tile=tile)
                B = t.info()["bucket_slots"]
                have = 0
                for lf in loads:
                    n_lf = int(lf * S)
                    lo = int((lf - 0.05) * S)
                    # fill to lf - 0.05 untimed, then time the 5% slice
                    if lo > have:
                        t.insert(keys[have:lo], vals[have:lo])
                    # the slice's scan cost before it is inserted (as the default line counts it),
                    # one line per probe step (T = 8, or B when smaller)
                    t.set_tile(min(8, B))
                    ic, _ = t.probe_cost(keys[lo:min(n_lf, lo + (1 << 18))])
                    t.set_tile(tile)
                    a, b, c, d, e = (torch.cuda.Event(enable_timing=True) for _ in range(5))
                    a.record()
                    st = t.insert(keys[lo:n_lf], vals[lo:n_lf], return_status=True)
                    b.record()
                    pos = keys[:n_lf][torch.randint(0, n_lf, (nq,), device=dev,
                                                    generator=torch.Generator(device=dev).manual_seed(lg))]
                    c.record()
                    t.query(pos)
                    d.record()
                    t.query(neg)
                    e.record()
                    torch.cuda.synchronize()
                    have = n_lf
                    fails = int((st == ws.FAIL_FULL).sum().item())
                    t.set_tile(min(8, B))
                    pc, _ = t.probe_cost(pos[: 1 << 18])
                    nc, _ = t.probe_cost(neg[: 1 << 18])
                    t.set_tile(tile)
                    sec = lambda x: float((x.cpu().numpy().view(np.uint64) & np.uint64(0xFFFFFFFF)).mean())
                    ics, pcs, ncs = sec(ic), sec(pc), sec(nc)
                    ins_ms, qp_ms, qn_ms = a.elapsed_time(b), c.elapsed_time(d), d.elapsed_time(e)
                    ins_b = ics * 32 + 32 + (32 if meta else 0) + 16
                    ins_gbs = (n_lf - lo) * ins_b / ins_ms / 1e6
                    qp_gbs = nq * (pcs * 32 + 16) / qp_ms / 1e6
                    qn_gbs = nq * (ncs * 32 + 16) / qn_ms / 1e6
                    rec = {"slots": S, "design": name, "tile": tile, "load": lf,
                           "insert_gops": round((n_lf - lo) / ins_ms / 1e6, 3),
                           "query_pos_gops": round(nq / qp_ms / 1e6, 3),
                           "query_neg_gops": round(nq / qn_ms / 1e6, 3),
                           "insert_gbs": round(ins_gbs, 1), "query_pos_gbs": round(qp_gbs, 1),
                           "query_neg_gbs": round(qn_gbs, 1),
                           "insert_sectors": round(ics, 3), "query_pos_sectors": round(pcs, 3),
                           "query_neg_sectors": round(ncs, 3),
                           "peak_gbs": den, "peak_kind": "L2 read (measured)" if in_l2 else "HBM copy (measured)",
                           "frac_insert": round(ins_gbs / den, 4), "frac_query_pos": round(qp_gbs / den, 4),
                           "frac_query_neg": round(qn_gbs / den, 4),
                           "insert_failures": fails, "count": t.count()}
                    out.write(json.dumps(rec) + "\n")
                    out.flush()
                t.close()
                torch.cuda.empty_cache()
    out.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = bench_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.sweep:
        sweep(args)
        return
    if args.workload == "batched":
        print(json.dumps(bench_batched(args)), flush=True)
        return
    if args.workload == "phased":
        print(json.dumps(bench_phased(args)), flush=True)
        return
    if args.workload == "aging":
        print(json.dumps(bench_aging(args)), flush=True)
        return
    if args.workload == "serve":
        print(json.dumps(bench_serve(args)), flush=True)
        return
    if args.workload == "mixed":
        batches = make_mixed_batches()  # host pool first: no GPU context exists yet
        print(json.dumps(bench_mixed(args, batches)), flush=True)
        return
    extra = world == 1 and not args.no_extra
    peaks = read_peaks() if extra else None  # before the tables take the memory
    res = bench_ours(args, rank, world, access_peak=peaks["hbm_rand128_gaccess_s"] if peaks else None)
    if extra:
        import torch
        torch.cuda.empty_cache()
        res["read_peaks"] = peaks
        if peaks.get("l2_peak_gbs"):
            res["l2_resident"] = bench_l2_leg(args, rank, world, peaks)
        res["batched"] = bench_batched(args, n_tables=1024, reps=5, tune_reps=1)
        torch.cuda.empty_cache()
        res["serve"] = bench_serve(args, n_req=args.serve_requests, reps=3)
        torch.cuda.empty_cache()
        batches = make_mixed_batches()  # spawn-started pool: safe after the GPU context exists
        res["mixed"] = bench_mixed(args, batches)
        del batches
        torch.cuda.empty_cache()
    if rank == 0:
        if not args.no_cpu:
            res["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
            res["cpu_baseline_sharded"] = cpu_baseline_sharded(args.cpu_seconds)
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
