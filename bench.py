#!/usr/bin/env python
"""Benchmark of the COMPASS hot path on GB300: one step = the push-down Fast-AGMS build of
every attribute-level sketch of a query's tables (one batched build), the magnitude
presort and cross ranks, the sketch-merging estimate of every connected sub-plan, the
learned combiner's inference over the sub-plan row estimates, and the join-order
enumeration (Algorithm 1) over the combined estimates; replayed as one CUDA graph.

Workload (N = 1): the 5-table cyclic join graph shaped like the paper's running example
(F1 36M, F2 4.5M, D1 2.5M, D2 134k, D3 4M rows; Zipf(1.1) foreign keys; point, subset
and 20% range predicates; d = 11, w = 4096; 19 connected sub-plans), synthetic.
Under torchrun every rank runs its own independent query (its own data seed): weak
scaling, no collective.  `--impl reference` times the single-threaded CPU oracle on a
bounded sample of the same workload.

Prints one JSON line on rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sketched tuples/s"
UNIT = "tuples/s"
INT_ISSUE_PEAK = 152 * 4 * 32 * 2.070e9   # 32-bit integer instructions/s: one warp instruction per SMSP per clock
# Algorithmic cost of one CW-61 bucket + sign evaluation: 4 products of 61-bit field elements
# (16 32x32->64-bit partial products) plus folds, reductions and the counter atomic.
CW_INSTR = 60
# Algorithmic cost of one exact 128-bit add or multiply-by-64-bit: 4 limbs, carries included.
OP128_INSTR = 8


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=["scale", "five_table"],
                    help="scale: the 1e9-row fact table configuration (the headline); five_table: the paper's "
                         "running example at full size")
    ap.add_argument("--scale", type=float, default=1.0, help="row-count scale of the workload (1.0 = full)")
    ap.add_argument("--no-extras", action="store_true",
                    help="measure the headline workload only (no five-table or batched-enumeration keys)")
    ap.add_argument("--w", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every step eagerly instead of replaying it as one captured CUDA graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--c3-rows-scale", type=float, default=1.0,
                    help="row-count factor of the batched-enumeration extra (1.0: rows in [1e4, 1e8])")
    ap.add_argument("--phases", action="store_true", help="print a per-phase breakdown on stderr")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuned launch shapes: read if it has this workload's, else written")
    ap.add_argument("--case", default=None,
                    choices=["estimate_small", "estimate_full", "build_f1", "build_five", "batched", "batched_full",
                             "scale",
                             "partition", "offline_sample", "cached", "star17", "shapes"],
                    help="run one small profiling case instead of the benchmark (for ncu captures)")
    return ap.parse_args()


def estimate_ops(n_tables, eu, ev, masks, d, w) -> int:
    """Exact 128-bit integer operations (multiplies and adds) of the sketch-merging
    contraction as the estimate kernel evaluates it: spanning tree from the lowest table,
    one operation per non-leaf table, every conditioning value of a cyclic sub-plan."""
    total = 0
    for m in masks:
        tabs = [t for t in range(n_tables) if (m >> t) & 1]
        if len(tabs) < 2:
            continue
        es = [e for e in range(len(eu)) if (m >> eu[e]) & 1 and (m >> ev[e]) & 1]
        root = tabs[0]
        order, seen, parent, tree = [root], {root}, {root: -1}, set()
        h = 0
        while h < len(order):
            t = order[h]
            h += 1
            for e in es:
                o = ev[e] if eu[e] == t else (eu[e] if ev[e] == t else None)
                if o is None or o in seen:
                    continue
                seen.add(o)
                parent[o] = e
                tree.add(e)
                order.append(o)
        cond = [e for e in es if e not in tree]
        deg = {t: sum(1 for e in es if t in (eu[e], ev[e])) for t in tabs}
        per_c = per_row = 0
        for t in order:
            if t != root and deg[t] == 1:
                continue
            kinds = []
            for e in es:
                if t not in (eu[e], ev[e]):
                    continue
                if e == parent[t]:
                    kinds.append("out")
                elif e in tree:
                    child = ev[e] if eu[e] == t else eu[e]
                    kinds.append("leaf" if (child != root and deg[child] == 1) else "slot")
                else:
                    kinds.append("cond")
            nc = [k for k in kinds if k in ("leaf", "slot")]
            per_row += w * kinds.count("leaf")                  # leaf suffix sums, once per item
            per_c += w * kinds.count("slot")                    # message suffix sums
            per_c += len(nc) * w * (len(nc) + 1)                # s*m, threshold products, prefix add
            if "out" in kinds:
                per_c += w * (2 * len(nc) + 1)                  # output: products, prefix adds, final add
        total += d * (per_row + (w if cond else 1) * per_c)
    return total


def triangle_plan(n_tables, eu, ev, mask):
    """(U, V, W, e*, eU, eV) when the sub-plan's only cycle is a triangle U-W-V closed by
    the conditioned edge e* = U-V (BFS spanning tree from the lowest table, edges in id
    order) and every other table is a leaf of U, V or W; else None.  Same rule as the
    estimate planner."""
    es = [e for e in range(len(eu)) if (mask >> eu[e]) & 1 and (mask >> ev[e]) & 1]
    tabs = [t for t in range(n_tables) if (mask >> t) & 1]
    order, seen, tree = [tabs[0]], {tabs[0]}, set()
    h = 0
    while h < len(order):
        t = order[h]
        h += 1
        for e in es:
            o = ev[e] if eu[e] == t else (eu[e] if ev[e] == t else None)
            if o is None or o in seen:
                continue
            seen.add(o)
            tree.add(e)
            order.append(o)
    cond = [e for e in es if e not in tree]
    if len(cond) != 1:
        return None
    es_ = cond[0]
    a, b = eu[es_], ev[es_]
    other = lambda e, t: ev[e] if eu[e] == t else eu[e]
    for w_ in tabs:
        if w_ in (a, b):
            continue
        ea = [e for e in tree if w_ in (eu[e], ev[e]) and other(e, w_) == a]
        eb = [e for e in tree if w_ in (eu[e], ev[e]) and other(e, w_) == b]
        if ea and eb:
            for t in tabs:
                if t in (a, b, w_):
                    continue
                inc = [e for e in es if t in (eu[e], ev[e])]
                if len(inc) != 1 or other(inc[0], t) not in (a, b, w_):
                    return None
            return a, b, w_, es_, ea[0], eb[0]
    return None


def triangle_ops(dw, masks):
    """Exact 128-bit operations of the triangle path for the triangle sub-plans of `masks`,
    and of the generic path for the others.  Per triangle sketch row, with G distinct
    row-side clamp ranks, L_n leaves at node n and nq conditioning values:
      preparation  sum_leaves 3w + 6 messages x w (1 + 2 L_n) + 4 nq + 4 w
      sweep        w (6 (G + 1) + 16 G + 4)   (per column: batch sums, group terms, total)
    G is computed here from the sketches with the kernel's rules (row side = the endpoint
    whose conditioned sketch row has fewer distinct magnitudes)."""
    wl = dw.wl
    nt, eu, ev, d, w = len(wl.tables), wl.edge_u, wl.edge_v, wl.d, wl.w
    generic = [m for m in masks if triangle_plan(nt, eu, ev, m) is None]
    ops = estimate_ops(nt, eu, ev, generic, d, w)
    sk = {}

    def sketch(e, t):
        key = (e, t)
        if key not in sk:
            sk[key] = dw.sketch(e, 0 if eu[e] == t else 1).cpu().numpy().astype(np.int64)
        return sk[key]

    n_tri = 0
    for m in masks:
        tp = triangle_plan(nt, eu, ev, m)
        if tp is None:
            continue
        n_tri += 1
        a, b, W, es_, ea, eb = tp
        es = [e for e in range(len(eu)) if (m >> eu[e]) & 1 and (m >> ev[e]) & 1]
        leaves = [sum(1 for e in es if t in (eu[e], ev[e])) - 2 for t in (a, b, W)]
        for r in range(d):
            cu, cv = np.abs(sketch(es_, a)[r]), np.abs(sketch(es_, b)[r])
            distinct = lambda x: int(np.count_nonzero(np.diff(np.sort(x))))
            R, par, tie = (b, eb, eb < es_) if distinct(cv) < distinct(cu) else (a, ea, ea < es_)
            sr, sc = sketch(es_, R)[r], sketch(es_, a if R == b else b)[r]
            live = (sr != 0) & (sc != 0)
            srt = np.sort(np.abs(sketch(par, R)[r]))
            ranks = np.searchsorted(srt, np.abs(sr[live]), side="right" if tie else "left")
            G, nq = int(np.unique(ranks).size), int(live.sum())
            prep = sum(3 * w * L for L in leaves) + sum(2 * w * (1 + 2 * L) for L in leaves) + 4 * nq + 4 * w
            ops += prep + w * (6 * (G + 1) + 16 * G + 4)
    return ops, n_tri, len(generic)


def build_work(wl, dw, dedupe: bool, unique: bool = True):
    """CW evaluations the batched build must do, by the path each key column takes:
    a column declared unique is hashed once per surviving row; a key column of a table
    with >= 2^18 rows (dedupe on) is aggregated when its surviving keys span no more values
    than its count array (the declared domain, else the power of two at or above
    min(rows, 2^27)): one evaluation per distinct surviving key; every other column one per
    surviving row.  Each per sketch row of each sketch on the column.  Survivors and
    distinct keys are counted on the device (torch, outside any timed region)."""
    import torch
    total, distinct = 0, {}
    for ti, (t, dt) in enumerate(zip(wl.tables, dw.tables)):
        if not t.key_col:
            continue
        keep = torch.ones(t.n_rows, dtype=torch.bool, device=dw.device)
        for q in t.preds:
            v = dt.cols[q.col].to(torch.int64)
            if q.op == 0:
                keep &= (v >= q.lo) & (v < q.hi)
            elif q.op == 1:
                keep &= v == q.lo
            else:
                bm = dt.bitmaps[t.preds.index(q)].to(torch.int64)
                inb = (v >= 0) & (v < q.nbits)
                vv = torch.where(inb, v, torch.zeros_like(v))
                keep &= inb & (((bm[vv >> 5] >> (vv & 31)) & 1) == 1)
        n_surv = int(keep.sum().item())
        meta = list(getattr(t, "col_meta", None) or []) + [None] * len(t.cols)
        for c in sorted(set(t.key_col)):
            pairs = t.key_col.count(c) * wl.d
            m = meta[c]
            if unique and m is not None and m[0] == "unique" and wl.w <= 65536:
                total += n_surv * pairs
                continue
            agg = False
            if dedupe and t.n_rows >= (1 << 18) and n_surv:
                kept = dt.cols[c][keep]
                lo, hi = int(kept.min().item()), int(kept.max().item())
                if m is not None and 0 < m[2] - m[1] <= (1 << 27):
                    agg = m[1] <= lo and hi < m[2]
                else:
                    cap = 1 << max(0, (min(t.n_rows, 1 << 27) - 1).bit_length())
                    agg = hi - lo < cap
            if agg:
                nd = int(torch.unique(kept).numel())
                distinct[f"{t.name}.col{c}"] = nd
                total += nd * pairs
            else:
                total += n_surv * pairs
    return total, distinct


def _kernel_traffic(name: str):
    """DRAM bytes (read + write) per launch of the kernels of `name` (a phase), summed, from
    the committed ncu capture; None if a source file changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "counters.json")) as f:
            c = json.load(f)[name]
        for src, sha in c["sources"].items():
            path = os.path.join(ROOT, "paper_2102_02440_gb300", "csrc", src)
            if hashlib.sha256(open(path, "rb").read()).hexdigest() != sha:
                return None
        return c["dram_bytes_per_launch"]
    except Exception:
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ms_local: float, world: int):
    """Weak-scaling aggregate: every rank processes units_per_rank units; the job takes
    as long as its slowest rank.  Returns (units per second of the whole job, max ms)."""
    ms_max = _max_over_ranks(ms_local, world)
    return units_per_rank * world / (ms_max / 1e3), ms_max


def workload(a, rank: int, device="cuda"):
    """The benchmark's workload, drawn on the device.  scale (the default): the scale
    configuration, a 1e9-row fact table with int64 Zipf(1.2) keys over 1e8 and 1e6 and two
    int32 predicates at 10% combined selectivity, joined with 1e8- and 1e6-row dimension
    tables (int64 primary keys), d = 15, w = 65536.  five_table: the 5-table cyclic graph of
    the paper's running example at full scale, d = 11, w = 4096.  Every rank draws its own
    data (weak scaling)."""
    from paper_2102_02440_gb300 import datagen as G
    if a.workload == "scale":
        f = a.scale
        return G.scale_workload_device(n_fact=int(1e9 * f), n_d1=int(1e8 * f), n_d2=max(int(1e6 * min(f, 1.0)), 1000),
                                       seed=20210209 + rank, device=device)
    return G.five_table_device(scale=a.scale, w=a.w, data_seed=20210205 + rank, device=device)


def host_sample(wl, frac: float):
    """The first `frac` of every table's rows as host (numpy) columns: the same graph,
    predicates and declarations, for the CPU oracle."""
    from paper_2102_02440_gb300 import datagen as G
    tabs = []
    for t in wl.tables:
        n = max(1, int(t.n_rows * frac))
        cols = [c[:n].cpu().numpy() if hasattr(c, "cpu") else np.ascontiguousarray(c[:n]) for c in t.cols]
        tabs.append(G.Table(t.name, cols, t.preds, t.key_col, t.edge_id, list(getattr(t, "col_meta", []) or [])))
    return G.Workload(f"{wl.name} first {frac:.4%}", tabs, wl.edge_u, wl.edge_v, wl.d, wl.w, wl.hash_seed,
                      wl.data_seed)


# ----------------------------------------------------------------------- CPU oracle leg

def _oracle_calibrate(wl, hp):
    """Seconds of oracle build per row of the workload (mean over its tables, by rows)."""
    from oracle import oracle as orc
    per = 0.0
    for t in wl.tables:
        n = min(t.n_rows, 20_000)
        h = host_sample_table(t, n)
        t0 = time.perf_counter()
        orc.build_sketch(h, hp, wl.d, wl.w)
        per += (time.perf_counter() - t0) / n * t.n_rows
    return per / max(wl.total_rows, 1)


def host_sample_table(t, n: int):
    from paper_2102_02440_gb300 import datagen as G
    cols = [c[:n].cpu().numpy() if hasattr(c, "cpu") else np.ascontiguousarray(c[:n]) for c in t.cols]
    return G.Table(t.name, cols, t.preds, t.key_col, t.edge_id)


def oracle_step(hwl, hp, masks, estimate: bool = True):
    """The oracle (single-threaded, as it stands) on a host workload: the push-down build
    of every sketch, then (estimate) the estimate of every sub-plan.  Returns seconds."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    built = [orc.build_sketch(t, hp, hwl.d, hwl.w) for t in hwl.tables]
    if estimate:
        sk = [tuple(built[hwl.sketch_of(e, end)[0]][0][hwl.sketch_of(e, end)[1]] for end in range(2))
              for e in range(hwl.n_edges)]
        surv = np.array([n for _, n in built], np.int64)
        for m in masks:
            orc.estimate(hwl.edge_u, hwl.edge_v, sk, surv, hwl.d, hwl.w, int(m))
    return time.perf_counter() - t0


def cpu_baseline(wl, masks, budget_s: float = 12.0):
    """The oracle on a bounded row sample of every table (the first rows, in proportion to
    table size): build of every sketch and estimate of every sub-plan; tuples/s and the
    sample description."""
    from oracle import oracle as orc
    orc.build()
    hp = orc.hash_params(wl.hash_seed, wl.n_edges, wl.d)
    frac = min(1.0, budget_s / max(_oracle_calibrate(wl, hp) * wl.total_rows * 1.3, 1e-9))
    hwl = host_sample(wl, frac)
    dt = oracle_step(hwl, hp, masks)
    rows = hwl.total_rows
    return {"value": rows / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {frac:.4%} of every table's rows ({rows} rows): push-down build of all "
                      f"{sum(len(t.key_col) for t in wl.tables)} sketches (d={wl.d} w={wl.w}) and the estimate "
                      f"of all {len(masks)} sub-plans on them, {dt:.1f} s"}


def cpu_baseline_all_cores(wl, budget_s: float = 6.0):
    """The same oracle (unchanged, single-threaded code) run as one instance per host core over
    row partitions of a bounded sample, merged by addition (sketches are linear, Sec. 2): each
    thread calls the oracle's C build on its rows (the call releases the interpreter lock), and
    the per-thread counters are summed.  Returns tuples/s over the sample with cores = threads
    (build only)."""
    import threading as th

    from oracle import oracle as orc
    orc.build()
    n_thr = max(1, os.cpu_count() or 1)
    hp = orc.hash_params(wl.hash_seed, wl.n_edges, wl.d)
    frac = min(1.0, budget_s * n_thr / max(_oracle_calibrate(wl, hp) * wl.total_rows * 1.5, 1e-9))
    hwl = host_sample(wl, frac)
    ns = [t.n_rows for t in hwl.tables]
    parts = [[(t, (ns[i] * j) // n_thr, (ns[i] * (j + 1)) // n_thr) for i, t in enumerate(hwl.tables)]
             for j in range(n_thr)]
    out = [[(np.zeros((len(t.key_col), wl.d, wl.w), np.int32), np.zeros(1, np.int64)) for t in hwl.tables]
           for _ in range(n_thr)]

    def work(j):
        for i, (t, b, e) in enumerate(parts[j]):
            if e > b:
                orc.build_sketch(t, hp, wl.d, wl.w, b, e, accumulate=out[j][i])

    t0 = time.perf_counter()
    threads = [th.Thread(target=work, args=(j,)) for j in range(n_thr)]
    for x in threads:
        x.start()
    for x in threads:
        x.join()
    for i in range(len(hwl.tables)):   # merge by addition (int32 counters wrap exactly)
        for j in range(1, n_thr):
            out[0][i][0][...] = (out[0][i][0].astype(np.int64) + out[j][i][0]).astype(np.int32)
            out[0][i][1][0] += out[j][i][1][0]
    dt = time.perf_counter() - t0
    rows = sum(ns)
    return {"value": rows / dt, "unit": UNIT, "cores": n_thr, "kind": "oracle",
            "sample": f"first {frac:.4%} of every table's rows ({rows} rows) in {n_thr} row partitions, one "
                      f"oracle build per core, counters merged by addition, {dt:.1f} s"}


def run_reference(a):
    """The reference arm: the oracle (single-threaded C++, as it stands) on the host cores,
    each step a bounded row sample of the same workload (build of every sketch + estimate of
    every sub-plan), sized so that the whole run ends within a few minutes."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2102_02440_gb300 import datagen as G
    orc.build()
    wl = workload(a, 0)
    masks = G.connected_subplans(len(wl.tables), wl.edge_u, wl.edge_v)
    hp = orc.hash_params(wl.hash_seed, wl.n_edges, wl.d)
    budget = max(1.0, min(4.0, 150.0 / max(a.steps + a.warmup, 1)))
    frac = min(1.0, budget / max(_oracle_calibrate(wl, hp) * wl.total_rows * 1.3, 1e-9))
    hwl = host_sample(wl, frac)
    del wl
    secs = []
    for k in range(a.warmup + a.steps):
        dt = oracle_step(hwl, hp, masks)
        if k >= a.warmup:
            secs.append(dt)
    ms = statistics.mean(secs) * 1e3
    v = hwl.total_rows / (ms / 1e3)
    sample = (f"first {frac:.4%} of every table's rows ({hwl.total_rows} rows): push-down build of all "
              f"{sum(len(t.key_col) for t in hwl.tables)} sketches and the estimate of all {len(masks)} sub-plans")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": hwl.name, "sample_of": workload_name(a), "rows_per_step": hwl.total_rows,
                       "sample": sample, "step": "one oracle pass over the sample (ms_per_step is that pass)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name(a) -> str:
    if a.workload == "scale":
        f = a.scale
        return (f"scale: fact {int(1e9 * f)} rows (int64 Zipf(1.2) keys over {int(1e8 * f)} and "
                f"{max(int(1e6 * min(f, 1.0)), 1000)}, 10% predicates), dimensions {int(1e8 * f)} and "
                f"{max(int(1e6 * min(f, 1.0)), 1000)} rows, d15 w65536")
    return f"five_table scale={a.scale} d11 w{a.w}"


# ----------------------------------------------------------------------- GPU leg

def cw_peak(dev, d: int, n_pairs: int):
    """Measured rate of the build's hash arithmetic on this GPU (cmp_microbench_cw: no
    memory traffic, no counter updates), evaluations/s, for both forms: shared powers and
    Horner.  Median of 5 timed launches after a warm-up."""
    import torch

    from paper_2102_02440_gb300 import compass as K
    hp = K.hash_params_u64(0xC0FFEE, 1, min(max(n_pairs, 1), 64)).reshape(-1)
    hd = torch.from_numpy(hp.view(np.int64)).to(dev)
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    n_keys = 1 << 26
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for form, name in ((0, "shared_powers"), (1, "horner")):
        np_ = min(max(n_pairs, 1), 64)
        K.cmp_microbench_cw(hd.data_ptr(), np_, n_keys, 65536, form, out.data_ptr(), K.stream_handle())
        ts = []
        for _ in range(5):
            s.record()
            K.cmp_microbench_cw(hd.data_ptr(), np_, n_keys, 65536, form, out.data_ptr(), K.stream_handle())
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        res[name] = n_keys * np_ / (statistics.median(ts) / 1e3)
    return res


def measure(a, wl, dev, world: int, rank: int, headline: bool):
    """One workload's step, timed: the batched build, presort + cross ranks, the estimate of
    every connected sub-plan, the learned combiner and the enumeration, captured as one CUDA
    graph and replayed.  Returns the fields of the bench line (headline) or of an extra key."""
    import torch

    from paper_2102_02440_gb300 import autotune as AT
    from paper_2102_02440_gb300 import compass as K
    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P

    dw = P.DeviceWorkload(wl, device=dev)
    masks = G.connected_subplans(len(wl.tables), wl.edge_u, wl.edge_v)
    # launch shapes picked by the autotuner on this workload (outside the timed region)
    cfg_build, tuned_build = AT.tune_build(dw, reps=2, cache_path=a.tune_cache)
    sig = f"estimate d{wl.d} w{wl.w} tables{len(wl.tables)} masks{','.join(str(m) for m in masks)}"
    cfg_est, tuned_est = AT.tune_estimate(lambda c: P.DeviceEstimator(dw, masks, cfg=c), reps=1,
                                          cache_path=a.tune_cache, signature=sig)
    est = P.DeviceEstimator(dw, masks, cfg=cfg_est)
    stream = torch.cuda.Stream(dev)  # a side stream: CUDA graphs cannot capture the legacy default stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    # learned combiner over every sub-plan's row estimates; self-join sizes of the two
    # sketches of each two-table sub-plan (its training domain), zero elsewhere: one
    # cmp_sketch_f2 launch over every sketch (the tables' counters are one buffer), then the
    # features pick each sub-plan's two sketches by index
    n_sub = len(masks)
    comb, comb_src = P.Combiner.for_sketches(wl.d, wl.w, device=dev)
    # the network serves two-table sub-plans (its training domain) with its stored rule; the
    # others keep the median, and so does every sub-plan when no trained weights exist for d
    # (the untrained network still runs, its output unused)
    use_median_at = float(comb_src.get("use_median_at", 1.0))
    trained = not str(comb_src.get("weights", "")).startswith("untrained")
    eligible = torch.from_numpy(np.array([trained and bin(int(m)).count("1") == 2 for m in masks], np.uint8)).to(dev)
    n_sk = dw.counters_all.shape[0]
    f2_all = torch.zeros(n_sk, dtype=torch.float64, device=dev)
    feat = torch.empty((n_sub, wl.d + 2), dtype=torch.float32, device=dev)
    y_mlp = torch.empty(n_sub, dtype=torch.float32, device=dev)
    est_comb = torch.empty(n_sub, dtype=torch.float64, device=dev)
    first_sketch = np.cumsum([0] + [t.k for t in dw.tables])
    f2_idx_host = np.full((n_sub, 2), -1, np.int32)
    for q, m in enumerate(masks):
        if bin(m).count("1") == 2:
            tu, tv = [t for t in range(len(wl.tables)) if (m >> t) & 1]
            e = next(e for e in range(wl.n_edges) if {wl.edge_u[e], wl.edge_v[e]} == {tu, tv})
            for end in range(2):
                t, si = wl.sketch_of(e, end)
                f2_idx_host[q, end] = first_sketch[t] + si
    f2_idx = torch.from_numpy(f2_idx_host).to(dev)

    def combiner(s):
        K.cmp_sketch_f2(dw.counters_all.data_ptr(), n_sk, wl.d, wl.w, f2_all.data_ptr(), s)
        K.cmp_mlp_features_indexed(est.row_est.data_ptr(), n_sub, wl.d, f2_all.data_ptr(), f2_idx.data_ptr(),
                                   feat.data_ptr(), s)
        K.cmp_mlp_infer(comb.params.data_ptr(), wl.d + 2, comb.nh, comb.skip, feat.data_ptr(), n_sub,
                        y_mlp.data_ptr(), s)
        K.cmp_mlp_combine_ex(est.est.data_ptr(), y_mlp.data_ptr(), eligible.data_ptr(), n_sub, use_median_at,
                             est_comb.data_ptr(), s)

    # join-order enumeration (Algorithm 1, max_plans = 10) over the combined estimates
    enum = P.Enumerator(est.graphs, np.zeros(n_sub, np.int32), masks, device=dev)

    def step(evs=None):
        s = K.stream_handle(stream)
        if evs:
            evs[0].record(stream)
        dw.build_batched(cfg_build, stream=stream)
        if evs:
            evs[1].record(stream)
        est.presort(stream=stream)
        if evs:
            evs[2].record(stream)
        est.estimate(stream=stream)
        if evs:
            evs[3].record(stream)
        combiner(s)
        if evs:
            evs[4].record(stream)
        enum.run(est_comb, stream=stream)
        if evs:
            evs[5].record(stream)

    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            step()
    torch.cuda.synchronize(dev)
    dw.check_status()
    # the whole step captured once as a CUDA graph (the same launches, replayed without
    # per-launch host overhead); its outputs must equal the eager step's bit for bit
    graph = None
    if not a.no_graph:
        eager_out = (est.row_est.clone(), est.est.clone(), est_comb.clone(), enum.order.clone())
        with torch.cuda.stream(stream):
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                step()
            for _ in range(a.warmup):
                graph.replay()
        torch.cuda.synchronize(dev)
        dw.check_status()
        if not (torch.equal(eager_out[3], enum.order) and torch.equal(eager_out[0], est.row_est) and
                torch.equal(eager_out[1].nan_to_num(-1.0), est.est.nan_to_num(-1.0)) and
                torch.equal(eager_out[2].nan_to_num(-1.0), est_comb.nan_to_num(-1.0))):
            raise RuntimeError("graph replay of the step differs from the eager step")

    def timed_step(ev0, ev1):
        ev0.record(stream)
        if graph is not None:
            graph.replay()
        else:
            step()
        ev1.record(stream)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(a.steps)]
    sampler = ClockSampler(dev.index if dev.index is not None else 0) if headline else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    _barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(a.steps):
            flush.zero_()                        # evict the previous step's inputs from L2
            timed_step(*evs[k])
    torch.cuda.synchronize(dev)
    _barrier(world)
    clocks = sampler.stop() if sampler else None
    dw.check_status()
    ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    # per-phase split from eager steps with events between the phases (outside the timing)
    pevs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(a.steps)]
    with torch.cuda.stream(stream):
        for k in range(a.steps):
            flush.zero_()
            step(pevs[k])
    torch.cuda.synchronize(dev)
    per = [[e[i].elapsed_time(e[i + 1]) for i in range(5)] for e in pevs]
    rows = wl.total_rows
    value, ms_max = whole_job_rate(rows, ms, world)
    phase = {n: statistics.mean(p[i] for p in per)
             for i, n in enumerate(("build", "presort", "estimate", "combiner", "enumerate"))}

    # roofline of the dominant phase, the batched build: HBM-bound on the columns it reads,
    # with the hashing it must do against the measured rate of the same arithmetic beside it
    surv = dw.survivors.cpu().numpy()
    updates = int(sum(int(surv[i]) * len(t.key_col) * wl.d for i, t in enumerate(wl.tables)))
    cw_evals, distinct = build_work(wl, dw, dedupe=bool(tuned_build["cfg"].get("dedupe", 1)))
    hbm_peak, peak_kind = _peaks()
    col_bytes = wl.column_bytes()
    build_s = phase["build"] / 1e3
    peaks = cw_peak(dev, wl.d, max(len(t.key_col) for t in wl.tables) * wl.d)
    alu_s = cw_evals / max(peaks.values())
    tkey = "build_scale" if wl.d == 15 else "build_five_table"
    roof = {"bound": "hbm", "achieved": col_bytes / build_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "frac": col_bytes / build_s / 1e9 / hbm_peak, "traffic": _kernel_traffic(tkey),
            "peak_kind": peak_kind,
            "kernel": "the batched build (one cmp_sketch_build_batched call: zeroing, key counting (two launches "
                      "when presence bitmaps are built beside counted tables), presence check, unique-key "
                      "hashing, presence-bitmap hashing, row kernel, hashing of the counted keys)",
            "traffic_source": "profiles/counters.json (ncu DRAM bytes of every kernel of one build; the 1e9-row "
                              "figure scaled x10 from its 10% case), null if a build source changed since",
            "algorithmic": f"{col_bytes} bytes: every referenced column read once ({rows} rows)",
            "alu": {"cw_evaluations": cw_evals, "tuple_updates": updates, "distinct_keys": distinct,
                    "achieved_evals_per_s": cw_evals / build_s,
                    "measured_peak_evals_per_s": peaks,
                    "frac": alu_s / build_s,
                    "peak_source": "cmp_microbench_cw on this GPU (the same arithmetic, no memory traffic)"}}
    est_ops, n_tri_sub, n_gen_sub = triangle_ops(dw, masks)
    est_s = phase["estimate"] / 1e3
    out = {"value": value, "ms_per_step": ms_max, "rows_per_step": rows, "phases_ms": phase,
           "subplans": len(masks), "subplan_estimates_per_s": len(masks) / est_s,
           "build_only_tuples_per_s": rows / build_s, "roofline": roof,
           "estimate_ops": {"exact_128bit_ops": est_ops, "ops_per_s": est_ops / est_s,
                            "triangle_subplans": n_tri_sub, "other_subplans": n_gen_sub},
           "plan": {"order": [wl.tables[t].name for t in enum.plans()[0][0]], "cost": enum.plans()[0][1],
                    "search": dict(zip(("complete_plans", "extensions", "pruned"), enum.plans()[0][2]))},
           "autotuned": {"build": tuned_build["cfg"], "estimate": tuned_est["cfg"]},
           "combiner": comb_src, "survivors": [int(x) for x in surv],
           "config": {"workload": wl.name, "rows_per_step": rows, "tables": len(wl.tables),
                      "sketches": sum(len(t.key_col) for t in wl.tables), "d": wl.d, "w": wl.w,
                      "subplans": len(masks), "column_bytes": col_bytes,
                      "l2": "256 MB buffer written between steps, outside the per-step events; inputs "
                            f"{col_bytes / 1e9:.2f} GB",
                      "step": "one captured CUDA graph replayed per step" if graph is not None else "eager launches",
                      "phases": "from eager steps with events between phases",
                      "parallelism": f"replicas x{world} (independent queries)"}}
    if clocks is not None:
        out["clocks"] = clocks

    # end to end through the public API: pinned host columns -> device, path, estimates -> host
    if headline and not a.no_e2e:
        host_cols = []
        for t in dw.tables:
            hc = []
            for c in t.cols:
                h = torch.empty(c.shape, dtype=c.dtype, pin_memory=True)
                h.copy_(c)
                hc.append(h)
            host_cols.append(hc)
        h2d = sum(c.numel() * c.element_size() for tc in host_cols for c in tc)
        out_host = torch.empty(n_sub, dtype=torch.float64).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_up = torch.cuda.Event(enable_timing=True)
        tms, tups = [], []
        with torch.cuda.stream(stream):
            for k in range(min(a.warmup, 2) + a.steps):
                flush.zero_()
                e0.record(stream)
                dw.upload(host_cols, stream=stream)
                e_up.record(stream)
                if graph is not None:
                    graph.replay()
                else:
                    step()
                out_host.copy_(est_comb, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                if k >= min(a.warmup, 2):
                    tms.append(e0.elapsed_time(e1))
                    tups.append(e0.elapsed_time(e_up))
        e2e_ms = _max_over_ranks(statistics.mean(tms), world)
        up_ms = statistics.mean(tups)
        out["e2e"] = {"value": rows * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(out_host.numel() * 8), "ms_per_step": e2e_ms,
                      "h2d_ms": up_ms, "h2d_gbs": h2d / (up_ms / 1e3) / 1e9}
        del host_cols
    if headline and rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, masks)
        out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(wl)
    # our kernel launches per step: build (zeroing; clearing + counting with aggregated key
    # columns; the unique-key kernel; the row kernel when it has items; hashing of the counted
    # keys; the presence-bitmap kernel), presort (one launch for w <= 16384, else chunks + 3
    # merges + split per 64 rows) and cross ranks, estimate (int64 items + int128 recompute for
    # tree sub-plans, 3 triangle launches, finalize, the exact tier), combiner (4), enumeration (1)
    h = dw._plan[0][0] if dw._plan else None
    info = P.build_plan_info(dw)
    # presort and cross ranks of the tables the plan reads sorted, per run of consecutive tables
    presort_l = 0
    for _lo, _rlo, run in P.presort_runs(dw, only=est.sorted_tables()):
        n_rows_sorted = sum(dw.tables[i].k for i in run) * wl.d
        if n_rows_sorted:
            presort_l += (1 if wl.w <= 16384 else 5 * ((n_rows_sorted + 63) // 64)) + 1
    # (the exact tier: two passes and its finalize, which return at once when no row is queued)
    est_l = (2 if n_gen_sub > sum(1 for m in masks if bin(m).count("1") == 1) else 0) + (3 if n_tri_sub else 0) + 1 + 3
    out["gpu_launches_per_step"] = info["launches"] + presort_l + est_l + 4 + 1
    return out


def measure_batched(a, dev):
    """The batched-enumeration configuration on the device: 64 synthetic graphs (chains,
    stars, cycles of 4..17 tables, rows log-uniform in [1e4, 1e8], Zipf 0.5..1.5 keys over
    1e5, ~50% of tables with a point or range predicate), d = 11, w = 1024.  Build of every
    table in one batched launch vs one launch per table; the estimate of every connected
    sub-plan in one plan (cached subtree messages and the star lattice on), replayed as a
    CUDA graph, vs one plan launch per sub-plan (timed on a sample of 2000)."""
    import torch

    from paper_2102_02440_gb300 import compass as K
    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    t0 = time.perf_counter()
    graphs = G.graph_batch_device(64, 4, 17, rows_lo=10_000, rows_hi=100_000_000, d=11, w=1024, device=dev,
                                  rows_scale=a.c3_rows_scale)
    gen_s = time.perf_counter() - t0
    gb = P.GraphBatch(graphs, device=dev)
    sg, sm = [], []
    for gi, g in enumerate(graphs):
        ms_ = G.connected_subplans(len(g.tables), g.edge_u, g.edge_v)
        sg += [gi] * len(ms_)
        sm += ms_
    sg, sm = np.array(sg, np.int32), np.array(sm, np.uint64)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    ms_build_b = timed(gb.build_batched)
    ms_build_t = timed(gb.build_per_table)
    gb.build_batched()
    gb.presort()
    reuse = K.cmp_estimate_cfg.make(threads=256, ctas_per_sm=4, cond_chunk=16,
                                    flags=K.CMP_EST_CACHE_MESSAGES | K.CMP_EST_STAR_LATTICE)
    plan = gb.plan(sg, sm, reuse)
    st = torch.cuda.Stream(dev)
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        plan.run(stream=st)
        st.synchronize()
        g_est = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_est, stream=st):
            plan.run(stream=st)
        ms_est_b = timed(lambda: (g_est.replay(), st.synchronize()))
    # the same plan without the exact tier beyond int128 (its sub-plans beyond int128 NaN)
    plan_nw = gb.plan(sg, sm, K.cmp_estimate_cfg.make(threads=256, ctas_per_sm=4, cond_chunk=16,
                                                      flags=K.CMP_EST_CACHE_MESSAGES | K.CMP_EST_STAR_LATTICE |
                                                      K.CMP_EST_NO_WIDE))
    ms_est_nw = timed(plan_nw.run, 1)
    nan_nw = torch.isnan(plan_nw.est).cpu().numpy()
    n_nan_nw = int(nan_nw.sum())
    n_cyc_nw = 0  # of those, the sub-plans with a cycle (as many edges as tables, or more)
    for q in np.flatnonzero(nan_nw):
        g, m = graphs[sg[q]], int(sm[q])
        inner = sum(1 for u, v in zip(g.edge_u, g.edge_v) if (m >> u) & 1 and (m >> v) & 1)
        n_cyc_nw += int(inner >= bin(m).count("1"))
    del plan_nw
    gb.dw.status.zero_()
    rng = np.random.default_rng(0)
    samp = rng.choice(sm.size, min(2000, sm.size), replace=False)
    plans = [gb.plan(sg[q:q + 1], sm[q:q + 1]) for q in samp]
    ms_est_1 = timed(lambda: [p.run() for p in plans], 1)
    n_nan = int(torch.isnan(plan.est).sum().item())
    gb.dw.status.zero_()
    return {"workload": f"64 graphs, {len(gb.wl.tables)} tables, {gb.total_rows} rows, {int(sm.size)} sub-plans, "
                        f"d11 w1024 (rows log-uniform in [1e4, 1e8] x {a.c3_rows_scale})",
            "generation_s": gen_s, "column_bytes": gb.wl.column_bytes(),
            "build_ms": {"batched_one_launch": ms_build_b, "per_table_launches": ms_build_t,
                         "speedup": ms_build_t / ms_build_b, "tuples_per_s": gb.total_rows / (ms_build_b / 1e3)},
            "estimate": {"one_plan_graph_replayed_ms": ms_est_b, "subplan_estimates_per_s": sm.size / (ms_est_b / 1e3),
                         "per_subplan_launches_per_s": samp.size / (ms_est_1 / 1e3),
                         "speedup": (sm.size / (ms_est_b / 1e3)) / (samp.size / (ms_est_1 / 1e3)),
                         "flags": "CMP_EST_CACHE_MESSAGES | CMP_EST_STAR_LATTICE, 256 threads x 4 CTAs/SM, chunk 16",
                         "subplans_nan": n_nan,
                         "without_exact_tier": {"ms": ms_est_nw, "subplans_beyond_int128": n_nan_nw,
                                                "of_which_cyclic": n_cyc_nw}}}


def run_ours(a):
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload(a, rank, device=dev)
    r = measure(a, wl, dev, world, rank, headline=True)
    del wl
    torch.cuda.empty_cache()
    extras = {}
    if not a.no_extras and world == 1:
        from paper_2102_02440_gb300 import datagen as G
        a5 = argparse.Namespace(**vars(a))
        a5.workload, a5.scale, a5.w = "five_table", 1.0, 4096
        wl5 = G.five_table_device(scale=1.0, w=4096, data_seed=20210205 + rank, device=dev)
        m5 = measure(a5, wl5, dev, world, rank, headline=False)
        extras["five_table"] = {k: m5[k] for k in ("value", "ms_per_step", "phases_ms", "subplan_estimates_per_s",
                                                    "build_only_tuples_per_s", "roofline", "plan", "config",
                                                    "estimate_ops", "gpu_launches_per_step")}
        del wl5, m5
        torch.cuda.empty_cache()
        extras["batched_enumeration"] = measure_batched(a, dev)
        torch.cuda.empty_cache()
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": r["config"],
                "roofline": r["roofline"], "cpu_baseline": r.get("cpu_baseline"), "e2e": r.get("e2e"),
                "clocks": r.get("clocks"), "gpu_launches": r["gpu_launches_per_step"] * a.steps,
                "phases_ms": r["phases_ms"], "subplan_estimates_per_s": r["subplan_estimates_per_s"],
                "build_only_tuples_per_s": r["build_only_tuples_per_s"], "estimate_ops": r["estimate_ops"],
                "plan": r["plan"], "autotuned": r["autotuned"], "combiner": r["combiner"],
                "survivors": r["survivors"], **extras}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_case(a):
    """Profiling cases (one GPU, under 1 GB on the device): the estimate of all 19 sub-plans
    of the five-table graph at w = 4096 on sketches of the tables at 5% scale (estimate_small)
    or full scale (estimate_full, the benchmark's sketches); the single-table fused build of
    the 36M-row F1 table alone (3 sketches, d = 11, w = 4096, per-tuple path); the
    benchmark's batched build of all five tables (build_five); or the star lattice over all
    65,535 sub-plans of one 17-table star (rows log-uniform in [1e4, 1e5], d = 11, w = 1024;
    star17)."""
    import torch

    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.case in ("estimate_small", "estimate_full"):
        wl = G.five_table(scale=0.05 if a.case == "estimate_small" else 1.0, w=4096)
        dw = P.DeviceWorkload(wl)
        dw.build_batched()
        est = P.DeviceEstimator(dw, G.connected_subplans(5, wl.edge_u, wl.edge_v))
        est.presort()
        fn = est.estimate
    elif a.case == "star17":
        from paper_2102_02440_gb300 import compass as K
        g = G.graph_batch(1, 17, 17, rows_lo=10_000, rows_hi=100_000, d=11, w=1024, kinds=("star",))
        dw = P.DeviceWorkload(g[0])
        dw.build_batched()
        est = P.DeviceEstimator(dw, G.connected_subplans(17, g[0].edge_u, g[0].edge_v),
                                cfg=K.cmp_estimate_cfg.make(flags=K.CMP_EST_STAR_LATTICE))
        est.presort()
        fn = est.estimate
    elif a.case == "build_f1":
        full = G.five_table(scale=1.0, w=4096)
        wl = G.Workload("F1 only", [full.tables[0]], [0] * 5, [0] * 5, 11, 4096, full.hash_seed, 0)
        dw = P.DeviceWorkload(wl)
        fn = dw.build
    else:  # build_five: the benchmark's batched build (key aggregation on F1, F2, D1, D3)
        wl = G.five_table(scale=1.0, w=4096)
        dw = P.DeviceWorkload(wl)
        fn = dw.build_batched
    for r in range(2):
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        print(f"{a.case} rep {r}: {s.elapsed_time(e):.3f} ms", flush=True)
    if a.case == "star17":  # the largest leaf subsets leave int128 in some rows: NaN, reported
        print(f"star17: {int(torch.isnan(est.est).sum().item())} of {est.est.numel()} sub-plans beyond int128",
              flush=True)
        dw.status.zero_()
    dw.check_status()


def run_batched(a):
    """Batched enumeration: 64 synthetic graphs (chains, stars, cycles of 4..17 tables, rows
    log-uniform in [1e4, 1e6], Zipf 0.5..1.5 keys over 1e5, ~50% of tables with a point or
    range predicate), d = 11, w = 1024.  Times, on one GPU:
      build: one batched launch for every table vs one launch per table;
      estimate: one plan over every connected sub-plan (cached subtree messages and the star
        lattice on) vs one plan launch per sub-plan (timed on a random sample of sub-plans,
        reported per sub-plan);
      the batched build + presort + estimate captured in one CUDA graph vs eager."""
    import torch

    from paper_2102_02440_gb300 import compass as K
    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    graphs = G.graph_batch(64, 4, 17, rows_lo=10_000, rows_hi=1_000_000, d=11, w=1024)
    gb = P.GraphBatch(graphs)
    sg, sm = [], []
    for gi, g in enumerate(graphs):
        ms = G.connected_subplans(len(g.tables), g.edge_u, g.edge_v)
        sg += [gi] * len(ms)
        sm += ms
    sg, sm = np.array(sg, np.int32), np.array(sm, np.uint64)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    ms_build_b = timed(gb.build_batched)
    ms_build_t = timed(gb.build_per_table)
    gb.build_batched()
    gb.presort()
    # one plan over every sub-plan, with the reuse across sub-plans on (cached subtree
    # messages and the star lattice) and the launch shape `--case shapes` measured fastest
    # here (256 threads, four CTAs per SM, 16 conditioning values per item); the
    # per-sub-plan comparison plans one sub-plan each
    reuse = K.cmp_estimate_cfg.make(threads=256, ctas_per_sm=4, cond_chunk=16,
                                    flags=K.CMP_EST_CACHE_MESSAGES | K.CMP_EST_STAR_LATTICE)
    plan = gb.plan(sg, sm, reuse)
    ms_est_b = timed(plan.run, 3)
    rng = np.random.default_rng(0)
    samp = rng.choice(sm.size, min(2000, sm.size), replace=False)
    plans = [gb.plan(sg[q:q + 1], sm[q:q + 1]) for q in samp]
    ms_est_1 = timed(lambda: [p.run() for p in plans], 3)
    # whole batched sequence: eager vs one CUDA graph
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())

    def seq():
        gb.build_batched(stream=st)
        gb.presort(stream=st)
        plan.run(stream=st)

    with torch.cuda.stream(st):
        seq()
        st.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            seq()
        ms_eager = timed(lambda: (seq(), st.synchronize()))
        ms_graph = timed(lambda: (graph.replay(), st.synchronize()))
    # sub-plans whose exact row estimates leave int128 (long chains of large tables) are NaN
    # with CMP_EOVERFLOW in the status word; count them instead of failing
    n_ovf = int(torch.isnan(plan.est).sum().item())
    gb.dw.status.zero_()
    # join-order enumeration of every graph in one launch (Algorithm 1, max_plans = 10 and 1)
    enum_ms, enum_stats = {}, {}
    for mp in (10, 1):
        en = P.Enumerator(gb.graph_structs(), sg, sm, cfg=K.cmp_enum_cfg.make(max_plans=mp, max_nodes=1 << 20))
        enum_ms[f"max_plans_{mp}"] = timed(lambda: en.run(plan.est), 5)
        res = en.plans()
        enum_stats[f"max_plans_{mp}"] = {"plans_found": sum(1 for o, c, st in res if o),
                                         "extensions": sum(st[1] for o, c, st in res),
                                         "complete_plans": sum(st[0] for o, c, st in res),
                                         "status": int(en.status.item())}
    n_tables = len(gb.wl.tables)
    line = {"case": "batched enumeration", "graphs": len(graphs), "tables": n_tables, "rows": gb.total_rows,
            "subplans": int(sm.size), "d": 11, "w": 1024,
            "build_ms": {"batched_one_launch": ms_build_b, "per_table_launches": ms_build_t,
                         "speedup": ms_build_t / ms_build_b},
            "estimate": {"flags": "CMP_EST_CACHE_MESSAGES | CMP_EST_STAR_LATTICE", "threads": 256,
                         "ctas_per_sm": 4, "cond_chunk": 16,
                         "batched_one_plan_ms": ms_est_b, "batched_subplans_per_s": sm.size / (ms_est_b / 1e3),
                         "per_subplan_launches_subplans_per_s": samp.size / (ms_est_1 / 1e3),
                         "per_subplan_sample": int(samp.size),
                         "speedup": (sm.size / (ms_est_b / 1e3)) / (samp.size / (ms_est_1 / 1e3))},
            "sequence_ms": {"eager": ms_eager, "cuda_graph": ms_graph},
            "subplans_beyond_int128": n_ovf,
            "enumeration_ms": enum_ms, "enumeration": enum_stats,
            "kinds": {k: sum(1 for g in graphs if g.name.startswith(k)) for k in ("chain", "star", "cycle")}}
    print(json.dumps(line), flush=True)


def run_scale(a):
    """The scale configuration (1e9-row fact, int64 keys, d = 15, w = 65536, drawn on the
    device): batched build of the three tables, presort + cross ranks, estimates of every
    connected sub-plan; per-phase CUDA-event times over 3 timed repetitions."""
    import torch

    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    f = a.scale
    wl = G.scale_workload_device(n_fact=int(1e9 * f), n_d1=int(1e8 * f), n_d2=max(int(1e6 * min(f, 1.0)), 1000))
    dw = P.DeviceWorkload(wl)
    masks = G.connected_subplans(3, wl.edge_u, wl.edge_v)
    est = P.DeviceEstimator(dw, masks)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ts = []
    for k in range(4):
        ev[0].record()
        dw.build_batched()
        ev[1].record()
        est.presort()
        ev[2].record()
        est.estimate()
        ev[3].record()
        torch.cuda.synchronize()
        if k:
            ts.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
    dw.check_status()
    ph = {n: statistics.median(t[i] for t in ts) for i, n in enumerate(("build", "presort", "estimate"))}
    surv = dw.survivors.cpu().numpy()
    rows, col_bytes = wl.total_rows, wl.column_bytes()
    evals = int(sum(int(surv[i]) * len(t.key_col) * wl.d for i, t in enumerate(wl.tables)))
    hbm_peak, kind = _peaks()
    step = sum(ph.values())
    print(json.dumps({"case": "scale", "workload": wl.name, "rows": rows, "column_bytes": col_bytes,
                      "survivors": [int(x) for x in surv], "phases_ms": ph,
                      "tuples_per_s_step": rows / (step / 1e3), "build_tuples_per_s": rows / (ph["build"] / 1e3),
                      "build_hbm": {"achieved_gbs": col_bytes / (ph["build"] / 1e3) / 1e9, "peak_gbs": hbm_peak,
                                    "frac": col_bytes / (ph["build"] / 1e3) / 1e9 / hbm_peak, "peak_kind": kind},
                      "build_alu": {"cw_evaluations": evals,
                                    "frac": evals * CW_INSTR / (ph["build"] / 1e3) / INT_ISSUE_PEAK},
                      "estimates": est.est.cpu().numpy().tolist()}), flush=True)


def chain_join_size(wl) -> int:
    """Exact size of D2 |x| F2 |x| D1 (tables 3, 1, 2 over edges e0, e1) of the five-table
    workload, from the columns on the host: per F2 tuple, the number of selected D2 tuples
    with its keyword key times the number of selected D1 tuples with its movie key."""
    def counts(t, col, dom):
        tb = wl.tables[t]
        keep = np.ones(tb.n_rows, bool)
        for q in tb.preds:
            v = tb.cols[q.col].astype(np.int64)
            keep &= (q.lo <= v) & (v < q.hi) if q.op == 0 else (v == q.lo)
        return np.bincount(tb.cols[col][keep].astype(np.int64), minlength=dom)
    f2 = wl.tables[1]
    kw = counts(3, 0, int(max(f2.cols[0].max(), wl.tables[3].cols[0].max())) + 1)
    mv = counts(2, 0, int(max(f2.cols[1].max(), wl.tables[2].cols[0].max())) + 1)
    return int((kw[f2.cols[0].astype(np.int64)] * mv[f2.cols[1].astype(np.int64)]).sum())


def run_partition(a):
    """Sketch partitioning (Sec. 4.1) on the k - mk - t chain of the five-table workload at
    full scale: D2 |x| F2 |x| D1 over edges e0 (keyword) and e1 (movie), F2 with the 2-axis
    tensor.  For two width configurations, equal memory (64 x 64 counters per F2 row: the
    4096 buckets of a 1-D row rearranged, so D2 and D1 get 64 buckets) and equal width
    (4096 x 4096: the merged sketches' width on both edges), the build of the three
    partitioned sketches and the contraction estimate are timed with CUDA events (median of
    10 after 3 warm-ups); the estimate is compared with the exact join size and with the
    merged 1-D estimate of the same sub-plan (w = 4096)."""
    import torch

    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    wl = G.five_table(scale=a.scale, w=4096)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    mask = (1 << 3) | (1 << 1) | (1 << 2)
    est_m = P.DeviceEstimator(dw, [mask])
    est_m.presort()
    est_m.estimate()
    torch.cuda.synchronize()
    merged = float(est_m.est.item())
    exact = chain_join_size(wl)
    hbm_peak, kind = _peaks()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=10, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    def qerr(x):
        return max(x, 1.0) / max(exact, 1.0) if x >= exact else max(exact, 1.0) / max(x, 1.0)

    configs = {}
    for name, widths in (("equal_memory_64x64", [64, 64]), ("equal_width_4096x4096", [4096, 4096])):
        pj = P.PartitionedJoin(wl, [3, 1, 2], [0, 1], widths, cols_dev=[dw.tables[t].cols for t in (3, 1, 2)],
                               hash_dev=dw.hash_dev)
        ms_build = timed(pj.build)
        ms_est = timed(pj.estimate)
        if int(pj.status.item()) != 0:
            raise RuntimeError(f"device status {int(pj.status.item())}")
        surv = [int(x) for x in pj.survivors.cpu().numpy()]
        est = float(pj.est.item())
        tensor_bytes = sum(x.numel() * 4 for x in pj.tensors)
        evals = sum(n * len(ax) * wl.d for n, ax in zip(surv, pj.axes))
        configs[name] = {
            "widths": widths, "tensor_bytes": tensor_bytes, "survivors": surv,
            "build_ms": ms_build, "estimate_ms": ms_est, "estimate": est, "q_error": qerr(est),
            "build_alu": {"cw_evaluations": evals, "frac": evals * CW_INSTR / (ms_build / 1e3) / INT_ISSUE_PEAK},
            "estimate_hbm": {"bytes": tensor_bytes, "achieved_gbs": tensor_bytes / (ms_est / 1e3) / 1e9,
                             "peak_gbs": hbm_peak, "frac": tensor_bytes / (ms_est / 1e3) / 1e9 / hbm_peak,
                             "peak_kind": kind},
        }
        del pj
        torch.cuda.empty_cache()
    print(json.dumps({"case": "partition", "workload": wl.name, "join": "D2 |x| F2 |x| D1 (e0, e1)", "d": wl.d,
                      "exact": exact, "merged_1d_w4096": {"estimate": merged, "q_error": qerr(merged)},
                      "partitioned": configs}), flush=True)


def two_way_sizes(wl):
    """Exact size of every single-edge join of the workload (its two-table sub-plans), from
    the columns on the host: per edge, the dot product of the two endpoints' selected key
    histograms."""
    def keep(t):
        tb = wl.tables[t]
        m = np.ones(tb.n_rows, bool)
        for q in tb.preds:
            v = tb.cols[q.col].astype(np.int64)
            if q.op == 0:
                m &= (q.lo <= v) & (v < q.hi)
            elif q.op == 1:
                m &= v == q.lo
            else:
                inb = (v >= 0) & (v < q.nbits)
                bits = np.zeros(tb.n_rows, bool)
                vv = v[inb]
                bits[inb] = ((q.bitmap[vv >> 5] >> (vv & 31).astype(np.uint32)) & 1) == 1
                m &= bits
        return m
    masks = [keep(t) for t in range(len(wl.tables))]
    out = {}
    for e in range(wl.n_edges):
        cols = []
        for end in range(2):
            t, s = wl.sketch_of(e, end)
            cols.append(wl.tables[t].cols[wl.tables[t].key_col[s]][masks[t]].astype(np.int64))
        n = int(max(c.max() if c.size else 0 for c in cols)) + 1
        out[(1 << wl.edge_u[e]) | (1 << wl.edge_v[e])] = int(
            (np.bincount(cols[0], minlength=n).astype(np.int64) * np.bincount(cols[1], minlength=n)).sum())
    return out


def run_offline_sample(a):
    """Two build options of Sec. 2 "Workflow" on the five-table workload (full scale, d = 11,
    w = 4096), each timed as build + presort + estimate of all 19 sub-plans (median of 5
    after a warm-up, CUDA events):
      offline: F1 and F2 have no predicates, so their sketches, presort and cross ranks are
        built once (untimed) and plugged into every query; the per-query work is D1, D2 and
        D3 only.  The estimates must equal the all-online ones bit for bit.
      sample: every table's sketches over a Bernoulli row sample at rate p (1, 0.1, 0.01),
        estimates scaled by 1 / p per table; q-errors of the five two-table sub-plans against
        their exact sizes."""
    import torch

    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    wl = G.five_table(scale=a.scale, w=4096)
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    def query(dw, est):
        def run():
            dw.build_batched()
            est.presort()
            est.estimate()
        return run

    dw = P.DeviceWorkload(wl)
    est = P.DeviceEstimator(dw, masks)
    ms_online = timed(query(dw, est))
    ref = est.est.clone()
    cols = [t.cols for t in dw.tables]
    dwo = P.DeviceWorkload(wl, cols_dev=cols, offline=[0, 1])
    dwo.build_offline()
    esto = P.DeviceEstimator(dwo, masks)
    ms_offline = timed(query(dwo, esto))
    same = bool(torch.equal(esto.est, ref)) or bool(torch.equal(torch.nan_to_num(esto.est), torch.nan_to_num(ref)))
    del dwo, esto
    exact = two_way_sizes(wl)
    pair_q = {m: q for q, m in enumerate(masks) if int(m) in exact}

    def qerr(x, t):
        x, t = max(float(x), 1.0), max(float(t), 1.0)
        return max(x / t, t / x)

    sample = {}
    for rate in (1.0, 0.1, 0.01):
        dws = P.DeviceWorkload(wl, cols_dev=cols, sample_rates=[rate] * 5)
        ests = P.DeviceEstimator(dws, masks)
        ms = timed(query(dws, ests))
        dws.check_status()
        ev = ests.est.cpu().numpy()
        qs = [qerr(ev[q], exact[int(m)]) for m, q in pair_q.items()]
        sample[f"rate_{rate}"] = {"ms": ms, "survivors": [int(x) for x in dws.survivors.cpu().numpy()],
                                  "two_way_q_error": {"median": float(np.median(qs)), "max": float(max(qs))},
                                  "two_way": {bin(int(m)): [float(ev[q]), exact[int(m)]] for m, q in pair_q.items()}}
        del dws, ests
        torch.cuda.empty_cache()
    print(json.dumps({"case": "offline_sample", "workload": wl.name, "subplans": len(masks),
                      "online_ms": ms_online,
                      "offline": {"tables": ["F1", "F2"], "per_query_ms": ms_offline,
                                  "speedup": ms_online / ms_offline, "estimates_identical": same},
                      "sample": sample}), flush=True)


def run_cached(a):
    """Reuse across the sub-plans of an enumeration (Sec. 4.2 (n+1)-D from n-D merges, Sec. 5
    caches of merged sketches and products) on the batched-enumeration graph set (64 chains,
    stars and cycles of 4..17 tables, d = 11, w = 1024): the estimate of the chain graphs'
    sub-plans, the star graphs' sub-plans and every sub-plan, planned plain, with cached
    subtree messages (CMP_EST_CACHE_MESSAGES), with the star lattice (CMP_EST_STAR_LATTICE)
    and with both.  Plan counts come from cmp_estimate_plan_stats; CUDA-event times are
    medians of 3 after one warm-up; every plan's outputs are compared bit for bit with the
    plain plan's."""
    import torch

    from paper_2102_02440_gb300 import compass as K
    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    graphs = G.graph_batch(64, 4, 17, rows_lo=10_000, rows_hi=1_000_000, d=11, w=1024)
    gb = P.GraphBatch(graphs)
    sg, sm, kind = [], [], []
    for gi, g in enumerate(graphs):
        for m in G.connected_subplans(len(g.tables), g.edge_u, g.edge_v):
            sg.append(gi)
            sm.append(m)
            kind.append(g.name.rstrip("0123456789"))
    sg, sm, kind = np.array(sg, np.int32), np.array(sm, np.uint64), np.array(kind)
    gb.build_batched()
    gb.presort()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    flags = {"plain": 0, "cache": K.CMP_EST_CACHE_MESSAGES, "lattice": K.CMP_EST_STAR_LATTICE,
             "cache_lattice": K.CMP_EST_CACHE_MESSAGES | K.CMP_EST_STAR_LATTICE}
    out = {}
    for name, sel in (("chain_graphs", kind == "chain"), ("star_graphs", kind == "star"),
                      ("all_subplans", np.ones(sm.size, bool))):
        res, ref = {"subplans": int(sel.sum())}, None
        for fname, fl in flags.items():
            plan = gb.plan(sg[sel], sm[sel], K.cmp_estimate_cfg.make(flags=fl))
            ms = timed(plan.run)
            torch.cuda.synchronize()
            st = K.cmp_estimate_plan_stats(plan.host.ctypes.data)
            r = {"ms": ms, "subplans_per_s": float(sel.sum()) / (ms / 1e3), "ops": int(st.n_ops),
                 "cached_messages": int(st.n_jobs), "levels": int(st.n_levels), "star_families": int(st.n_star),
                 "star_subplans": int(st.n_star_sub), "lattice_entries": int(st.n_star_entries),
                 "ws_bytes": int(plan.ws.numel())}
            if ref is None:
                ref = plan
            else:
                na, nb = torch.isnan(ref.est), torch.isnan(plan.est)
                both = ~na & ~nb
                r["identical"] = bool(torch.equal(ref.row_est[both], plan.row_est[both]) and torch.equal(na, nb) and
                                      torch.equal(ref.est[both], plan.est[both]))
                # rows where an intermediate value left int128 may be flagged by one evaluation only
                r["nan_in_one_only"] = int((na ^ nb).sum().item())
                r["finite_mismatch"] = int(((ref.est != plan.est) & both).sum().item() +
                                           ((ref.row_est != plan.row_est).any(-1).any(-1) & both).sum().item())
                r["speedup"] = res["plain"]["ms"] / ms
                del plan
            res[fname] = r
        out[name] = res
        del ref
    gb.dw.status.zero_()
    print(json.dumps({"case": "reuse across sub-plans", "graphs": len(graphs), "d": 11, "w": 1024, **out}),
          flush=True)


def run_shapes(a):
    """Estimate launch shapes on the batched-enumeration graph set (64 graphs, 381,253
    sub-plans, d = 11, w = 1024), every sub-plan in one plan with both reuse flags: threads
    per CTA, resident CTAs per SM and conditioning values per item.  CUDA-event medians of 3
    after one warm-up; every shape's outputs compared bit for bit with the first."""
    import torch

    from paper_2102_02440_gb300 import compass as K
    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    graphs = G.graph_batch(64, 4, 17, rows_lo=10_000, rows_hi=1_000_000, d=11, w=1024)
    gb = P.GraphBatch(graphs)
    sg, sm = [], []
    for gi, g in enumerate(graphs):
        ms = G.connected_subplans(len(g.tables), g.edge_u, g.edge_v)
        sg += [gi] * len(ms)
        sm += ms
    gb.build_batched()
    gb.presort()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flags = K.CMP_EST_CACHE_MESSAGES | K.CMP_EST_STAR_LATTICE
    out, ref = [], None
    for th, cps, ch in ((1024, 1, 64), (256, 4, 64), (256, 4, 16), (512, 1, 64), (256, 2, 64)):
        plan = gb.plan(sg, sm, K.cmp_estimate_cfg.make(threads=th, ctas_per_sm=cps, cond_chunk=ch, flags=flags))
        plan.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            s.record()
            plan.run()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        r = {"threads": th, "ctas_per_sm": cps, "cond_chunk": ch, "ms": statistics.median(ts),
             "subplans_per_s": len(sm) / (statistics.median(ts) / 1e3)}
        if ref is None:
            ref = plan
        else:
            ok = ~torch.isnan(ref.est)
            r["identical"] = bool(torch.equal(torch.isnan(ref.est), torch.isnan(plan.est)) and
                                  torch.equal(ref.est[ok], plan.est[ok]) and torch.equal(ref.row_est[ok], plan.row_est[ok]))
        out.append(r)
    gb.dw.status.zero_()
    print(json.dumps({"case": "estimate launch shapes", "subplans": len(sm), "shapes": out}), flush=True)


def main():
    a = _args()
    if a.case == "batched":
        run_batched(a)
    elif a.case == "batched_full":  # the batched-enumeration extra of the benchmark line, alone
        import torch
        print(json.dumps({"case": "batched enumeration at full rows",
                          **measure_batched(a, torch.device("cuda", 0))}), flush=True)
    elif a.case == "cached":
        run_cached(a)
    elif a.case == "shapes":
        run_shapes(a)
    elif a.case == "scale":
        run_scale(a)
    elif a.case == "partition":
        run_partition(a)
    elif a.case == "offline_sample":
        run_offline_sample(a)
    elif a.case:
        run_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
