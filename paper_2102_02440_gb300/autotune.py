"""Launch-shape autotuner for the build and the estimate.

Times candidate cmp_build_cfg / cmp_estimate_cfg shapes on the caller's own workload with
CUDA events, checks that every candidate produces bit-identical outputs (the results do
not depend on the launch shape), and returns the fastest.  Choices can be cached in a
JSON file keyed by a workload signature (d, w, widest table, row count, key width,
predicate share), so a later run with a similar workload skips the search.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import compass as K

BUILD_CANDIDATES = [
    dict(mode=1, threads=512, tile_rows=2048, dedupe=1),
    dict(mode=1, threads=1024, tile_rows=4096, dedupe=1),
    dict(mode=1, threads=512, tile_rows=2048, dedupe=0),
    dict(mode=2, threads=1024, tile_rows=4096, dedupe=1),
    dict(mode=2, threads=512, tile_rows=2048, dedupe=1),
    dict(mode=2, threads=1024, tile_rows=4096, dedupe=0),
    dict(mode=2, threads=1024, tile_rows=2048, dedupe=1, ctas_per_sm=1),
]

ESTIMATE_CANDIDATES = [
    dict(threads=1024, ctas_per_sm=1, cond_chunk=64),
    dict(threads=1024, ctas_per_sm=2, cond_chunk=64),
    dict(threads=512, ctas_per_sm=2, cond_chunk=64),
    dict(threads=512, ctas_per_sm=4, cond_chunk=64),
    dict(threads=1024, ctas_per_sm=1, cond_chunk=16),
    dict(threads=1024, ctas_per_sm=1, cond_chunk=256),
    dict(threads=256, ctas_per_sm=4, cond_chunk=64),
    dict(threads=256, ctas_per_sm=4, cond_chunk=16),
]


def build_signature(dw) -> str:
    k = max((t.k for t in dw.tables), default=0)
    rows = sum(t.n_rows for t in dw.tables)
    int64 = any(c.dtype == torch.int64 for t in dw.tables for c in t.cols)
    preds = sum(1 for t in dw.wl.tables if t.preds) / max(len(dw.tables), 1)
    return f"build d{dw.d} w{dw.w} k{k} rows2^{int(math.log2(max(rows, 1)))} key{'64' if int64 else '32'} " \
           f"pred{round(preds, 1)}"


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def _save(path, cache):
    if path:
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def tune_build(dw, candidates=None, reps: int = 3, cache_path: str | None = None):
    """Fastest batched-build shape for DeviceWorkload `dw`.  Returns (cmp_build_cfg, report)."""
    sig = build_signature(dw)
    cache = _load(cache_path)
    if sig in cache:
        return K.cmp_build_cfg.make(**cache[sig]["cfg"]), cache[sig]
    report, ref, best = [], None, None
    for cand in candidates or BUILD_CANDIDATES:
        cfg = K.cmp_build_cfg.make(**cand)
        try:
            dw._plan = None
            dw.encode_batched(cfg)
        except K.CompassError:
            report.append({"cfg": cand, "ms": None, "why": "rejected by the library"})
            continue
        ms = _time(lambda: dw.build_batched(cfg), reps)
        out = [t.counters.clone() for t in dw.tables] + [dw.survivors.clone()]
        if ref is None:
            ref = out
        elif not all(torch.equal(a, b) for a, b in zip(ref, out)):
            raise RuntimeError(f"launch shape {cand} changed the sketches")
        report.append({"cfg": cand, "ms": ms})
        if best is None or ms < best[1]:
            best = (cand, ms)
    dw._plan = None
    entry = {"cfg": best[0], "ms": best[1], "signature": sig, "tried": report}
    cache[sig] = entry
    _save(cache_path, cache)
    return K.cmp_build_cfg.make(**best[0]), entry


def tune_estimate(make_estimator, candidates=None, reps: int = 3, cache_path: str | None = None,
                  signature: str | None = None):
    """Fastest estimate shape; make_estimator(cfg) must return an object with presort()
    (called once), estimate() and est / row_est tensors.  Returns (cmp_estimate_cfg, report).
    With cache_path and signature (a description of the plan's sizes), a cached choice is
    reused without timing."""
    cache = _load(cache_path) if signature else {}
    if signature and signature in cache:
        return K.cmp_estimate_cfg.make(**cache[signature]["cfg"]), cache[signature]
    report, ref, best = [], None, None
    for cand in candidates or ESTIMATE_CANDIDATES:
        cfg = K.cmp_estimate_cfg.make(**cand)
        est = make_estimator(cfg)
        if ref is None:
            est.presort()
        ms = _time(est.estimate, reps)
        out = (est.est.clone(), est.row_est.clone())
        if ref is None:
            ref = out
        elif not (torch.equal(ref[0].nan_to_num(-1.0), out[0].nan_to_num(-1.0)) and torch.equal(ref[1], out[1])):
            raise RuntimeError(f"launch shape {cand} changed the estimates")
        report.append({"cfg": cand, "ms": ms})
        if best is None or ms < best[1]:
            best = (cand, ms)
        del est
    entry = {"cfg": best[0], "ms": best[1], "tried": report}
    if signature:
        entry["signature"] = signature
        cache[signature] = entry
        _save(cache_path, cache)
    return K.cmp_estimate_cfg.make(**best[0]), entry
