"""Trains the learned combiner on the GPU at the learned-combiner configuration's full size
and writes its checkpoint (paper_2102_02440_gb300/checkpoints/combiner_d{d}.bin, read by
Combiner.for_sketches) with a JSON summary beside it.

Data: n_pairs independent two-table joins drawn on the device (rows log-uniform in [1e4,
1e7] per table, key domain log-uniform in [1e3, 1e6] per pair, Zipf exponent uniform in
[0.5, 1.5] per table, own permutation of the domain per table; datagen.join_pairs_device),
in batches; every pair labelled with its exact join size by the oracle's histogram dot
product (host threads; the C call releases the interpreter lock).  Sketches: d rows, w
buckets, one hash family (seed 0xC0FFEE + 3) for every batch; features as
cmp_mlp_features (sorted, median-centred log row estimates and log self-join sizes).

Split by pair index 80/10/10.  The network (hidden 64, skip connection from the median row
feature, zero-initialised output so that it starts as the median) is trained full-batch
with the library's forward/backward/Adam kernels (Huber loss in log space), keeping the
parameters with the best validation mean log q-error.  Two combination rules are compared
on the validation split: the network everywhere, and the network only where the median is
below one tuple; the better (lower median q-error, then lower mean log q-error) is stored
as the checkpoint's rule.  Test-split q-errors of the network, the chosen rule and the
plain median are recorded in the summary.

Usage (on a GPU): python tests/train_combiner.py [--pairs 100000] [--d 11] [--w 4096]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SEED = 20210208
HASH_SEED = 0xC0FFEE + 3
BATCH = 250          # pairs drawn per device generator call
NH = 64
ROWS = (10_000, 10_000_000)
DOMS = (1_000, 1_000_000)


def qerr(est, exact):
    a = np.maximum(np.asarray(est, np.float64), 1.0)
    b = np.maximum(np.asarray(exact, np.float64), 1.0)
    return np.maximum(a / b, b / a)


def batch_seed(b: int) -> int:
    return SEED + 7919 * b


def pair_batch(b: int, d: int, w: int, orc, pool, device="cuda"):
    """Pairs [b BATCH, (b + 1) BATCH): features [BATCH][d + 2], plain medians, exact sizes."""
    import torch

    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    keys, off, meta = G.join_pairs_device(BATCH, ROWS[0], ROWS[1], dom_lo=DOMS[0], dom_hi=DOMS[1],
                                          seed=batch_seed(b), device=device)
    host = keys.cpu().numpy()
    dom = meta["domain"]
    labels = list(pool.map(lambda i: orc.join2_dense(host[off[2 * i]:off[2 * i + 1]],
                                                      host[off[2 * i + 1]:off[2 * i + 2]], int(dom[2 * i])),
                           range(BATCH)))
    pb = P.PairBatch(None, d=d, w=w, hash_seed=HASH_SEED, device_keys=keys, offsets=off, device=device)
    pb.build()
    pb.prepare_estimate()
    pb.estimate()
    feat = pb.features()
    torch.cuda.synchronize()
    pb.dw.check_status()
    out = (feat.cpu().numpy().copy(), pb.est.cpu().numpy().copy(), np.array(labels, np.float64),
           int(off[-1]))
    del pb, keys
    torch.cuda.empty_cache()
    return out


def dataset(n_pairs: int, d: int, w: int, first_batch: int = 0, log=print):
    from oracle import oracle as orc
    orc.build()
    feats, meds, exact, rows = [], [], [], 0
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as pool:
        for b in range(first_batch, first_batch + n_pairs // BATCH):
            f, m, e, r = pair_batch(b, d, w, orc, pool)
            feats.append(f)
            meds.append(m)
            exact.append(e)
            rows += r
            if (b - first_batch) % 40 == 0:
                log(f"batch {b}: {rows} rows so far, {time.time() - t0:.0f} s")
    return np.concatenate(feats), np.concatenate(meds), np.concatenate(exact), rows


def main():
    import torch

    from paper_2102_02440_gb300 import pipeline as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=100_000)
    ap.add_argument("--d", type=int, default=11)
    ap.add_argument("--w", type=int, default=4096)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--out", default=P.CHECKPOINT_DIR)
    a = ap.parse_args()
    n = a.pairs - a.pairs % (10 * BATCH)
    t0 = time.time()
    feat, med, exact, rows = dataset(n, a.d, a.w)
    gen_s = time.time() - t0
    i_tr, i_va = int(0.8 * n), int(0.9 * n)
    dev = "cuda"
    x = torch.from_numpy(feat).to(dev)
    y = torch.from_numpy((np.log1p(exact) / 32.0).astype(np.float32)).to(dev)
    m_dev = torch.from_numpy(med).to(dev)
    comb = P.Combiner(a.d + 2, NH, seed=1, device=dev, skip=a.d // 2, init_scale=0.0)
    x_tr, y_tr = x[:i_tr].contiguous(), y[:i_tr].contiguous()

    def predict(lo, hi, rule):
        yy = comb.infer(x[lo:hi].contiguous())
        out = torch.empty(hi - lo, dtype=torch.float64, device=dev)
        from paper_2102_02440_gb300 import compass as K
        K.cmp_mlp_combine_ex(m_dev[lo:hi].contiguous().data_ptr(), yy.data_ptr(), 0, hi - lo, rule, out.data_ptr(),
                             K.stream_handle())
        return out.cpu().numpy()

    rules = {"network everywhere": float("inf"), "network below one tuple": 1.0}
    best = {r: (np.inf, None) for r in rules}
    for it in range(1, a.iters + 1):
        comb.train_step(x_tr, y_tr, lr=3e-4, huber_delta=0.001)
        if it % 200 == 0:
            for r, thr in rules.items():
                q = float(np.mean(np.log(qerr(predict(i_tr, i_va, thr), exact[i_tr:i_va]))))
                if q < best[r][0]:
                    best[r] = (q, comb.params.clone(), comb.m.clone(), comb.v.clone(), it)
    val = {}
    for r, thr in rules.items():
        comb.params.copy_(best[r][1])
        qv = qerr(predict(i_tr, i_va, thr), exact[i_tr:i_va])
        val[r] = (float(np.median(qv)), float(np.mean(np.log(qv))))
    chosen = min(rules, key=lambda r: val[r])
    q_mean, p, mm, vv, it_best = best[chosen]
    comb.params.copy_(p)
    comb.m.copy_(mm)
    comb.v.copy_(vv)
    comb.step = it_best
    qt = qerr(predict(i_va, n, rules[chosen]), exact[i_va:])
    qm = qerr(med[i_va:], exact[i_va:])

    def stats(q):
        return {"median": float(np.median(q)), "p90": float(np.percentile(q, 90)), "p99": float(np.percentile(q, 99))}

    summary = {"pairs": n, "rows": rows, "d": a.d, "w": a.w, "hash_seed": HASH_SEED, "seed": SEED, "batch": BATCH,
               "split": [i_tr, i_va - i_tr, n - i_va], "rule": chosen, "use_median_at": rules[chosen],
               "best_iteration": it_best, "validation": {r: {"median_q": v[0], "mean_log_q": v[1]} for r, v in val.items()},
               "test_q_error": {"combined": stats(qt), "plain_median": stats(qm)},
               "test_pairs_median_below_one": int((med[i_va:] < 1.0).sum()), "generation_s": gen_s,
               "labels": "oracle join2_dense (histogram dot product) on every pair"}
    os.makedirs(a.out, exist_ok=True)
    path = os.path.join(a.out, f"combiner_d{a.d}.bin")
    comb.save(path, {k: summary[k] for k in ("pairs", "w", "rule", "use_median_at", "test_q_error", "hash_seed")},
              seed=1)
    with open(os.path.join(a.out, f"combiner_d{a.d}.json"), "w") as f:
        json.dump(summary, f, indent=1, sort_keys=True)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
