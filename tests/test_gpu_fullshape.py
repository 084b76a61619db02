"""Oracle parity of the five-table workload at the benchmark's own shape: full scale (47M
rows), d = 11, w = 4096, built by the batched build with the tables' declarations (unique
dimension keys, foreign-key domains) and estimated by the plan the benchmark replays.
One sampled sketch row: every sketch's counters on that row are recomputed by the oracle's
hash from the surviving keys, and the exact row estimates of all 19 connected sub-plans
(the 15 trees on the generic path with its int64 -> int128 recompute, the 4 triangle
sub-plans on the triangle path) are compared with the oracle's on those d = 1 slices.  The
same plan with cached subtree messages, and cmp_estimate_noalloc (whose 44 triangle rows
exceed its array and run in waves), must give the same integers."""
import threading

import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROW = 5  # the sampled sketch row


def _keep(t):
    m = np.ones(t.n_rows, bool)
    for q in t.preds:
        v = t.cols[q.col].astype(np.int64)
        if q.op == G.RANGE:
            m &= (q.lo <= v) & (v < q.hi)
        elif q.op == G.EQ:
            m &= v == q.lo
        else:
            inb = (v >= 0) & (v < q.nbits)
            bits = np.zeros(t.n_rows, bool)
            vv = v[inb]
            bits[inb] = ((q.bitmap[vv >> 5] >> (vv & 31).astype(np.uint32)) & 1) == 1
            m &= bits
    return m


@pytest.fixture(scope="module")
def bench_shape():
    wl = G.five_table(scale=1.0, w=4096)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    dw.check_status()
    return wl, dw, masks, est


def test_sampled_row_counters_and_survivors(orc, bench_shape):
    wl, dw, _, _ = bench_shape
    surv = dw.survivors.cpu().numpy()
    for ti, t in enumerate(wl.tables):
        keep = _keep(t)
        assert int(surv[ti]) == int(keep.sum()), t.name
        for s in range(len(t.key_col)):
            keys = t.cols[t.key_col[s]][keep].astype(np.int64)
            b, sg = orc.hash_eval(dw.hash_u64[t.edge_id[s], ROW], wl.w, keys)
            want = np.bincount(b, weights=sg, minlength=wl.w).astype(np.int64)
            got = dw.tables[ti].counters[s, ROW].cpu().numpy().astype(np.int64)
            assert np.array_equal(got, want), (t.name, s)


def test_all_subplans_on_the_sampled_row_match_oracle(orc, bench_shape):
    wl, dw, masks, est = bench_shape
    sk = [tuple(dw.sketch(e, end)[ROW:ROW + 1].cpu().numpy() for end in range(2)) for e in range(wl.n_edges)]
    surv = dw.survivors.cpu().numpy()
    rows = est.row_values()
    assert len(masks) == 19
    refs = [None] * len(masks)

    def work(qs):
        for q in qs:
            refs[q] = orc.estimate(wl.edge_u, wl.edge_v, sk, surv, 1, wl.w, int(masks[q]))

    # the oracle's C calls release the interpreter lock: the four triangle sub-plans (minutes
    # each at w = 4096) run side by side
    cyc = [q for q, m in enumerate(masks) if (m & 0b111) == 0b111]
    assert len(cyc) == 4
    groups = [[q] for q in cyc] + [[q for q in range(len(masks)) if q not in cyc]]
    threads = [threading.Thread(target=work, args=(g,)) for g in groups]
    for x in threads:
        x.start()
    for x in threads:
        x.join()
    for q, m in enumerate(masks):
        if bin(m).count("1") == 1:
            assert rows[q][ROW] == int(surv[int(m).bit_length() - 1])
        assert rows[q][ROW] == refs[q].rows[0], (bin(m), rows[q][ROW], refs[q].rows[0])


def test_cached_messages_and_noalloc_equal_the_plan(bench_shape):
    wl, dw, masks, est = bench_shape
    cached = P.DeviceEstimator(dw, masks, cfg=K.cmp_estimate_cfg.make(flags=K.CMP_EST_CACHE_MESSAGES))
    cached.estimate()
    torch.cuda.synchronize()
    dw.check_status()
    assert torch.equal(cached.row_est, est.row_est) and torch.equal(cached.est, est.est)
    assert est.ws.numel() > K.CMP_NOALLOC_WS_BYTES   # the triangle rows cannot all fit: waves
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        out = torch.full_like(est.est, float("nan"))
        rows = torch.full_like(est.row_est, -1)
        K.cmp_estimate_noalloc(est.plan_host.ctypes.data, est.plan_dev.data_ptr(), out.data_ptr(), rows.data_ptr(),
                               status.data_ptr(), K.stream_handle())
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out, est.est) and torch.equal(rows, est.row_est)
