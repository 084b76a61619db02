"""Batched enumeration workload (many chains, stars and cycles): one build launch for
every table of every graph, one estimate plan for every connected sub-plan of every
graph, and the same work captured in a CUDA graph and replayed.  Results must equal
per-table builds, per-graph plans and, on samples, the oracle."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    graphs = G.graph_batch(24, n_lo=3, n_hi=8, rows_lo=500, rows_hi=30_000, d=5, w=256, seed=31)
    gb = P.GraphBatch(graphs)
    gb.build_batched()
    gb.presort()
    sub_graph, sub_mask = [], []
    for gi, g in enumerate(graphs):
        ms = G.connected_subplans(len(g.tables), g.edge_u, g.edge_v)
        sub_graph += [gi] * len(ms)
        sub_mask += ms
    plan = gb.plan(sub_graph, sub_mask)
    plan.run()
    torch.cuda.synchronize()
    gb.dw.check_status()
    return graphs, gb, np.array(sub_graph), np.array(sub_mask, np.uint64), plan


def test_batched_build_equals_per_table_build(batch):
    graphs, gb, *_ = batch
    ref = [t.counters.clone() for t in gb.dw.tables]
    surv = gb.dw.survivors.clone()
    gb.build_per_table()
    torch.cuda.synchronize()
    for a, t in zip(ref, gb.dw.tables):
        assert torch.equal(a, t.counters)
    assert torch.equal(surv, gb.dw.survivors)


def test_sampled_tables_match_oracle(orc, batch):
    graphs, gb, *_ = batch
    rng = np.random.default_rng(0)
    for ti in rng.choice(len(gb.wl.tables), 12, replace=False):
        t = gb.wl.tables[ti]
        c, n = orc.build_sketch(t, gb.dw.hash_u64, gb.d, gb.w)
        assert int(gb.dw.survivors[ti].item()) == n
        assert np.array_equal(gb.dw.tables[ti].counters.cpu().numpy()[:len(t.key_col)], c)


def test_one_plan_equals_per_graph_plans_and_oracle(orc, batch):
    graphs, gb, sg, sm, plan = batch
    est_all = plan.est.cpu().numpy()
    rows_all = plan.row_est.cpu().numpy()
    rng = np.random.default_rng(1)
    for gi in rng.choice(len(graphs), 6, replace=False):
        idx = np.nonzero(sg == gi)[0]
        p1 = gb.plan(sg[idx], sm[idx])
        p1.run()
        torch.cuda.synchronize()
        assert np.array_equal(p1.est.cpu().numpy(), est_all[idx])
        assert np.array_equal(p1.row_est.cpu().numpy(), rows_all[idx])
        g = graphs[gi]
        toff, eoff = gb.table_off[gi], gb.edge_off[gi]
        # the oracle's own build of the graph's tables (the batch's hash parameters)
        built = [orc.build_sketch(gb.wl.tables[toff + t], gb.dw.hash_u64, gb.d, gb.w) for t in range(len(g.tables))]
        sk = []
        for e in range(g.n_edges):
            ends = [gb.wl.sketch_of(e + eoff, end) for end in range(2)]
            sk.append(tuple(built[t - toff][0][si] for t, si in ends))
        surv = np.array([n for _, n in built], np.int64)
        for q in rng.choice(idx, min(6, idx.size), replace=False):
            ref = orc.estimate(g.edge_u, g.edge_v, sk, surv, gb.d, gb.w, int(sm[q]))
            r = rows_all[q]
            got = [int(np.uint64(r[i, 0])) + (int(r[i, 1]) << 64) for i in range(gb.d)]
            assert got == ref.rows and est_all[q] == ref.est


def test_cuda_graph_capture_and_replay(batch):
    graphs, gb, sg, sm, plan = batch
    ref_c = [t.counters.clone() for t in gb.dw.tables]
    ref_e = plan.est.clone()
    for t in gb.dw.tables:
        t.counters.fill_(7)
    plan.est.fill_(-1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gb.build_batched(stream=s)           # warm the launch attributes outside capture
        gb.presort(stream=s)
        plan.run(stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            gb.build_batched(stream=s)
            gb.presort(stream=s)
            plan.run(stream=s)
    for t in gb.dw.tables:
        t.counters.fill_(-3)
    plan.est.fill_(0)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for a, t in zip(ref_c, gb.dw.tables):
        assert torch.equal(a, t.counters)
    assert torch.equal(ref_e, plan.est)


def test_upload_from_host_then_build_equals_resident_build():
    """DeviceWorkload.upload (host columns copied on several streams, the caller's stream
    waiting for all of them) followed by the batched build gives the same counters and
    survivor counts as the build over the columns the workload uploaded itself; the columns
    are overwritten with zeros first so that a missed part would show."""
    rng = np.random.default_rng(8)
    wl = G.random_graph_workload(rng, 5, 1, 1_000, 300_000, 5000, d=3, w=512, pred_prob=0.5, hash_seed=8)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    torch.cuda.synchronize()
    ref = [t.counters.clone() for t in dw.tables]
    ref_surv = dw.survivors.clone()
    host = [[c.cpu().pin_memory() for c in t.cols] for t in dw.tables]
    for t in dw.tables:
        for c in t.cols:
            c.zero_()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for n_streams in (1, 3, 4):
            dw.upload(host, n_streams=n_streams, stream=st)
            dw.build_batched(stream=st)
            st.synchronize()
            for t, r in zip(dw.tables, ref):
                assert torch.equal(t.counters, r)
            assert torch.equal(dw.survivors, ref_surv)
