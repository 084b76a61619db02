"""GPU parity of the estimate with cached subtree messages (CMP_EST_CACHE_MESSAGES: an
(n+1)-table sub-plan extends the cached message of an n-table subtree, Sec. 4.2 / Sec. 5):
exact int128 row estimates and identical doubles against the oracle and bit for bit against
the plan without the cache, on chains, trees, stars, cycles with tails, many graphs in one
plan, the five-table workload and rows beyond int128."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

CACHE = K.cmp_estimate_cfg.make(flags=K.CMP_EST_CACHE_MESSAGES)


def _oracle_check(orc, dw, est, masks):
    wl = dw.wl
    built = [orc.build_sketch(t, dw.hash_u64, wl.d, wl.w) for t in wl.tables]
    sk = [tuple(built[wl.sketch_of(e, end)[0]][0][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(dw.n_edges)]
    surv = np.array([n for _, n in built], np.int64)
    rows = est.row_values()
    e_gpu = est.est.cpu().numpy()
    for q, m in enumerate(masks):
        ref = orc.estimate(wl.edge_u, wl.edge_v, sk, surv, wl.d, wl.w, int(m))
        assert rows[q] == ref.rows, (q, bin(m))
        assert e_gpu[q] == ref.est, (q, bin(m), e_gpu[q], ref.est)


def _run(dw, masks, cfg, graph_of=None):
    est = P.DeviceEstimator(dw, masks, graph_of, cfg=cfg)
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    return est


def _same(a, b):
    assert torch.equal(a.row_est, b.row_est)
    assert torch.equal(torch.nan_to_num(a.est, nan=-7.0), torch.nan_to_num(b.est, nan=-7.0))


GRAPHS = {
    "chain9": ([0, 1, 2, 3, 4, 5, 6, 7], [1, 2, 3, 4, 5, 6, 7, 8], 9),
    "chain9_shuffled": ([4, 7, 0, 2, 8, 1, 5, 6], [7, 0, 2, 8, 1, 5, 6, 3], 9),
    "tree": ([0, 0, 1, 1, 2, 3, 3], [1, 2, 3, 4, 5, 6, 7], 8),
    "star_centre3": ([3, 3, 3, 3, 3], [0, 1, 2, 4, 5], 6),
    "caterpillar": ([1, 2, 3, 1, 2, 3, 4], [2, 3, 4, 0, 5, 6, 7], 8),
    "cycle5+tails": ([0, 1, 2, 3, 4, 2, 6], [1, 2, 3, 4, 0, 5, 2], 7),
}


def _workload(rng, eu, ev, nt, d, w, seed):
    tabs = []
    for t in range(nt):
        n = int(rng.integers(50, 2500))
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if eu[e] == t or ev[e] == t:
                cols.append(G.zipf_keys(rng, n, 200, float(rng.uniform(0.6, 1.4))))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    return G.Workload("g", tabs, eu, ev, d, w, seed, 0)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("w", [16, 257])
def test_cached_messages_match_oracle_and_plain_plan(orc, name, w):
    eu, ev, nt = GRAPHS[name]
    rng = np.random.default_rng(sum(map(ord, name)) + w)
    dw = P.DeviceWorkload(_workload(rng, eu, ev, nt, 3, w, 11 + w))
    dw.build()
    masks = G.connected_subplans(nt, eu, ev)
    plain = _run(dw, masks, None)
    cached = _run(dw, masks, CACHE)
    dw.check_status()
    st = K.cmp_estimate_plan_stats(cached.plan_host.ctypes.data)
    if name.startswith("chain") or name in ("tree", "caterpillar"):
        assert st.n_jobs > 0
    _same(cached, plain)
    _oracle_check(orc, dw, cached, masks)


def test_many_graphs_one_cached_plan_and_replay():
    rng = np.random.default_rng(21)
    graphs = []
    for gi in range(3):
        eu, ev, nt = GRAPHS[["chain9", "tree", "caterpillar"][gi]]
        graphs.append(_workload(rng, eu, ev, nt, 5, 64, 100 + gi))
    gb = P.GraphBatch(graphs)
    gb.build_batched()
    gb.presort()
    sg, sm = [], []
    for gi, g in enumerate(graphs):
        ms = G.connected_subplans(len(g.tables), g.edge_u, g.edge_v)
        sg += [gi] * len(ms)
        sm += ms
    pc = gb.plan(sg, sm, CACHE)
    pp = gb.plan(sg, sm)
    pc.run()
    pp.run()
    first = pc.est.clone()
    pc.run()
    torch.cuda.synchronize()
    assert torch.equal(pc.est, first) and torch.equal(pc.est, pp.est) and torch.equal(pc.row_est, pp.row_est)
    assert int(gb.dw.status.item()) == 0


def test_five_table_workload_cached(orc):
    wl = G.five_table(scale=0.005, w=256)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    cached = _run(dw, masks, CACHE)
    plain = _run(dw, masks, None)
    dw.check_status()
    _same(cached, plain)
    _oracle_check(orc, dw, cached, masks)


def test_rows_beyond_int128_are_flagged_through_the_cache():
    """A 16-table chain of one-row tables with counters at 2^31 - 1 in sketch row 0 and small
    values in row 1, with the exact tier off: the long sub-plans leave int128 in row 0 (NaN
    with CMP_EOVERFLOW), including those that read an overflowed cached message; both plans
    agree on every estimate, and on every exact row of the sub-plans that stay in range."""
    n = 16
    eu, ev = list(range(n - 1)), list(range(1, n))
    rng = np.random.default_rng(3)
    tabs = []
    for t in range(n):
        cols, kc, ei = [], [], []
        for e in range(n - 1):
            if eu[e] == t or ev[e] == t:
                cols.append(np.array([int(rng.integers(0, 100))], np.int32))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    dw = P.DeviceWorkload(G.Workload("raw", tabs, eu, ev, 3, 32, 1, 0))
    dw.survivors.fill_(1)
    for t in dw.tables:
        a = rng.integers(-20, 21, size=tuple(t.counters.shape)).astype(np.int32)
        a[:, 0, :] = 2 ** 31 - 1
        t.counters.copy_(torch.from_numpy(a))
    masks = G.connected_subplans(n, eu, ev)
    dw.status.zero_()
    no_wide = K.CMP_EST_NO_WIDE      # the int128 path's own flagging (the exact tier: test_gpu_wide)
    cached = _run(dw, masks, K.cmp_estimate_cfg.make(flags=K.CMP_EST_CACHE_MESSAGES | no_wide))
    st_c = int(dw.status.item())
    dw.status.zero_()
    plain = _run(dw, masks, K.cmp_estimate_cfg.make(flags=no_wide))
    st_p = int(dw.status.item())
    assert st_c == st_p == K.CMP_EOVERFLOW
    nan_c = torch.isnan(cached.est)
    assert torch.equal(nan_c, torch.isnan(plain.est)) and 0 < int(nan_c.sum()) < len(masks)
    ok = ~nan_c
    assert torch.equal(cached.est[ok], plain.est[ok]) and torch.equal(cached.row_est[ok], plain.row_est[ok])
    # the longest chains are the ones out of range
    sizes = np.array([bin(int(m)).count("1") for m in masks])
    assert sizes[nan_c.cpu().numpy()].min() > sizes[ok.cpu().numpy()].min()
