"""GPU parity of the star lattice (CMP_EST_STAR_LATTICE: every leaf subset of a star family
from one table of cached products, Sec. 5): exact int128 row estimates and identical doubles
against the generic contraction and the oracle, for 3 to 16 leaf edges (B side only, A side
with one and with several blocks), ragged widths, mixed plans with chains and cycles, the
message cache at the same time, and rows beyond int128."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

STAR = K.cmp_estimate_cfg.make(flags=K.CMP_EST_STAR_LATTICE)


def _star_workload(rng, n_leaves, d, w, rows_lo, rows_hi, seed, domain=200):
    eu, ev = [0] * n_leaves, list(range(1, n_leaves + 1))
    tabs = []
    for t in range(n_leaves + 1):
        n = int(rng.integers(rows_lo, rows_hi + 1))
        cols, kc, ei = [], [], []
        for e in range(n_leaves):
            if eu[e] == t or ev[e] == t:
                cols.append(G.zipf_keys(rng, n, domain, float(rng.uniform(0.6, 1.4))))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    return G.Workload(f"star{n_leaves}", tabs, eu, ev, d, w, seed, 0)


def _run(dw, masks, cfg):
    dw.status.zero_()
    est = P.DeviceEstimator(dw, masks, cfg=cfg)
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    return est, int(dw.status.item())


def _oracle(orc, dw):
    wl = dw.wl
    built = [orc.build_sketch(t, dw.hash_u64, wl.d, wl.w) for t in wl.tables]
    sk = [tuple(built[wl.sketch_of(e, end)[0]][0][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(dw.n_edges)]
    return sk, np.array([n for _, n in built], np.int64)


@pytest.mark.parametrize("n_leaves,w,sample", [(3, 16, None), (5, 257, None), (8, 1024, None), (9, 100, None),
                                               (12, 64, 300), (14, 33, 200), (16, 16, 150)])
def test_star_lattice_matches_generic_and_oracle(orc, n_leaves, w, sample):
    rng = np.random.default_rng(100 * n_leaves + w)
    # small tables for many leaves keep every row of every subset inside int128
    hi = 3000 if n_leaves <= 8 else 40
    dw = P.DeviceWorkload(_star_workload(rng, n_leaves, 3, w, 5, hi, 7 + w))
    dw.build()
    masks = G.connected_subplans(n_leaves + 1, dw.wl.edge_u, dw.wl.edge_v)
    lat, st1 = _run(dw, masks, STAR)
    gen, st2 = _run(dw, masks, None)
    info = K.cmp_estimate_plan_stats(lat.plan_host.ctypes.data)
    assert info.n_star == 1 and info.n_star_sub == 2 ** n_leaves - 1
    assert st1 == st2 == 0
    assert torch.equal(lat.row_est, gen.row_est) and torch.equal(lat.est, gen.est)
    sk, surv = _oracle(orc, dw)
    qs = range(len(masks)) if sample is None else np.random.default_rng(1).choice(len(masks), sample, replace=False)
    rows = lat.row_values()
    e = lat.est.cpu().numpy()
    for q in qs:
        ref = orc.estimate(dw.wl.edge_u, dw.wl.edge_v, sk, surv, 3, w, int(masks[q]))
        assert rows[q] == ref.rows and e[q] == ref.est, (q, bin(int(masks[q])))


def test_star_lattice_in_a_mixed_plan_with_the_cache():
    """Stars, chains and cycles of several graphs in one plan, with and without both flags:
    every estimate identical."""
    graphs = G.graph_batch(12, 4, 7, rows_lo=50, rows_hi=2000, d=5, w=128, seed=77)
    gb = P.GraphBatch(graphs)
    gb.build_batched()
    gb.presort()
    sg, sm = [], []
    for gi, g in enumerate(graphs):
        ms = G.connected_subplans(len(g.tables), g.edge_u, g.edge_v)
        sg += [gi] * len(ms)
        sm += ms
    both = K.cmp_estimate_cfg.make(flags=K.CMP_EST_STAR_LATTICE | K.CMP_EST_CACHE_MESSAGES)
    plans = [gb.plan(sg, sm), gb.plan(sg, sm, STAR), gb.plan(sg, sm, both)]
    assert K.cmp_estimate_plan_stats(plans[1].host.ctypes.data).n_star >= 1
    for p in plans:
        p.run()
    plans[2].run()   # replay
    torch.cuda.synchronize()
    assert int(gb.dw.status.item()) == 0 and not bool(torch.isnan(plans[0].est).any())
    for p in plans[1:]:
        assert torch.equal(p.est, plans[0].est) and torch.equal(p.row_est, plans[0].row_est)


def test_star_rows_beyond_int128():
    """One-row leaf tables of a 10-leaf star, counters at 2^31 - 1 in sketch row 0 (every
    product is huge) and small elsewhere, with the exact tier off: the large subsets leave
    int128 in row 0 and are NaN with CMP_EOVERFLOW on both evaluations; the others are
    identical."""
    n = 10
    rng = np.random.default_rng(4)
    eu, ev = [0] * n, list(range(1, n + 1))
    tabs = []
    for t in range(n + 1):
        cols, kc, ei = [], [], []
        for e in range(n):
            if eu[e] == t or ev[e] == t:
                cols.append(np.array([int(rng.integers(0, 100))], np.int32))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    dw = P.DeviceWorkload(G.Workload("raw", tabs, eu, ev, 3, 32, 1, 0))
    dw.survivors.fill_(1)
    for t in dw.tables:
        a = rng.integers(1, 21, size=tuple(t.counters.shape)).astype(np.int32)
        a[:, 0, :] = 2 ** 31 - 1
        t.counters.copy_(torch.from_numpy(a))
    masks = G.connected_subplans(n + 1, eu, ev)
    no_wide = K.CMP_EST_NO_WIDE      # the int128 path's own flagging (the exact tier: test_gpu_wide)
    lat, st1 = _run(dw, masks, K.cmp_estimate_cfg.make(flags=K.CMP_EST_STAR_LATTICE | no_wide))
    gen, st2 = _run(dw, masks, K.cmp_estimate_cfg.make(flags=no_wide))
    assert st1 == st2 == K.CMP_EOVERFLOW
    nan = torch.isnan(lat.est)
    assert torch.equal(nan, torch.isnan(gen.est)) and 0 < int(nan.sum()) < len(masks)
    ok = ~nan
    assert torch.equal(lat.est[ok], gen.est[ok]) and torch.equal(lat.row_est[ok], gen.row_est[ok])
