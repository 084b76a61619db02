"""Key aggregation of the batched build (each key column's survivors counted per distinct
key, then every distinct key hashed once per (sketch, row) with its count): counters and
survivor counts must equal the per-tuple build and the oracle bit for bit, in every
launch shape, for negative and int64 keys, predicates, key ranges too wide for the count
array (run-time fallback to the per-row path), empty and fully filtered tables, key
columns shared by several sketches or also filtered on, and plan replays."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

ON = dict(aggregate=1)
SHAPES = [
    dict(),
    dict(mode=1, pairs_per_slab=3, threads=256, tile_rows=512),
    dict(mode=2, threads=1024, tile_rows=4096),
    dict(mode=1, threads=512, tile_rows=2048, ctas_per_sm=1),
]


def _oracle(orc, wl, hp):
    return [orc.build_sketch(t, hp, wl.d, wl.w) for t in wl.tables]


def _build(wl, cfg):
    dw = P.DeviceWorkload(wl)
    for t in dw.tables:
        t.counters.fill_(77)  # stale contents must be overwritten
    dw.survivors.fill_(-3)
    dw.build_batched(cfg)
    torch.cuda.synchronize()
    dw.check_status()
    return dw


def _same(dw, ref):
    surv = dw.survivors.cpu().numpy()
    for i, (t, (c, n)) in enumerate(zip(dw.tables, ref)):
        assert int(surv[i]) == n, (t.name, int(surv[i]), n)
        if t.k:
            got = t.counters.cpu().numpy()
            assert np.array_equal(got, c), (t.name, np.argwhere(got != c)[:5])


def _workload(seed, w=512, d=5):
    """Tables of every kind the aggregation must handle, one edge per sketch."""
    rng = np.random.default_rng(seed)
    n = 40_000
    tabs, eu, ev = [], [], []

    def edge():
        eu.append(0)
        ev.append(0)
        return len(eu) - 1

    # Zipf foreign keys (many duplicates), two sketches on one column, one on another,
    # the second key column also filtered on
    k1 = G.zipf_keys(rng, n, 3000, 1.1)
    k2 = G.zipf_keys(rng, n, 500, 0.8)
    tabs.append(G.Table("fk", [k1, k2], [G.Pred(1, G.RANGE, 10, 400)], [0, 0, 1], [edge(), edge(), edge()]))
    # negative int32 keys around zero, an EQ predicate on another column
    k3 = (G.zipf_keys(rng, n, 2000, 1.0) - 1000).astype(np.int32)
    c3 = rng.integers(0, 4, n).astype(np.int32)
    tabs.append(G.Table("neg", [k3, c3], [G.Pred(1, G.EQ, 2)], [0], [edge()]))
    # int64 keys at large offsets with a narrow range, and a primary key column
    k4 = (G.zipf_keys(rng, n, 5000, 1.2).astype(np.int64) + (1 << 40))
    pk = rng.permutation(n).astype(np.int64) - (1 << 62)
    tabs.append(G.Table("i64", [k4, pk], [], [0, 1], [edge(), edge()]))
    # key range wider than the table's row count: the count array is too small at run time
    wide = (rng.integers(0, 4, n).astype(np.int64) * (1 << 33)).astype(np.int64)
    tabs.append(G.Table("wide", [wide], [], [0], [edge()]))
    # every row filtered out; and an empty table
    k6 = G.zipf_keys(rng, n, 100, 1.0)
    tabs.append(G.Table("none", [k6, k6.copy()], [G.Pred(1, G.RANGE, 500, 600)], [0], [edge()]))
    tabs.append(G.Table("empty", [np.zeros(0, np.int32)], [], [0], [edge()]))
    # a single distinct key (count = survivors of the whole table)
    tabs.append(G.Table("one", [np.full(n, -7, np.int32)], [], [0, 0], [edge(), edge()]))
    return G.Workload("agg", tabs, eu, ev, d, w, 4242 + seed, seed)


@pytest.mark.parametrize("si", range(len(SHAPES)))
def test_aggregated_build_matches_oracle_and_per_row(orc, si):
    wl = _workload(si)
    ref = _oracle(orc, wl, P.DeviceWorkload(wl).hash_u64)
    on = _build(wl, K.cmp_build_cfg.make(**SHAPES[si], **ON))
    _same(on, ref)
    off = _build(wl, K.cmp_build_cfg.make(**SHAPES[si], aggregate=0))
    _same(off, ref)
    on.build_batched()  # replay: the count arrays are cleared by the plan itself
    torch.cuda.synchronize()
    _same(on, ref)


@pytest.mark.parametrize("w", [1, 7, 4096])
def test_aggregated_build_odd_widths(orc, w):
    wl = _workload(10 + w, w=w, d=3)
    _same(_build(wl, K.cmp_build_cfg.make(**ON)), _oracle(orc, wl, P.DeviceWorkload(wl).hash_u64))


def test_auto_aggregation_five_table(orc):
    """The benchmark's tables at 5% scale: F1 (1.8M rows) and F2 (225k) are above and
    below the automatic threshold of 2^18 rows."""
    wl = G.five_table(scale=0.05, w=4096)
    auto = _build(wl, None)
    off = _build(wl, K.cmp_build_cfg.make(aggregate=0))
    for a, b in zip(auto.tables, off.tables):
        assert torch.equal(a.counters, b.counters)
    assert torch.equal(auto.survivors, off.survivors)
    ref = orc.build_sketch(wl.tables[0], auto.hash_u64, wl.d, wl.w)
    assert np.array_equal(auto.tables[0].counters.cpu().numpy(), ref[0])
    assert int(auto.survivors[0].item()) == ref[1]


def test_graph_batch_aggregated_equals_per_table(orc):
    graphs = G.graph_batch(8, n_lo=3, n_hi=6, rows_lo=20_000, rows_hi=400_000, d=5, w=256, seed=7)
    gb = P.GraphBatch(graphs)
    gb.build_batched(K.cmp_build_cfg.make(**ON))
    torch.cuda.synchronize()
    gb.dw.check_status()
    ref = [t.counters.clone() for t in gb.dw.tables]
    surv = gb.dw.survivors.clone()
    gb.build_per_table()
    torch.cuda.synchronize()
    for a, t in zip(ref, gb.dw.tables):
        assert torch.equal(a, t.counters)
    assert torch.equal(surv, gb.dw.survivors)
