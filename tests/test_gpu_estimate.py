"""GPU parity of presort + sketch-merging estimate against the oracle: exact int128 row
estimates and identical doubles (one rounding of the same exact median), on chains,
stars, cycles, parallel edges, single tables, many graphs in one plan, and the
five-table cyclic workload."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu


def _oracle_inputs(orc, dw):
    """The oracle's own build of every table: sketches[e] = (u-side, v-side) as numpy
    [d, w], and the survivor counts.  The device build must equal it (checked here too)."""
    wl = dw.wl
    built = [orc.build_sketch(t, dw.hash_u64, wl.d, wl.w) for t in wl.tables]
    for (c, n), t in zip(built, dw.tables):
        if t.k:
            assert np.array_equal(t.counters.cpu().numpy(), c)
    sk = []
    for e in range(dw.n_edges):
        sk.append(tuple(built[wl.sketch_of(e, end)[0]][0][wl.sketch_of(e, end)[1]] for end in range(2)))
    return sk, np.array([n for _, n in built], np.int64)


def _check(orc, dw, est, masks, brute=False):
    torch.cuda.synchronize()
    dw.check_status()
    sk, surv = _oracle_inputs(orc, dw)
    rows = est.row_values()
    e_gpu = est.est.cpu().numpy()
    for q, m in enumerate(masks):
        ref = orc.estimate(dw.wl.edge_u, dw.wl.edge_v, sk, surv, dw.d, dw.w, int(m), brute=brute)
        assert rows[q] == ref.rows, (q, bin(m), rows[q], ref.rows)
        assert e_gpu[q] == ref.est, (q, bin(m), e_gpu[q], ref.est)


def test_presort_orders_by_magnitude_then_bucket():
    rng = np.random.default_rng(0)
    for w in (1, 2, 5, 64, 1023, 4096, 16384, 16385, 40000, 65536):
        C = torch.from_numpy(rng.integers(-7, 8, size=(3, w)).astype(np.int32)).cuda()
        C[0, 0] = -(2 ** 31) + 1
        a = torch.empty_like(C)
        p = torch.empty_like(C)
        nb = K.cmp_presort_ws_bytes(3, w)
        ws = torch.empty(max(nb, 16), dtype=torch.uint8, device="cuda")
        K.cmp_presort(C.data_ptr(), 3, w, a.data_ptr(), p.data_ptr(), ws.data_ptr(), nb, K.stream_handle())
        torch.cuda.synchronize()
        Cn = C.cpu().numpy().astype(np.int64)
        for r in range(3):
            want = sorted(range(w), key=lambda j: (abs(Cn[r, j]), j))
            assert p[r].cpu().numpy().tolist() == want
            assert np.array_equal(a[r].cpu().numpy().view(np.uint32), np.abs(Cn[r, want]).astype(np.uint32))


GRAPHS = {
    "chain5": ([0, 1, 2, 3], [1, 2, 3, 4], 5),
    "star5": ([0, 0, 0, 0], [1, 2, 3, 4], 5),
    "triangle": ([0, 1, 0], [1, 2, 2], 3),
    "cycle4+tail": ([0, 1, 2, 3, 3], [1, 2, 3, 0, 4], 5),
    "parallel": ([0, 0, 1], [1, 1, 2], 3),
    "tree": ([0, 0, 1, 1, 2], [1, 2, 3, 4, 5], 6),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("w", [3, 16, 257])
def test_random_graphs_all_connected_subplans(orc, name, w):
    eu, ev, nt = GRAPHS[name]
    rng = np.random.default_rng(sum(map(ord, name)) + w)
    tabs = []
    for t in range(nt):
        n = int(rng.integers(50, 3000))
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if eu[e] == t or ev[e] == t:
                cols.append(G.zipf_keys(rng, n, 300, float(rng.uniform(0.6, 1.4))))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    wl = G.Workload(name, tabs, eu, ev, 3, w, 77 + w, 0)
    dw = P.DeviceWorkload(wl)
    dw.build()
    masks = G.connected_subplans(nt, eu, ev)
    est = P.DeviceEstimator(dw, masks)
    # the plan reads only the sorted rows of P.sorted_tables: the others' presort and cross-rank
    # buffers hold zeros (in-bounds, wrong) and must not change a row
    for buf in (dw.abs_all, dw.perm_all, dw.ranks_all):
        buf.zero_()
    assert len(est.sorted_tables()) < nt or name in ("triangle", "parallel", "cycle4+tail")
    est.presort()
    est.estimate()
    _check(orc, dw, est, masks, brute=(w == 3 and len(eu) <= 5))
    pairs = [m for m in masks if bin(m).count("1") <= 2]  # roots of the two-table sub-plans only
    est2 = P.DeviceEstimator(dw, pairs)
    for buf in (dw.abs_all, dw.perm_all, dw.ranks_all):
        buf.zero_()
    est2.presort()
    est2.estimate()
    _check(orc, dw, est2, pairs)


@pytest.mark.parametrize("shape", [dict(threads=256, ctas_per_sm=4), dict(threads=256, ctas_per_sm=4, cond_chunk=16),
                                   dict(threads=128, ctas_per_sm=8, cond_chunk=7), dict(threads=512, ctas_per_sm=1),
                                   dict(threads=1024, ctas_per_sm=2, cond_chunk=300)])
def test_launch_shapes_give_identical_estimates(orc, shape):
    """Every launch shape (the 1024-, 512- and 256-thread register budgets, ragged conditioning
    chunks) gives the same exact rows on cycles of 4 to 7 tables, trees and the cached
    messages, equal to the oracle."""
    rng = np.random.default_rng(31)
    wls = [G.random_graph_workload(rng, n, 1, 50, 1500, 200, d=3, w=97, pred_prob=0.3, hash_seed=n) for n in (4, 7)]
    eu, ev = [0, 1, 2, 3, 4, 5], [1, 2, 3, 4, 5, 0]
    tabs = []
    for t in range(6):
        n = int(rng.integers(50, 1500))
        cols, kc, ei = [], [], []
        for e in range(6):
            if eu[e] == t or ev[e] == t:
                cols.append(G.zipf_keys(rng, n, 200, 1.0))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"C{t}", cols, [], kc, ei))
    wls.append(G.Workload("cycle6", tabs, eu, ev, 3, 97, 5, 0))
    for wl in wls:
        dw = P.DeviceWorkload(wl)
        dw.build()
        masks = G.connected_subplans(len(wl.tables), wl.edge_u, wl.edge_v)
        ref = P.DeviceEstimator(dw, masks)
        ref.presort()
        ref.estimate()
        cfg = K.cmp_estimate_cfg.make(flags=K.CMP_EST_CACHE_MESSAGES, **shape)
        est = P.DeviceEstimator(dw, masks, cfg=cfg)
        est.presort()
        est.estimate()
        torch.cuda.synchronize()
        dw.check_status()
        assert torch.equal(est.row_est, ref.row_est) and torch.equal(est.est, ref.est)
        _check(orc, dw, est, masks)


def test_two_way_full_size_workload(orc):
    wl = G.two_way()
    dw = P.DeviceWorkload(wl)
    dw.build()
    est = P.DeviceEstimator(dw, [0b11, 0b01, 0b10])
    est.presort()
    est.estimate()
    _check(orc, dw, est, [0b11, 0b01, 0b10])


def test_many_graphs_one_plan_and_replay(orc):
    rng = np.random.default_rng(5)
    dws, masks, gof = [], [], []
    for gi in range(4):
        wl = G.random_graph_workload(rng, 5, gi % 2, 100, 4000, 500, d=5, w=64, pred_prob=0.5, hash_seed=gi)
        dw = P.DeviceWorkload(wl)
        dw.build()
        dws.append(dw)
        ms = G.connected_subplans(5, wl.edge_u, wl.edge_v)
        masks += ms
        gof += [gi] * len(ms)
    est = P.DeviceEstimator(dws, masks, gof)
    est.presort()
    est.estimate()
    first = est.est.clone()
    est.estimate()
    assert torch.equal(first, est.est)
    torch.cuda.synchronize()
    off = 0
    rows = est.row_values()
    for gi, dw in enumerate(dws):
        sk, surv = _oracle_inputs(orc, dw)
        for q in range(off, off + gof.count(gi)):
            ref = orc.estimate(dw.wl.edge_u, dw.wl.edge_v, sk, surv, 5, 64, masks[q])
            assert rows[q] == ref.rows and float(est.est[q]) == ref.est
        off += gof.count(gi)


def test_five_table_reduced_scale_all_subplans(orc):
    wl = G.five_table(scale=0.005, w=256)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    assert len(masks) == 19
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    _check(orc, dw, est, masks)


def test_rejections():
    wl = G.two_way(n_r=100, n_s=100)
    dw = P.DeviceWorkload(wl)
    dw.build()
    with pytest.raises(K.CompassError):
        P.DeviceEstimator(dw, [0b100])      # beyond n_tables
    with pytest.raises(K.CompassError):
        P.DeviceEstimator(dw, [0])
    wl2 = G.Workload("2cyc", [G.Table(f"T{t}", [np.zeros(4, np.int32)] * 4, [], [0, 1, 2, 3][:k], e)
                              for t, (k, e) in enumerate([(2, [0, 2]), (2, [0, 1]), (2, [1, 2])])],
                     [0, 1, 0], [1, 2, 2], 2, 16, 1, 0)
    dw2 = P.DeviceWorkload(wl2)
    dw2.build()
    P.DeviceEstimator(dw2, [0b111])          # one cycle: supported


def test_cross_ranks_multi_windows_at_full_width():
    """w = 65536: many 2048-position segments per row.  A sketch of widely spread magnitudes
    against one of magnitudes 0..3 (many ties): some segments' windows in the other row are
    empty, some hold most of the row (beyond the shared-memory window: the searches read the
    row in global memory).  Every rank equals the definition (np.searchsorted, ties broken
    by edge id) and the per-table kernel's."""
    rng = np.random.default_rng(21)
    d, w = 2, 65536
    C = np.stack([rng.integers(-30000, 30001, size=(d, w)), rng.integers(-3, 4, size=(d, w))]).astype(np.int32)
    Cd = torch.from_numpy(C).cuda()
    a = torch.empty_like(Cd)
    p = torch.empty_like(Cd)
    need = K.cmp_presort_ws_bytes(2 * d, w)
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device="cuda")
    K.cmp_presort(Cd.data_ptr(), 2 * d, w, a.data_ptr(), p.data_ptr(), ws.data_ptr(), need, K.stream_handle())
    edges = [5, 2]
    multi = torch.full((4, d, w), -7, dtype=torch.int32, device="cuda")
    K.cmp_cross_ranks_multi(a.data_ptr(), p.data_ptr(), [2], edges, d, w, multi.data_ptr(), K.stream_handle())
    one = torch.full((4, d, w), -9, dtype=torch.int32, device="cuda")
    K.cmp_cross_ranks(a.data_ptr(), p.data_ptr(), 2, d, w, edges, one.data_ptr(), K.stream_handle())
    torch.cuda.synchronize()
    assert torch.equal(one, multi)
    A = a.cpu().numpy().view(np.uint32).reshape(2, d, w)
    R = multi.cpu().numpy().reshape(2, 2, d, w)
    for x in range(2):
        for y in range(2):
            for i in range(d):
                if x == y:
                    inv = np.empty(w, np.int64)
                    inv[p.cpu().numpy()[x, i]] = np.arange(w)
                    assert np.array_equal(R[x, y, i], inv)
                else:
                    side = "right" if edges[y] < edges[x] else "left"
                    assert np.array_equal(R[x, y, i], np.searchsorted(A[y, i], A[x, i], side=side))


def test_cross_ranks_multi_equals_per_table():
    """One launch for several tables (0 to 16 sketches each, consecutive blocks) gives the
    ranks of one cmp_cross_ranks call per table."""
    rng = np.random.default_rng(12)
    d, w = 3, 300
    ks = [2, 0, 1, 3, 16, 1]
    total = sum(ks)
    C = torch.from_numpy(rng.integers(-9, 10, size=(total, d, w)).astype(np.int32)).cuda()
    a = torch.empty_like(C)
    p = torch.empty_like(C)
    K.cmp_presort(C.data_ptr(), total * d, w, a.data_ptr(), p.data_ptr(), 0, 0, K.stream_handle())
    edges = [int(e) for k in ks for e in rng.permutation(40)[:k]]
    multi = torch.full((sum(k * k for k in ks), d, w), -7, dtype=torch.int32, device="cuda")
    K.cmp_cross_ranks_multi(a.data_ptr(), p.data_ptr(), ks, edges, d, w, multi.data_ptr(), K.stream_handle())
    off = roff = e = 0
    for k in ks:
        if k:
            one = torch.full((k * k, d, w), -9, dtype=torch.int32, device="cuda")
            K.cmp_cross_ranks(a[off:].data_ptr(), p[off:].data_ptr(), k, d, w, edges[e:e + k], one.data_ptr(),
                              K.stream_handle())
            torch.cuda.synchronize()
            assert torch.equal(one, multi[roff:roff + k * k])
        off, roff, e = off + k, roff + k * k, e + k


@pytest.mark.parametrize("w", [16384, 20011])
def test_wide_star_roots_split_over_chunks(orc, w):
    """At w >= 16384 a tree whose only operation is a root with two or more inputs (a star)
    is split into chunks of the root's sorted positions, each recomputing the leaf suffix
    sums; ragged chunk ends at w = 20011.  Its rows equal the oracle's, beside unsplit
    sub-plans (pairs, a chain through the root) in the same plan."""
    eu, ev, nt = [0, 0, 0, 3], [1, 2, 3, 4], 5
    rng = np.random.default_rng(w)
    tabs = []
    for t in range(nt):
        n = int(rng.integers(20_000, 200_000))
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if t in (eu[e], ev[e]):
                cols.append(G.zipf_keys(rng, n, 50_000, float(rng.uniform(0.6, 1.3))))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    wl = G.Workload("star_wide", tabs, eu, ev, 3, w, 4711 + w, 0)
    dw = P.DeviceWorkload(wl)
    dw.build()
    masks = [0b00111, 0b01011, 0b01111, 0b00011, 0b11001, 0b11111, 0b11000]
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    _check(orc, dw, est, masks)
