"""Sub-plans with two or three independent cycles (Sec. 4.2: the merged tensors of every
table contracted over all of the sub-plan's edges): the non-tree edges of the BFS tree
are conditioned together, one conditioning value per assignment of their buckets (w^rho
of them, split into chunks), each a tree contraction.  Exact int128 rows and the double
estimate must equal the oracle's on every connected sub-plan of graphs with two cycles,
three cycles (K4), parallel edges, two triangles sharing a table, a cycle with a chord;
at several widths and conditioning chunks, on real builds (Zipf keys, ties)."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

GRAPHS = {
    "two_cycles": ([0, 1, 2, 0, 3], [1, 2, 0, 3, 1], 4),
    "k4": ([0, 0, 0, 1, 1, 2], [1, 2, 3, 2, 3, 3], 4),
    "triple_parallel": ([0, 0, 0, 1], [1, 1, 1, 2], 3),
    "bowtie+leaf": ([0, 1, 2, 0, 3, 4, 2], [1, 2, 0, 3, 4, 0, 5], 6),
    "chord+tail": ([0, 1, 2, 3, 0, 3], [1, 2, 3, 0, 2, 4], 5),
}


def _workload(name, w, seed):
    eu, ev, nt = GRAPHS[name]
    rng = np.random.default_rng(seed)
    tabs = []
    for t in range(nt):
        n = int(rng.integers(50, 2000))
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if t in (eu[e], ev[e]):
                cols.append(G.zipf_keys(rng, n, 200, float(rng.uniform(0.6, 1.4))))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    return G.Workload(name, tabs, eu, ev, 3, w, 91 + w, 0)


def _oracle_rows(orc, dw, masks):
    wl = dw.wl
    built = [orc.build_sketch(t, dw.hash_u64, wl.d, wl.w) for t in wl.tables]
    for (c, _), t in zip(built, dw.tables):
        assert np.array_equal(t.counters.cpu().numpy(), c)
    sk = [tuple(built[wl.sketch_of(e, end)[0]][0][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(dw.n_edges)]
    surv = np.array([n for _, n in built], np.int64)
    return [orc.estimate(wl.edge_u, wl.edge_v, sk, surv, wl.d, wl.w, int(m)) for m in masks]


def _rho(eu, ev, m):
    inner = sum(1 for u, v in zip(eu, ev) if (m >> u) & 1 and (m >> v) & 1)
    return inner - bin(m).count("1") + 1


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("w", [3, 16, 45])
def test_multi_cycle_subplans_match_oracle(orc, name, w):
    eu, ev, nt = GRAPHS[name]
    dw = P.DeviceWorkload(_workload(name, w, sum(map(ord, name)) + w))
    dw.build()
    masks = G.connected_subplans(nt, eu, ev)
    assert max(_rho(eu, ev, m) for m in masks) >= 2
    refs = _oracle_rows(orc, dw, masks)
    for cfg in (None, K.cmp_estimate_cfg.make(cond_chunk=7),
                K.cmp_estimate_cfg.make(threads=128, ctas_per_sm=8, cond_chunk=300, flags=K.CMP_EST_GENERIC_ONLY)):
        dw.status.zero_()
        est = P.DeviceEstimator(dw, masks, cfg=cfg)
        est.presort()
        est.estimate()
        torch.cuda.synchronize()
        dw.check_status()
        rows = est.row_values()
        e = est.est.cpu().numpy()
        for q, ref in enumerate(refs):
            assert rows[q] == ref.rows, (name, w, bin(masks[q]), rows[q], ref.rows)
            assert e[q] == ref.est, (name, w, bin(masks[q]))


def test_cycle_ranks_interleaved_in_one_plan(orc):
    """K4's sub-plans in one plan, largest first: trees, one cycle (the triangle path),
    three cycles (64,000 conditioning values per row), their items interleaved; a ragged
    conditioning chunk."""
    w = 40
    eu, ev, nt = GRAPHS["k4"]
    dw = P.DeviceWorkload(_workload("k4", w, 5))
    dw.build()
    masks = G.connected_subplans(nt, eu, ev)
    refs = _oracle_rows(orc, dw, masks)
    order = list(range(len(masks)))[::-1]
    est = P.DeviceEstimator(dw, [masks[q] for q in order], cfg=K.cmp_estimate_cfg.make(cond_chunk=33))
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    dw.check_status()
    rows = est.row_values()
    e = est.est.cpu().numpy()
    for i, q in enumerate(order):
        assert rows[i] == refs[q].rows, bin(masks[q])
        assert e[i] == refs[q].est
