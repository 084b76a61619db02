"""GPU parity of join-order enumeration (Algorithm 1, Sec. 5) against the oracle: best
plan, cost and search counters identical, on the paper's JOB 6a walk-through, on random
graphs with synthetic estimate tables (all max_plans settings, many graphs in one launch),
end to end on sketches (the GPU estimate then the GPU search, against the oracle estimate
then the oracle search), and the missing-estimate and search-budget statuses."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from oracle import enumerate as E
from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

_keep = []


def _graph(n, eu, ev, card):
    ne = len(eu)
    a = (C.c_int32 * max(ne, 1))(*eu)
    b = (C.c_int32 * max(ne, 1))(*ev)
    surv = torch.tensor(card, dtype=torch.int64, device="cuda")
    _keep.extend([a, b, surv])
    return K.cmp_graph(n, ne, a, b, None, None, None, None, None, surv.data_ptr())


def _run(graphs, subs, est_host, max_plans, max_nodes=0):
    """subs: list of (graph index, mask); est_host: matching estimates."""
    sg = [g for g, _ in subs]
    sm = [m for _, m in subs]
    en = P.Enumerator(graphs, sg, sm, cfg=K.cmp_enum_cfg.make(max_plans=max_plans, max_nodes=max_nodes))
    est = torch.tensor(est_host, dtype=torch.float64, device="cuda")
    en.run(est)
    torch.cuda.synchronize()
    return en.plans(), int(en.status.item())


def _connected(n, eu, ev):
    adj = [0] * n
    for u, v in zip(eu, ev):
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    out = []
    for m in range(1, 1 << n):
        if bin(m).count("1") < 2:
            continue
        first = (m & -m).bit_length() - 1
        seen, todo = 1 << first, [first]
        while todo:
            t = todo.pop()
            nb = adj[t] & m & ~seen
            seen |= nb
            todo += [x for x in range(n) if (nb >> x) & 1]
        if seen == m:
            out.append(m)
    return out


def _oracle(n, eu, ev, est, card, max_plans):
    best, cost, st, _ = E.enumerate_plans(n, eu, ev, est, card, max_plans=0 if max_plans == -1 else max_plans)
    return (tuple(best) if best else (), cost, (st["plans"], st["nodes"], st["pruned"]))


def test_job6a_walkthrough_on_device():
    names = ["mk", "k", "t", "ci", "n"]
    eu, ev, est, card = [], [], {}, [0] * 5
    for line in open("tests/golden/job6a_enumeration.txt"):
        f = line.split("#")[0].split()
        if f and f[0] == "edges":
            for e in f[1:]:
                u, v = map(int, e.split("-"))
                eu.append(u)
                ev.append(v)
        elif f and f[0] == "est":
            est[sum(1 << names.index(x) for x in f[1].split(","))] = float(f[2])
        elif f and f[0] == "card":
            card[names.index(f[1])] = int(f[2])
    masks = sorted(est)
    got, st = _run([_graph(5, eu, ev, card)], [(0, m) for m in masks], [est[m] for m in masks], 2)
    assert st == 0
    order, cost, stats = got[0]
    assert [names[v] for v in order] == ["k", "mk", "ci", "n", "t"] and cost == 703298.0
    assert got[0] == _oracle(5, eu, ev, est, card, 2)


@pytest.mark.parametrize("max_plans", [1, 2, 10, -1])
def test_random_graphs_match_oracle(max_plans):
    rng = np.random.default_rng(100 + max_plans)
    graphs, subs, est_host, ref = [], [], [], []
    for gi in range(40):
        n = int(rng.integers(1, 9))
        eu, ev = [], []
        for t in range(1, n):
            eu.append(int(rng.integers(0, t)))
            ev.append(t)
        for _ in range(int(rng.integers(0, 3)) if n > 1 else 0):
            a, b = rng.choice(n, 2, replace=False)
            eu.append(int(a))
            ev.append(int(b))
        card = [int(x) for x in rng.integers(0, 10_000, n)]
        est = {}
        for m in _connected(n, eu, ev):
            r = rng.random()   # ties, zeros, NaN, negatives and a wide range of magnitudes
            est[m] = (float(rng.integers(0, 4)) if r < 0.3 else float("nan") if r < 0.33 else
                      -float(rng.integers(1, 9)) if r < 0.36 else float(rng.lognormal(8, 4)))
        graphs.append(_graph(n, eu, ev, card))
        for m in sorted(est):
            subs.append((gi, m))
            est_host.append(est[m])
        ref.append(_oracle(n, eu, ev, est, card, max_plans))
    got, st = _run(graphs, subs, est_host, max_plans)
    assert st == 0
    for gi, (g, r) in enumerate(zip(got, ref)):
        assert g[0] == r[0] and g[2] == r[2], (gi, g, r)
        assert g[1] == r[1] or (math.isinf(g[1]) and math.isinf(r[1]))


def test_end_to_end_on_sketches(orc):
    """GPU estimate + GPU search against oracle estimate + oracle search, on the five-table
    graph at reduced size: the estimates agree exactly, so the plans must too."""
    wl = G.five_table(scale=0.005, w=256)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    multi = [m for m in masks if bin(m).count("1") >= 2]
    en = P.Enumerator(est.graphs, np.zeros(len(masks), np.int32), masks, cfg=K.cmp_enum_cfg.make(max_plans=-1))
    en.run(est.est)
    torch.cuda.synchronize()
    dw.check_status()
    built = [orc.build_sketch(t, dw.hash_u64, wl.d, wl.w) for t in wl.tables]   # the oracle's own build
    sk = [tuple(built[wl.sketch_of(e, end)[0]][0][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(dw.n_edges)]
    surv = np.array([n for _, n in built], np.int64)
    ref_est = {m: orc.estimate(wl.edge_u, wl.edge_v, sk, surv, wl.d, wl.w, m).est for m in multi}
    ref = _oracle(5, wl.edge_u, wl.edge_v, ref_est, [int(x) for x in surv], -1)
    assert en.plans()[0] == ref


def test_missing_estimate_and_budget_statuses():
    eu, ev = [0, 1, 2], [1, 2, 3]   # chain of 4
    est = {m: 1.0 for m in _connected(4, eu, ev)}
    masks = sorted(est)
    g = _graph(4, eu, ev, [1, 2, 3, 4])
    # the full sub-plan's estimate left out: unreachable complete plans, CMP_EUNSUPPORTED
    got, st = _run([g], [(0, m) for m in masks if m != 0b1111], [1.0] * (len(masks) - 1), -1)
    assert st == K.CMP_EUNSUPPORTED and got[0][0] == () and math.isinf(got[0][1])
    # a search budget of 3 prefix extensions: stops with CMP_ETIMEOUT
    got, st = _run([g], [(0, m) for m in masks], [1.0] * len(masks), -1, max_nodes=3)
    assert st == K.CMP_ETIMEOUT and got[0][2][1] == 3
