"""Pins of the enumeration oracle (Algorithm 1, Sec. 5) and of the L1 permutation
distance (Sec. 6.2): the paper's JOB 6a walk-through and L1 example, exhaustive
enumeration against brute force over all connected left-deep orders, max_plans = 1
against a greedy left-deep search, and the readings for NaN and negative estimates."""
import math
import os

import numpy as np

from oracle import enumerate as E

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ["mk", "k", "t", "ci", "n"]


def _job6a():
    eu, ev, est, card, facts = [], [], {}, [0] * 5, []
    for line in open(os.path.join(HERE, "golden", "job6a_enumeration.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "edges":
            for e in line[1:]:
                u, v = map(int, e.split("-"))
                eu.append(u)
                ev.append(v)
        elif line[0] == "est":
            est[sum(1 << NAMES.index(x) for x in line[1].split(","))] = float(line[2])
        elif line[0] == "card":
            card[NAMES.index(line[1])] = int(line[2])
        else:
            facts.append(line)
    return eu, ev, est, card, facts


def test_job6a_walkthrough():
    eu, ev, est, card, facts = _job6a()
    deg = [0] * 5
    for u, v in zip(eu, ev):
        deg[u] += 1
        deg[v] += 1
    best, cost, stats, trace = E.enumerate_plans(5, eu, ev, est, card, max_plans=2)
    plans = [(o, c) for kind, o, c in trace if kind == "plan"]
    pruned = {o for kind, o, c in trace if kind == "pruned"}
    for f in facts:
        if f[0] == "order":
            assert [NAMES[v] for v in E.source_order(5, card, deg)] == f[1:]
        elif f[0] == "plan":
            order = tuple(NAMES.index(x) for x in f[1:-1])
            assert (order, float(f[-1])) in plans
        elif f[0] == "pruned":
            assert tuple(NAMES.index(x) for x in f[1:]) in pruned
        elif f[0] == "best":
            assert [NAMES[v] for v in best] == f[1:-1] and cost == float(f[-1])
    # the plans in the walk-through's order; n's enumeration stops at max_plans = 2
    assert [tuple(NAMES[v] for v in o) for o, c in plans] == [
        ("n", "ci", "t", "mk", "k"), ("n", "ci", "mk", "k", "t"), ("k", "mk", "ci", "n", "t"),
        ("mk", "k", "ci", "n", "t")]
    assert ("abort", (4,), 0.0) in trace
    # from ci everything is pruned: no complete plan starts there
    assert all(o[0] != 3 for o, c in plans)


def test_l1_permutation_distance():
    *_, facts = _job6a()
    for f in facts:
        if f[0] == "l1":
            t = [float(x) for x in f[1].split(",")]
            s = [float(x) for x in f[2].split(",")]
            assert E.l1_permutation_distance(t, s) == int(f[3])
    # Sec. 6.2's 2- and 3-way rows keep the true order: distance 0
    assert E.l1_permutation_distance([14, 486, 3e5, 6e6, 215e6], [3e3, 7.5e3, 6.4e6, 14e6, 397e6]) == 0
    assert E.l1_permutation_distance([11, 61, 1242, 1e4, 17e6], [6.7e3, 35e3, 7e5, 1.5e6, 8.7e9]) == 0
    assert E.l1_permutation_distance([1, 2, 3], [3, 2, 1]) == 4


def _connected_masks(n, eu, ev):
    adj = [0] * n
    for u, v in zip(eu, ev):
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    out = []
    for m in range(1, 1 << n):
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


def _random_graph(rng, n, extra):
    eu, ev = [], []
    for t in range(1, n):
        eu.append(int(rng.integers(0, t)))
        ev.append(t)
    for _ in range(extra):
        a, b = rng.choice(n, 2, replace=False)
        eu.append(int(a))
        ev.append(int(b))
    return eu, ev


def test_exhaustive_equals_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(60):
        n = int(rng.integers(2, 7))
        eu, ev = _random_graph(rng, n, int(rng.integers(0, 3)))
        est = {m: float(rng.choice([rng.integers(0, 50), rng.uniform(0, 1e6)])) for m in _connected_masks(n, eu, ev)}
        card = [int(x) for x in rng.integers(1, 1000, n)]
        best, cost, stats, _ = E.enumerate_plans(n, eu, ev, est, card, max_plans=0)
        bb, bc = E.brute_force_best(n, eu, ev, est)
        assert cost == bc, (trial, cost, bc)
        # the reported order is connected-left-deep and has that cost
        mask, c = 1 << best[0], 0.0
        for v in best[1:]:
            mask |= 1 << v
            c += est[mask]
        assert sorted(best) == list(range(n)) and c == cost


def test_one_plan_per_source_is_greedy_from_each_source():
    rng = np.random.default_rng(2)
    for trial in range(40):
        n = int(rng.integers(2, 8))
        eu, ev = _random_graph(rng, n, int(rng.integers(0, 3)))
        est = {m: float(rng.uniform(0, 1e6)) for m in _connected_masks(n, eu, ev)}
        card = [int(x) for x in rng.integers(1, 1000, n)]
        best, cost, stats, trace = E.enumerate_plans(n, eu, ev, est, card, max_plans=1)
        adj = [0] * n
        for u, v in zip(eu, ev):
            adj[u] |= 1 << v
            adj[v] |= 1 << u
        # greedy left-deep search from the first source
        deg = [sum(1 for u, v in zip(eu, ev) if t in (u, v)) for t in range(n)]
        s = E.source_order(n, card, deg)[0]
        order, mask, c = [s], 1 << s, 0.0
        while len(order) < n:
            nb = 0
            for t in order:
                nb |= adj[t]
            cand = [v for v in range(n) if (nb >> v) & 1 and not (mask >> v) & 1]
            v = min(cand, key=lambda v: (est[mask | (1 << v)], v))
            order.append(v)
            mask |= 1 << v
            c += est[mask]
        first_plan = next(o for kind, o, _ in trace if kind == "plan")
        assert first_plan == tuple(order)
        assert cost <= c


def test_nan_and_negative_estimates():
    # chain 0-1-2: prefix {0,1} NaN (beyond the exact range) counts as +inf, {1,2} < 0 as 0
    eu, ev = [0, 1], [1, 2]
    est = {0b011: float("nan"), 0b110: -5.0, 0b111: 10.0}
    best, cost, _, _ = E.enumerate_plans(3, eu, ev, est, [5, 5, 5], max_plans=0)
    assert cost == 10.0 and best in ((1, 2, 0), (2, 1, 0))
    assert E._est(est, 0b011) == math.inf and E._est(est, 0b110) == 0.0
