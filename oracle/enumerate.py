"""Oracle (test infrastructure only; the product path never imports it): join-order
enumeration over sketch estimates (Sec. 5, Algorithm 1) and the L1 permutation distance
of Sec. 6.2, written from the paper's description as plain single-threaded Python.

Readings (where the paper is silent):
- The cost of a left-deep plan is the sum of the estimates of its join prefixes of two or
  more tables; the first table adds nothing.  (With the first table's cardinality added,
  the paper's walk-through of JOB 6a could not enumerate mk-k-ci-n-t from mk, nor find it
  equal in cost to k-mk-ci-n-t.)
- f(v) = alpha * card(v) / max card + beta * deg(v) / max deg (a zero maximum gives 0),
  card(v) = the table's exact selected count, deg(v) = the number of join edges at v.
  Sources are taken in increasing f(v), ties by table id; candidates in increasing
  estimate, ties by table id.
- A source's enumeration ends ("abort") when it has completed max_plans plans; max_plans
  = 0 means no limit.  Pruning is strict (cost > min_cost returns) and so is the update
  (cost < min_cost), so of equal-cost plans the first found is kept.
- An estimate that is NaN (beyond the exact range) counts as +inf and a negative one as 0.

Every step is logged in `trace` as (event, order tuple, cost) so that tests can follow
the walk-through."""
from __future__ import annotations

import math


def _est(est, mask: int) -> float:
    v = est[mask]
    if v != v:  # NaN
        return math.inf
    return max(v, 0.0)


def source_order(n: int, card, deg, alpha: float = 0.5, beta: float = 0.5) -> list:
    """Vertices sorted by f(v) (Algorithm 1, line 7), ties by id."""
    mc = max(card) if n else 0
    md = max(deg) if n else 0

    def f(v):
        a = (float(card[v]) / float(mc)) if mc > 0 else 0.0
        b = (float(deg[v]) / float(md)) if md > 0 else 0.0
        return alpha * a + beta * b

    return sorted(range(n), key=lambda v: (f(v), v))


def enumerate_plans(n: int, edge_u, edge_v, est, card, alpha: float = 0.5, beta: float = 0.5,
                    max_plans: int = 10):
    """Algorithm 1 over a join graph of n tables.  est maps a connected sub-plan mask (bit t
    = table t, two or more tables) to its estimate.  Returns (best order, min cost, stats,
    trace); stats = dict(plans, nodes, pruned)."""
    adj = [0] * n
    deg = [0] * n
    for u, v in zip(edge_u, edge_v):
        adj[u] |= 1 << v
        adj[v] |= 1 << u
        deg[u] += 1
        deg[v] += 1
    full = (1 << n) - 1
    state = {"min": math.inf, "best": None, "plans": 0, "nodes": 0, "pruned": 0}
    trace = []

    class Abort(Exception):
        pass

    def dfs(order, mask, cost, per_source):
        # the caller added this prefix's estimate; line 17: early pruning
        if cost > state["min"]:
            state["pruned"] += 1
            trace.append(("pruned", tuple(order), cost))
            return
        if mask == full:
            trace.append(("plan", tuple(order), cost))
            state["plans"] += 1
            if cost < state["min"]:
                state["min"] = cost
                state["best"] = tuple(order)
            per_source[0] += 1
            if max_plans and per_source[0] == max_plans:
                raise Abort()
            return
        nb = 0
        for t in order:
            nb |= adj[t]
        cand = [v for v in range(n) if (nb >> v) & 1 and not (mask >> v) & 1]
        e = {v: _est(est, mask | (1 << v)) for v in cand}
        for v in sorted(cand, key=lambda v: (e[v], v)):
            state["nodes"] += 1
            dfs(order + [v], mask | (1 << v), cost + e[v], per_source)

    for s in source_order(n, card, deg, alpha, beta):
        per_source = [0]
        trace.append(("source", (s,), 0.0))
        try:
            dfs([s], 1 << s, 0.0, per_source)
        except Abort:
            trace.append(("abort", (s,), 0.0))
    stats = {"plans": state["plans"], "nodes": state["nodes"], "pruned": state["pruned"]}
    return state["best"], state["min"], stats, trace


def brute_force_best(n: int, edge_u, edge_v, est):
    """Minimum cost over every left-deep order whose every prefix is connected (no cross
    products), by enumerating all permutations; ties: the lexicographically first order."""
    import itertools
    adj = [0] * n
    for u, v in zip(edge_u, edge_v):
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    best, best_cost = None, math.inf
    for perm in itertools.permutations(range(n)):
        mask, cost, ok = 1 << perm[0], 0.0, True
        for v in perm[1:]:
            nb = 0
            for t in range(n):
                if (mask >> t) & 1:
                    nb |= adj[t]
            if not (nb >> v) & 1:
                ok = False
                break
            mask |= 1 << v
            cost += _est(est, mask)
        if ok and cost < best_cost:
            best, best_cost = perm, cost
    return best, best_cost


def l1_permutation_distance(true_sizes, est_sizes) -> int:
    """Sec. 6.2: with the sub-plans ranked by true size (the correct order) and by estimate,
    the sum over sub-plans of |position by estimate - position by true size|.  Ties in
    either ranking are broken by the sub-plan's index."""
    n = len(true_sizes)
    by_true = sorted(range(n), key=lambda i: (true_sizes[i], i))
    by_est = sorted(range(n), key=lambda i: (est_sizes[i], i))
    pos_true = {q: k for k, q in enumerate(by_true)}
    pos_est = {q: k for k, q in enumerate(by_est)}
    return sum(abs(pos_est[q] - pos_true[q]) for q in range(n))
