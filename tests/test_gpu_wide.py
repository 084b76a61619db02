"""The exact tier beyond int128 of the estimate (rows whose value, or an intermediate of
their evaluation, leave int128, evaluated again modulo 16 primes with a magnitude bound
and rebuilt by Garner's algorithm): every row of such a sub-plan must equal the oracle's
arbitrary-precision row, and the estimate its correctly rounded exact median, on every
evaluation path that hands rows to the tier (generic, cached messages, star lattice,
triangle), with cancellations and large magnitudes; rows whose bound reaches 2^990 stay
NaN with CMP_EOVERFLOW."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu


def _one_row_tables(eu, ev, n, d, w):
    """One-row tables (counters overwritten by the test), survivors 1."""
    rng = np.random.default_rng(0)
    tabs = []
    for t in range(n):
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if t in (eu[e], ev[e]):
                cols.append(np.array([int(rng.integers(0, 100))], np.int32))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    dw = P.DeviceWorkload(G.Workload("raw", tabs, eu, ev, d, w, 1, 0))
    dw.survivors.fill_(1)
    return dw


def _fill(dw, fn):
    dw.host_counters = []
    for t in dw.tables:
        a = fn(tuple(t.counters.shape)).astype(np.int32)
        dw.host_counters.append(a)
        t.counters.copy_(torch.from_numpy(a))


def _oracle(orc, dw, masks):
    wl = dw.wl
    sk = [tuple(dw.host_counters[wl.sketch_of(e, end)[0]][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(dw.n_edges)]
    surv = np.ones(len(wl.tables), np.int64)
    return [orc.estimate(wl.edge_u, wl.edge_v, sk, surv, dw.d, dw.w, int(m)) for m in masks]


def _run(dw, masks, flags=0, cond_chunk=0):
    dw.status.zero_()
    est = P.DeviceEstimator(dw, masks, cfg=K.cmp_estimate_cfg.make(flags=flags, cond_chunk=cond_chunk))
    est.presort()
    est.estimate_wide()
    torch.cuda.synchronize()
    return est, int(dw.status.item())


def _check_exact(orc, dw, masks, flags_list, cond_chunk=0):
    refs = _oracle(orc, dw, masks)
    beyond = sum(1 for r in refs if any(abs(v) >= 1 << 127 for v in r.rows))
    assert beyond > 0                                   # the tier has work to do
    for flags in flags_list:
        est, st = _run(dw, masks, flags, cond_chunk)
        assert st == 0, (flags, st)
        rows = est.wide_values()
        e = est.est.cpu().numpy()
        for q, ref in enumerate(refs):
            assert rows[q] == ref.rows, (flags, bin(int(masks[q])))
            assert e[q] == ref.est, (flags, bin(int(masks[q])), e[q], ref.est)
    return refs


def test_chain_beyond_int128_generic_and_cached(orc):
    """A 16-table chain of one-row tables with counters at 2^31 - 1 in sketch row 0 and small
    signed values in the others: the long sub-plans leave int128 in row 0, some through a
    cached subtree message."""
    n = 16
    eu, ev = list(range(n - 1)), list(range(1, n))
    dw = _one_row_tables(eu, ev, n, 3, 32)
    rng = np.random.default_rng(3)

    def f(shape):
        a = rng.integers(-20, 21, size=shape)
        a[:, 0, :] = 2 ** 31 - 1
        return a
    _fill(dw, f)
    masks = G.connected_subplans(n, eu, ev)
    _check_exact(orc, dw, masks, [0, K.CMP_EST_CACHE_MESSAGES, K.CMP_EST_GENERIC_ONLY])


def test_star_beyond_int128_lattice_and_generic(orc):
    """A 10-leaf star of one-row tables, counters at 2^31 - 1 in sketch row 0: the large leaf
    subsets leave int128 on the lattice and on the generic path."""
    n = 10
    eu, ev = [0] * n, list(range(1, n + 1))
    dw = _one_row_tables(eu, ev, n + 1, 3, 32)
    rng = np.random.default_rng(4)

    def f(shape):
        a = rng.integers(1, 21, size=shape)
        a[:, 0, :] = 2 ** 31 - 1
        return a
    _fill(dw, f)
    masks = G.connected_subplans(n + 1, eu, ev)
    _check_exact(orc, dw, masks, [K.CMP_EST_STAR_LATTICE, 0])


def test_triangle_beyond_int128(orc):
    """A triangle with three leaves, counters at 2^31 - 1: every row beyond int128, on the
    triangle path and the generic path."""
    eu, ev = [0, 1, 0, 0, 1, 2], [1, 2, 2, 3, 4, 5]
    dw = _one_row_tables(eu, ev, 6, 3, 32)
    _fill(dw, lambda shape: np.full(shape, 2 ** 31 - 1))
    _check_exact(orc, dw, [0b111111, 0b000111, 0b001111], [0, K.CMP_EST_GENERIC_ONLY])


@pytest.mark.parametrize("huge", [[1, 2, 3], [1, 2, 3, 4], [1, 2, 3, 4, 5]])
def test_star_rows_on_the_lattice_or_generic(orc, huge):
    """A 10-leaf star (w = 8), sketch row 0 at 2^31 - 1 on the edges in `huge` and small
    elsewhere: 1 to 5, 68 or 202 of its leaf subsets leave int128 in row 0.  With the star
    lattice, below the break-even count those rows run the generic contraction; above it the
    family's lattice runs again modulo each needed prime and as a bound, its entries summed
    into the rows.  Rows equal the oracle's either way."""
    n = 10
    eu, ev = [0] * n, list(range(1, n + 1))
    dw = _one_row_tables(eu, ev, n + 1, 3, 8)
    rng = np.random.default_rng(4)
    host = [rng.integers(1, 4, size=tuple(t.counters.shape)) for t in dw.tables]
    for e in huge:
        for end in range(2):
            t, k = dw.wl.sketch_of(e, end)
            host[t][k, 0, :] = 2 ** 31 - 1
    dw.host_counters = [a.astype(np.int32) for a in host]
    for t, a in zip(dw.tables, dw.host_counters):
        t.counters.copy_(torch.from_numpy(a))
    masks = G.connected_subplans(n + 1, eu, ev)
    _check_exact(orc, dw, masks, [K.CMP_EST_STAR_LATTICE, 0])


def test_split_star_root_beyond_int128(orc):
    """A three-leaf star at w = 16384 (its root split into chunks of sorted positions) with
    counters near 2^31 - 1: every row leaves int128, and the exact tier evaluates it as one
    unit per chunk."""
    eu, ev = [0, 0, 0], [1, 2, 3]
    dw = _one_row_tables(eu, ev, 4, 3, 16384)
    rng = np.random.default_rng(8)

    def f(shape):
        return rng.choice(np.array([2 ** 31 - 1, -(2 ** 31 - 1), 2 ** 31 - 3, 0, 7]), size=shape)
    _fill(dw, f)
    _check_exact(orc, dw, [0b1111, 0b0111], [0, K.CMP_EST_GENERIC_ONLY])


def test_cancelling_signs_and_ties(orc):
    """Random counters of both signs near +-2^31, with zeros and equal magnitudes (ties),
    on a cycle with a leaf and a chain: products far beyond int128 whose sums cancel; even d
    (the median is the mean of the two middle rows)."""
    eu, ev = [0, 1, 2, 3, 0, 4, 5, 6, 7], [1, 2, 3, 0, 4, 5, 6, 7, 8]
    dw = _one_row_tables(eu, ev, 9, 4, 24)
    rng = np.random.default_rng(9)

    def f(shape):
        a = rng.choice(np.array([-(2 ** 31 - 1), -(2 ** 31 - 7), 0, 2 ** 31 - 7, 2 ** 31 - 1, -3, 5]), size=shape)
        return a
    _fill(dw, f)
    masks = [m for m in G.connected_subplans(9, eu, ev) if bin(m).count("1") >= 5]
    _check_exact(orc, dw, masks, [0, K.CMP_EST_GENERIC_ONLY, K.CMP_EST_CACHE_MESSAGES])


@pytest.mark.parametrize("cond_chunk", [1, 7, 64])
def test_cycles_split_into_conditioning_chunks(orc, cond_chunk):
    """A 5-cycle with a leaf and a 4-cycle, w = 100: each row of a cyclic sub-plan beyond
    int128 is evaluated by the tier as one unit per conditioning chunk (100, 15 or 2 of
    them, the last one ragged), whose residues and bounds are summed per row."""
    eu, ev = [0, 1, 2, 3, 4, 0, 6, 7, 8, 9], [1, 2, 3, 4, 0, 5, 7, 8, 9, 6]
    n = 10
    dw = _one_row_tables(eu, ev, n, 3, 100)
    rng = np.random.default_rng(cond_chunk)

    def f(shape):
        a = rng.choice(np.array([-(2 ** 31 - 1), 2 ** 31 - 1, 2 ** 31 - 5, 0, -9, 4]), size=shape)
        return a
    _fill(dw, f)
    masks = [m for m in G.connected_subplans(n, eu, ev) if bin(m).count("1") >= 4]
    assert 0b0000111111 in masks and 0b1111000000 in masks  # both cycles
    _check_exact(orc, dw, masks, [0, K.CMP_EST_GENERIC_ONLY], cond_chunk=cond_chunk)


def test_multi_cycle_beyond_int128(orc):
    """Two and three independent cycles (a 4-cycle with a chord and a tail, K4 beside it)
    with counters near +-2^31: the rows leave int128 and the tier conditions on every
    assignment of the non-tree edges, one unit per chunk."""
    eu, ev = [0, 1, 2, 3, 0, 3, 5, 5, 5, 6, 6, 7], [1, 2, 3, 0, 2, 4, 6, 7, 8, 7, 8, 8]
    n = 9
    dw = _one_row_tables(eu, ev, n, 3, 12)
    rng = np.random.default_rng(21)

    def f(shape):
        return rng.choice(np.array([-(2 ** 31 - 1), 2 ** 31 - 1, 2 ** 31 - 9, 0, -5, 3]), size=shape)
    _fill(dw, f)
    masks = [m for m in G.connected_subplans(n, eu, ev) if bin(m).count("1") >= 4]
    assert 0b11111 in masks and 0b111100000 in masks
    _check_exact(orc, dw, masks, [0, K.CMP_EST_GENERIC_ONLY], cond_chunk=10)


def test_beyond_the_exact_tier_is_reported(orc):
    """A 34-table chain at 2^31 - 1 everywhere: its row exceeds 2^990 (the bound of the
    tier), so its estimate is NaN with CMP_EOVERFLOW; a 20-table part of it (about 2^620) is
    exact."""
    n = 34
    eu, ev = list(range(n - 1)), list(range(1, n))
    dw = _one_row_tables(eu, ev, n, 1, 2)
    _fill(dw, lambda shape: np.full(shape, 2 ** 31 - 1))
    full, part = (1 << n) - 1, (1 << 20) - 1
    refs = _oracle(orc, dw, [full, part])
    assert abs(refs[0].rows[0]) > 1 << 990 and (1 << 127) < abs(refs[1].rows[0]) < 1 << 990
    est, st = _run(dw, [full, part])
    assert st == K.CMP_EOVERFLOW
    e = est.est.cpu().numpy()
    assert np.isnan(e[0]) and e[1] == refs[1].est
    assert est.wide_values()[1] == refs[1].rows


def test_in_range_plans_skip_the_tier_and_equal_no_wide(orc):
    """A workload whose rows all stay in int128: the tier queues nothing, and the results
    equal those with the tier off bit for bit."""
    rng = np.random.default_rng(5)
    wl = G.random_graph_workload(rng, 6, 1, 500, 20_000, 2000, d=5, w=256, pred_prob=0.5, hash_seed=5)
    dw = P.DeviceWorkload(wl)
    dw.build()
    masks = G.connected_subplans(6, wl.edge_u, wl.edge_v)
    a, st = _run(dw, masks, 0)
    b, st2 = _run(dw, masks, K.CMP_EST_NO_WIDE)
    assert st == st2 == 0
    assert torch.equal(a.est, b.est) and torch.equal(a.row_est, b.row_est)
    rows = a.row_values()
    assert a.wide_values() == rows
