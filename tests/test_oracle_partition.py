"""Pins of the partitioned-sketch oracle (Sec. 4.1, sketch partitioning): the tensor a tuple
updates is indexed by its per-edge buckets and the update is the product of its per-edge
signs; the estimate of a tree-shaped join is the full contraction of the tables' tensors
and it is unbiased.  Each pin checks the oracle against something it does not compute
itself: the 1-D oracle sketch, an exact histogram, the brute-force join, numpy's einsum,
the definition as a sum over bucket assignments, or a sample mean over hash seeds."""
import numpy as np
import pytest

from paper_2102_02440_gb300 import datagen as G


@pytest.fixture(scope="module")
def part(orc):
    from oracle import partition
    return partition


def _table(rng, n, k, dom=60, preds=True, int64=False, neg=False):
    dt = np.int64 if int64 else np.int32
    cols = []
    for _ in range(k):
        c = G.zipf_keys(rng, n, dom, float(rng.uniform(0.5, 1.4)), dt)
        if neg:
            c = (c - dom // 2).astype(dt)
        cols.append(c)
    cols.append(G.uniform_col(rng, n, 0, 1000))
    cols.append(G.uniform_col(rng, n, -5, 40))
    pr = []
    if preds:
        pr = [G.Pred(k, G.RANGE, 100, 800), G.Pred(k + 1, G.IN, 0, 0, G.bitmap_of([0, 2, 3, 7, 11, 30, 31, 32], 40), 40)]
    return G.Table("t", cols, pr, list(range(k)), list(range(k)))


def _identity(n_edges, d):
    hp = np.zeros((n_edges, d, 6), np.uint64)
    hp[..., 0] = 1  # h(x) = x mod w, xi = +1
    return hp


def test_selection_matches_1d_oracle_and_loop(orc, part):
    rng = np.random.default_rng(1)
    for int64 in (False, True):
        t = _table(rng, 4000, 2, int64=int64)
        keep = part.selected(t)
        _, n1 = orc.build_sketch(t, orc.hash_params(3, 2, 1), 1, 16)
        assert int(keep.sum()) == n1
        for r in range(0, t.n_rows, 97):   # plain loop over the conjunction
            v, c = int(t.cols[2][r]), int(t.cols[3][r])
            want = 100 <= v < 800 and c in (0, 2, 3, 7, 11, 30, 31, 32)
            assert bool(keep[r]) == want


@pytest.mark.parametrize("w", [1, 7, 64, 1000])
def test_one_axis_is_the_1d_sketch(orc, part, w):
    rng = np.random.default_rng(w)
    t = _table(rng, 3000, 3, dom=400, int64=w == 7, neg=w == 64)
    hp = orc.hash_params(11, 3, 5)
    full, n_full = orc.build_sketch(t, hp, 5, w)
    for s in range(3):
        ts = G.Table("t", t.cols, t.preds, [t.key_col[s]], [t.edge_id[s]])
        got, n = part.build_partitioned(ts, hp, 5, [w])
        assert n == n_full
        assert np.array_equal(got, full[s])


def test_zero_axes_hold_the_selected_count(part, orc):
    rng = np.random.default_rng(4)
    t = _table(rng, 2500, 1)
    t0 = G.Table("t", t.cols, t.preds, [], [])
    got, n = part.build_partitioned(t0, orc.hash_params(1, 1, 3), 3, [])
    assert got.shape == (3, 1) and (got[:, 0] == n).all() and n == int(part.selected(t).sum())


def test_identity_hash_gives_the_joint_histogram(part):
    """h(x) = x and xi = +1 with widths covering the key domains: entry [x1, x2] counts the
    selected tuples with keys (x1, x2), row-major with the last axis contiguous."""
    rng = np.random.default_rng(7)
    t = _table(rng, 5000, 2, dom=30)
    widths = [37, 31]
    got, _ = part.build_partitioned(t, _identity(2, 2), 2, widths)
    keep = part.selected(t)
    hist = np.zeros((37, 31), np.int64)
    for a, b in zip(t.cols[0][keep], t.cols[1][keep]):
        hist[int(a), int(b)] += 1
    for i in range(2):
        assert np.array_equal(got[i].reshape(37, 31), hist)


def test_update_is_the_product_of_the_axis_signs(part):
    """xi = parity sign of x (c1 = 1) on both axes: entry [x1, x2] = (-1)^(x1 + x2) count;
    on one axis only, (-1)^x1 count; c0 = 1 on one axis negates every entry."""
    rng = np.random.default_rng(8)
    t = _table(rng, 4000, 2, dom=20, preds=False)
    hist = np.zeros((20, 21), np.int64)
    for a, b in zip(t.cols[0], t.cols[1]):
        hist[int(a), int(b)] += 1
    sa = np.where(np.arange(20) % 2 == 0, 1, -1)[:, None]
    sb = np.where(np.arange(21) % 2 == 0, 1, -1)[None, :]
    hp = _identity(2, 1)
    hp[0, 0, 3] = 1
    hp[1, 0, 3] = 1
    got, _ = part.build_partitioned(t, hp, 1, [20, 21])
    assert np.array_equal(got[0].reshape(20, 21), hist * sa * sb)
    hp[1, 0, 3] = 0
    got, _ = part.build_partitioned(t, hp, 1, [20, 21])
    assert np.array_equal(got[0].reshape(20, 21), hist * sa)
    hp[0, 0, 3] = 0
    hp[0, 0, 2] = 1
    got, _ = part.build_partitioned(t, hp, 1, [20, 21])
    assert np.array_equal(got[0].reshape(20, 21), -hist)


def test_linear_over_row_ranges(orc, part):
    rng = np.random.default_rng(9)
    t = _table(rng, 3001, 3, dom=200, int64=True, neg=True)
    hp = orc.hash_params(5, 3, 4)
    whole, n = part.build_partitioned(t, hp, 4, [5, 8, 3])
    a, na = part.build_partitioned(t, hp, 4, [5, 8, 3], 0, 1234)
    b, nb = part.build_partitioned(t, hp, 4, [5, 8, 3], 1234, None)
    assert na + nb == n
    assert np.array_equal(whole, (a.astype(np.int64) + b).astype(np.int32))


def _random_tree(rng, nt):
    eu, ev = [], []
    for t in range(1, nt):
        eu.append(int(rng.integers(0, t)))
        ev.append(t)
    perm = rng.permutation(nt - 1)
    return [eu[i] for i in perm], [ev[i] for i in perm]


def _axes(nt, eu, ev, rng):
    dims = []
    for t in range(nt):
        inc = [e for e in range(len(eu)) if t in (eu[e], ev[e])]
        dims.append([inc[i] for i in rng.permutation(len(inc))])
    return dims


def _einsum(eu, ev, width, dims, tensors, d):
    letters = "abcdefghijklmnopqrstuvwxyz"
    spec = ",".join("".join(letters[e] for e in ax) for ax in dims) + "->"
    out = []
    for i in range(d):
        ops = [np.asarray(tensors[t][i], np.int64).reshape([width[e] for e in ax]) for t, ax in enumerate(dims)]
        out.append(int(np.einsum(spec, *ops)))
    return out


@pytest.mark.parametrize("seed", range(8))
def test_contraction_equals_definition_and_einsum(part, seed):
    rng = np.random.default_rng(seed)
    nt = int(rng.integers(2, 6))
    eu, ev = _random_tree(rng, nt)
    dims = _axes(nt, eu, ev, rng)
    width = [int(rng.integers(1, 5)) for _ in eu]
    d = 3
    tensors = []
    for ax in dims:
        size = int(np.prod([width[e] for e in ax]))
        tensors.append(rng.integers(-9, 10, size=(d, size)))
    part.check_tree(nt, eu, ev, dims)
    rows, oor = part.contract_seq(eu, ev, width, dims, tensors, d)
    assert not any(oor)
    assert rows == part.contract_brute(eu, ev, width, dims, tensors, d)
    assert rows == _einsum(eu, ev, width, dims, tensors, d)


def _chain_workload(rng, n_mid=6000):
    """k - mk - t shaped chain: table 0 (keyword-like, point predicate on a code), table 1
    (movie_keyword-like, two key columns), table 2 (title-like, range predicate)."""
    kw, mv = 40, 90
    k = G.Table("k", [np.arange(kw, dtype=np.int32), G.uniform_col(rng, kw, 0, 4)], [G.Pred(1, G.RANGE, 0, 2)],
                [0], [0])
    mk = G.Table("mk", [G.zipf_keys(rng, n_mid, kw, 1.1), G.zipf_keys(rng, n_mid, mv, 0.9)], [], [0, 1], [0, 1])
    t = G.Table("t", [np.arange(mv, dtype=np.int32), G.uniform_col(rng, mv, 0, 100)], [G.Pred(1, G.RANGE, 10, 70)],
                [0], [1])
    return [k, mk, t], [0, 1], [1, 2], kw, mv


def test_identity_hash_estimate_is_the_exact_join(orc, part):
    rng = np.random.default_rng(12)
    tabs, eu, ev, kw, mv = _chain_workload(rng)
    hp = _identity(2, 2)
    width = [kw, mv]
    sk = [part.build_partitioned(tb, hp, 2, [width[e] for e in tb.edge_id])[0] for tb in tabs]
    dims = [tb.edge_id for tb in tabs]
    rows, oor = part.contract_seq(eu, ev, width, dims, sk, 2)
    keep = [part.selected(tb) for tb in tabs]
    keys = [(tabs[0].cols[0][keep[0]], tabs[1].cols[0][keep[1]]), (tabs[1].cols[1][keep[1]], tabs[2].cols[0][keep[2]])]
    # join_brute takes one key column per (edge, endpoint): table 1's two columns are aligned
    exact = orc.join_brute(eu, ev, [int(k.sum()) for k in keep], keys, 0b111)
    assert rows == [exact, exact] and not any(oor)
    assert part.median_to_double(rows) == float(exact)


def test_identity_hash_star_and_four_axes(orc, part):
    """A 4-axis centre table joined to four dimension tables (a star): the exact join size."""
    rng = np.random.default_rng(13)
    doms = [5, 7, 4, 6]
    n = 300
    centre = G.Table("c", [G.zipf_keys(rng, n, dm, 0.8) for dm in doms], [], [0, 1, 2, 3], [0, 1, 2, 3])
    dims_t = [G.Table(f"d{e}", [G.zipf_keys(rng, 9, dm, 0.5)], [], [0], [e]) for e, dm in enumerate(doms)]
    tabs = [centre] + dims_t
    eu, ev = [0, 0, 0, 0], [1, 2, 3, 4]
    hp = _identity(4, 1)
    sk = [part.build_partitioned(tb, hp, 1, [doms[e] for e in tb.edge_id])[0] for tb in tabs]
    rows, _ = part.contract_seq(eu, ev, doms, [tb.edge_id for tb in tabs], sk, 1)
    keys = [(centre.cols[e], dims_t[e].cols[0]) for e in range(4)]
    exact = orc.join_brute(eu, ev, [tb.n_rows for tb in tabs], keys, 0b11111)
    assert rows == [exact]


def test_unbiased_over_hash_seeds(orc, part):
    """E[row estimate] = exact join size (Sec. 4.1): the mean of 400 independent rows (40
    seeds x 10 rows) is within 4.5 standard errors of the brute-force size."""
    rng = np.random.default_rng(14)
    tabs, eu, ev, kw, mv = _chain_workload(rng, 1500)
    keep = [part.selected(tb) for tb in tabs]
    keys = [(tabs[0].cols[0][keep[0]], tabs[1].cols[0][keep[1]]), (tabs[1].cols[1][keep[1]], tabs[2].cols[0][keep[2]])]
    exact = orc.join_brute(eu, ev, [int(k.sum()) for k in keep], keys, 0b111)
    width = [8, 16]
    vals = []
    for seed in range(40):
        hp = orc.hash_params(1000 + seed, 2, 10)
        sk = [part.build_partitioned(tb, hp, 10, [width[e] for e in tb.edge_id])[0] for tb in tabs]
        rows, _ = part.contract_seq(eu, ev, width, [tb.edge_id for tb in tabs], sk, 10)
        vals += rows
    vals = np.array(vals, np.float64)
    se = vals.std(ddof=1) / np.sqrt(vals.size)
    assert exact > 0 and abs(vals.mean() - exact) < 4.5 * se


def test_out_of_range_rule(part):
    """Chain 0 - 1 - 2 - 3, widths (2, 8, 2), big = 2^31 - 1 in tables 1..3.  The message
    into the root is 16 big^3 per entry.  Row 0: root (big, -big): each product 16 big^4 is
    beyond int128 although the sum is 0.  Row 1: root (2^30, 2^30): the products 2^34 big^3
    fit, their sum 2^35 big^3 does not.  Row 2: all ones, 32."""
    big = (1 << 31) - 1
    eu, ev = [0, 1, 2], [1, 2, 3]
    dims = [[0], [0, 1], [1, 2], [2]]
    width = [2, 8, 2]
    d = 3
    tensors = [np.ones((d, 2), object), np.ones((d, 16), object), np.ones((d, 16), object), np.ones((d, 2), object)]
    for t in (1, 2, 3):
        tensors[t][0] = big
        tensors[t][1] = big
    tensors[0][0] = [big, -big]
    tensors[0][1] = [1 << 30, 1 << 30]
    rows, oor = part.contract_seq(eu, ev, width, dims, tensors, d)
    assert 2 ** 34 * big ** 3 < 1 << 127 <= 16 * big ** 4
    assert oor == [True, True, False]
    assert rows == [0, 2 ** 35 * big ** 3, 32]


def test_check_tree_rejects(part):
    with pytest.raises(ValueError):
        part.check_tree(3, [0, 1, 0], [1, 2, 2], [[0, 2], [0, 1], [1, 2]])   # a cycle
    with pytest.raises(ValueError):
        part.check_tree(3, [0], [1], [[0], [0], []])                          # not spanning
    with pytest.raises(ValueError):
        part.check_tree(3, [0, 1], [1, 2], [[0], [0], [1]])                   # missing axis
