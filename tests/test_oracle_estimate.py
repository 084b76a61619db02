"""Pins of the oracle's estimate (Sec. 3.2: per-row inner product then median;
Sec. 4.2: sketch merging by minimum absolute value, iterated over a table's joins;
Sec. 4.1: the 3-table contraction sum over i, j of sk_k[i] * M[i, j] * sk_t[j])."""
import itertools
import os

import numpy as np
import pytest

from paper_2102_02440_gb300 import datagen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sk(rng, d, w, lo=-6, hi=7):
    return rng.integers(lo, hi, size=(d, w)).astype(np.int32)


def test_worked_merge_values(orc):
    """Sec. 4.2 example: merge[0,0] = -2 for (3, -2) and merge[0,2] = 0 for (3, 0).
    A chain k - mk - t whose end sketches are unit vectors reads one merged bucket."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "merge_worked_example.txt")) if ln[0] != "#"]
    w = 3
    for a, b, i, j, want in ([int(v) for v in r] for r in rows):
        mk1 = np.zeros((1, w), np.int32)
        mk2 = np.zeros((1, w), np.int32)
        mk1[0, i] = a
        mk2[0, j] = b
        mk2[0, (j + 1) % w] = 9     # other buckets must not leak in
        k = np.zeros((1, w), np.int32)
        k[0, i] = 1
        t = np.zeros((1, w), np.int32)
        t[0, j] = 1
        # tables: 0 = k, 1 = mk, 2 = t; e0 = k-mk (mk's first join), e1 = mk-t
        sketches = [(k, mk1), (mk2, t)]
        for brute in (False, True):
            r = orc.estimate([0, 1], [1, 2], sketches, [1, 1, 1], 1, w, 0b111, brute=brute)
            assert r.rows == [want]


def test_merge_tie_keeps_the_first_sketch(orc):
    """The merge equation takes sk_mk1[i] when |sk_mk1[i]| <= |sk_mk2[j]|: on a tie in
    magnitude with opposite signs the first (lower edge id) sketch's value is kept."""
    w = 2
    k = np.array([[1, 0]], np.int32)
    t = np.array([[0, 1]], np.int32)
    for a, b in ((3, -3), (-3, 3), (0, 0), (-5, 5)):
        mk1 = np.array([[a, 7]], np.int32)
        mk2 = np.array([[7, b]], np.int32)
        r = orc.estimate([0, 1], [1, 2], [(k, mk1), (mk2, t)], [1, 1, 1], 1, w, 0b111)
        assert r.rows == [a]


def _merge2(s1, s2):
    """Merged 2-D sketch of Sec. 4.2: s1[i] where |s1[i]| <= |s2[j]|, else s2[j]."""
    a = np.abs(s1)[:, None] <= np.abs(s2)[None, :]
    return np.where(a, s1[:, None], s2[None, :]).astype(object)


def test_three_chain_equals_explicit_double_sum(orc):
    rng = np.random.default_rng(1)
    d, w = 3, 17
    k, mk1, mk2, t = (_sk(rng, d, w, -40, 41) for _ in range(4))
    sketches = [(k, mk1), (mk2, t)]
    r = orc.estimate([0, 1], [1, 2], sketches, [1, 1, 1], d, w, 0b111)
    for i in range(d):
        M = _merge2(mk1[i].astype(object), mk2[i].astype(object))
        want = int(np.dot(k[i].astype(object), M.dot(t[i].astype(object))))
        assert r.rows[i] == want


def test_two_way_is_inner_product_and_median(orc):
    rng = np.random.default_rng(2)
    for d in (1, 2, 5, 6):
        A, B = _sk(rng, d, 64, -1000, 1000), _sk(rng, d, 64, -1000, 1000)
        r = orc.estimate([0], [1], [(A, B)], [10, 20], d, 64, 0b11)
        want = [int(np.dot(A[i].astype(np.int64), B[i].astype(np.int64))) for i in range(d)]
        assert r.rows == want
        srt = sorted(want)
        med = srt[d // 2] if d % 2 else (srt[d // 2 - 1] + srt[d // 2]) / 2
        assert r.est == float(med)


def test_single_table_is_exact_count(orc):
    A = np.ones((3, 8), np.int32)
    r = orc.estimate([0], [1], [(A, A)], [123, 456], 3, 8, 0b10)
    assert r.rows == [456] * 3 and r.est == 456.0


GRAPHS = {
    "chain4": ([0, 1, 2], [1, 2, 3], 4),
    "star5": ([0, 0, 0, 0], [1, 2, 3, 4], 5),
    "triangle": ([0, 1, 0], [1, 2, 2], 3),
    "cycle4": ([0, 1, 2, 3], [1, 2, 3, 0], 4),
    "parallel": ([0, 0, 1], [1, 1, 2], 3),
    "tri+tail": ([0, 1, 2, 2], [1, 2, 0, 3], 4),
    "two_cycles": ([0, 1, 2, 0, 3], [1, 2, 0, 3, 1], 4),
    "k4": ([0, 0, 0, 1, 1, 2], [1, 2, 3, 2, 3, 3], 4),          # three independent cycles
    "triple_parallel": ([0, 0, 0, 1], [1, 1, 1, 2], 3),         # two, on one pair of tables
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_message_passing_equals_brute_force(orc, name):
    eu, ev, nt = GRAPHS[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    w = 3 if len(eu) >= 5 else 4
    d = 2
    for trial in range(3):
        lo, hi = (-3, 4) if trial < 2 else (0, 5)       # ties and zeros are frequent
        sketches = [(_sk(rng, d, w, lo, hi), _sk(rng, d, w, lo, hi)) for _ in eu]
        for mask in G.connected_subplans(nt, eu, ev, 2):
            a = orc.estimate(eu, ev, sketches, [1] * nt, d, w, mask)
            b = orc.estimate(eu, ev, sketches, [1] * nt, d, w, mask, brute=True)
            assert a.rows == b.rows, (mask, a.rows, b.rows)
            assert a.est == b.est


def test_brute_force_definition_on_a_tiny_star(orc):
    """Independent restatement of the definition for one star sub-plan (w=2)."""
    rng = np.random.default_rng(3)
    w, d = 2, 1
    c = [_sk(rng, d, w) for _ in range(3)]    # centre's sketches on e0, e1, e2
    leaf = [_sk(rng, d, w) for _ in range(3)]
    sketches = [(c[e], leaf[e]) for e in range(3)]
    r = orc.estimate([0, 0, 0], [1, 2, 3], sketches, [1] * 4, d, w, 0b1111, brute=True)
    tot = 0
    for j in itertools.product(range(w), repeat=3):
        vals = [int(c[e][0, j[e]]) for e in range(3)]
        m = min(range(3), key=lambda e: (abs(vals[e]), e))
        tot += vals[m] * int(leaf[0][0, j[0]]) * int(leaf[1][0, j[1]]) * int(leaf[2][0, j[2]])
    assert r.rows == [tot]


def test_big_values_promote_beyond_int128(orc):
    """A long chain of large counters exceeds 2^127; exact result vs Python integers."""
    n = 9
    eu, ev = list(range(n - 1)), list(range(1, n))
    w = 2
    big = np.full((1, w), 2_000_000_000, np.int32)
    sketches = [(big, big) for _ in eu]
    r = orc.estimate(eu, ev, sketches, [1] * n, 1, w, (1 << n) - 1)
    # all merged entries are 2e9 (ties keep the first): sum over 2^(n-1) assignments of 2e9^n
    want = (2_000_000_000 ** n) * (w ** (n - 1))
    assert r.rows == [want]
    assert r.est == float(want)
    # exact big integers round once, to nearest even
    for v in (want, -want, want + 1, (1 << 200) + (1 << 147), (1 << 200) + (1 << 147) + 1, 3 ** 150):
        assert orc.dec_to_double(v) == float(v)


def test_identity_hash_two_way_is_exact_join(orc):
    rng = np.random.default_rng(4)
    w = 512
    a = G.zipf_keys(rng, 3000, w, 1.0)
    b = G.zipf_keys(rng, 5000, w, 1.3)
    hp = np.zeros((1, 3, 6), np.uint64)
    hp[..., 0] = 1
    A, na = orc.build_sketch(G.Table("a", [a], [], [0], [0]), hp, 3, w)
    B, nb = orc.build_sketch(G.Table("b", [b], [], [0], [0]), hp, 3, w)
    r = orc.estimate([0], [1], [(A[0], B[0])], [na, nb], 3, w, 0b11)
    exact = orc.join2(a, b)
    assert r.rows == [exact] * 3
    assert exact == int(np.dot(np.bincount(a, minlength=w).astype(np.int64),
                               np.bincount(b, minlength=w).astype(np.int64)))


def test_identity_hash_merged_estimate_overestimates(orc):
    """Sec. 4.2 says merging is likely to overestimate; with identity hashes and
    non-negative counts min(f1[i], f2[j]) >= joint(i, j), so it provably does."""
    rng = np.random.default_rng(5)
    w = 64
    for trial in range(5):
        n = [400, 600, 500]
        k = G.zipf_keys(rng, n[0], w, 1.1)
        mk_a = G.zipf_keys(rng, n[1], w, 1.1)
        mk_b = G.zipf_keys(rng, n[1], w, 0.9)
        t = G.zipf_keys(rng, n[2], w, 1.2)
        hp = np.zeros((2, 1, 6), np.uint64)
        hp[..., 0] = 1
        K, _ = orc.build_sketch(G.Table("k", [k], [], [0], [0]), hp, 1, w)
        MK, _ = orc.build_sketch(G.Table("mk", [mk_a, mk_b], [], [0, 1], [0, 1]), hp, 1, w)
        T, _ = orc.build_sketch(G.Table("t", [t], [], [0], [1]), hp, 1, w)
        r = orc.estimate([0, 1], [1, 2], [(K[0], MK[0]), (MK[1], T[0])], n, 1, w, 0b111)
        exact = orc.join_brute([0, 1], [1, 2], n, [(k, mk_a), (mk_b, t)], 0b111)
        assert r.rows[0] >= exact


def test_join_brute_matches_join2(orc):
    rng = np.random.default_rng(6)
    a = rng.integers(0, 30, 200)
    b = rng.integers(0, 30, 300)
    assert orc.join_brute([0], [1], [200, 300], [(a, b)], 0b11) == orc.join2(a, b)
    assert orc.join2(a, b) == int(sum((a == v).sum() * (b == v).sum() for v in range(30)))


def test_unbiased_two_way_over_seeds(orc):
    """Sec. 3.2: the per-row Fast-AGMS inner product is unbiased.  Mean over 400 seeds
    (one row each) lies within 4 standard errors of the exact join size."""
    rng = np.random.default_rng(7)
    a = G.zipf_keys(rng, 2000, 5000, 1.0)
    b = G.zipf_keys(rng, 3000, 5000, 1.0)
    exact = orc.join2(a, b)
    vals = []
    M, w = 400, 64
    for s in range(M):
        hp = orc.hash_params(1000 + s, 1, 1)
        A, _ = orc.build_sketch(G.Table("a", [a], [], [0], [0]), hp, 1, w)
        B, _ = orc.build_sketch(G.Table("b", [b], [], [0], [0]), hp, 1, w)
        vals.append(orc.estimate([0], [1], [(A[0], B[0])], [0, 0], 1, w, 0b11).rows[0])
    vals = np.array(vals, np.float64)
    se = vals.std(ddof=1) / np.sqrt(M)
    assert abs(vals.mean() - exact) < 4 * se, (vals.mean(), exact, se)


def test_w1_reduces_to_agms_product(orc):
    """w = 1: every tuple lands in the single bucket; the estimate is the basic AGMS
    product of two sums of signs (Sec. 3.1)."""
    rng = np.random.default_rng(8)
    a = rng.integers(0, 100, 500)
    b = rng.integers(0, 100, 700)
    hp = orc.hash_params(5, 1, 3)
    A, _ = orc.build_sketch(G.Table("a", [a], [], [0], [0]), hp, 3, 1)
    B, _ = orc.build_sketch(G.Table("b", [b], [], [0], [0]), hp, 3, 1)
    r = orc.estimate([0], [1], [(A[0], B[0])], [0, 0], 3, 1, 0b11)
    for i in range(3):
        sa = int(orc.hash_eval(hp[0, i], 1, a)[1].sum())
        sb = int(orc.hash_eval(hp[0, i], 1, b)[1].sum())
        assert r.rows[i] == sa * sb


def test_rejects_disconnected_and_bad_masks(orc):
    A = np.ones((1, 4), np.int32)
    with pytest.raises(ValueError):
        orc.estimate([0], [1], [(A, A)], [1, 1, 1], 1, 4, 0b101)   # tables 0 and 2 not adjacent
    with pytest.raises(ValueError):
        orc.estimate([0], [1], [(A, A)], [1, 1], 1, 4, 0b100)      # bit beyond n_tables
    with pytest.raises(ValueError):
        orc.estimate([0], [1], [(A, A)], [1, 1], 1, 4, 0)


def _star_regrouped(centre, leaf, edges):
    """Row estimates of the star over leaf edges `edges` (ascending) by the regrouping the
    star lattice evaluates: for every edge a, every bucket r of the centre's sketch on a is the
    merged value where |s_a[r]| is the minimum (strictly below the lower-id edges, at most the
    higher-id ones), and the leaves b contribute their sums over the buckets allowed on their
    side: E = sum_a sum_r s_a[r] m_a[r] prod_{b != a} f_ab(|s_a[r]|)."""
    d, w = centre[edges[0]].shape
    rows = []
    for i in range(d):
        tot = 0
        for a in edges:
            for r in range(w):
                sa = int(centre[a][i, r])
                if sa == 0:
                    continue
                tau = abs(sa)
                term = sa * int(leaf[a][i, r])
                for b in edges:
                    if b == a:
                        continue
                    mag = np.abs(centre[b][i].astype(np.int64))
                    ok = mag > tau if b < a else mag >= tau
                    term *= int(leaf[b][i][ok].astype(np.int64).sum())
                tot += term
        rows.append(tot)
    return rows


def test_star_regrouping_equals_the_merged_contraction(orc):
    """The identity behind the star lattice: a star's row estimate is a sum over its leaf edges
    a and the centre's buckets r of s_a[r] m_a[r] times, per other leaf b, b's sketch summed
    over the buckets whose centre value keeps a the first minimum.  Checked on every leaf subset
    of 4- and 5-leaf stars with small values (many ties and zeros) against the oracle's merged
    contraction, and on the brute-force definition for one of them."""
    rng = np.random.default_rng(17)
    for n_leaves, w in ((4, 5), (5, 4)):
        eu, ev = [0] * n_leaves, list(range(1, n_leaves + 1))
        centre = [_sk(rng, 2, w, -3, 4) for _ in range(n_leaves)]
        leaf = [_sk(rng, 2, w, -3, 4) for _ in range(n_leaves)]
        sketches = [(centre[e], leaf[e]) for e in range(n_leaves)]
        surv = [1] * (n_leaves + 1)
        for bits in range(1, 1 << n_leaves):
            edges = [e for e in range(n_leaves) if (bits >> e) & 1]
            mask = 1 | sum(1 << (e + 1) for e in edges)
            want = orc.estimate(eu, ev, sketches, surv, 2, w, mask).rows
            assert _star_regrouped(centre, leaf, edges) == want, (n_leaves, bits)
        full = (1 << (n_leaves + 1)) - 1
        if n_leaves == 4:
            assert orc.estimate(eu, ev, sketches, surv, 2, w, full, brute=True).rows == \
                _star_regrouped(centre, leaf, list(range(n_leaves)))


def _merge2(x, y):
    """Merged 2-D sketch of a table with sketches x (lower edge id) and y (Sec. 4.2): the value
    of smaller magnitude, x on ties."""
    X, Y = np.meshgrid(x.astype(np.int64), y.astype(np.int64), indexing="ij")
    return np.where(np.abs(X) <= np.abs(Y), X, Y).astype(object)


def test_subtree_message_is_shared_by_the_sub_plans_containing_it(orc):
    """The reading behind cached messages: on the chain 0-1-2-3-4 (edge i joins i and i+1), the
    message of the subtree {2, 3, 4} over edge 1 (its merged sketches contracted with each other,
    one value per bucket of table 2's sketch on edge 1) is the same array inside every sub-plan
    that contains the subtree.  Built once from the definition, it gives the oracle's exact row
    estimates of both {1, 2, 3, 4} and {0, 1, 2, 3, 4}."""
    rng = np.random.default_rng(23)
    w, n = 5, 5
    eu, ev = list(range(n - 1)), list(range(1, n))
    # sk[t][e]: table t's sketch on edge e (one row)
    sk = {t: {} for t in range(n)}
    for e in range(n - 1):
        sk[e][e] = _sk(rng, 1, w, -4, 5)[0]
        sk[e + 1][e] = _sk(rng, 1, w, -4, 5)[0]
    sketches = [(sk[e][e][None, :], sk[e + 1][e][None, :]) for e in range(n - 1)]
    surv = [1] * n
    # message of {3, 4} over edge 2, then of {2, 3, 4} over edge 1, bucket by bucket
    m34 = np.array([sum(int(v) for v in _merge2(sk[3][2], sk[3][3])[j] * sk[4][3].astype(object))
                    for j in range(w)], dtype=object)
    m234 = np.array([sum(_merge2(sk[2][1], sk[2][2])[j] * m34) for j in range(w)], dtype=object)
    # {1, 2, 3, 4}: table 1 is a leaf on edge 1
    want1 = orc.estimate(eu, ev, sketches, surv, 1, w, 0b11110).rows[0]
    assert int(sum(sk[1][1].astype(object) * m234)) == want1
    # {0, 1, 2, 3, 4}: table 1 merges edges 0 and 1, table 0 is a leaf on edge 0
    m1 = _merge2(sk[1][0], sk[1][1])
    got = sum(int(sk[0][0][i]) * int(sum(m1[i] * m234)) for i in range(w))
    assert got == orc.estimate(eu, ev, sketches, surv, 1, w, 0b11111).rows[0]


@pytest.mark.parametrize("n,c,w", [(3, 2 ** 31 - 1, 2), (20, 2 ** 31 - 1, 2), (34, 2 ** 31 - 1, 2), (40, -(2 ** 31), 3),
                                   (12, 7, 5)])
def test_constant_chains_have_their_closed_form(orc, n, c, w):
    """A chain of n tables whose every counter is c: every merged value is c (ties keep it),
    so each of the w^(n-1) bucket assignments contributes c^n and E = c^n w^(n-1) exactly;
    the values reach 2^1300, far beyond int128 (and beyond a double), and the median of equal
    rows is that value rounded once."""
    eu, ev = list(range(n - 1)), list(range(1, n))
    sk = [tuple(np.full((2, w), c, np.int32) for _ in range(2)) for _ in range(n - 1)]
    r = orc.estimate(eu, ev, sk, np.ones(n, np.int64), 2, w, (1 << n) - 1)
    want = c ** n * w ** (n - 1)
    assert r.rows == [want, want]
    # one rounding to double; beyond the largest finite double that is an infinity
    assert r.est == (float(want) if abs(want) < 2 ** 1024 - 2 ** 970 else float("inf") * (1 if want > 0 else -1))


def test_constant_star_has_its_closed_form(orc):
    """A root with 12 leaves, every counter -(2^31 - 1): E = c^13 w^12."""
    k, c, w = 12, -(2 ** 31 - 1), 3
    eu, ev = [0] * k, list(range(1, k + 1))
    sk = [tuple(np.full((1, w), c, np.int32) for _ in range(2)) for _ in range(k)]
    r = orc.estimate(eu, ev, sk, np.ones(k + 1, np.int64), 1, w, (1 << (k + 1)) - 1)
    assert r.rows == [c ** (k + 1) * w ** k]


def test_join2_dense_equals_the_sort_merge_join(orc):
    """The histogram dot product over a known domain (the labeller of the learned
    combiner's training joins) equals the sort-merge join size, and brute force on small
    inputs: skewed keys, disjoint key sets, one shared key, empty sides, keys at both ends of
    the domain; a key outside the domain is refused."""
    rng = np.random.default_rng(12)
    cases = []
    for dom in (1, 7, 1000, 100_000):
        a = G.zipf_keys(rng, int(rng.integers(1, 5000)), dom, 1.3)
        b = G.zipf_keys(rng, int(rng.integers(1, 5000)), dom, 0.6)
        cases.append((a, b, dom))
    cases.append((np.arange(0, 100, 2, dtype=np.int32), np.arange(1, 100, 2, dtype=np.int32), 100))  # disjoint
    cases.append((np.full(3000, 41, np.int32), np.full(2000, 41, np.int32), 42))                    # one key
    cases.append((np.zeros(0, np.int32), np.arange(10, dtype=np.int32), 10))                        # empty
    cases.append((np.array([0, 9, 9], np.int32), np.array([9, 0, 0, 5], np.int32), 10))              # the ends
    for a, b, dom in cases:
        want = orc.join2(a, b)
        assert orc.join2_dense(a, b, dom) == want
        if a.size * b.size <= 10_000_000:
            assert want == int((a[:, None].astype(np.int64) == b[None, :]).sum())
    with pytest.raises(ValueError):
        orc.join2_dense(np.array([3, 10], np.int32), np.array([3], np.int32), 10)
