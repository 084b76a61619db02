"""Pins of the oracle's push-down build (Sec. 2 "Partitioned query execution": only
tuples satisfying the selection update the sketch; Sec. 3.2: C[i][h_i(x)] += xi_i(x);
Sec. 2 "Sketches": mergeable by addition)."""
import os

import numpy as np
import pytest

from paper_2102_02440_gb300 import datagen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _filter_brute(t):
    keep = np.ones(t.n_rows, bool)
    for q in t.preds:
        v = t.cols[q.col].astype(np.int64)
        if q.op == G.RANGE:
            keep &= (q.lo <= v) & (v < q.hi)
        elif q.op == G.EQ:
            keep &= v == q.lo
        else:
            inb = (v >= 0) & (v < q.nbits)
            bits = np.zeros(t.n_rows, bool)
            vv = v[inb]
            bits[inb] = (q.bitmap[vv >> 5] >> (vv & 31).astype(np.uint32)) & 1 == 1
            keep &= bits
    return keep


def test_hand_example(orc):
    lines = [ln.split() for ln in open(os.path.join(GOLDEN, "hand_build.txt")) if ln.strip() and ln[0] != "#"]
    for blk in range(0, len(lines), 4):
        params = np.array([int(v) for v in lines[blk][1:]], np.uint64).reshape(1, 1, 6)
        w = int(lines[blk + 1][1])
        keys = np.array([int(v) for v in lines[blk + 2][1:]], np.int64)
        want = [int(v) for v in lines[blk + 3][1:]]
        t = G.Table("h", [keys], [], [0], [0])
        c, n = orc.build_sketch(t, params, 1, w)
        assert c[0, 0].tolist() == want
        assert n == len(keys)


def _tiny_table(rng, n, preds=True, int64=False):
    dt = np.int64 if int64 else np.int32
    key = G.zipf_keys(rng, n, 500, 1.2, dt)
    key2 = G.zipf_keys(rng, n, 50, 0.7, dt)
    p = G.uniform_col(rng, n, 0, 1000)
    code = G.uniform_col(rng, n, -5, 40)
    pr = []
    if preds:
        pr = [G.Pred(2, G.RANGE, 100, 700), G.Pred(3, G.IN, 0, 0, G.bitmap_of([0, 3, 5, 8, 13, 21, 34], 40), 40)]
    return G.Table("t", [key, key2, p, code], pr, [0, 1, 0], [0, 1, 2])


@pytest.mark.parametrize("int64", [False, True])
def test_survivors_and_sum_of_signs(orc, int64):
    rng = np.random.default_rng(5)
    t = _tiny_table(rng, 3000, True, int64)
    d, w = 5, 64
    hp = orc.hash_params(11, 3, d)
    c, n = orc.build_sketch(t, hp, d, w)
    keep = _filter_brute(t)
    assert n == int(keep.sum())
    # per row: sum of counters = sum of the survivors' signs; |counters| sum <= survivors
    for s in range(3):
        keys = t.cols[t.key_col[s]][keep].astype(np.int64)
        for i in range(d):
            b, sg = orc.hash_eval(hp[t.edge_id[s], i], w, keys)
            assert int(c[s, i].sum()) == int(sg.sum())
            want = np.zeros(w, np.int64)
            np.add.at(want, b, sg)
            assert np.array_equal(c[s, i], want)
        assert np.abs(c[s]).sum(axis=1).max() <= n


def test_linearity_partitions_merge_by_addition(orc):
    rng = np.random.default_rng(6)
    t = _tiny_table(rng, 5001)
    d, w = 3, 32
    hp = orc.hash_params(12, 3, d)
    whole, n = orc.build_sketch(t, hp, d, w)
    acc = (np.zeros_like(whole), np.zeros(1, np.int64))
    for lo, hi in ((0, 1234), (1234, 1235), (1235, 4000), (4000, 5001)):
        orc.build_sketch(t, hp, d, w, lo, hi, accumulate=acc)
    assert np.array_equal(acc[0], whole) and int(acc[1][0]) == n


def test_identity_hash_gives_exact_histogram(orc):
    # a=1, b=0, c*=0: h(x) = x for 0 <= x < w, xi = +1, so counters are the histogram
    rng = np.random.default_rng(7)
    w = 256
    keys = G.zipf_keys(rng, 10_000, w, 1.1)
    hp = np.zeros((1, 2, 6), np.uint64)
    hp[..., 0] = 1
    t = G.Table("t", [keys], [], [0], [0])
    c, n = orc.build_sketch(t, hp, 2, w)
    hist = np.bincount(keys, minlength=w)
    assert np.array_equal(c[0, 0], hist) and np.array_equal(c[0, 1], hist)


def test_int32_and_int64_keys_hash_identically(orc):
    rng = np.random.default_rng(8)
    k32 = G.uniform_col(rng, 4000, -(1 << 31), (1 << 31) - 1)
    hp = orc.hash_params(13, 1, 4)
    a, _ = orc.build_sketch(G.Table("a", [k32], [], [0], [0]), hp, 4, 128)
    b, _ = orc.build_sketch(G.Table("b", [k32.astype(np.int64)], [], [0], [0]), hp, 4, 128)
    assert np.array_equal(a, b)


def test_predicate_edge_cases(orc):
    v = np.array([-(1 << 31), -1, 0, 1, 299, 300, (1 << 31) - 1], np.int32)
    t = G.Table("p", [v], [G.Pred(0, G.RANGE, G.INT64_MIN, 300)], [0], [0])
    hp = orc.hash_params(1, 1, 1)
    assert orc.build_sketch(t, hp, 1, 8)[1] == 5
    t.preds = [G.Pred(0, G.EQ, 299)]
    assert orc.build_sketch(t, hp, 1, 8)[1] == 1
    t.preds = [G.Pred(0, G.IN, 0, 0, G.bitmap_of([0, 1, 31], 32), 32)]   # negatives and >= nbits excluded
    assert orc.build_sketch(t, hp, 1, 8)[1] == 2
    t.preds = [G.Pred(0, G.RANGE, 5, 5)]                                 # empty range
    c, n = orc.build_sketch(t, hp, 1, 8)
    assert n == 0 and not c.any()


def test_empty_table_and_rejections(orc):
    hp = orc.hash_params(1, 1, 2)
    t = G.Table("e", [np.zeros(0, np.int32)], [], [0], [0])
    c, n = orc.build_sketch(t, hp, 2, 16)
    assert n == 0 and not c.any()
    with pytest.raises(ValueError):
        orc.build_sketch(G.Table("bad", [np.zeros(3, np.int32)], [], [1], [0]), hp, 2, 16)
    with pytest.raises(ValueError):
        orc.build_sketch(G.Table("bad", [np.zeros(3, np.int32)], [], [0], [5]), hp, 2, 16)
