"""Pins of the row-sample oracle (Sec. 2 "Workflow": sketches over a sample).  The per-row
trial is SplitMix64 output r, checked against the oracle's C++ generator (itself pinned to
the published outputs); the threshold arithmetic, the kept fraction, nesting and seed
independence; and the scaled two-way estimate is unbiased over sample seeds."""
import numpy as np
import pytest

from paper_2102_02440_gb300 import datagen as G


@pytest.fixture(scope="module")
def smp(orc):
    from oracle import sample
    return sample


@pytest.mark.parametrize("seed", [0, 1234567, 2 ** 64 - 1, 0xC0FFEE])
def test_trials_are_the_splitmix64_stream(orc, smp, seed):
    assert [int(v) for v in smp.splitmix64_at(seed, np.arange(257))] == orc.splitmix64(seed, 257)
    # counter-based: any position on its own
    assert int(smp.splitmix64_at(seed, [1000])[0]) == orc.splitmix64(seed, 1001)[1000]


def test_thresholds(smp):
    assert smp.keep_threshold(1.0) == 0 and smp.keep_threshold(0.0) == 0
    assert smp.keep_threshold(0.5) == 1 << 63
    assert smp.keep_threshold(0.25) == 1 << 62
    assert smp.keep_threshold(2.0 ** -70) == 1
    assert smp.keep_threshold(0.1) == int(0.1 * 2.0 ** 64)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(ValueError):
            smp.keep_threshold(bad)


def test_kept_fraction_nesting_and_seeds(smp):
    n = 200_000
    for p in (0.5, 0.1, 0.01):
        m = smp.sample_mask(n, 42, smp.keep_threshold(p))
        assert abs(m.sum() - n * p) < 5 * np.sqrt(n * p * (1 - p))
    lo = smp.sample_mask(n, 42, smp.keep_threshold(0.1))
    hi = smp.sample_mask(n, 42, smp.keep_threshold(0.3))
    assert not (lo & ~hi).any()
    other = smp.sample_mask(n, 43, smp.keep_threshold(0.1))
    both = (lo & other).sum()
    assert abs(both - n * 0.01) < 5 * np.sqrt(n * 0.01)   # independent seeds: p^2 overlap
    assert smp.sample_mask(10, 5, 0).all()


def test_scale(smp):
    rates = [0.5, 1.0, 0.25, 0.0]
    assert smp.scale_of(0b1111, rates) == 8.0
    assert smp.scale_of(0b0010, rates) == 1.0
    assert smp.scale_of(0b0101, [0.1, 1.0, 0.3]) == (1.0 * (1.0 / 0.1)) * (1.0 / 0.3)


def test_sampled_table_keeps_order_and_predicates(smp):
    rng = np.random.default_rng(2)
    t = G.Table("t", [np.arange(1000, dtype=np.int32), G.uniform_col(rng, 1000, 0, 10)], [G.Pred(1, G.RANGE, 0, 5)],
                [0], [0])
    s = smp.sampled_table(t, 9, 0.2)
    m = smp.sample_mask(1000, 9, smp.keep_threshold(0.2))
    assert np.array_equal(s.cols[0], np.flatnonzero(m)) and s.preds is t.preds


def _two_tables(rng):
    r = G.Table("R", [G.zipf_keys(rng, 3000, 200, 1.0)], [], [0], [0])
    s = G.Table("S", [G.zipf_keys(rng, 4000, 200, 0.8)], [], [0], [0])
    return r, s


def _scaled_rows(orc, smp, r, s, hp, d, w, seed, p):
    rs = smp.sampled_table(r, 1000 + seed, p)
    ss = smp.sampled_table(s, 5000 + seed, p)
    cr, nr = orc.build_sketch(rs, hp, d, w)
    cs, ns = orc.build_sketch(ss, hp, d, w)
    est = orc.estimate([0], [1], [(cr[0], cs[0])], [nr, ns], d, w, 0b11)
    return [v * smp.scale_of(0b11, [p, p]) for v in est.rows]


def test_scaled_rows_are_unbiased_for_fixed_hashes(orc, smp):
    """With the hash functions fixed, the expected scaled row estimate over independent 30%
    samples is the full tables' row estimate (the sample enters the counters linearly)."""
    rng = np.random.default_rng(11)
    r, s = _two_tables(rng)
    d, w = 3, 64
    hp = orc.hash_params(77, 1, d)
    cr, nr = orc.build_sketch(r, hp, d, w)
    cs, ns = orc.build_sketch(s, hp, d, w)
    full = orc.estimate([0], [1], [(cr[0], cs[0])], [nr, ns], d, w, 0b11).rows
    vals = np.array([_scaled_rows(orc, smp, r, s, hp, d, w, seed, 0.3) for seed in range(300)], np.float64)
    se = vals.std(axis=0, ddof=1) / np.sqrt(vals.shape[0])
    assert (np.abs(vals.mean(axis=0) - np.array(full, np.float64)) < 4.5 * se).all()


def test_scaled_two_way_estimate_is_unbiased(orc, smp):
    """Over hash functions and samples together, the scaled row estimate is unbiased for
    the exact join size: 80 trials x 9 rows within 4.5 standard errors."""
    rng = np.random.default_rng(12)
    r, s = _two_tables(rng)
    exact = orc.join2(r.cols[0], s.cols[0])
    d, w = 9, 64
    vals = []
    for seed in range(80):
        vals += _scaled_rows(orc, smp, r, s, orc.hash_params(300 + seed, 1, d), d, w, seed, 0.3)
    vals = np.array(vals, np.float64)
    se = vals.std(ddof=1) / np.sqrt(vals.size)
    assert abs(vals.mean() - exact) < 4.5 * se
