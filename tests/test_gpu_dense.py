"""Presence-bitmap columns of the batched build: a unique key column with a declared domain
in a table without predicates is marked in a bitmap by the counting pass and hashed in
domain order, its bucket and sign residues advanced by finite differences.  Counters and
survivors must equal the oracle's bit for bit: dense and sparse domains (up to four times
the rows), ragged domain ends, domains crossing 0, crossing p = 2^61 - 1 and at both ends
of int64, int32 slabs of several pairs, packed 16-bit slabs, odd widths, two sketches on
one column, a presence column beside counted and unique columns; and the run-time fallback
to the per-row path when the declaration does not hold (a repeated key, a key outside the
domain)."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1
PRIME = (1 << 61) - 1


def _build(wl, cfg=None):
    dw = P.DeviceWorkload(wl)
    for t in dw.tables:
        t.counters.fill_(77)  # stale contents must be overwritten
    dw.survivors.fill_(-3)
    dw.build_batched(cfg)
    torch.cuda.synchronize()
    dw.check_status()
    return dw


def _check(orc, wl, dw):
    surv = dw.survivors.cpu().numpy()
    for i, t in enumerate(wl.tables):
        c, n = orc.build_sketch(t, dw.hash_u64, wl.d, wl.w)
        assert int(surv[i]) == n, (t.name, int(surv[i]), n)
        got = dw.tables[i].counters.cpu().numpy()
        assert np.array_equal(got, c), (t.name, np.argwhere(got != c)[:5])


def _one(name, keys, lo, hi, d, w, sketches=1, seed=0):
    t = G.Table(name, [keys], [], [0] * sketches, list(range(sketches)), [("unique", lo, hi)])
    return G.Workload(name, [t], [0] * sketches, [0] * sketches, d, w, 4242 + seed, seed)


def _domain_keys(rng, lo, span, n, dtype=np.int64):
    """n distinct keys of [lo, lo + span), shuffled (Python ints: no int64 overflow)."""
    off = rng.choice(span, n, replace=False) if n < span else rng.permutation(span)
    return np.array([lo + int(o) for o in off], dtype=np.int64).astype(dtype)


@pytest.mark.parametrize("w,d", [(1024, 5), (65536, 3), (40001, 2), (3000, 4)])
def test_dense_permutation_matches_oracle(orc, w, d):
    """A permutation of a ragged domain [0, n) (n not a multiple of the 256-key run)."""
    rng = np.random.default_rng(w)
    n = 700_001
    wl = _one("pk", rng.permutation(n).astype(np.int32), 0, n, d, w, seed=w)
    dw = _build(wl)
    assert P.build_plan_info(dw)["n_presence"] == 1
    _check(orc, wl, dw)


@pytest.mark.parametrize("case", ["sparse", "neg", "prime", "top", "bottom", "offset"])
def test_dense_domain_edges(orc, case):
    """Sparse domains (a quarter of the keys present) and domains whose keys cross 0, cross
    the field prime, or sit at the ends of int64: consecutive keys keep consecutive
    residues, so the differences run through every crossing."""
    rng = np.random.default_rng(sum(map(ord, case)))
    n = 200_000
    if case == "sparse":
        lo, span = 12345, 4 * n
    elif case == "neg":
        lo, span = -n // 2 - 77, n + 300
    elif case == "prime":
        lo, span = PRIME - n // 2, n + 1000
    elif case == "top":
        lo, span = I64_MAX - (n + 500), n + 500
    elif case == "bottom":
        lo, span = I64_MIN, n + 33
    else:
        lo, span = (1 << 40) + 3, n + 256
    keys = _domain_keys(rng, lo, span, n)
    for w, d in ((65536, 2), (1024, 3)):
        wl = _one(case, keys, lo, lo + span, d, w, sketches=2, seed=len(case))
        dw = _build(wl)
        assert P.build_plan_info(dw)["n_presence"] == 1, case
        _check(orc, wl, dw)


def test_dense_fallback_when_the_declaration_fails(orc):
    """A repeated key, or a key outside the declared domain, makes the presence column
    inactive at run time: the row kernel hashes it, and the counters stay exact."""
    rng = np.random.default_rng(7)
    n = 300_000
    keys = rng.permutation(n).astype(np.int64)
    dup = keys.copy()
    dup[123] = dup[456]
    out = keys.copy()
    out[999] = n + 5
    for name, k in (("dup", dup), ("out", out)):
        for w in (1024, 65536):
            wl = _one(name, k, 0, n, 3, w)
            dw = _build(wl)
            assert P.build_plan_info(dw)["n_presence"] == 1
            _check(orc, wl, dw)


def test_dense_beside_counted_and_unique_columns(orc):
    """One plan with a presence column (two sketches), a foreign-key column counted per key
    (declared domain), a unique column of a filtered table (the unique-key kernel) and the
    same keys in an unfiltered table (a second presence column)."""
    rng = np.random.default_rng(11)
    n = 400_000
    pk = rng.permutation(n).astype(np.int64) - 1000
    fk = G.zipf_keys(rng, 3 * n, n, 1.1).astype(np.int64) - 1000
    p = rng.integers(0, 1000, 3 * n).astype(np.int32)
    pk2 = rng.permutation(n).astype(np.int32)
    q = rng.integers(0, 1000, n).astype(np.int32)
    tabs = [G.Table("D", [pk], [], [0, 0], [0, 1], [("unique", -1000, n - 1000)]),
            G.Table("F", [fk, p], [G.Pred(1, G.RANGE, 0, 400)], [0, 0], [0, 1], [("domain", -1000, n - 1000), None]),
            G.Table("E", [pk2, q], [G.Pred(1, G.RANGE, 100, 900)], [0], [2], [("unique", 0, n), None]),
            G.Table("E2", [pk2], [], [0], [2], [("unique", 0, n)])]
    for w in (2048, 65536):
        wl = G.Workload("mixed", tabs, [0, 0, 2], [1, 1, 3], 4, w, 99, 1)
        dw = _build(wl)
        info = P.build_plan_info(dw)
        assert info["n_presence"] == 2 and info["n_unique_slabs"] > 0
        _check(orc, wl, dw)
        # the same counters with the unique paths off
        off = _build(wl, K.cmp_build_cfg.make(unique=-1))
        assert P.build_plan_info(off)["n_presence"] == 0
        for x, y in zip(dw.tables, off.tables):
            assert torch.equal(x.counters, y.counters)


@pytest.mark.parametrize("w", [1024, 65536])
def test_dense_beside_the_second_counting_launch(orc, w):
    """Presence columns and counted columns without a unique-key kernel: the counting pass
    runs in two launches (the presence tables first), the dense kernel's first part beside
    the second one (256 threads, one CTA per SM) and the rest of each item's runs after it
    (512 threads).  Counters equal the oracle's; the plan has two more launches than the
    single pass."""
    rng = np.random.default_rng(w + 5)
    n = 300_000
    pk = rng.permutation(n).astype(np.int64)
    fk = G.zipf_keys(rng, 2_000_000, n, 1.2).astype(np.int64)
    p = rng.integers(0, 1000, 2_000_000).astype(np.int32)
    tabs = [G.Table("D", [pk], [], [0], [0], [("unique", 0, n)]),
            G.Table("F", [fk, p], [G.Pred(1, G.RANGE, 0, 300)], [0], [0], [("domain", 0, n), None])]
    wl = G.Workload("split", tabs, [0], [1], 4, w, 31, 2)
    dw = _build(wl)
    info = P.build_plan_info(dw)
    assert info["n_presence"] == 1 and info["n_unique_slabs"] == 0
    # zeroing, clearing, two counting launches, the presence check, dense in two parts, row
    # kernel, hashing
    assert info["launches"] == 9
    _check(orc, wl, dw)
