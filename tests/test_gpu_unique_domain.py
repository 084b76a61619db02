"""The batched build's column declarations (cmp_col.flags): key columns declared unique
(hashed once per surviving row by the shared-memory slab kernel, int32 or packed 16-bit
counters) and key columns with a declared domain (count arrays sized to it, keys outside
it sending the column back to the per-row path).  Counters and survivor counts must equal
the oracle's bit for bit whether the declarations hold or not, in every launch shape,
with predicates, negative and int64 keys, and buckets whose 16-bit halves wrap many
times within one item."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(),
    dict(mode=1, pairs_per_slab=3, threads=256, tile_rows=512),
    dict(mode=2, threads=1024, tile_rows=4096),
]


def _build(wl, cfg, hints=True, hp=None):
    dw = P.DeviceWorkload(wl, hints=hints)
    if hp is not None:
        dw.hash_u64 = hp
        dw.hash_dev.copy_(torch.from_numpy(np.ascontiguousarray(hp).reshape(-1).view(np.int64)))
    for t in dw.tables:
        t.counters.fill_(77)  # stale contents must be overwritten
    dw.survivors.fill_(-3)
    dw.build_batched(cfg)
    torch.cuda.synchronize()
    dw.check_status()
    return dw


def _same(dw, ref):
    surv = dw.survivors.cpu().numpy()
    for i, (t, (c, n)) in enumerate(zip(dw.tables, ref)):
        assert int(surv[i]) == n, (t.name, int(surv[i]), n)
        if t.k:
            got = t.counters.cpu().numpy()
            assert np.array_equal(got, c), (t.name, np.argwhere(got != c)[:5])


def _workload(seed, w=512, d=5, n=300_000):
    rng = np.random.default_rng(seed)
    tabs, eu, ev = [], [], []

    def edge():
        eu.append(0)
        ev.append(0)
        return len(eu) - 1

    # primary keys: int32 permutation with a range predicate; negative int64 keys; a
    # unique column next to a foreign-key column in one table; a unique key column that
    # also carries the predicate
    pk = rng.permutation(n).astype(np.int32)
    p = rng.integers(0, 1000, n).astype(np.int32)
    tabs.append(G.Table("pk32", [pk, p], [G.Pred(1, G.RANGE, 100, 700)], [0, 0], [edge(), edge()],
                        [("unique", 0, n), None]))
    pk64 = rng.permutation(n).astype(np.int64) - (1 << 50)
    tabs.append(G.Table("pk64", [pk64], [], [0], [edge()], [("unique", -(1 << 50), -(1 << 50) + n)]))
    fk = G.zipf_keys(rng, n, 4000, 1.1)
    pk2 = (rng.permutation(n).astype(np.int64) * 3 + 5)
    tabs.append(G.Table("mixed", [fk, pk2], [], [0, 1, 1], [edge(), edge(), edge()],
                        [("domain", 0, 4000), ("unique", 5, 3 * n + 5)]))
    pk3 = rng.permutation(n).astype(np.int32)
    tabs.append(G.Table("pkpred", [pk3], [G.Pred(0, G.RANGE, 1000, 50_000)], [0], [edge()],
                        [("unique", 0, n)]))
    # declared domains that hold, that the surviving keys leave (run-time fallback), and a
    # domain declared on a column of negative keys
    fk2 = G.zipf_keys(rng, n, 2000, 1.0)
    tabs.append(G.Table("dom_ok", [fk2], [], [0], [edge()], [("domain", 0, 2000)]))
    fk3 = G.zipf_keys(rng, n, 3000, 1.0)
    tabs.append(G.Table("dom_bad", [fk3], [], [0], [edge()], [("domain", 0, 1000)]))
    fk4 = (G.zipf_keys(rng, n, 5000, 1.2).astype(np.int64) - 2500)
    tabs.append(G.Table("dom_neg", [fk4], [], [0], [edge()], [("domain", -2500, 2500)]))
    # a "unique" declaration that does not hold: repeated keys must still be counted
    dup = rng.integers(0, 50, n).astype(np.int32)
    tabs.append(G.Table("dup", [dup], [], [0], [edge()], [("unique", 0, 50)]))
    tabs.append(G.Table("empty", [np.zeros(0, np.int32)], [], [0], [edge()], [("unique", 0, 1)]))
    return G.Workload("declared", tabs, eu, ev, d, w, 777 + seed, seed)


@pytest.mark.parametrize("si", range(len(SHAPES)))
@pytest.mark.parametrize("w", [512, 65536])
def test_declared_columns_match_oracle(orc, si, w):
    if w > 16384 and SHAPES[si].get("mode") == 1:
        pytest.skip("shared-memory slabs of the row kernel hold at most 16384-bucket rows")
    wl = _workload(si, w=w, d=3)
    ref = [orc.build_sketch(t, P.DeviceWorkload(wl).hash_u64, wl.d, wl.w) for t in wl.tables]
    for cfg in (K.cmp_build_cfg.make(**SHAPES[si]), K.cmp_build_cfg.make(**SHAPES[si], aggregate=1),
                K.cmp_build_cfg.make(**SHAPES[si], unique=-1)):
        _same(_build(wl, cfg), ref)
    _same(_build(wl, K.cmp_build_cfg.make(**SHAPES[si]), hints=False), ref)


def test_unique_int32_slabs_of_many_pairs(orc):
    """w = 4096: 22 pairs of one unique column in int32 slabs of several pairs each."""
    rng = np.random.default_rng(3)
    n = 500_000
    pk = rng.permutation(n).astype(np.int32)
    p = rng.integers(0, 1000, n).astype(np.int32)
    t = G.Table("D", [pk, p], [G.Pred(1, G.RANGE, 0, 200)], [0, 0], [0, 1], [("unique", 0, n), None])
    wl = G.Workload("slabs", [t], [0, 0], [0, 0], 11, 4096, 99, 3)
    ref = [orc.build_sketch(t, P.DeviceWorkload(wl).hash_u64, wl.d, wl.w)]
    _same(_build(wl, None), ref)


def test_packed_halves_wrap_exactly(orc):
    """Identity buckets (a = 1, b = 0: h(x) = x mod w) and constant signs (+1 on row 0, -1
    on row 1): 40,000 keys congruent to 10 and 40,000 congruent to 11 mod w = 65536 land
    in the two halves of one shared-memory word within one item, so both halves wrap
    (carries into the high half, borrows below zero) many times; the rest of the 6M keys
    are distinct and spread."""
    w, n = 65536, 6_000_000
    rng = np.random.default_rng(11)
    k = np.arange(40_000, dtype=np.int64) * w
    keys = np.concatenate([k + 10, k + 11, (1 << 40) + rng.permutation(n - 80_000).astype(np.int64)])
    t = G.Table("U", [keys], [], [0], [0], [("unique", 0, 1 << 41)])
    wl = G.Workload("wrap", [t], [0], [0], 2, w, 5, 5)
    hp = np.zeros((1, 2, 6), np.uint64)
    hp[:, :, 0] = 1          # a = 1, b = 0
    hp[0, 1, 2] = 1          # row 1: c0 = 1, every sign -1
    ref = [orc.build_sketch(t, hp, wl.d, wl.w)]
    assert ref[0][0][0, 0, 10] >= 40_000 and ref[0][0][0, 1, 11] <= -40_000
    _same(_build(wl, None, hp=hp), ref)
    _same(_build(wl, K.cmp_build_cfg.make(unique=-1), hp=hp), ref)


def test_odd_width_packed_last_half(orc):
    """w = 40001 (odd, packed): the last word's high half has no bucket."""
    wl = _workload(21, w=40001, d=2, n=200_000)
    ref = [orc.build_sketch(t, P.DeviceWorkload(wl).hash_u64, wl.d, wl.w) for t in wl.tables]
    _same(_build(wl, None), ref)


def test_five_table_declarations_equal_plain_build(orc):
    """The benchmark's tables at 5% scale with and without their declarations."""
    wl = G.five_table(scale=0.05, w=4096)
    a = _build(wl, None)
    b = _build(wl, None, hints=False)
    for x, y in zip(a.tables, b.tables):
        assert torch.equal(x.counters, y.counters)
    assert torch.equal(a.survivors, b.survivors)
    for i in (2, 3):  # D1 (unique key, range predicate), D2 (unique key, point predicate)
        ref = orc.build_sketch(wl.tables[i], a.hash_u64, wl.d, wl.w)
        assert np.array_equal(a.tables[i].counters.cpu().numpy(), ref[0])
        assert int(a.survivors[i].item()) == ref[1]


@pytest.mark.parametrize("dom", [(0, 1), (-(1 << 62), 1 << 62)])
@pytest.mark.parametrize("w", [65536, 40001, 4096])
def test_unique_extreme_keys(orc, w, dom):
    """int64 keys at the ends of the field and of int64 (0, -1, p - 1, p, p + 1, -p,
    INT64_MIN, INT64_MAX, 2^31 - 1, 2^31, ...) in a unique column, mixed with random keys,
    so that both the small-key and the general arithmetic run in the same warps.  With the
    domain [0, 1) the column is a presence column whose keys leave the domain (the per-row
    fallback); with the domain of 2^63 keys it goes to the unique-key kernel."""
    p = (1 << 61) - 1
    ext = [0, 1, -1, p - 1, p, p + 1, -p, -p - 1, 2 * p, 2 * p + 1, (1 << 31) - 1, 1 << 31, -(1 << 31),
           (1 << 62) + 3, -(1 << 63), (1 << 63) - 1, (1 << 63) - 2, -(1 << 63) + 1]
    rng = np.random.default_rng(w)
    rand = rng.choice(np.arange(1 << 40, (1 << 40) + 10_000_000, dtype=np.int64), 200_000, replace=False)
    small = rng.permutation(100_000).astype(np.int64) + 10
    keys = np.concatenate([np.array(ext, np.int64), rand, small])
    rng.shuffle(keys)
    t = G.Table("X", [keys], [], [0, 0], [0, 1], [("unique", dom[0], dom[1])])
    wl = G.Workload("extreme", [t], [0, 0], [0, 0], 5, w, 31, 1)
    ref = [orc.build_sketch(t, P.DeviceWorkload(wl).hash_u64, wl.d, wl.w)]
    _same(_build(wl, None), ref)
