"""Host-side tests of the C ABI: the library loads, exports every symbol the header
declares, and rejects bad arguments before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def K():
    from paper_2102_02440_gb300 import build_lib, compass
    build_lib.build()
    return compass


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(cmp_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(K):
    L = K.lib()
    declared = _declared()
    assert len(declared) >= 7
    missing = [n for n in declared if getattr(L, n, None) is None]
    assert not missing, missing


def test_status_strings(K):
    assert K.status_str(0) == "ok"
    assert "invalid" in K.status_str(-1)
    assert K.lib().cmp_abi_version() == K.CMP_ABI_VERSION == 7


def test_hash_params_match_oracle_generator(K, orc):
    for seed, ne, d in ((0, 1, 1), (0xC0FFEE, 5, 11), (2**63 + 5, 3, 64)):
        assert np.array_equal(K.hash_params_u64(seed, ne, d), orc.hash_params(seed, ne, d))
    with pytest.raises(K.CompassError):
        K.cmp_hash_params(1, 1, 0)
    with pytest.raises(K.CompassError):
        K.cmp_hash_params(1, 1, 65)


def _desc(K, n_rows=10, ncols=1, preds=(), key_col=(0,), edge_id=(0,), dtype=0, flags=0, dom=(0, 0)):
    cols = (K.cmp_col * max(ncols, 1))(*[K.cmp_col(0x1000 * (i + 1), dtype, flags, dom[0], dom[1])
                                         for i in range(ncols)])
    pr = (K.cmp_pred * max(len(preds), 1))(*preds)
    kc = (C.c_int32 * max(len(key_col), 1))(*key_col)
    ei = (C.c_int32 * max(len(edge_id), 1))(*edge_id)
    t = K.cmp_table(n_rows, ncols, len(preds), len(key_col), 0, cols, pr, kc, ei)
    t._keep = (cols, pr, kc, ei)
    return t


@pytest.mark.parametrize("case", ["d0", "d65", "w0", "rows_neg", "rows_big", "bad_keycol", "bad_edge",
                                  "bad_dtype", "bad_pred_col", "bad_pred_op", "in_no_bitmap", "null_counters",
                                  "too_many_sketches", "bad_col_flags", "empty_domain"])
def test_build_rejects_bad_arguments(K, case):
    d, w, ne = 4, 64, 2
    t = _desc(K)
    if case == "d0":
        d = 0
    elif case == "d65":
        d = 65
    elif case == "w0":
        w = 0
    elif case == "rows_neg":
        t.n_rows = -1
    elif case == "rows_big":
        t.n_rows = 2 ** 31
    elif case == "bad_keycol":
        t = _desc(K, key_col=(3,))
    elif case == "bad_edge":
        t = _desc(K, edge_id=(2,))
    elif case == "bad_dtype":
        t = _desc(K, dtype=7)
    elif case == "bad_pred_col":
        t = _desc(K, preds=[K.cmp_pred(5, 0, 0, 1, None, 0)])
    elif case == "bad_pred_op":
        t = _desc(K, preds=[K.cmp_pred(0, 9, 0, 1, None, 0)])
    elif case == "in_no_bitmap":
        t = _desc(K, preds=[K.cmp_pred(0, 2, 0, 0, None, 100)])
    elif case == "too_many_sketches":
        t = _desc(K, key_col=tuple([0] * 17), edge_id=tuple([0] * 17))
    elif case == "bad_col_flags":
        t = _desc(K, flags=4)
    elif case == "empty_domain":
        t = _desc(K, flags=K.CMP_COL_DOMAIN, dom=(5, 5))
    counters = 0 if case == "null_counters" else 0x2000
    st = K.lib().cmp_sketch_build(C.byref(t), d, w, 0x3000, ne, counters, 0x4000, 0x5000, None, None)
    assert st == K.CMP_EINVAL


def test_build_rejects_bad_cfg(K):
    t = _desc(K)
    for cfg in (K.cmp_build_cfg.make(threads=48), K.cmp_build_cfg.make(tile_rows=100),
                K.cmp_build_cfg.make(mode=3), K.cmp_build_cfg.make(threads=128, tile_rows=4096, dedupe=1)):
        st = K.lib().cmp_sketch_build(C.byref(t), 4, 64, 0x3000, 2, 0x2000, 0x4000, 0x5000, C.byref(cfg), None)
        assert st == K.CMP_EINVAL


def test_column_declarations_plan_host_logic(K):
    """A declared domain sizes the count array to the domain (instead of the power of two
    at or above the row count); a unique column needs no count array at all, and the
    unique path can be switched off; bad unique settings are rejected."""
    n = 10_000_000
    plain = K.cmp_build_plan_bytes([_desc(K, n_rows=n)], 11, 1024, None)[1]
    assert plain >= (1 << 24) * 4                      # next power of two at or above 10M slots
    dom = K.cmp_build_plan_bytes([_desc(K, n_rows=n, flags=K.CMP_COL_DOMAIN, dom=(-50, 1000))], 11, 1024,
                                 None)[1]
    assert 1050 * 4 <= dom < 1 << 20
    wide = K.cmp_build_plan_bytes([_desc(K, n_rows=n, flags=K.CMP_COL_DOMAIN, dom=(0, 1 << 40))], 11, 1024,
                                  None)[1]
    assert wide == plain                               # a domain beyond 2^27 values is not used
    uniq = [_desc(K, n_rows=n, flags=K.CMP_COL_UNIQUE)]
    assert K.cmp_build_plan_bytes(uniq, 11, 1024, None)[1] == 0
    assert K.cmp_build_plan_bytes(uniq, 11, 65536, None)[1] == 0       # packed 16-bit slabs
    assert K.cmp_build_plan_bytes(uniq, 11, 1 << 18, None)[1] == plain  # too wide: aggregated instead
    assert K.cmp_build_plan_bytes(uniq, 11, 1024, K.cmp_build_cfg.make(unique=-1))[1] == plain
    for bad in (K.cmp_build_cfg.make(unique=2), K.cmp_build_cfg.make(unique=-2)):
        with pytest.raises(K.CompassError) as ei:
            K.cmp_build_plan_bytes(uniq, 11, 1024, bad)
        assert ei.value.status == K.CMP_EINVAL
    nb, _ = K.cmp_build_plan_bytes(uniq, 11, 1024, None)
    buf = np.zeros(nb, np.uint8)
    K.cmp_build_plan_encode(uniq, 11, 1024, 1, [0x2000], 0x4000, None, buf.ctypes.data, nb)


def test_presence_columns_plan_host_logic(K):
    """A unique column with a declared domain of at most four times its table's rows, in a
    table without predicates or sample, becomes a presence bitmap: one bit per domain key
    (whole 256-key runs) in the workspace, one more launch (the dense kernel), no unique-key
    slab.  A predicate, a wider domain, no domain, or the unique paths switched off leave it
    to the other paths."""
    n = 1_000_000
    flags = K.CMP_COL_UNIQUE | K.CMP_COL_DOMAIN

    def stats(tabs, cfg=None, w=1024):
        nb, wb = K.cmp_build_plan_bytes(tabs, 11, w, cfg)
        buf = np.zeros(nb, np.uint8)
        K.cmp_build_plan_encode(tabs, 11, w, 1, [0x2000] * len(tabs), 0x4000, cfg, buf.ctypes.data, nb)
        return K.cmp_build_plan_stats(buf.ctypes.data), wb

    dense, wb = stats([_desc(K, n_rows=n, flags=flags, dom=(5, 5 + 4 * n))])
    assert dense.n_presence == 1 and dense.n_agg == 1 and dense.n_unique_slabs == 0
    assert 4 * n // 8 <= wb < 4 * n // 8 + 4096
    ragged, wb2 = stats([_desc(K, n_rows=n, flags=flags, dom=(-7, n - 7 + 1))])
    assert ragged.n_presence == 1 and wb2 >= (n // 256 + 1) * 32
    # zeroing, clearing, counting, the presence check, the row kernel (the run-time fallback), the
    # dense kernel
    assert dense.launches == 6
    packed, _ = stats([_desc(K, n_rows=n, flags=flags, dom=(0, n))], w=65536)
    assert packed.n_presence == 1
    # with a counted table beside it: the counting pass in two launches (presence first), the
    # dense kernel in two parts (its share beside the second counting launch, then the rest)
    fk = _desc(K, n_rows=4 * n, flags=K.CMP_COL_DOMAIN, dom=(0, n))
    split, _ = stats([fk, _desc(K, n_rows=n, flags=flags, dom=(0, n))])
    assert split.n_presence == 1 and split.n_agg == 2 and split.launches == 9
    # a scan long enough to cover the whole walk (its bytes against the walk's key x row steps):
    # the dense kernel stays in one part beside it
    fk_long = _desc(K, n_rows=80 * n, flags=K.CMP_COL_DOMAIN, dom=(0, n))
    whole, _ = stats([fk_long, _desc(K, n_rows=n, flags=flags, dom=(0, n))])
    assert whole.n_presence == 1 and whole.launches == 8
    rng = K.cmp_pred(0, K.CMP_RANGE, 0, 100, None, 0)
    for t, cfg in ((_desc(K, n_rows=n, flags=flags, dom=(0, 4 * n + 1)), None),
                   (_desc(K, n_rows=n, flags=flags, dom=(0, n), preds=(rng,)), None),
                   (_desc(K, n_rows=n, flags=K.CMP_COL_UNIQUE), None),
                   (_desc(K, n_rows=n, flags=flags, dom=(0, n)), K.cmp_build_cfg.make(unique=-1))):
        st, _ = stats([t], cfg)
        assert st.n_presence == 0


def test_batched_plan_encoding_host_logic(K):
    """Plan sizing and encoding run on the host; the blob is self-describing."""
    tabs = [_desc(K, n_rows=n, key_col=(0, 0), edge_id=(0, 1)) for n in (0, 1, 5000, 10_000_000)]
    nb, wb = K.cmp_build_plan_bytes(tabs, 11, 1024, None)
    assert nb > 0
    # key aggregation (auto: tables of >= 2^18 rows): one count array for the 10M-row table
    assert wb >= 10_000_000 * 4
    assert K.cmp_build_plan_bytes(tabs, 11, 1024, K.cmp_build_cfg.make(aggregate=0))[1] == 0
    assert K.cmp_build_plan_bytes(tabs, 11, 1024, K.cmp_build_cfg.make(aggregate=1))[1] > wb  # also the 5000-row table
    for bad in (K.cmp_build_cfg.make(aggregate=1, dedupe=0), K.cmp_build_cfg.make(aggregate=2)):
        with pytest.raises(K.CompassError) as ei:
            K.cmp_build_plan_bytes(tabs, 11, 1024, bad)
        assert ei.value.status == K.CMP_EINVAL
    buf = np.zeros(nb, np.uint8)
    with pytest.raises(K.CompassError):
        K.cmp_build_plan_encode(tabs, 11, 1024, 2, [0x1000] * 4, 0x2000, None, buf.ctypes.data, nb - 16)
    with pytest.raises(K.CompassError):   # edge id 1 beyond n_edges = 1
        K.cmp_build_plan_encode(tabs, 11, 1024, 1, [0x1000] * 4, 0x2000, None, buf.ctypes.data, nb)
    K.cmp_build_plan_encode(tabs, 11, 1024, 2, [0x1000] * 4, 0x2000, None, buf.ctypes.data, nb)
    hdr = buf[:8].view(np.uint64)[0]
    assert hdr == 0x434D504255494C44
    # a workspace below the plan's requirement is rejected before anything is enqueued
    assert K.lib().cmp_sketch_build_batched(buf.ctypes.data, 0x1000, 0x2000, 0x4000, wb - 1, 0x3000,
                                            None) == K.CMP_EWORKSPACE
    assert K.lib().cmp_sketch_build_batched(buf.ctypes.data, 0x1000, 0x2000, None, 0, 0x3000,
                                            None) == K.CMP_EWORKSPACE
    # cmp_sketch_build_batched rejects a blob that is not a plan
    junk = np.zeros(nb, np.uint8)
    assert K.lib().cmp_sketch_build_batched(junk.ctypes.data, 0x1000, 0x2000, None, 0, 0x3000,
                                            None) == K.CMP_EINVAL


def _graph(K, eu, ev, nt):
    ne = len(eu)
    arr = lambda v: (C.c_int32 * max(ne, 1))(*v)
    ptrs = (C.c_void_p * max(2 * ne, 1))(*[0x10000 + 0x100 * i for i in range(2 * ne)])
    slots = (C.c_int32 * max(2 * ne, 1))(*([0] * (2 * ne)))
    g = K.cmp_graph(nt, ne, arr(eu), arr(ev), ptrs, ptrs, ptrs, ptrs, slots, 0x9000)
    g._keep = (ptrs, slots)
    return g


def test_estimate_plan_host_logic(K):
    """Planning is host-only: connectivity, cycle rank and sizes need no GPU."""
    tri = _graph(K, [0, 1, 0], [1, 2, 2], 3)
    pb, wb = K.cmp_estimate_plan_bytes([tri], 11, 4096, [0, 0, 0, 0], [0b111, 0b011, 0b001, 0b110])
    assert pb > 0 and wb > 0
    buf = np.zeros(pb, np.uint8)
    K.cmp_estimate_plan_encode([tri], 11, 4096, [0] * 4, [0b111, 0b011, 0b001, 0b110], buf.ctypes.data, pb)
    assert buf[:8].view(np.uint64)[0] == 0x434D504553544D54
    with pytest.raises(K.CompassError) as ei:     # 0 and 2 are adjacent (e2), 1 is not in the set: fine
        K.cmp_estimate_plan_bytes([_graph(K, [0, 1], [1, 2], 3)], 11, 64, [0], [0b101])
    assert ei.value.status == K.CMP_EINVAL        # chain 0-1-2 without 1 is disconnected
    k4 = _graph(K, [0, 0, 0, 1, 1, 2], [1, 2, 3, 2, 3, 3], 4)
    K.cmp_estimate_plan_bytes([k4], 5, 64, [0], [0b1111])   # three independent cycles: 64^3 values
    with pytest.raises(K.CompassError) as ei:
        K.cmp_estimate_plan_bytes([k4], 5, 2048, [0], [0b1111])
    assert ei.value.status == K.CMP_EUNSUPPORTED  # 2048^3 conditioning values exceed int32
    K.cmp_estimate_plan_bytes([k4], 5, 2048, [0], [0b0111])   # one cycle
    k5 = _graph(K, [0, 0, 0, 0, 1, 1, 1, 2, 2, 3], [1, 2, 3, 4, 2, 3, 4, 3, 4, 4], 5)
    with pytest.raises(K.CompassError) as ei:
        K.cmp_estimate_plan_bytes([k5], 5, 4, [0], [0b11111])
    assert ei.value.status == K.CMP_EUNSUPPORTED  # six independent cycles (at most three)
    K.cmp_estimate_plan_bytes([k5], 5, 4, [0], [0b01111])   # its K4: three
    for bad in ([0], [1 << 4], [0b10000]):
        with pytest.raises(K.CompassError):
            K.cmp_estimate_plan_bytes([k4], 5, 64, [0], bad)
    with pytest.raises(K.CompassError):
        K.cmp_estimate_plan_bytes([k4], 5, 64, [3], [0b11])    # graph index out of range
    with pytest.raises(K.CompassError):
        K.cmp_estimate_plan_bytes([_graph(K, [0], [0], 2)], 5, 64, [0], [0b1])   # self-loop
    junk = np.zeros(256, np.uint8)
    assert K.lib().cmp_estimate(junk.ctypes.data, 0x10, 0x10, 1 << 20, 0x10, None, None, None) == K.CMP_EINVAL


def test_estimate_plan_triangle_path_host_logic(K):
    """Sub-plans whose only cycle is a triangle (other tables leaves of it) are planned on
    the triangle path, which changes the workspace; trees, longer cycles and rows wider
    than 16384 are not; CMP_EST_GENERIC_ONLY turns it off; other flag bits are rejected."""
    g = _graph(K, [0, 1, 0, 0, 1, 3], [1, 2, 2, 3, 4, 5], 6)   # triangle 0-1-2, leaves 3, 4; 5 hangs off 3
    gen = K.cmp_estimate_cfg.make(flags=K.CMP_EST_GENERIC_ONLY)

    def ws(mask, w=4096, cfg=None):
        return K.cmp_estimate_plan_bytes([g], 11, w, [0], [mask], cfg)[1]

    for m in (0b000111, 0b001111, 0b011111):          # triangle plus leaves
        assert ws(m) != ws(m, cfg=gen)
    for m in (0b000011, 0b011011, 0b111011):          # trees
        assert ws(m) == ws(m, cfg=gen)
    assert ws(0b111111) == ws(0b111111, cfg=gen)      # table 5 is not a leaf of the triangle
    assert ws(0b000111, w=16385) == ws(0b000111, w=16385, cfg=gen)
    c4 = _graph(K, [0, 1, 2, 3], [1, 2, 3, 0], 4)
    assert (K.cmp_estimate_plan_bytes([c4], 5, 64, [0], [0b1111])[1] ==
            K.cmp_estimate_plan_bytes([c4], 5, 64, [0], [0b1111], gen)[1])
    with pytest.raises(K.CompassError) as ei:
        K.cmp_estimate_plan_bytes([g], 11, 64, [0], [0b111], K.cmp_estimate_cfg.make(flags=16))
    assert ei.value.status == K.CMP_EINVAL


def _plan_stats(K, graphs, d, w, sg, sm, flags=0):
    cfg = K.cmp_estimate_cfg.make(flags=flags)
    pb, wb = K.cmp_estimate_plan_bytes(graphs, d, w, sg, sm, cfg)
    buf = np.zeros(pb, np.uint8)
    K.cmp_estimate_plan_encode(graphs, d, w, sg, sm, buf.ctypes.data, pb, cfg)
    return K.cmp_estimate_plan_stats(buf.ctypes.data), wb


@pytest.mark.parametrize("n", [2, 3, 4, 5, 9, 17])
def test_estimate_plan_cached_messages_on_chains(K, n):
    """Cached subtree messages on the chain 0-1-...-(n-1) with every connected sub-plan.
    Each sub-path [i..j] is rooted at i and its child subtree is [i+1..j] over edge i.  The
    message of [a..j] (a >= 2, j > a) has two users, the sub-plan [a-1..j] and the message of
    [a-1..j], so (n-2)(n-3)/2 messages are cached, at levels j - a - 1 (n - 3 launches).  The
    operations fall from sum_L (n-L+1)(L-1) (every non-leaf table of every sub-plan) to one per
    sub-plan and cached message, plus one for each sub-plan [0..j] with j >= 2 (its child
    [1..j] has a single user and stays inline)."""
    from paper_2102_02440_gb300 import datagen as G
    g = _graph(K, list(range(n - 1)), list(range(1, n)), n)
    sm = G.connected_subplans(n, list(range(n - 1)), list(range(1, n)))
    sg = [0] * len(sm)
    d = 5
    plain, wb0 = _plan_stats(K, [g], d, 64, sg, sm)
    cached, wb1 = _plan_stats(K, [g], d, 64, sg, sm, K.CMP_EST_CACHE_MESSAGES)
    n_jobs = (n - 2) * (n - 3) // 2 if n >= 3 else 0
    assert plain.n_jobs == 0 and plain.n_levels == 0
    assert plain.n_ops == sum((n - L + 1) * (L - 1) for L in range(2, n + 1))
    assert cached.n_jobs == n_jobs and cached.n_job_items == n_jobs * d
    assert cached.n_levels == max(n - 3, 0)
    n_sub_multi = n * (n - 1) // 2
    assert cached.n_ops == n_sub_multi + max(n - 2, 0) + n_jobs
    assert cached.n_items == plain.n_items + n_jobs * d and cached.n_sub == plain.n_sub == len(sm)
    assert wb1 >= 16 * n_jobs * d * 64   # the cache: 16 bytes per bucket and row of every cached message


def test_estimate_plan_cached_messages_shapes(K):
    """Stars rooted at their centre cache nothing (every child is a leaf); a star whose centre
    is not the lowest id has one user per subtree and caches nothing either.  A cycle's
    cyclic sub-plan is never cached, its paths are.  Many graphs: messages of different
    graphs are distinct even on equal table sets."""
    from paper_2102_02440_gb300 import datagen as G
    for eu, ev, nt in (([0, 0, 0, 0], [1, 2, 3, 4], 5), ([2, 2, 2, 2], [0, 1, 3, 4], 5)):
        sm = G.connected_subplans(nt, eu, ev)
        st, _ = _plan_stats(K, [_graph(K, eu, ev, nt)], 3, 64, [0] * len(sm), sm, K.CMP_EST_CACHE_MESSAGES)
        assert st.n_jobs == 0 and st.n_levels == 0
    # cycle 0-1-2-3-4-0: arcs are chains whose lowest id may sit inside them
    eu, ev = [0, 1, 2, 3, 4], [1, 2, 3, 4, 0]
    sm = G.connected_subplans(5, eu, ev)
    c5 = _graph(K, eu, ev, 5)
    plain, _ = _plan_stats(K, [c5], 3, 64, [0] * len(sm), sm)
    cached, _ = _plan_stats(K, [c5], 3, 64, [0] * len(sm), sm, K.CMP_EST_CACHE_MESSAGES)
    assert cached.n_jobs > 0 and cached.n_ops < plain.n_ops
    only_cycle, _ = _plan_stats(K, [c5], 3, 64, [0], [0b11111], K.CMP_EST_CACHE_MESSAGES)
    assert only_cycle.n_jobs == 0
    two, _ = _plan_stats(K, [c5, c5], 3, 64, [0] * len(sm) + [1] * len(sm), sm + sm, K.CMP_EST_CACHE_MESSAGES)
    assert two.n_jobs == 2 * cached.n_jobs and two.n_ops == 2 * cached.n_ops
    with pytest.raises(K.CompassError):
        K.cmp_estimate_plan_stats(np.zeros(256, np.uint8).ctypes.data)


def test_estimate_plan_star_families(K):
    """CMP_EST_STAR_LATTICE host logic.  A star with centre 0 and K leaves asked for every
    leaf subset is one family of 2^K - 1 stars with K 2^(K-1) lattice entries per row; asked
    for its two-table sub-plans only it is too sparse (K 2^(K-1) > 2 sum |S|^2) and stays on
    the generic path; fewer than three leaf edges never form a family; a centre that is not
    the lowest id roots the sub-plans with a leaf, which are then no stars; chains have none."""
    from paper_2102_02440_gb300 import datagen as G
    d = 3
    for n_leaves in (3, 4, 8, 16):
        eu, ev = [0] * n_leaves, list(range(1, n_leaves + 1))
        g = _graph(K, eu, ev, n_leaves + 1)
        sm = G.connected_subplans(n_leaves + 1, eu, ev)
        st, wb = _plan_stats(K, [g], d, 64, [0] * len(sm), sm, K.CMP_EST_STAR_LATTICE)
        assert st.n_star == 1 and st.n_star_sub == 2 ** n_leaves - 1
        assert st.n_star_entries == d * n_leaves * 2 ** (n_leaves - 1)
        assert wb >= 17 * st.n_star_entries + 8 * d * n_leaves * 65
        plain, _ = _plan_stats(K, [g], d, 64, [0] * len(sm), sm)
        assert plain.n_star == 0 and st.n_ops < plain.n_ops and st.n_items < plain.n_items
        pairs = [m for m in sm if bin(m).count("1") == 2]
        sp, _ = _plan_stats(K, [g], d, 64, [0] * len(pairs), pairs, K.CMP_EST_STAR_LATTICE)
        assert sp.n_star == 0                              # K 2^(K-1) > 2 K
    two = _graph(K, [0, 0], [1, 2], 3)
    st, _ = _plan_stats(K, [two], d, 64, [0] * 3, [0b011, 0b101, 0b111], K.CMP_EST_STAR_LATTICE)
    assert st.n_star == 0
    c3 = _graph(K, [3, 3, 3, 3, 3], [0, 1, 2, 4, 5], 6)
    sm = G.connected_subplans(6, [3, 3, 3, 3, 3], [0, 1, 2, 4, 5])
    st, _ = _plan_stats(K, [c3], d, 64, [0] * len(sm), sm, K.CMP_EST_STAR_LATTICE)
    assert st.n_star == 0                          # rooted at 3 only without 0, 1, 2: two leaf edges
    ch = _graph(K, list(range(8)), list(range(1, 9)), 9)
    sm = G.connected_subplans(9, list(range(8)), list(range(1, 9)))
    st, _ = _plan_stats(K, [ch], d, 64, [0] * len(sm), sm, K.CMP_EST_STAR_LATTICE | K.CMP_EST_CACHE_MESSAGES)
    assert st.n_star == 0 and st.n_jobs == 21


def test_estimate_plan_reuse_flags_on_random_graphs(K):
    """Both reuse flags on random graphs with parallel edges and extra cycles, every connected
    sub-plan or a random subset of them: planning succeeds or fails exactly as without the
    flags; with them the sub-plan count is unchanged, operations never grow, and every
    sub-plan is a single table, a star of a family, or has its own items."""
    from paper_2102_02440_gb300 import datagen as G
    rng = np.random.default_rng(5)
    both = K.CMP_EST_CACHE_MESSAGES | K.CMP_EST_STAR_LATTICE
    for trial in range(12):
        nt = int(rng.integers(3, 9))
        eu, ev = [], []
        for t in range(1, nt):
            eu.append(int(rng.integers(0, t)))
            ev.append(t)
        for _ in range(int(rng.integers(0, 2))):
            u, v = rng.choice(nt, 2, replace=False)
            eu.append(int(u))
            ev.append(int(v))
        g = _graph(K, eu, ev, nt)
        sm = G.connected_subplans(nt, eu, ev)
        if trial % 2:
            sm = [m for m in sm if rng.random() < 0.5] or sm[:1]
        try:
            plain, _ = _plan_stats(K, [g], 3, 64, [0] * len(sm), sm)
        except K.CompassError as e:
            with pytest.raises(K.CompassError) as ei:
                _plan_stats(K, [g], 3, 64, [0] * len(sm), sm, both)
            assert ei.value.status == e.status
            continue
        reuse, _ = _plan_stats(K, [g], 3, 64, [0] * len(sm), sm, both)
        assert reuse.n_sub == plain.n_sub == len(sm)
        assert reuse.n_ops <= plain.n_ops and reuse.n_star_sub <= len(sm)
        assert reuse.n_job_items == 3 * reuse.n_jobs


def test_cross_ranks_multi_rejections(K):
    ks = (C.c_int32 * 2)(2, 17)
    e = (C.c_int32 * 19)(*range(19))
    assert K.lib().cmp_cross_ranks_multi(0x10, 0x10, 2, ks, e, 3, 64, 0x10, None) == K.CMP_EINVAL  # k > 16
    ks = (C.c_int32 * 2)(2, 1)
    assert K.lib().cmp_cross_ranks_multi(0x10, 0x10, 2, ks, e, 0, 64, 0x10, None) == K.CMP_EINVAL  # d < 1
    assert K.lib().cmp_cross_ranks_multi(None, 0x10, 2, ks, e, 3, 64, 0x10, None) == K.CMP_EINVAL
    assert K.lib().cmp_cross_ranks_multi(0x10, 0x10, 2, None, e, 3, 64, 0x10, None) == K.CMP_EINVAL
    assert K.lib().cmp_cross_ranks_multi(0x10, 0x10, 0, None, None, 3, 64, None, None) == K.CMP_OK  # nothing


def test_features_indexed_rejections(K):
    assert K.lib().cmp_mlp_features_indexed(0x10, 4, 0, 0x10, 0x10, 0x10, None) == K.CMP_EINVAL   # d < 1
    assert K.lib().cmp_mlp_features_indexed(0x10, 4, 11, 0x10, None, 0x10, None) == K.CMP_EINVAL  # no index
    assert K.lib().cmp_mlp_features_indexed(None, 0, 11, None, None, None, None) == K.CMP_OK       # nothing


def test_enumeration_plan_host_logic(K):
    """Enumeration plans are encoded on the host: edges, one estimate per sub-plan."""
    g = _graph(K, [0, 1], [1, 2], 3)
    pb, wb = K.cmp_enum_plan_bytes([g], [0, 0, 0], [0b011, 0b110, 0b111])
    assert pb > 0 and wb > 0
    buf = np.zeros(pb, np.uint8)
    K.cmp_enum_plan_encode([g], [0, 0, 0], [0b011, 0b110, 0b111], buf.ctypes.data, pb)
    for sg, sm in (([0, 0], [0b011, 0b011]),      # the same sub-plan twice
                   ([1], [0b011]),                # graph index out of range
                   ([0], [0b1000]),               # table beyond the graph
                   ([0], [0])):                   # empty sub-plan
        with pytest.raises(K.CompassError) as ei:
            K.cmp_enum_plan_bytes([g], sg, sm)
        assert ei.value.status == K.CMP_EINVAL
    with pytest.raises(K.CompassError):
        K.cmp_enum_plan_encode([g], [0, 0, 0], [0b011, 0b110, 0b111], buf.ctypes.data, pb - 8)
    bad = K.cmp_enum_cfg.make(max_plans=-2)
    assert K.lib().cmp_enumerate(buf.ctypes.data, 0x1000, 0x1000, C.byref(bad), 0x1000, wb, 0x1000, 0x1000, 0x1000,
                                 None, None) == K.CMP_EINVAL
    assert K.lib().cmp_enumerate(buf.ctypes.data, 0x1000, 0x1000, None, 0x1000, wb - 1, 0x1000, 0x1000, 0x1000,
                                 None, None) == K.CMP_EWORKSPACE


def test_presort_rejections(K):
    assert K.lib().cmp_presort(0x10, 4, 0, 0x10, 0x10, None, 0, None) == K.CMP_EINVAL
    assert K.lib().cmp_presort(0x10, 4, 1 << 15, 0x10, 0x10, None, 0, None) == K.CMP_EWORKSPACE
    assert K.cmp_presort_ws_bytes(4, 1 << 15) == 2 * 4 * (1 << 15) * 8
    assert K.cmp_presort_ws_bytes(1000, 65536) == 2 * 64 * 65536 * 8
    assert K.cmp_presort_ws_bytes(1000, 4096) == 0
    assert K.lib().cmp_presort(None, 4, 64, 0x10, 0x10, None, 0, None) == K.CMP_EINVAL


def test_partitioned_build_rejects_bad_arguments(K):
    """Host checks of cmp_part_build (nothing is launched)."""
    L = K.lib()

    def call(t, widths, ne=5, counters=0x2000, cfg=None):
        wa = (C.c_int32 * max(len(widths), 1))(*widths) if widths is not None else None
        return L.cmp_part_build(C.byref(t), 4, wa, 0x3000, ne, counters, 0x4000, C.byref(cfg) if cfg else None, None)

    two = _desc(K, ncols=2, key_col=(0, 1), edge_id=(0, 1))
    assert call(_desc(K, key_col=(0,) * 5, edge_id=(0, 1, 2, 3, 4)), [2] * 5) == K.CMP_EINVAL   # > 4 axes
    assert call(_desc(K, ncols=2, key_col=(0, 1), edge_id=(1, 1)), [4, 4]) == K.CMP_EINVAL      # repeated edge
    assert call(two, [0, 4]) == K.CMP_EINVAL
    assert call(two, [4, (1 << 20) + 1]) == K.CMP_EINVAL
    assert call(two, [65536, 65536]) == K.CMP_EINVAL                                             # > 2^31 - 1
    assert call(two, None) == K.CMP_EINVAL
    assert call(two, [4, 4], counters=0) == K.CMP_EINVAL
    assert call(two, [4, 4], ne=1) == K.CMP_EINVAL                                               # edge id >= n_edges
    for cfg in (K.cmp_part_build_cfg.make(threads=48), K.cmp_part_build_cfg.make(tile_rows=100),
                K.cmp_part_build_cfg.make(mode=3), K.cmp_part_build_cfg.make(rows_per_cta=-1)):
        assert call(two, [4, 4], cfg=cfg) == K.CMP_EINVAL
    # shared-memory mode with a tensor row larger than a CTA's shared memory
    assert call(two, [1 << 10, 1 << 10], cfg=K.cmp_part_build_cfg.make(mode=1)) == K.CMP_EINVAL


def test_partitioned_estimate_plan_host_logic(K):
    """Workspace of the contraction order and the tree checks (host only)."""
    j, keep = K.part_join([0, 1], [1, 2], [5, 7], [[0], [0, 1], [1]], [0x1000, 0x2000, 0x3000])
    # flags (256 B), table 1 contracted on its last axis with table 2: [3][5] int128 (256 B),
    # then the root with table 1's message: [3][1] (256 B)
    assert K.cmp_part_estimate_ws_bytes(j, 3) == 768
    j1, k1 = K.part_join([], [], [], [[]], [0x1000])
    assert K.cmp_part_estimate_ws_bytes(j1, 11) == 256
    # 4-axis centre as the root: four contractions, [d][w0 w1 w2] ... [d][1]
    j4, k4 = K.part_join([0, 0, 0, 0], [1, 2, 3, 4], [2, 3, 4, 5], [[0, 1, 2, 3], [0], [1], [2], [3]],
                         [0x1000 * (i + 1) for i in range(5)])
    per = [2 * 3 * 4, 2 * 3, 2, 1]
    assert K.cmp_part_estimate_ws_bytes(j4, 1) == 256 + sum(((16 * p + 255) // 256) * 256 for p in per)
    bad = [
        ([0, 1, 0], [1, 2, 2], [2, 2, 2], [[0, 2], [0, 1], [1, 2]]),    # a cycle (3 edges, 3 tables)
        ([0, 1], [1, 0], [2, 2], [[0, 1], [0, 1], []]),                 # not connected
        ([0, 1], [1, 2], [2, 2], [[0], [0, 0], [1]]),                   # repeated axis
        ([0, 1], [1, 2], [2, 2], [[1], [0, 1], [0]]),                   # axis not incident
        ([0, 1], [1, 2], [2, 2], [[0], [0], [1]]),                      # missing axis
        ([0, 1], [1, 2], [0, 2], [[0], [0, 1], [1]]),                   # width 0
        ([0, 1], [1, 1], [2, 2], [[0], [0, 1], [1]]),                   # self-loop
    ]
    for eu, ev, w, ax in bad:
        jb, kb = K.part_join(eu, ev, w, ax, [0x1000, 0x2000, 0x3000])
        with pytest.raises(K.CompassError):
            K.cmp_part_estimate_ws_bytes(jb, 3)
    jn, kn = K.part_join([0, 1], [1, 2], [5, 7], [[0], [0, 1], [1]], [0x1000, 0, 0x3000])
    with pytest.raises(K.CompassError):
        K.cmp_part_estimate_ws_bytes(jn, 3)
    for d in (0, 65):
        with pytest.raises(K.CompassError):
            K.cmp_part_estimate_ws_bytes(j, d)
    j5, k5 = K.part_join([0] * 5, [1, 2, 3, 4, 5], [2] * 5, [[0, 1, 2, 3, 4], [0], [1], [2], [3], [4]],
                         [0x1000] * 6)
    with pytest.raises(K.CompassError):
        K.cmp_part_estimate_ws_bytes(j5, 3)                              # > 4 axes
    # workspace too small / misaligned: rejected before any launch
    assert K.lib().cmp_part_estimate(C.byref(j), 3, 0x10000, 512, 0x2000, None, None, None) == K.CMP_EWORKSPACE
    assert K.lib().cmp_part_estimate(C.byref(j), 3, 0x10010, 768, 0x2000, None, None, None) == K.CMP_EINVAL


def test_sample_rate_rejections(K):
    """Row-sample rates outside [0, 1] (or NaN) are rejected on the host by the builds, the
    estimate plan and the partitioned estimate."""
    L = K.lib()
    for bad in (-0.5, 1.5, float("nan")):
        t = _desc(K)
        t.sample_rate = bad
        assert L.cmp_sketch_build(C.byref(t), 4, 64, 0x3000, 2, 0x2000, 0x4000, 0x5000, None, None) == K.CMP_EINVAL
        n, ws = C.c_size_t(0), C.c_size_t(0)
        assert L.cmp_build_plan_bytes((K.cmp_table * 1)(t), 1, 4, 64, None, C.byref(n), C.byref(ws)) == K.CMP_EINVAL
        wa = (C.c_int32 * 1)(8)
        assert L.cmp_part_build(C.byref(t), 4, wa, 0x3000, 2, 0x2000, 0x4000, None, None) == K.CMP_EINVAL
        j, keep = K.part_join([0], [1], [4], [[0], [0]], [0x1000, 0x2000], [0.5, bad])
        with pytest.raises(K.CompassError):
            K.cmp_part_estimate_ws_bytes(j, 3)
    j, keep = K.part_join([0], [1], [4], [[0], [0]], [0x1000, 0x2000], [0.5, 1.0])
    assert K.cmp_part_estimate_ws_bytes(j, 3) > 0


def test_estimate_plan_sample_rates(K):
    g = _graph(K, [0, 1], [1, 2], 3)
    rates = (C.c_double * 3)(0.5, 1.0, 0.25)
    g.sample_rate = rates
    pb, wb = K.cmp_estimate_plan_bytes([g], 5, 64, [0, 0], [0b111, 0b001])
    assert pb > 0
    for bad in (-1.0, 2.0, float("nan")):
        rates[1] = bad
        with pytest.raises(K.CompassError):
            K.cmp_estimate_plan_bytes([g], 5, 64, [0], [0b111])


def test_sorted_tables_rule():
    """Host rule of the tables whose sorted rows an estimate plan reads: the lowest table id
    of every multi-table sub-plan and every table joined to two or more others in one."""
    from paper_2102_02440_gb300 import datagen as G
    from paper_2102_02440_gb300 import pipeline as P
    chain = ([0, 1, 2, 3], [1, 2, 3, 4])
    assert P.sorted_tables(5, *chain, G.connected_subplans(5, *chain)) == {0, 1, 2, 3}
    star = ([0, 0, 0, 0], [1, 2, 3, 4])
    assert P.sorted_tables(5, *star, G.connected_subplans(5, *star)) == {0}
    back = ([4, 4, 4, 4], [0, 1, 2, 3])  # the centre has the highest id
    assert P.sorted_tables(5, *back, [0b10001, 0b10010]) == {0, 1}
    assert P.sorted_tables(5, *back, [0b10011]) == {0, 4}
    assert P.sorted_tables(5, *back, [0b00001, 0b10000]) == set()  # single tables read no sketch


def test_estimate_plan_items_of_split_roots_and_cycle_ranks(K):
    """Work items per sketch row: one for a tree; kRootSplit (8) for a tree whose only
    operation is a root with two or more inputs once w >= 16384 (a star's sorted positions
    in chunks), not for a two-table sub-plan; ceil(w^rho / chunk) for rho conditioned edges."""
    d = 5
    star = _graph(K, [0, 0, 0], [1, 2, 3], 4)
    for w, per_star in ((8192, 1), (16384, 8), (65536, 8)):
        st, _ = _plan_stats(K, [star], d, w, [0, 0, 0], [0b1111, 0b0111, 0b0011])
        assert st.n_items == d * (2 * per_star + 1), (w, st.n_items)
    chain = _graph(K, [0, 1], [1, 2], 3)   # rooted at table 0: two operations, never split
    st, _ = _plan_stats(K, [chain], d, 65536, [0], [0b111])
    assert st.n_items == d
    k4 = _graph(K, [0, 0, 0, 1, 1, 2], [1, 2, 3, 2, 3, 3], 4)
    for mask, rho in ((0b1111, 3), (0b0111, 1)):
        cfg = K.cmp_estimate_cfg.make(cond_chunk=1000, flags=K.CMP_EST_GENERIC_ONLY)
        pb, _ = K.cmp_estimate_plan_bytes([k4], d, 64, [0], [mask], cfg)
        buf = np.zeros(pb, np.uint8)
        K.cmp_estimate_plan_encode([k4], d, 64, [0], [mask], buf.ctypes.data, pb, cfg)
        st = K.cmp_estimate_plan_stats(buf.ctypes.data)
        assert st.n_items == d * -(-64 ** rho // 1000), (rho, st.n_items)
