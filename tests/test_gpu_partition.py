"""GPU parity of the partitioned sketches (Sec. 4.1).  cmp_part_build against the oracle's
build, bit for bit: 0 to 4 axes, shared-memory and global modes, several row groups,
power-of-two and other widths, int32 / int64 / negative / wide keys, every predicate kind,
empty tables and ragged tiles.  cmp_part_estimate against the oracle's exact contraction:
random trees on host-drawn tensors, both contraction forms and team sizes, and the int128
range rule.  Then the k - mk - t chain of the five-table workload end to end, and at full
size in the benchmark's two width configurations (sampled rows)."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def part(orc):
    from oracle import partition
    return partition


def _hash_dev(hp):
    return torch.from_numpy(np.ascontiguousarray(hp, np.uint64).reshape(-1).view(np.int64)).cuda()


def _gpu_build(t, hp, d, widths, cfg=None):
    dt = P.DeviceTable(t, d, 1, torch.device("cuda"))
    size = int(np.prod(widths)) if widths else 1
    out = torch.full((d, size), 7, dtype=torch.int32, device="cuda")   # overwritten by the build
    surv = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    hd = _hash_dev(hp)
    K.cmp_part_build(dt.desc, d, list(widths), hd.data_ptr(), hp.shape[0], out.data_ptr(), surv.data_ptr(), cfg,
                     K.stream_handle())
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(surv.item())


def _table(rng, n, k, dom, int64=False, neg=False, preds=True, wide=False):
    dt = np.int64 if int64 or wide else np.int32
    cols = []
    for _ in range(k):
        c = G.zipf_keys(rng, n, dom, float(rng.uniform(0.5, 1.4)), dt)
        if neg:
            c = (c - dom // 2).astype(dt)
        if wide:   # keys on both sides of 2^31: warps mix the narrow and the full hash path
            c = (c.astype(np.int64) * 7919 + np.where(rng.random(n) < 0.5, 0, 1 << 40)).astype(np.int64)
        cols.append(c)
    cols.append(G.uniform_col(rng, n, 0, 1000))
    cols.append(G.uniform_col(rng, n, -5, 40))
    cols.append(G.uniform_col(rng, n, 0, 9, np.int64))
    pr = []
    if preds:
        pr = [G.Pred(k, G.RANGE, 50, 900), G.Pred(k + 1, G.IN, 0, 0, G.bitmap_of([0, 1, 3, 7, 11, 31, 32], 40), 40),
              G.Pred(k + 2, G.EQ, 4, 0)] if rng.random() < 0.5 else [G.Pred(k, G.RANGE, 0, 700)]
    return G.Table("t", cols, pr, list(range(k)), list(range(k)))


BUILD_CASES = [  # seed, rows, widths, d, int64, neg, wide, preds, cfg
    (0, 1000, [], 3, False, False, False, True, None),
    (1, 5000, [64], 5, False, False, False, True, None),
    (2, 5000, [100], 4, True, True, False, True, dict(mode=2)),
    (3, 20000, [64, 64], 11, False, False, False, False, None),
    (4, 20000, [37, 53], 11, True, False, False, True, dict(mode=1)),
    (5, 20000, [64, 64], 11, False, False, False, True, dict(mode=2)),
    (6, 30001, [8, 16, 4], 7, False, True, False, True, None),
    (7, 30001, [5, 7, 9], 7, True, True, False, True, dict(mode=2, rows_per_cta=2)),
    (8, 12345, [4, 4, 4, 4], 3, False, False, False, True, None),
    (9, 12345, [3, 5, 2, 7], 3, True, True, False, False, dict(mode=1, rows_per_cta=1)),
    (10, 0, [8, 8], 3, False, False, False, True, None),
    (11, 70000, [512, 512], 2, False, False, False, True, None),
    (12, 40000, [16, 32], 11, False, False, True, True, dict(mode=1, rows_per_cta=3)),
    (13, 9999, [48, 48], 5, False, False, False, True, dict(threads=64, tile_rows=128)),
    (14, 9999, [1], 2, False, False, False, True, None),
    (15, 3000, [1 << 20], 2, False, False, False, True, None),
    (16, 25000, [2048, 1024], 1, True, False, True, True, None),
]


@pytest.mark.parametrize("seed,n,widths,d,int64,neg,wide,preds,cfg", BUILD_CASES)
def test_build_matches_oracle(part, orc, seed, n, widths, d, int64, neg, wide, preds, cfg):
    rng = np.random.default_rng(seed)
    t = _table(rng, n, len(widths), 300, int64, neg, preds, wide)
    hp = orc.hash_params(100 + seed, max(len(widths), 1), d)
    want, n_want = part.build_partitioned(t, hp, d, widths)
    got, n_got = _gpu_build(t, hp, d, widths, K.cmp_part_build_cfg.make(**cfg) if cfg else None)
    assert n_got == n_want
    assert np.array_equal(got, want)


def test_launch_shapes_give_identical_tensors(orc):
    rng = np.random.default_rng(30)
    t = _table(rng, 50000, 2, 2000)
    hp = orc.hash_params(7, 2, 11)
    ref, _ = _gpu_build(t, hp, 11, [64, 64])
    for cfg in (dict(mode=1, rows_per_cta=4), dict(mode=2), dict(mode=2, rows_per_cta=1, ctas_per_sm=1),
                dict(threads=256, tile_rows=1024), dict(mode=1, ctas_per_sm=2, rows_per_cta=2)):
        got, _ = _gpu_build(t, hp, 11, [64, 64], K.cmp_part_build_cfg.make(**cfg))
        assert np.array_equal(got, ref), cfg


def test_one_axis_equals_the_1d_build(orc):
    rng = np.random.default_rng(31)
    t = _table(rng, 40000, 3, 5000, int64=True)
    hp = orc.hash_params(9, 3, 5)
    dt = P.DeviceTable(t, 5, 1000, torch.device("cuda"))
    surv = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hd = _hash_dev(hp)
    K.cmp_sketch_build(dt.desc, 5, 1000, hd.data_ptr(), 3, dt.counters.data_ptr(), surv.data_ptr(), st.data_ptr(),
                       None, K.stream_handle())
    torch.cuda.synchronize()
    full = dt.counters.cpu().numpy()
    for s in range(3):
        ts = G.Table("t", t.cols, t.preds, [t.key_col[s]], [t.edge_id[s]])
        got, n = _gpu_build(ts, hp, 5, [1000])
        assert np.array_equal(got, full[s]) and n == int(surv.item())


# ------------------------------------------------------------------ estimate

def _tree(rng, nt):
    eu, ev = [], []
    for t in range(1, nt):
        eu.append(int(rng.integers(0, t)))
        ev.append(t)
    perm = rng.permutation(nt - 1)
    eu, ev = [eu[i] for i in perm], [ev[i] for i in perm]
    axes = []
    for t in range(nt):
        inc = [e for e in range(len(eu)) if t in (eu[e], ev[e])]
        axes.append([inc[i] for i in rng.permutation(len(inc))])
    return eu, ev, axes


def _run_estimate(eu, ev, widths, axes, host_tensors, d):
    dev = [torch.from_numpy(np.ascontiguousarray(x, np.int32)).cuda() for x in host_tensors]
    j, keep = K.part_join(eu, ev, widths, axes, [x.data_ptr() for x in dev])
    nb = K.cmp_part_estimate_ws_bytes(j, d)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    est = torch.empty(1, dtype=torch.float64, device="cuda")
    row = torch.empty((d, 2), dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    K.cmp_part_estimate(j, d, ws.data_ptr(), nb, est.data_ptr(), row.data_ptr(), st.data_ptr(), K.stream_handle())
    torch.cuda.synchronize()
    r = row.cpu().numpy()
    rows = [int(r[i, 1]) * (1 << 64) + int(np.uint64(r[i, 0])) for i in range(d)]
    return rows, float(est.item()), int(st.item())


def _check(part, eu, ev, widths, axes, tensors, d):
    rows, est, st = _run_estimate(eu, ev, widths, axes, tensors, d)
    ref, oor = part.contract_seq(eu, ev, widths, axes, tensors, d)
    for i in range(d):
        if not oor[i]:
            assert rows[i] == ref[i], i
    if any(oor):
        assert st == K.CMP_EOVERFLOW and np.isnan(est)
    else:
        assert st == 0 and est == part.median_to_double(ref)
    return oor


EST_CASES = [  # seed, tables, max width, value bound, d
    (0, 1, 1, 1000, 3), (1, 2, 50, 1000, 5), (2, 3, 40, 2 ** 31 - 1, 4), (3, 5, 6, 100, 3),
    (4, 6, 4, 2 ** 31 - 1, 7), (5, 4, 30, 10, 2), (6, 7, 3, 5, 6), (7, 5, 9, 2 ** 20, 11), (8, 3, 64, 1, 1),
]


@pytest.mark.parametrize("seed,nt,wmax,vmax,d", EST_CASES)
def test_estimate_matches_oracle_on_random_trees(part, seed, nt, wmax, vmax, d):
    rng = np.random.default_rng(seed)
    eu, ev, axes = _tree(rng, nt)
    widths = [int(rng.integers(1, wmax + 1)) for _ in eu]
    tensors = []
    for ax in axes:
        size = int(np.prod([widths[e] for e in ax])) if ax else 1
        x = rng.integers(-vmax - (1 if vmax == 2 ** 31 - 1 else 0), vmax + 1, size=(d, size))
        x[rng.random(x.shape) < 0.2] = 0
        tensors.append(x)
    _check(part, eu, ev, widths, axes, tensors, d)


@pytest.mark.parametrize("shape", ["dot_warp", "dot_warp_unaligned", "dot_cta", "col", "col_narrow", "col_wide_in"])
def test_contraction_forms(part, shape):
    """One launch shape each: B == 1 with a warp per output (vector loads or not), B == 1 with
    a CTA per output, B > 1 with full and partial 32-wide column blocks, int128 inputs."""
    rng = np.random.default_rng(sum(map(ord, shape)))
    d = 3
    if shape in ("dot_warp", "dot_warp_unaligned"):      # table 1 [3000 (parent), w (child)]
        w = 12 if shape == "dot_warp" else 13
        eu, ev, widths, axes = [0, 1], [1, 2], [3000, w], [[0], [0, 1], [1]]
    elif shape == "dot_cta":                              # root [5000] . leaf [5000]
        eu, ev, widths, axes = [0], [1], [5000], [[0], [0]]
    elif shape == "col":                                  # table 1 [w (child), 100 (parent)]
        eu, ev, widths, axes = [0, 1], [1, 2], [100, 40], [[0], [1, 0], [1]]
    elif shape == "col_narrow":                           # B = 5 < 32
        eu, ev, widths, axes = [0, 1], [1, 2], [5, 300], [[0], [1, 0], [1]]
    else:                                                 # chain of 2-axis tables: int128 messages
        eu, ev, widths, axes = [0, 1, 2], [1, 2, 3], [70, 33, 50], [[0], [1, 0], [2, 1], [2]]
    lim = 2 ** 20 if shape == "col_wide_in" else 2 ** 31    # four tables: keep every row inside int128
    tensors = []
    for ax in axes:
        size = int(np.prod([widths[e] for e in ax]))
        tensors.append(rng.integers(-lim, lim, size=(d, size)))
    oor = _check(part, eu, ev, widths, axes, tensors, d)
    assert not any(oor)


@pytest.mark.parametrize("rows,w,d", [(1300, 1500, 2), (2500, 1024, 1), (1220, 4100, 2)])
def test_bulk_streamed_rows(part, rows, w, d):
    """Long int32 rows of the middle table streamed through shared memory by bulk copies
    (at least 16 rows per SM): row lengths that are and are not whole 4096-byte chunks, and
    output counts that do not divide evenly among the warps."""
    rng = np.random.default_rng(rows + w)
    eu, ev, widths, axes = [0, 1], [1, 2], [rows, w], [[0], [0, 1], [1]]
    tensors = [rng.integers(-2 ** 31, 2 ** 31, size=(d, rows)), rng.integers(-2 ** 31, 2 ** 31, size=(d, rows * w)),
               rng.integers(-2 ** 31, 2 ** 31, size=(d, w))]
    assert not any(_check(part, eu, ev, widths, axes, tensors, d))


def test_out_of_range_rows(part):
    """The oracle's range rule on the device: a product beyond int128 with a zero sum, a sum
    beyond int128 of in-range products, and an in-range row."""
    big = (1 << 31) - 1
    eu, ev = [0, 1, 2], [1, 2, 3]
    axes = [[0], [0, 1], [1, 2], [2]]
    widths = [2, 8, 2]
    d = 3
    tensors = [np.ones((d, 2), np.int64), np.ones((d, 16), np.int64), np.ones((d, 16), np.int64),
               np.ones((d, 2), np.int64)]
    for t in (1, 2, 3):
        tensors[t][0] = big
        tensors[t][1] = big
    tensors[0][0] = [big, -big]
    tensors[0][1] = [1 << 30, 1 << 30]
    rows, est, st = _run_estimate(eu, ev, widths, axes, tensors, d)
    assert st == K.CMP_EOVERFLOW and np.isnan(est) and rows[2] == 32


def test_large_chain_row(part):
    """A [2048][2048] middle tensor (one sketch row): the streaming dot form at scale."""
    rng = np.random.default_rng(40)
    eu, ev, widths, axes = [0, 1], [1, 2], [2048, 2048], [[0], [0, 1], [1]]
    tensors = [rng.integers(-3000, 3000, size=(1, 2048)), rng.integers(-2 ** 31, 2 ** 31, size=(1, 2048 * 2048)),
               rng.integers(-2 ** 20, 2 ** 20, size=(1, 2048))]
    _check(part, eu, ev, widths, axes, tensors, 1)


# ----------------------------------------------------------- chain end to end

def _oracle_chain(orc, part, wl, widths, sel_rows):
    hp = orc.hash_params(wl.hash_seed, wl.n_edges, wl.d)[:, sel_rows, :]
    out = []
    for t in (3, 1, 2):
        src = wl.tables[t]
        sel = [s for s, e in enumerate(src.edge_id) if e in (0, 1)]
        tt = G.Table(src.name, src.cols, src.preds, [src.key_col[s] for s in sel], [src.edge_id[s] for s in sel])
        x, n = part.build_partitioned(tt, hp, len(sel_rows), [widths[src.edge_id[s]] for s in sel])
        out.append((x, n))
    return out


@pytest.mark.parametrize("scale,widths", [(0.02, [64, 64]), (0.02, [256, 128]), (1.0, [64, 64])])
def test_five_table_chain_matches_oracle(orc, part, scale, widths):
    wl = G.five_table(scale=scale, w=4096)
    pj = P.PartitionedJoin(wl, [3, 1, 2], [0, 1], widths)
    pj.build()
    pj.estimate()
    torch.cuda.synchronize()
    ref = _oracle_chain(orc, part, wl, widths, list(range(wl.d)))
    for i, (x, n) in enumerate(ref):
        assert np.array_equal(pj.tensors[i].cpu().numpy(), x)
        assert int(pj.survivors[i].item()) == n
    rows, oor = part.contract_seq([0, 1], [1, 2], widths, pj.axes, [x for x, _ in ref], wl.d)
    assert not any(oor) and pj.row_values() == rows
    assert int(pj.status.item()) == 0 and float(pj.est.item()) == part.median_to_double(rows)


def test_five_table_chain_full_width_sampled_row(orc, part):
    """The benchmark's equal-width configuration (4096 x 4096 per row, full scale): sketch
    row 5 of every tensor and its row estimate against the oracle."""
    wl = G.five_table(scale=1.0, w=4096)
    widths = [4096, 4096]
    pj = P.PartitionedJoin(wl, [3, 1, 2], [0, 1], widths)
    pj.build()
    pj.estimate()
    torch.cuda.synchronize()
    ref = _oracle_chain(orc, part, wl, widths, [5])
    for i, (x, n) in enumerate(ref):
        assert np.array_equal(pj.tensors[i][5:6].cpu().numpy(), x)
        assert int(pj.survivors[i].item()) == n
    rows, oor = part.contract_seq([0, 1], [1, 2], widths, pj.axes, [x for x, _ in ref], 1)
    assert not oor[0] and pj.row_values()[5] == rows[0]


def test_bulk_wait_that_runs_out_reports_timeout(part):
    """The bounded mbarrier wait of the bulk-streamed contraction, given a budget of 0 polls:
    every warp's first wait gives up, the launch writes CMP_ETIMEOUT to the status word and
    returns (each warp first drains its copies in flight); the context stays usable and the
    same join estimated next with the default bound gives the oracle's rows."""
    rng = np.random.default_rng(77)
    rows, w, d = 2500, 1024, 1   # int32 rows of >= 1024 entries, >= 16 per SM: the bulk path
    eu, ev, widths, axes = [0, 1], [1, 2], [rows, w], [[0], [0, 1], [1]]
    tensors = [rng.integers(-2 ** 20, 2 ** 20, size=(d, rows)), rng.integers(-2 ** 20, 2 ** 20, size=(d, rows * w)),
               rng.integers(-2 ** 20, 2 ** 20, size=(d, w))]
    dev = [torch.from_numpy(np.ascontiguousarray(x, np.int32)).cuda() for x in tensors]
    j, keep = K.part_join(eu, ev, widths, axes, [x.data_ptr() for x in dev])
    nb = K.cmp_part_estimate_ws_bytes(j, d)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    est = torch.empty(1, dtype=torch.float64, device="cuda")
    row = torch.empty((d, 2), dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    K.cmp_part_estimate_ex(j, d, ws.data_ptr(), nb, est.data_ptr(), row.data_ptr(), st.data_ptr(), 0,
                           K.stream_handle())
    torch.cuda.synchronize()
    assert int(st.item()) == K.CMP_ETIMEOUT
    assert not any(_check(part, eu, ev, widths, axes, tensors, d))   # a fresh, default-bound run
    with pytest.raises(K.CompassError) as ei:                      # a budget below -1 is refused
        K.cmp_part_estimate_ex(j, d, ws.data_ptr(), nb, est.data_ptr(), row.data_ptr(), st.data_ptr(), -2,
                               K.stream_handle())
    assert ei.value.status == K.CMP_EINVAL
