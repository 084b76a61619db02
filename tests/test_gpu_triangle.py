"""GPU parity of the triangle path of the estimate (sub-plans whose only cycle is a
triangle, every other table a leaf of it): exact row estimates against the oracle and
against the generic path (one tree contraction per conditioning value), on raw sketch
values with many ties and zeros, both choices of the row side, empty query sets, widths
from 1 to the path's maximum and past it, and int128 overflow."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

GENERIC = K.cmp_estimate_cfg.make(flags=K.CMP_EST_GENERIC_ONLY)


def _graph(rng, nt):
    """Triangle on three tables plus nt - 3 leaves, random edge ids and table labels."""
    eu, ev = [0, 1, 0], [1, 2, 2]
    for t in range(3, nt):
        eu.append(int(rng.integers(0, 3)))
        ev.append(t)
    order = rng.permutation(len(eu))
    lab = rng.permutation(nt)
    return [int(lab[eu[i]]) for i in order], [int(lab[ev[i]]) for i in order]


def _raw_workload(rng, eu, ev, nt, d, w):
    """A DeviceWorkload of one-row tables whose counters are then overwritten."""
    tabs = []
    for t in range(nt):
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if eu[e] == t or ev[e] == t:
                cols.append(np.array([int(rng.integers(0, 100))], np.int32))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    dw = P.DeviceWorkload(G.Workload("raw", tabs, eu, ev, d, w, 1, 0))
    dw.survivors.fill_(1)
    return dw


def _fill(dw, rng, lo, hi, zero_p):
    """Counters drawn on the host (kept in dw.host_counters for the oracle) and uploaded."""
    dw.host_counters = []
    for t in dw.tables:
        a = rng.integers(lo, hi + 1, size=tuple(t.counters.shape), dtype=np.int64)
        a[rng.random(a.shape) < zero_p] = 0
        a = a.astype(np.int32)
        dw.host_counters.append(a)
        t.counters.copy_(torch.from_numpy(a))


def _set_row(dw, t, s, r, values):
    """Overwrite one counter row on the host copy and the device."""
    dw.host_counters[t][s, r] = values
    dw.tables[t].counters[s, r] = torch.from_numpy(np.ascontiguousarray(dw.host_counters[t][s, r])).cuda()


def _run(dw, masks, cfg=None):
    dw.status.zero_()
    est = P.DeviceEstimator(dw, masks, cfg=cfg)
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    return est, int(dw.status.item())


def _oracle_rows(orc, dw, masks):
    """Oracle estimates on the host counters the test drew (every table survivor count 1)."""
    wl = dw.wl
    sk = [tuple(dw.host_counters[wl.sketch_of(e, end)[0]][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(dw.n_edges)]
    surv = np.ones(len(wl.tables), np.int64)
    return [orc.estimate(wl.edge_u, wl.edge_v, sk, surv, dw.d, dw.w, int(m)) for m in masks]


def _cyclic(masks, eu, ev):
    return [m for m in masks if sum(1 for e in range(len(eu)) if (m >> eu[e]) & 1 and (m >> ev[e]) & 1)
            == bin(m).count("1")]


CASES = [  # (seed, tables, width, value range, zero fraction)
    (0, 3, 1, 3, 0.3), (1, 3, 2, 1, 0.2), (2, 4, 3, 2, 0.5), (3, 5, 16, 3, 0.3), (4, 6, 33, 50, 0.1),
    (5, 7, 64, 1, 0.4), (6, 4, 255, 5, 0.2), (7, 5, 256, 1000, 0.0), (8, 6, 257, 2, 0.6),
    (9, 8, 100, 7, 0.3), (10, 3, 511, 1 << 20, 0.1), (11, 6, 1000, 3, 0.25),
]


@pytest.mark.parametrize("seed,nt,w,vmax,zp", CASES)
def test_triangle_rows_match_oracle_and_generic(orc, seed, nt, w, vmax, zp):
    rng = np.random.default_rng(seed)
    eu, ev = _graph(rng, nt)
    dw = _raw_workload(rng, eu, ev, nt, 3, w)
    _fill(dw, rng, -vmax, vmax, zp)
    masks = G.connected_subplans(nt, eu, ev)
    assert _cyclic(masks, eu, ev)
    tri, st = _run(dw, masks)
    gen, st2 = _run(dw, masks, GENERIC)
    assert st == 0 and st2 == 0
    assert torch.equal(tri.row_est, gen.row_est) and torch.equal(tri.est, gen.est)
    rows = tri.row_values()
    for q, ref in enumerate(_oracle_rows(orc, dw, masks)):
        assert rows[q] == ref.rows, (q, bin(masks[q]))
        assert float(tri.est[q]) == ref.est


def test_triangle_both_row_sides(orc):
    """The row side is chosen per sketch row (fewer distinct conditioned magnitudes);
    rows where either table wins must give the oracle's values."""
    rng = np.random.default_rng(21)
    eu, ev = [0, 1, 0, 2], [1, 2, 2, 3]       # triangle 0-1-2 (e* = 1-2 by BFS), leaf 3 on table 2
    dw = _raw_workload(rng, eu, ev, 4, 4, 200)
    _fill(dw, rng, -400, 400, 0.1)
    # e1 = 1-2 is conditioned: make table 1's side narrow on rows 0, 2 and table 2's on rows 1, 3
    t1, s1 = dw.wl.sketch_of(1, 0)
    t2, s2 = dw.wl.sketch_of(1, 1)
    for r in range(4):
        narrow = (t1, s1) if r % 2 == 0 else (t2, s2)
        _set_row(dw, narrow[0], narrow[1], r, rng.integers(-1, 2, size=200).astype(np.int32))
    masks = [0b0111, 0b1111]
    tri, st = _run(dw, masks)
    assert st == 0
    rows = tri.row_values()
    for q, ref in enumerate(_oracle_rows(orc, dw, masks)):
        assert rows[q] == ref.rows


def test_triangle_without_nonzero_conditioning_values(orc):
    rng = np.random.default_rng(3)
    eu, ev = [0, 1, 0], [1, 2, 2]
    dw = _raw_workload(rng, eu, ev, 3, 3, 64)
    _fill(dw, rng, -5, 5, 0.2)
    t, s = dw.wl.sketch_of(1, 0)        # conditioned edge e1 = 1-2
    _set_row(dw, t, s, 0, 0)             # row 0: no conditioning value survives
    row1 = np.zeros(64, np.int32)
    row1[17] = 3                         # row 1: exactly one
    _set_row(dw, t, s, 1, row1)
    tri, st = _run(dw, [0b111])
    assert st == 0
    ref = _oracle_rows(orc, dw, [0b111])[0]
    assert tri.row_values()[0] == ref.rows and ref.rows[0] == 0


@pytest.mark.parametrize("w", [4096, 4097, 16384, 16385])
def test_triangle_wide_rows_match_generic(w):
    """Up to the path's maximum width (16384) and past it (planned on the generic path)."""
    rng = np.random.default_rng(w)
    eu, ev = [0, 1, 0, 0, 1], [1, 2, 2, 3, 4]
    dw = _raw_workload(rng, eu, ev, 5, 2, w)
    _fill(dw, rng, -30, 30, 0.2)
    masks = [0b00111, 0b01111, 0b11111]
    tri, st = _run(dw, masks)
    gen, st2 = _run(dw, masks, GENERIC)
    assert st == 0 and st2 == 0
    assert torch.equal(tri.row_est, gen.row_est) and torch.equal(tri.est, gen.est)


def test_triangle_int128_overflow_is_reported(orc):
    """Counters at 2^31 - 1 on a triangle with three leaves, with the exact tier off: every
    row is beyond int128; the estimate is NaN with CMP_EOVERFLOW, as on the generic path."""
    rng = np.random.default_rng(9)
    eu, ev = [0, 1, 0, 0, 1, 2], [1, 2, 2, 3, 4, 5]
    dw = _raw_workload(rng, eu, ev, 6, 3, 32)
    _fill(dw, rng, 2 ** 31 - 1, 2 ** 31 - 1, 0.0)
    no_wide = K.CMP_EST_NO_WIDE      # the int128 path's own flagging (the exact tier: test_gpu_wide)
    tri, st = _run(dw, [0b111111], K.cmp_estimate_cfg.make(flags=no_wide))
    assert st == K.CMP_EOVERFLOW and np.isnan(float(tri.est[0]))
    gen, st2 = _run(dw, [0b111111], K.cmp_estimate_cfg.make(flags=K.CMP_EST_GENERIC_ONLY | no_wide))
    assert st2 == K.CMP_EOVERFLOW and np.isnan(float(gen.est[0]))
    ref = _oracle_rows(orc, dw, [0b111111])[0]
    assert all(abs(v) >= 2 ** 127 for v in ref.rows)


def test_five_table_full_width_triangle_vs_generic():
    """The benchmark's shape at full width (w = 4096, d = 11), reduced row counts: the four
    cyclic sub-plans on the triangle path equal the generic path bit for bit."""
    wl = G.five_table(scale=0.02, w=4096)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    tri, st = _run(dw, masks)
    gen, st2 = _run(dw, masks, GENERIC)
    assert st == 0 and st2 == 0
    assert len(_cyclic(masks, wl.edge_u, wl.edge_v)) == 4
    assert torch.equal(tri.row_est, gen.row_est) and torch.equal(tri.est, gen.est)
