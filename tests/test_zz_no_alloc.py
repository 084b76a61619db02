"""cmp_estimate_noalloc: the estimate for callers that cannot allocate device memory
(its workspace is a fixed array inside the library).  Its results must equal those of
cmp_estimate with a caller-provided workspace, on consecutive calls that reuse the same
array, and plans that do not fit must be rejected with CMP_EWORKSPACE.  This file is
collected last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu


def _workload(seed, w):
    rng = np.random.default_rng(seed)
    wl = G.random_graph_workload(rng, 6, 1, 500, 20_000, 2000, d=5, w=w, pred_prob=0.5, hash_seed=seed)
    dw = P.DeviceWorkload(wl)
    dw.build()
    masks = G.connected_subplans(6, wl.edge_u, wl.edge_v)
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    return dw, est


def _noalloc(est, status):
    out = torch.full_like(est.est, float("nan"))
    rows = torch.full_like(est.row_est, -1)
    K.cmp_estimate_noalloc(est.plan_host.ctypes.data, est.plan_dev.data_ptr(), out.data_ptr(), rows.data_ptr(),
                           status.data_ptr(), K.stream_handle())
    return out, rows


@pytest.mark.parametrize("w", [64, 1024])
def test_noalloc_matches_caller_workspace_on_consecutive_calls(w):
    dw, est = _workload(11 + w, w)
    est.estimate()
    ref_est, ref_rows = est.est.clone(), est.row_est.clone()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    a_est, a_rows = _noalloc(est, status)
    b_est, b_rows = _noalloc(est, status)       # second call reuses the array's old contents
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for e, r in ((a_est, a_rows), (b_est, b_rows)):
        assert torch.equal(e, ref_est)           # exact: one rounding of the same exact integers
        assert torch.equal(r, ref_rows)


def test_noalloc_then_another_plan():
    _, est1 = _workload(3, 256)
    _, est2 = _workload(4, 64)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for est in (est1, est2, est1):
        est.estimate()
        got, rows = _noalloc(est, status)
        torch.cuda.synchronize()
        assert torch.equal(got, est.est) and torch.equal(rows, est.row_est)
    assert int(status.item()) == 0


def _raw_workload(rng, eu, ev, nt, d, w, vmax=40, zero_p=0.2):
    """One-row tables whose counters are then overwritten with random values (ties and
    zeros included), so wide sketches cost no table data."""
    tabs = []
    for t in range(nt):
        cols, kc, ei = [], [], []
        for e in range(len(eu)):
            if t in (eu[e], ev[e]):
                cols.append(np.array([int(rng.integers(0, 100))], np.int32))
                kc.append(len(cols) - 1)
                ei.append(e)
        tabs.append(G.Table(f"T{t}", cols, [], kc, ei))
    dw = P.DeviceWorkload(G.Workload("raw", tabs, eu, ev, d, w, 1, 0))
    dw.survivors.fill_(1)
    for t in dw.tables:
        a = rng.integers(-vmax, vmax + 1, size=tuple(t.counters.shape), dtype=np.int64)
        a[rng.random(a.shape) < zero_p] = 0
        t.counters.copy_(torch.from_numpy(a.astype(np.int32)))
    return dw


def _tri_row_bytes(w, leaves):
    """Scratch bytes of one triangle row (sub-plan, sketch row) at width w with `leaves`
    leaves per node: the regions of the triangle path, each rounded up to 256 bytes."""
    al = lambda x: (x + 255) & ~255
    w1, nl = w + 1, 3 * leaves
    return (al(64) + al(96 * w) + al(48 * w) + al(8 * nl * w1) + al(16 * nl * w1) + al(8 * w) + al(48 * w1) +
            al(8 * w) + al(32 * w) + al(4 * w) + al(4 * w) + al(48 * w1) + al(4 * (w1 + 1)) + al(4 * (w1 + 1)))


def _noalloc_guarded(est, status, guard=8):
    """cmp_estimate_noalloc into output buffers followed by `guard` sentinel elements,
    which must come back untouched."""
    n, d = est.est.numel(), est.d
    out = torch.full((n + guard,), -7.25, dtype=torch.float64, device="cuda")
    rows = torch.full((n * d * 2 + guard,), 0x5A5A5A5A, dtype=torch.int64, device="cuda")
    K.cmp_estimate_noalloc(est.plan_host.ctypes.data, est.plan_dev.data_ptr(), out.data_ptr(), rows.data_ptr(),
                           status.data_ptr(), K.stream_handle())
    torch.cuda.synchronize()
    assert torch.all(out[n:] == -7.25) and torch.all(rows[n * d * 2:] == 0x5A5A5A5A)
    return out[:n], rows[:n * d * 2].view(n, d, 2)


def _check_against_workspace_path(dw, masks):
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    ref_est, ref_rows = est.est.clone(), est.row_est.clone()
    assert int(dw.status.item()) == 0
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):                            # the second call starts from the first's contents
        got, rows = _noalloc_guarded(est, status)
        assert int(status.item()) == 0
        assert torch.equal(got, ref_est) and torch.equal(rows, ref_rows)
    return est


def test_noalloc_triangle_only_plan_runs_its_rows_in_waves():
    """A plan whose only sub-plan is a triangle (no generic items) at w = 16384, d = 9: its
    nine triangle rows need more scratch than the array holds, so they run in waves."""
    rng = np.random.default_rng(5)
    dw = _raw_workload(rng, [0, 1, 0], [1, 2, 2], 3, 9, 16384)
    assert 9 * _tri_row_bytes(16384, 0) > K.CMP_NOALLOC_WS_BYTES
    est = _check_against_workspace_path(dw, [0b111])
    info = K.cmp_estimate_plan_stats(est.plan_host.ctypes.data)
    assert info.n_tri == 1 and info.n_items == 9 * (16384 // 256)   # one sweep item per 256 columns


def test_noalloc_generic_plan_with_shrunken_grid():
    """Tree sub-plans of a six-table chain at w = 16384: the persistent grid's CTA scratch
    areas exceed the array, so the call runs with fewer CTAs than the caller-workspace
    path."""
    rng = np.random.default_rng(6)
    eu, ev = [0, 1, 2, 3, 4], [1, 2, 3, 4, 5]
    dw = _raw_workload(rng, eu, ev, 6, 5, 16384, vmax=6)
    masks = G.connected_subplans(6, eu, ev)
    est = _check_against_workspace_path(dw, masks)
    info = K.cmp_estimate_plan_stats(est.plan_host.ctypes.data)
    # the caller-workspace path's workspace (every CTA's scratch) does not fit in the array
    assert info.n_tri == 0 and est.ws.numel() > K.CMP_NOALLOC_WS_BYTES


def test_noalloc_mixed_triangle_and_tree_plan_in_waves():
    """Triangle sub-plans with leaves next to tree sub-plans (every connected sub-plan of a
    triangle with two leaves), w = 16384, d = 7: both scratch kinds share the array, the
    grid shrinks and the triangle rows run in waves."""
    rng = np.random.default_rng(7)
    eu, ev = [0, 1, 0, 0, 2], [1, 2, 2, 3, 4]
    dw = _raw_workload(rng, eu, ev, 5, 7, 16384, vmax=10)
    masks = G.connected_subplans(5, eu, ev)
    est = _check_against_workspace_path(dw, masks)
    info = K.cmp_estimate_plan_stats(est.plan_host.ctypes.data)
    assert info.n_tri >= 4 and info.n_tri * 7 * _tri_row_bytes(16384, 0) > K.CMP_NOALLOC_WS_BYTES


def test_noalloc_rejects_plans_beyond_its_workspace():
    # 64 rows x 40k two-table sub-plans: the per-item partial sums alone exceed the array
    wl = G.two_way(n_r=1000, n_s=1000, d=64, w=16)
    dw = P.DeviceWorkload(wl)
    dw.build()
    est = P.DeviceEstimator(dw, [0b11] * 40_000)
    est.presort()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(K.CompassError) as ei:
        _noalloc(est, status)
    assert ei.value.status == K.CMP_EWORKSPACE
