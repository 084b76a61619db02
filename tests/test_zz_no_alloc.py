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
