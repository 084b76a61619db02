"""The learned combiner at the learned-combiner configuration's full size: the checkpoint
trained by tests/train_combiner.py (1e5 seeded joins of 1e4..1e7 rows per table, d = 11,
w = 4096, 80/10/10 split by pair index) is evaluated on its held-out test split, drawn
again from the same seeds, against the oracle's exact join sizes: with its stored rule the
combined estimate's median q-error is at or below the plain median's and its 90th
percentile below it; the checkpoint's recorded test figures are reproduced."""
import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import pipeline as P

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CKPT = os.path.join(P.CHECKPOINT_DIR, "combiner_d11.bin")


@pytest.mark.skipif(not os.path.exists(CKPT), reason="no trained checkpoint")
def test_trained_combiner_on_the_held_out_split(orc):
    import train_combiner as T
    comb, meta = P.Combiner.load(CKPT)
    n = meta["pairs"]
    b0, b1 = int(0.9 * n) // T.BATCH, n // T.BATCH
    feats, meds, exact = [], [], []
    with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as pool:
        for b in range(b0, b1):
            f, m, e, _ = T.pair_batch(b, 11, meta["w"], orc, pool)
            feats.append(f)
            meds.append(m)
            exact.append(e)
    feat, med, exact = np.concatenate(feats), np.concatenate(meds), np.concatenate(exact)
    x = torch.from_numpy(feat).cuda()
    y = comb.infer(x)
    m_dev = torch.from_numpy(med).cuda()
    out = torch.empty_like(m_dev)
    K.cmp_mlp_combine_ex(m_dev.data_ptr(), y.data_ptr(), 0, med.size, float(meta["use_median_at"]), out.data_ptr(),
                         K.stream_handle())
    ql, qm = T.qerr(out.cpu().numpy(), exact), T.qerr(med, exact)
    print(f"test split ({med.size} joins): combined median {np.median(ql):.4f} p90 {np.percentile(ql, 90):.2f} "
          f"p99 {np.percentile(ql, 99):.1f}; plain median {np.median(qm):.4f} p90 {np.percentile(qm, 90):.2f} "
          f"p99 {np.percentile(qm, 99):.1f}")
    assert np.median(ql) <= np.median(qm)
    assert np.percentile(ql, 90) < np.percentile(qm, 90)
    rec = meta["test_q_error"]["combined"]
    assert np.median(ql) == pytest.approx(rec["median"], rel=1e-9)
