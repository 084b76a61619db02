"""The autotuner picks the fastest launch shape among candidates that all give
bit-identical sketches and estimates, and reuses cached choices."""
import json

import pytest
import torch

from paper_2102_02440_gb300 import autotune as AT
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu


def test_tune_build_and_cache(tmp_path):
    wl = G.five_table(scale=0.01, w=1024)
    dw = P.DeviceWorkload(wl)
    path = str(tmp_path / "tune.json")
    cfg, rep = AT.tune_build(dw, reps=2, cache_path=path)
    assert rep["ms"] == min(r["ms"] for r in rep["tried"] if r["ms"] is not None)
    cache = json.load(open(path))
    assert AT.build_signature(dw) in cache
    cfg2, rep2 = AT.tune_build(dw, reps=2, cache_path=path)      # served from the cache
    assert rep2["cfg"] == rep["cfg"]
    dw.build_batched(cfg2)
    torch.cuda.synchronize()
    dw.check_status()


def test_tune_estimate_consistent():
    wl = G.five_table(scale=0.01, w=512)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    cfg, rep = AT.tune_estimate(lambda c: P.DeviceEstimator(dw, masks, cfg=c), reps=2)
    assert len(rep["tried"]) == len(AT.ESTIMATE_CANDIDATES)
