"""GPU parity of sketches over a row sample (Sec. 2 "Workflow").  The single-table,
batched (with and without key aggregation) and partitioned builds over a sample equal the
oracle's build of the sampled rows bit for bit, with their survivor counts; the estimates
of every sub-plan equal the oracle's estimate over the sampled sketches times the sample
scale, bit for bit, for the merged and the partitioned estimators."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu

SEED = 0x5A3B1E   # the pipeline's default sample seed base (table t uses SEED + t)


@pytest.fixture(scope="module")
def smp(orc):
    from oracle import sample
    return sample


def _table(rng, n, preds, int64=False):
    dt = np.int64 if int64 else np.int32
    cols = [G.zipf_keys(rng, n, 3000, 1.1, dt), G.zipf_keys(rng, n, 500, 0.7, dt), G.uniform_col(rng, n, 0, 1000)]
    pr = [G.Pred(2, G.RANGE, 100, 600)] if preds else []
    return G.Table("t", cols, pr, [0, 1, 0], [0, 1, 2])


@pytest.mark.parametrize("rate,preds,int64,cfg", [
    (0.5, False, False, None), (0.1, True, False, None), (0.01, True, True, dict(mode=2)),
    (0.3, False, True, dict(mode=1, dedupe=0)), (0.999, True, False, dict(threads=128, tile_rows=256)),
    (1.0, True, False, None)])
def test_single_table_build_over_a_sample(orc, smp, rate, preds, int64, cfg):
    rng = np.random.default_rng(int(rate * 1000) + preds)
    t = _table(rng, 60_000, preds, int64)
    d, w = 5, 512
    hp = orc.hash_params(3, 3, d)
    want, n_want = orc.build_sketch(smp.sampled_table(t, 77, rate), hp, d, w)
    dt = P.DeviceTable(t, d, w, torch.device("cuda"), sample_seed=77, sample_rate=rate)
    surv = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hd = torch.from_numpy(hp.reshape(-1).view(np.int64)).cuda()
    K.cmp_sketch_build(dt.desc, d, w, hd.data_ptr(), 3, dt.counters.data_ptr(), surv.data_ptr(), st.data_ptr(),
                       K.cmp_build_cfg.make(**cfg) if cfg else None, K.stream_handle())
    torch.cuda.synchronize()
    assert int(surv.item()) == n_want and int(st.item()) == 0
    assert np.array_equal(dt.counters.cpu().numpy(), want)


def _oracle(orc, smp, wl, rates, hash_u64):
    built = [orc.build_sketch(smp.sampled_table(t, SEED + i, rates[i]), hash_u64, wl.d, wl.w)
             for i, t in enumerate(wl.tables)]
    sk = [tuple(built[wl.sketch_of(e, end)[0]][0][wl.sketch_of(e, end)[1]] for end in range(2))
          for e in range(wl.n_edges)]
    return built, sk, np.array([n for _, n in built], np.int64)


@pytest.mark.parametrize("aggregate", [-1, 0, 1])
def test_batched_build_and_estimate_over_samples(orc, smp, aggregate):
    wl = G.five_table(scale=0.02, w=1024)
    rates = [0.1, 0.5, 1.0, 0.25, 0.0]
    dw = P.DeviceWorkload(wl, sample_rates=rates)
    dw.encode_batched(K.cmp_build_cfg.make(aggregate=aggregate))
    dw.build_batched()
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    torch.cuda.synchronize()
    dw.check_status()
    built, sk, surv = _oracle(orc, smp, wl, rates, dw.hash_u64)
    assert np.array_equal(dw.survivors.cpu().numpy(), surv)
    for (c, n), t in zip(built, dw.tables):
        assert np.array_equal(t.counters.cpu().numpy(), c)
    rows = est.row_values()
    e_gpu = est.est.cpu().numpy()
    for q, m in enumerate(masks):
        ref = orc.estimate(wl.edge_u, wl.edge_v, sk, surv, wl.d, wl.w, int(m))
        assert rows[q] == ref.rows
        want = ref.est * smp.scale_of(int(m), rates)
        assert e_gpu[q] == want or (np.isnan(e_gpu[q]) and np.isnan(want)), (bin(m), e_gpu[q], want)
    singles = [q for q, m in enumerate(masks) if bin(int(m)).count("1") == 1]
    assert singles and all(e_gpu[q] == surv[int(masks[q]).bit_length() - 1] *
                           smp.scale_of(int(masks[q]), rates) for q in singles)


def test_partitioned_build_and_estimate_over_samples(orc, smp):
    from oracle import partition as part
    wl = G.five_table(scale=0.02, w=4096)
    rates = [1.0, 0.2, 0.5, 0.7, 1.0]        # per workload table; the chain uses tables 3, 1, 2
    chain_rates = [rates[3], rates[1], rates[2]]
    pj = P.PartitionedJoin(wl, [3, 1, 2], [0, 1], [64, 32], sample_rates=chain_rates)
    pj.build()
    pj.estimate()
    torch.cuda.synchronize()
    hp = orc.hash_params(wl.hash_seed, wl.n_edges, wl.d)
    ref = []
    for i, t in enumerate((3, 1, 2)):
        src = smp.sampled_table(wl.tables[t], SEED + t, rates[t])
        x, n = part.build_partitioned(src, hp, wl.d, pj.table_widths(i))
        assert np.array_equal(pj.tensors[i].cpu().numpy(), x) and int(pj.survivors[i].item()) == n
        ref.append(x)
    rows, oor = part.contract_seq([0, 1], [1, 2], [64, 32], pj.axes, ref, wl.d)
    assert not any(oor) and pj.row_values() == rows
    assert float(pj.est.item()) == part.median_to_double(rows) * smp.scale_of(0b111, chain_rates)


def test_offline_tables_give_identical_estimates():
    """Offline sketches (Sec. 2 "Workflow"): F1 and F2 (no predicates) built once with their
    presort and cross ranks; every query then builds and presorts D1, D2, D3 only, and its
    estimates equal the all-online ones bit for bit, over two queries."""
    wl = G.five_table(scale=0.02, w=1024)
    masks = G.connected_subplans(5, wl.edge_u, wl.edge_v)
    dw = P.DeviceWorkload(wl)
    dw.build_batched()
    est = P.DeviceEstimator(dw, masks)
    est.presort()
    est.estimate()
    dwo = P.DeviceWorkload(wl, cols_dev=[t.cols for t in dw.tables], offline=[1, 0])
    assert dwo.storage_order == [2, 3, 4, 0, 1]
    dwo.build_offline()
    esto = P.DeviceEstimator(dwo, masks)
    for _ in range(2):
        dwo.build_batched()
        esto.presort()
        esto.estimate()
        torch.cuda.synchronize()
        assert torch.equal(esto.row_est, est.row_est)
        assert torch.equal(torch.nan_to_num(esto.est, nan=-1.0), torch.nan_to_num(est.est, nan=-1.0))
        assert torch.equal(dwo.survivors, dw.survivors)
    with pytest.raises(ValueError):
        P.DeviceWorkload(wl, offline=[2])     # D1 has a predicate
