"""GPU parity of the learned combiner against the oracle (self-join sizes, features,
forward pass, gradients, Adam), and the trained network against the plain median:
the median q-error of its estimates on held-out pairs must not exceed the median's."""
import numpy as np
import pytest
import torch

from paper_2102_02440_gb300 import compass as K
from paper_2102_02440_gb300 import datagen as G
from paper_2102_02440_gb300 import pipeline as P

pytestmark = pytest.mark.gpu
NH = 64


def _rows_as_int(row_est):
    r = row_est.cpu().numpy()
    lo = r[..., 0].astype(np.uint64).astype(object)
    hi = r[..., 1].astype(object)
    return hi * (1 << 64) + lo


def _features_ref(rows, f2a, f2b):
    """Definition of the features (see cmp_mlp_features), in float64 then float32."""
    n, d = rows.shape
    out = np.zeros((n, d + 2), np.float32)
    for q in range(n):
        v = np.float32(np.array(sorted(float(np.copysign(np.log1p(abs(float(e))), float(e))) for e in rows[q])) / 32.0)
        m = d // 2
        out[q, :d] = v - v[m]
        out[q, m] = v[m]
        out[q, d] = np.float32(np.log1p(max(f2a[q], 0.0)) / 32.0)
        out[q, d + 1] = np.float32(np.log1p(max(f2b[q], 0.0)) / 32.0)
    return out


@pytest.fixture(scope="module")
def small_pairs(orc):
    pairs = G.join_pairs(300, rows_lo=200, rows_hi=20_000, dom_lo=100, dom_hi=100_000, seed=7)
    pb = P.PairBatch(pairs, d=11, w=512, hash_seed=99)
    pb.build()
    pb.prepare_estimate()
    pb.estimate()
    pb.features()
    torch.cuda.synchronize()
    pb.dw.check_status()
    # the oracle's own build of every table (one sketch each): the reference inputs
    pb.oracle_counters = np.stack([orc.build_sketch(t, pb.dw.hash_u64, pb.d, pb.w)[0][0] for t in pb.dw.wl.tables])
    return pairs, pb


def _host_features(rng, n, nin):
    """Feature-like inputs drawn on the host: sorted centred log row values and two sizes."""
    x = rng.normal(0.0, 0.05, size=(n, nin)).astype(np.float32)
    x[:, (nin - 2) // 2] = rng.uniform(0.0, 0.8, n).astype(np.float32)
    x[:, -2:] = rng.uniform(0.0, 0.9, size=(n, 2)).astype(np.float32)
    return x


def test_device_counters_equal_oracle_build(small_pairs):
    _, pb = small_pairs
    assert np.array_equal(pb.counters.cpu().numpy(), pb.oracle_counters)


def test_self_join_sizes_exact(small_pairs):
    _, pb = small_pairs
    C = pb.oracle_counters.astype(object)
    f2 = pb.f2.cpu().numpy()
    for s in range(0, 2 * pb.n, 7):
        rows = sorted(int((C[s, i] ** 2).sum()) for i in range(pb.d))
        assert f2[s] == float(rows[pb.d // 2])


def test_two_way_estimates_match_oracle(orc, small_pairs):
    _, pb = small_pairs
    rows = _rows_as_int(pb.row_est)
    est = pb.est.cpu().numpy()
    C = pb.oracle_counters
    for q in range(0, pb.n, 13):
        ref = orc.estimate([0], [1], [(C[2 * q], C[2 * q + 1])], [0, 0], pb.d, pb.w, 0b11)
        assert list(rows[q]) == ref.rows and est[q] == ref.est


def test_features_match_definition(orc, small_pairs):
    """Features from the oracle's row estimates and self-join sizes (exact integers, one
    rounding) against the device features."""
    _, pb = small_pairs
    C = pb.oracle_counters
    rows = np.array([orc.estimate([0], [1], [(C[2 * q], C[2 * q + 1])], [0, 0], pb.d, pb.w, 0b11).rows
                     for q in range(pb.n)], dtype=object)

    def f2(c):
        r = sorted(int((c[i].astype(object) ** 2).sum()) for i in range(pb.d))
        return float(r[pb.d // 2])

    f2a = np.array([f2(C[2 * q]) for q in range(pb.n)])
    f2b = np.array([f2(C[2 * q + 1]) for q in range(pb.n)])
    ref = _features_ref(rows, f2a, f2b)
    np.testing.assert_allclose(pb.feat.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("skip", [-1, 5])
def test_forward_matches_oracle(orc, small_pairs, skip):
    _, pb = small_pairs
    comb = P.Combiner(pb.d + 2, NH, seed=3, skip=skip)
    x = _host_features(np.random.default_rng(4 + skip), pb.n, pb.d + 2)
    y = comb.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = orc.mlp_forward(pb.d + 2, NH, comb.params.cpu().numpy(), x, skip=skip)
    np.testing.assert_allclose(y, ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("skip,huber", [(-1, None), (5, None), (5, 0.01)])
def test_gradient_and_adam_match_oracle(orc, small_pairs, skip, huber):
    _, pb = small_pairs
    rng = np.random.default_rng(5)
    nin = pb.d + 2
    comb = P.Combiner(nin, NH, seed=4, skip=skip)
    xh = _host_features(rng, pb.n, nin)
    th = rng.standard_normal(pb.n).astype(np.float32) * 0.3 + 0.5
    x, t = torch.from_numpy(xh).cuda(), torch.from_numpy(th).cuda()
    p0 = comb.params.cpu().numpy().copy()
    comb.train_step(x, t, lr=1e-3, huber_delta=huber or 0.0)
    torch.cuda.synchronize()
    loss_ref, g_ref = orc.mlp_loss_grad(nin, NH, p0, xh, th, skip=skip, huber_delta=huber)
    g = comb.grad.cpu().numpy().astype(np.float64)
    assert abs(float(comb.loss.item()) - loss_ref) <= 1e-5 * abs(loss_ref) + 1e-7
    np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=1e-6 * np.abs(g_ref).max())
    p_ref, m, v = p0.copy(), np.zeros(p0.size), np.zeros(p0.size)
    orc.adam_step(p_ref, m, v, g, lr=1e-3, step=1)   # same gradient, fp64 update
    np.testing.assert_allclose(comb.params.cpu().numpy(), p_ref, rtol=0, atol=2e-6)


def test_training_is_deterministic(small_pairs):
    _, pb = small_pairs
    t = torch.linspace(0, 1, pb.n, device="cuda")
    outs = []
    for _ in range(2):
        comb = P.Combiner(pb.d + 2, NH, seed=8)
        for _ in range(20):
            comb.train_step(pb.feat, t, lr=3e-3)
        outs.append(comb.params.clone())
    assert torch.equal(outs[0], outs[1])


def qerr(est, true):
    e = np.maximum(est, 1.0)
    t = np.maximum(true, 1.0)
    return np.maximum(e / t, t / e)


def test_combine_rule():
    med = torch.tensor([5.0, 1.0, 0.99, 0.0, -3.0, 1e12], dtype=torch.float64, device="cuda")
    y = torch.tensor([0.1, 0.2, 0.3, 0.0, -0.5, 0.4], dtype=torch.float32, device="cuda")
    comb = P.Combiner(13, NH, seed=0)
    out = comb.combine(med, y).cpu().numpy()
    yd = y.double().cpu().numpy()
    want = [5.0, 1.0, np.expm1(32 * yd[2]), 0.0, 0.0, 1e12]
    np.testing.assert_allclose(out, want, rtol=1e-15)


@pytest.mark.slow
def test_learned_combiner_vs_median(orc):
    """Reduced learned-combiner workload: 20000 independent joins (rows log-uniform in
    [1e3, 2e4], domains log-uniform in [1e3, 1e6], Zipf 0.5..1.5, drawn on the device),
    d = 11, w = 4096, split 80/10/10; labels are the oracle's exact join sizes.  The
    network (skip connection from the median row feature, Huber loss in log space) is
    trained on the GPU by the library's kernels on the training pairs whose median row
    estimate is below one tuple, stopped on the validation split, and the combined
    estimate is judged on the test split against the plain median of the same sketches:
    median q-error at or below the median's, 90th percentile strictly below."""
    keys, off, _ = G.join_pairs_device(20_000, 1_000, 20_000, seed=20210208)
    host = keys.cpu().numpy()
    n = (len(off) - 1) // 2
    exact = np.array([orc.join2(host[off[2 * i]:off[2 * i + 1]], host[off[2 * i + 1]:off[2 * i + 2]])
                      for i in range(n)], np.float64)
    pb = P.PairBatch(None, d=11, w=4096, hash_seed=0xC0FFEE + 3, device_keys=keys, offsets=off)
    pb.build()
    pb.prepare_estimate()
    pb.estimate()
    feat = pb.features()
    torch.cuda.synchronize()
    pb.dw.check_status()
    a, b = int(0.8 * n), int(0.9 * n)
    y = torch.from_numpy((np.log1p(exact) / 32.0).astype(np.float32)).cuda()
    use = pb.est < 1.0                                   # where the combiner replaces the median
    tr = torch.arange(a, device="cuda")[use[:a]]
    comb = P.Combiner(pb.d + 2, NH, seed=1, skip=pb.d // 2, init_scale=0.0)
    x_tr, y_tr = feat[tr].contiguous(), y[tr].contiguous()

    def combined(lo, hi):
        yy = comb.infer(feat[lo:hi].contiguous())
        return comb.combine(pb.est[lo:hi].contiguous(), yy).cpu().numpy()

    best, best_p = np.median(qerr(combined(a, b), exact[a:b])), None
    for it in range(1, 3001):
        comb.train_step(x_tr, y_tr, lr=3e-4, huber_delta=0.001)
        if it % 250 == 0:
            q = np.mean(np.log(qerr(combined(a, b), exact[a:b])))
            if best_p is None or q < best:
                best, best_p = q, comb.params.clone()
    comb.params.copy_(best_p)
    learned = combined(b, n)
    median = pb.est.cpu().numpy()[b:]
    ql, qm = qerr(learned, exact[b:]), qerr(median, exact[b:])
    print(f"test q-error median/p90/p99: combiner {np.median(ql):.4f}/{np.percentile(ql, 90):.2f}/"
          f"{np.percentile(ql, 99):.1f}  plain median {np.median(qm):.4f}/{np.percentile(qm, 90):.2f}/"
          f"{np.percentile(qm, 99):.1f}")
    assert np.median(ql) <= np.median(qm)
    assert np.percentile(ql, 90) < np.percentile(qm, 90)


def test_features_indexed_equals_gathered():
    """cmp_mlp_features_indexed (self-join sizes of all sketches, picked by index) gives the
    features of cmp_mlp_features on the gathered per-sample arrays, -1 reading as 0."""
    rng = np.random.default_rng(8)
    n, d, n_sk = 500, 11, 7
    rows = torch.from_numpy(rng.integers(-(1 << 40), 1 << 40, size=(n, d, 2)).astype(np.int64)).cuda()
    rows[..., 1] = torch.where(rows[..., 0] < 0, -1, 0)   # sign-extended int128 values
    f2 = torch.from_numpy(rng.uniform(0, 1e12, n_sk)).cuda()
    idx = torch.from_numpy(rng.integers(-1, n_sk, size=(n, 2)).astype(np.int32)).cuda()
    a = torch.where(idx[:, 0] >= 0, f2[idx[:, 0].clamp(min=0).long()], torch.zeros((), dtype=torch.float64, device="cuda"))
    b = torch.where(idx[:, 1] >= 0, f2[idx[:, 1].clamp(min=0).long()], torch.zeros((), dtype=torch.float64, device="cuda"))
    ref = torch.empty((n, d + 2), dtype=torch.float32, device="cuda")
    got = torch.full_like(ref, float("nan"))
    K.cmp_mlp_features(rows.data_ptr(), n, d, a.contiguous().data_ptr(), b.contiguous().data_ptr(), ref.data_ptr(),
                       K.stream_handle())
    K.cmp_mlp_features_indexed(rows.data_ptr(), n, d, f2.data_ptr(), idx.data_ptr(), got.data_ptr(), K.stream_handle())
    torch.cuda.synchronize()
    assert torch.equal(ref, got)


@pytest.mark.parametrize("d,w", [(1, 1), (3, 100), (8, 777), (15, 65536), (16, 4096), (64, 300)])
def test_self_join_sizes_every_row_split(d, w):
    """cmp_sketch_f2 with rows spread over the CTAs of a cluster (fewer rows than CTAs, one
    each, several each, even d): the exact median of the exact row sums of squares, rounded
    once, for counters up to +-(2^31 - 1)."""
    rng = np.random.default_rng(d * 1000 + w)
    n = 5
    C = rng.integers(-(2 ** 31) + 1, 2 ** 31, size=(n, d, w), dtype=np.int64)
    C[:, :, 0] = 2 ** 31 - 1
    Cd = torch.from_numpy(C.astype(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    K.cmp_sketch_f2(Cd.data_ptr(), n, d, w, out.data_ptr(), K.stream_handle())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for s in range(n):
        rows = sorted(sum(int(v) * int(v) for v in C[s, i]) for i in range(d))
        want = float(rows[d // 2]) if d % 2 else float(rows[d // 2 - 1] + rows[d // 2]) / 2.0
        assert got[s] == want, (s, got[s], want)
