"""Pins of the oracle's learned combiner (not in the paper, which takes the median over
rows, Sec. 3.2): bfloat16 rounding, forward pass, gradients by finite differences, Adam."""
import numpy as np
import pytest

NIN, NH = 13, 64


def _params(rng):
    n = NH * NIN + 2 * NH + 1
    return (rng.standard_normal(n) * 0.3).astype(np.float32)


def test_bf16_round_nearest_even(orc):
    vals = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, 3.14159265, -2.71828, 1e-30, 65504.0,
                     np.inf, -np.inf], np.float32)
    got = orc.bf16_round(vals)
    u = vals.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    want = (((u + 0x7FFF + lsb) & 0xFFFF0000) & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    fin = np.isfinite(vals)
    assert np.array_equal(got[fin], want[fin])
    assert np.array_equal(got[~fin], vals[~fin])
    # 1 + 2^-8 is exactly half way between 1 and 1 + 2^-7: ties go to the even significand (1.0)
    assert got[1] == 1.0 and got[2] == 1.0078125
    assert np.isnan(orc.bf16_round(np.array([np.nan], np.float32))[0])


def test_forward_matches_numpy(orc):
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.standard_normal((50, NIN)).astype(np.float32)
    q = orc.bf16_round(p).astype(np.float64)
    W1 = q[:NH * NIN].reshape(NH, NIN)
    b1 = q[NH * NIN:NH * NIN + NH]
    W2 = q[NH * NIN + NH:NH * NIN + 2 * NH]
    b2 = q[-1]
    want = np.maximum(x.astype(np.float64) @ W1.T + b1, 0) @ W2 + b2
    np.testing.assert_allclose(orc.mlp_forward(NIN, NH, p, x), want, rtol=1e-12, atol=1e-12)


def test_skip_connection_adds_the_clamped_feature(orc):
    """y = max(x[skip], 0) + MLP(x): the difference to the no-skip output is exactly the
    clamped feature, and the gradient (no parameter on the skip path) is unchanged."""
    rng = np.random.default_rng(9)
    p = _params(rng)
    x = rng.standard_normal((30, NIN)).astype(np.float32)
    t = rng.standard_normal(30).astype(np.float32)
    y0 = orc.mlp_forward(NIN, NH, p, x)
    y5 = orc.mlp_forward(NIN, NH, p, x, skip=5)
    np.testing.assert_allclose(y5 - y0, np.maximum(x[:, 5].astype(np.float64), 0), rtol=0, atol=1e-12)
    # loss/grad with skip equal those without skip on targets shifted by the skip term
    l5, g5 = orc.mlp_loss_grad(NIN, NH, p, x, t, skip=5)
    t_shift = (t.astype(np.float64) - np.maximum(x[:, 5], 0)).astype(np.float32)
    l0, g0 = orc.mlp_loss_grad(NIN, NH, p, x, t_shift)
    assert abs(l5 - l0) < 1e-5 * max(l0, 1e-9) + 1e-9
    np.testing.assert_allclose(g5, g0, rtol=1e-4, atol=1e-7)


def _pattern(p, x):
    W1 = p[:NH * NIN].reshape(NH, NIN).astype(np.float64)
    b1 = p[NH * NIN:NH * NIN + NH].astype(np.float64)
    return (x.astype(np.float64) @ W1.T + b1) > 0


def test_gradient_by_central_differences(orc):
    """Gradient of the loss in the (bf16-rounded) parameters: perturb a parameter that
    is exactly representable in bf16 by a bf16-exact step and compare."""
    rng = np.random.default_rng(1)
    p = orc.bf16_round(_params(rng))
    x = rng.standard_normal((40, NIN)).astype(np.float32)
    t = rng.standard_normal(40).astype(np.float32)
    _, g = orc.mlp_loss_grad(NIN, NH, p, x, t)
    idx = list(rng.choice(p.size, 60, replace=False)) + [p.size - 1, NH * NIN + 3]
    checked = 0
    for i in idx:
        h = np.float32(2.0 ** (np.floor(np.log2(abs(p[i]) + 1e-3)) - 6))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        assert orc.bf16_round(pp)[i] == pp[i] and orc.bf16_round(pm)[i] == pm[i]
        if not (np.array_equal(_pattern(pp, x), _pattern(p, x)) and np.array_equal(_pattern(pm, x), _pattern(p, x))):
            continue        # the step crosses a ReLU kink: the loss is not one quadratic there
        checked += 1
        lp, _ = orc.mlp_loss_grad(NIN, NH, pp, x, t)
        lm, _ = orc.mlp_loss_grad(NIN, NH, pm, x, t)
        fd = (lp - lm) / (2 * float(h))   # exact for a quadratic, up to rounding
        assert abs(fd - g[i]) <= 1e-9 + 1e-7 * abs(g[i]), (i, fd, g[i])
    assert checked >= 40


def test_huber_gradient_by_central_differences(orc):
    """Huber loss (quadratic within delta, linear beyond): gradient vs central differences,
    with a step small enough that no residual crosses +-delta or a ReLU kink."""
    rng = np.random.default_rng(11)
    p = orc.bf16_round(_params(rng))
    x = rng.standard_normal((40, NIN)).astype(np.float32)
    t = rng.standard_normal(40).astype(np.float32)
    delta = 0.5
    _, g = orc.mlp_loss_grad(NIN, NH, p, x, t, skip=3, huber_delta=delta)
    y0 = orc.mlp_forward(NIN, NH, p, x, skip=3)
    checked = 0
    for i in list(rng.choice(p.size, 40, replace=False)) + [p.size - 1]:
        h = np.float32(2.0 ** (np.floor(np.log2(abs(p[i]) + 1e-3)) - 6))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        yp, ym = orc.mlp_forward(NIN, NH, pp, x, skip=3), orc.mlp_forward(NIN, NH, pm, x, skip=3)
        side = lambda y: np.sign(np.abs(y - t) - delta)
        if not (np.array_equal(side(yp), side(y0)) and np.array_equal(side(ym), side(y0))):
            continue
        if not (np.array_equal(_pattern(pp, x), _pattern(p, x)) and np.array_equal(_pattern(pm, x), _pattern(p, x))):
            continue
        checked += 1
        lp, _ = orc.mlp_loss_grad(NIN, NH, pp, x, t, skip=3, huber_delta=delta)
        lm, _ = orc.mlp_loss_grad(NIN, NH, pm, x, t, skip=3, huber_delta=delta)
        fd = (lp - lm) / (2 * float(h))
        assert abs(fd - g[i]) <= 1e-9 + 1e-6 * abs(g[i]), (i, fd, g[i])
    assert checked >= 20


def test_adam_first_step_moves_by_lr(orc):
    """Adam's bias-corrected first step is -lr * sign(g) (for |g| >> eps)."""
    p = np.array([1.0, -2.0, 0.5], np.float32)
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    orc.adam_step(p, m, v, g, lr=1e-2, step=1)
    np.testing.assert_allclose(p, [0.99, -1.99, 0.49], rtol=0, atol=1e-6)


def test_training_reduces_loss(orc):
    rng = np.random.default_rng(2)
    p = _params(rng) * 0.3
    x = rng.standard_normal((256, NIN)).astype(np.float32)
    t = (x[:, :3].sum(1) * 0.5).astype(np.float32)
    m, v = np.zeros(p.size), np.zeros(p.size)
    l0, _ = orc.mlp_loss_grad(NIN, NH, p, x, t)
    for step in range(1, 201):
        _, g = orc.mlp_loss_grad(NIN, NH, p, x, t)
        orc.adam_step(p, m, v, g, lr=3e-3, step=step)
    l1, _ = orc.mlp_loss_grad(NIN, NH, p, x, t)
    assert l1 < 0.2 * l0
