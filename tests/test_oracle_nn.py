"""Pins of the FP64 reference of the learned warm start (oracle/nn.py) to
things other than itself: PyTorch's BF16 conversion and convolution on the
CPU, PyTorch autograd, finite differences, adjoint identities and the mass
invariant of the projection."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import nn as onn


def _rng(seed=0):
    return np.random.default_rng(seed)


def _torch_conv(x, W, b):
    """x (n, h, w, cin), W (9, cout, cin) -> (n, h, w, cout) by torch conv2d (cross-correlation), float64."""
    cout, cin = W.shape[1], W.shape[2]
    wt = torch.from_numpy(W.reshape(3, 3, cout, cin).transpose(2, 3, 0, 1).copy())
    xt = torch.from_numpy(x.transpose(0, 3, 1, 2).copy())
    y = F.conv2d(xt, wt, torch.from_numpy(b) if b is not None else None, padding=1)
    return y.numpy().transpose(0, 2, 3, 1)


def test_bf16_round_matches_torch_conversion():
    r = _rng(1)
    a = np.concatenate([r.normal(0, 1, 5000), r.normal(0, 1e-3, 1000), r.normal(0, 1e4, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1.0078125, -3.5, 65504.0]])
    a32 = a.astype(np.float32)
    ref = torch.from_numpy(a32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(onn.bf16_round(a32), ref)
    # ties go to the even neighbour: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert onn.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert onn.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


@pytest.mark.parametrize("shape", [(1, 5, 7, 16, 32), (2, 8, 6, 32, 64), (1, 3, 3, 48, 32)])
def test_conv3x3_matches_torch_conv2d(shape):
    n, h, w, cin, cout = shape
    r = _rng(2)
    x = r.normal(0, 1, (n, h, w, cin))
    W = r.normal(0, 0.2, (9, cout, cin))
    b = r.normal(0, 0.1, cout)
    np.testing.assert_allclose(onn.conv3x3(x, W, b, bf16=False), _torch_conv(x, W, b), rtol=1e-12, atol=1e-12)
    # with rounding: the exact convolution of the rounded operands
    np.testing.assert_allclose(onn.conv3x3(x, W, b, bf16=True),
                               _torch_conv(onn.bf16_round(x), onn.bf16_round(W), b), rtol=1e-12, atol=1e-12)


def test_conv3x3_grads_match_autograd():
    r = _rng(3)
    n, h, w, cin, cout = 2, 6, 5, 16, 32
    x = r.normal(0, 1, (n, h, w, cin))
    W = r.normal(0, 0.2, (9, cout, cin))
    dy = r.normal(0, 1, (n, h, w, cout))
    xt = torch.tensor(x.transpose(0, 3, 1, 2), requires_grad=True)
    wt = torch.tensor(W.reshape(3, 3, cout, cin).transpose(2, 3, 0, 1), requires_grad=True)
    bt = torch.zeros(cout, dtype=torch.float64, requires_grad=True)
    y = F.conv2d(xt, wt, bt, padding=1)
    y.backward(torch.from_numpy(dy.transpose(0, 3, 1, 2).copy()))
    dx, dW, db = onn.conv3x3_grads(x, W, dy, bf16=False)
    np.testing.assert_allclose(dx, xt.grad.numpy().transpose(0, 2, 3, 1), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(dW, wt.grad.numpy().transpose(2, 3, 0, 1).reshape(9, cout, cin), rtol=1e-11,
                               atol=1e-11)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_pool_and_upsampling_adjoints():
    r = _rng(4)
    x = r.normal(0, 1, (2, 8, 6, 3))
    y = r.normal(0, 1, (2, 4, 3, 3))
    assert np.isclose(np.sum(onn.pool2(x) * y), np.sum(x * onn.pool2_adj(y)), rtol=1e-13)
    assert np.isclose(np.sum(onn.up2(y) * x), np.sum(y * onn.up2_adj(x)), rtol=1e-13)
    # pooling a constant keeps it; upsampling then pooling is the identity
    np.testing.assert_allclose(onn.pool2(np.full((1, 4, 4, 2), 3.5)), 3.5)
    np.testing.assert_allclose(onn.pool2(onn.up2(y)), y, rtol=1e-14)
    # pooling is the mean of each 2x2 block
    assert np.isclose(onn.pool2(x)[1, 2, 1, 0], x[1, 4:6, 2:4, 0].mean())


def test_layer_shapes_of_the_default_network():
    shapes = onn.layer_shapes([32, 64, 128, 256])
    assert len(shapes) == 15
    assert shapes[0] == (16, 32) and shapes[7] == (256, 256) and shapes[8] == (256, 128) and shapes[-1] == (32, 32)
    weights = sum(9 * ci * co + co for ci, co in shapes)
    assert 1.5e6 < weights < 2.0e6


def _tiny(seed=5, widths=(32, 64), n=1, h=8, w=8):
    r = _rng(seed)
    params = [(r.normal(0, np.sqrt(2.0 / (9 * ci)), (9, co, ci)), r.normal(0, 0.05, co))
              for ci, co in onn.layer_shapes(list(widths))]
    x = r.normal(0, 1, (n, h, w, 16))
    base = r.normal(0, 1, (n, h, w))
    target = r.normal(0, 1, (n, h, w))
    return params, x, base, target


def _loss(params, x, base, target, widths):
    out, _ = onn.forward(x, params, widths, bf16=False)
    return onn.mse_residual(out, base, target)[0] / base.size


def test_network_gradient_matches_finite_differences():
    widths = (32, 64)
    params, x, base, target = _tiny()
    out, cache = onn.forward(x, params, widths, bf16=False)
    _, dout = onn.mse_residual(out, base, target)
    grads = onn.backward(dout, params, widths, cache, bf16=False)
    r = _rng(6)
    eps = 1e-7          # below the smallest distance of a pre-activation to a ReLU kink (4e-5 here)
    for k in range(len(params)):
        for which in (0, 1):
            d = r.normal(0, 1, params[k][which].shape)
            plus = [list(p) for p in params]
            minus = [list(p) for p in params]
            plus[k][which] = params[k][which] + eps * d
            minus[k][which] = params[k][which] - eps * d
            fd = (_loss(plus, x, base, target, widths) - _loss(minus, x, base, target, widths)) / (2 * eps)
            # mse_residual's gradient is that of the mean squared error
            an = np.sum(grads[k][which] * d)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, which, fd, an)


def test_network_gradient_three_levels_matches_autograd():
    """A second, independent restatement of the whole network in torch autograd (float64)."""
    widths = (32, 64, 128)
    params, x, base, target = _tiny(seed=7, widths=widths, n=2, h=8, w=8)
    out, cache = onn.forward(x, params, widths, bf16=False)
    loss, dout = onn.mse_residual(out, base, target)
    grads = onn.backward(dout, params, widths, cache, bf16=False)

    Wt = [torch.tensor(W.reshape(3, 3, W.shape[1], W.shape[2]).transpose(2, 3, 0, 1), requires_grad=True)
          for W, _ in params]
    bt = [torch.tensor(b, requires_grad=True) for _, b in params]
    conv = lambda h, k: F.conv2d(h, Wt[k], bt[k], padding=1)
    h = torch.from_numpy(x.transpose(0, 3, 1, 2).copy())
    e, k = [], 0
    for l in range(3):
        if l:
            h = F.avg_pool2d(h, 2)
        h = torch.relu(conv(torch.relu(conv(h, k)), k + 1))
        e.append(h)
        k += 2
    d = e[-1]
    for l in (1, 0):
        s = torch.relu(conv(F.interpolate(d, scale_factor=2, mode="nearest"), k)) + e[l]
        d = torch.relu(conv(s, k + 1))
        k += 2
    o = conv(d, k)
    pred = torch.from_numpy(base) + o[:, 0]
    lt = ((pred - torch.from_numpy(target)) ** 2).sum()
    lt.backward()
    assert np.isclose(loss, lt.item(), rtol=1e-12)
    np.testing.assert_allclose(out, o.detach().numpy().transpose(0, 2, 3, 1), rtol=1e-10, atol=1e-12)
    P = base.size
    for k in range(len(params)):
        gW = Wt[k].grad.numpy().transpose(2, 3, 0, 1).reshape(grads[k][0].shape) / P
        np.testing.assert_allclose(grads[k][0], gW, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(grads[k][1], bt[k].grad.numpy() / P, rtol=1e-9, atol=1e-12)


def test_mse_residual_gradient():
    r = _rng(8)
    out = r.normal(0, 1, (2, 4, 5, 32))
    base, target = r.normal(0, 1, (2, 4, 5)), r.normal(0, 1, (2, 4, 5))
    loss, dout = onn.mse_residual(out, base, target)
    assert np.isclose(loss, np.sum((base + out[..., 0] - target) ** 2))
    assert np.all(dout[..., 1:] == 0)
    i = (1, 2, 3, 0)
    e = 1e-6
    o2 = out.copy()
    o2[i] += e
    fd = (onn.mse_residual(o2, base, target)[0] - loss) / e / base.size
    assert abs(fd - dout[i]) < 1e-5


def test_adam_first_step_moves_by_lr_times_sign():
    # at t = 1 the bias-corrected step is lr g / (|g| + eps)
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    w1, m, v = onn.adam(w, np.zeros(3), np.zeros(3), g, 1e-2, 0.9, 0.999, 1e-12, 1)
    np.testing.assert_allclose(w1, w - 1e-2 * np.sign(g), rtol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    # f(w) = |w - 3|^2: Adam with a decaying step converges to the minimiser
    w, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 3001):
        w, m, v = onn.adam(w, m, v, 2.0 * (w - 3.0), 0.1 / np.sqrt(t), 0.9, 0.999, 1e-8, t)
    np.testing.assert_allclose(w, 3.0, atol=1e-3)


def test_projection_restores_mass_and_bounds():
    r = _rng(9)
    n, h, w = 3, 16, 12
    phi0 = np.clip(r.normal(0, 0.4, (n, h, w)), 0, 1)
    phi1 = np.clip(r.uniform(0, 1, (n, h, w)), 0, 1 - phi0)
    hi = 1 - phi0
    for scale, bias in ((0.3, 0.0), (0.2, 0.15), (0.2, -0.15)):
        out0 = r.normal(bias, scale, (n, h, w))
        field = onn.project(out0, phi0, phi1)
        assert field.min() >= 0.0 and np.all(field <= hi + 1e-15)
        for i in range(n):
            assert np.isclose(field[i].sum(), phi1[i].sum(), rtol=1e-6), (scale, bias)
    # an exact prediction (in range, right mass) is returned unchanged
    np.testing.assert_allclose(onn.project(np.zeros_like(phi1), phi0, phi1), phi1, atol=1e-15)
    # a prediction clamped everywhere to 0 or hi has no room to move: the correction vanishes
    hard = onn.project(np.where(phi1 > 0.5, 5.0, -5.0), phi0, phi1)
    assert np.all((hard == 0.0) | np.isclose(hard, hi))


def test_projection_update_is_monotone_for_bounded_lambda():
    hi = 0.8
    q = np.linspace(0.0, hi, 2001)
    for lam in (-1.0, -0.5, 0.5, 1.0):
        v = q + lam * q * (hi - q) / hi
        assert np.all(np.diff(v) >= -1e-15) and v[0] == 0.0 and np.isclose(v[-1], hi) and v.min() >= 0 \
            and v.max() <= hi + 1e-15
