"""Warm-start kernels (include/lbm_nn.h) against the FP64 reference oracle/nn.py.

The reference applies the kernels' BF16 rounding to the same float32 inputs,
so the only differences left are the float32 accumulation order (bounded
relative to the sum of absolute products) and, in a whole network, the BF16
rounding decisions that float32-sized differences flip (measured against
the reference's own sensitivity)."""
import numpy as np
import pytest
import torch

from oracle import nn as onn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nn(lbm_lib):
    from paper_2311_05091_gb300 import _nn
    _nn.library()
    return _nn


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _bf16(nn, W32):
    """Device BF16 copy made by the library's own conversion."""
    src = _dev(W32)
    dst = torch.empty(src.shape, dtype=torch.bfloat16, device="cuda")
    nn.to_bf16(src.data_ptr(), dst.data_ptr(), src.numel())
    return dst


def _rng(seed):
    return np.random.default_rng(seed)


def test_bf16_conversion_is_round_to_nearest_even(nn):
    r = _rng(0)
    a = np.concatenate([r.normal(0, 1, 4096), [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -0.0, 3.0e38]]).astype(np.float32)
    got = _bf16(nn, a).float().cpu().numpy().astype(np.float64)
    assert np.array_equal(got, onn.bf16_round(a))


CONV_SHAPES = [(2, 13, 17, 16, 32, True), (1, 9, 64, 32, 64, False), (3, 8, 8, 64, 32, True),
               (1, 1, 1, 16, 32, False), (1, 33, 5, 48, 96, False), (2, 5, 130, 32, 128, True),
               (1, 7, 200, 16, 256, False), (2, 3, 40, 64, 64, True)]


@pytest.mark.parametrize("n,h,w,cin,cout,relu", CONV_SHAPES)
def test_conv3x3_forward(nn, n, h, w, cin, cout, relu):
    r = _rng(1)
    x = r.normal(0, 1, (n, h, w, cin)).astype(np.float32)
    W = r.normal(0, 0.2, (9, cout, cin)).astype(np.float32)
    b = r.normal(0, 0.1, cout).astype(np.float32)
    xd, bd, yd = _dev(x), _dev(b), torch.full((n, h, w, cout), np.nan, device="cuda")
    Wb = _bf16(nn, W)
    nn.conv3x3(xd.data_ptr(), Wb.data_ptr(), bd.data_ptr(), yd.data_ptr(), n, h, w, cin, cout, relu)
    got = yd.cpu().numpy().astype(np.float64)
    ref = onn.conv3x3(x, W, b.astype(np.float64), bf16=True)
    bound = onn.conv3x3(np.abs(onn.bf16_round(x)), np.abs(onn.bf16_round(W)), np.abs(b.astype(np.float64)),
                        bf16=False)
    if relu:
        ref = np.maximum(ref, 0.0)
    nn.check()                                        # no bounded wait gave up
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)


# cout <= 64 runs the kernel with the three kernel rows folded into M, cout >= 128 the one with a CTA per kernel row
WGRAD_SHAPES = [(2, 13, 17, 16, 32), (1, 70, 70, 32, 16), (1, 8, 8, 48, 32), (2, 40, 64, 64, 64), (1, 12, 70, 32, 128),
                (1, 9, 40, 48, 256), (1, 1, 3, 16, 16), (2, 2, 3, 16, 128)]   # the last two: images of one and two rows


@pytest.mark.parametrize("n,h,w,cin,cout", WGRAD_SHAPES)
def test_conv3x3_weight_and_data_gradients(nn, n, h, w, cin, cout):
    r = _rng(2)
    x = r.normal(0, 1, (n, h, w, cin)).astype(np.float32)
    dy = r.normal(0, 1, (n, h, w, cout)).astype(np.float32)
    W = r.normal(0, 0.2, (9, cout, cin)).astype(np.float32)
    dx_ref, dW_ref, db_ref = onn.conv3x3_grads(x, W, dy, bf16=True)
    xd, dyd = _dev(x), _dev(dy)
    dW = torch.full((9, cout, cin), np.nan, device="cuda")
    db = torch.full((cout,), np.nan, device="cuda")
    ws = nn.wgrad_workspace(n, h, w, cin, cout)
    work = torch.empty(ws, device="cuda")
    nn.conv3x3_wgrad(xd.data_ptr(), dyd.data_ptr(), dW.data_ptr(), db.data_ptr(), work.data_ptr(), ws, n, h, w, cin,
                     cout)
    xr, dyr = np.abs(onn.bf16_round(x)), np.abs(onn.bf16_round(dy))
    _, bound, _ = onn.conv3x3_grads(xr, np.zeros_like(W), dyr, bf16=False)
    got = dW.cpu().numpy()
    assert np.all(np.abs(got - dW_ref) <= 1e-5 * bound + 1e-30)
    np.testing.assert_allclose(db.cpu().numpy(), db_ref, rtol=1e-5, atol=1e-5 * np.abs(dy).sum(axis=(0, 1, 2)).max())
    # data gradient: the forward kernel with the flipped, transposed weights (needs cin % 32 == 0)
    if cin % 32 == 0:
        Wb = _bf16(nn, W)
        Wf = torch.empty((9, cin, cout), dtype=torch.bfloat16, device="cuda")
        nn.flip_transpose(Wb.data_ptr(), Wf.data_ptr(), cin, cout)
        wf_host = Wf.float().cpu().numpy()
        assert np.array_equal(wf_host, onn.bf16_round(W)[::-1].transpose(0, 2, 1))
        dx = torch.full((n, h, w, cin), np.nan, device="cuda")
        nn.conv3x3(dyd.data_ptr(), Wf.data_ptr(), 0, dx.data_ptr(), n, h, w, cout, cin, 0)
        bx = onn.conv3x3_grads(np.zeros_like(x), np.abs(onn.bf16_round(W)), dyr, bf16=False)[0]
        assert np.all(np.abs(dx.cpu().numpy() - dx_ref) <= 1e-5 * bx + 1e-30)


def test_wgrad_is_deterministic(nn):
    r = _rng(3)
    n, h, w, cin, cout = 2, 64, 80, 32, 64
    xd = _dev(r.normal(0, 1, (n, h, w, cin)))
    dyd = _dev(r.normal(0, 1, (n, h, w, cout)))
    ws = nn.wgrad_workspace(n, h, w, cin, cout)
    work = torch.empty(ws, device="cuda")
    outs = []
    for _ in range(2):
        dW = torch.empty((9, cout, cin), device="cuda")
        db = torch.empty((cout,), device="cuda")
        nn.conv3x3_wgrad(xd.data_ptr(), dyd.data_ptr(), dW.data_ptr(), db.data_ptr(), work.data_ptr(), ws, n, h, w,
                         cin, cout)
        outs.append((dW.cpu(), db.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("c", [32, 6])          # float4 path (c % 4 == 0) and the scalar path
def test_pooling_upsampling_relu_add_pack(nn, c):
    r = _rng(4)
    n, h, w = 2, 10, 14
    x = r.normal(0, 1, (n, h, w, c)).astype(np.float32)
    xd = _dev(x)                       # every device input is held by a name while kernels use it
    y = torch.empty((n, h // 2, w // 2, c), device="cuda")
    nn.pool2(xd.data_ptr(), y.data_ptr(), n, h, w, c)
    np.testing.assert_allclose(y.cpu().numpy(), onn.pool2(x.astype(np.float64)), rtol=1e-6, atol=1e-7)
    g = r.normal(0, 1, (n, h // 2, w // 2, c)).astype(np.float32)
    gd = _dev(g)
    gx = torch.empty((n, h, w, c), device="cuda")
    nn.pool2(gd.data_ptr(), gx.data_ptr(), n, h, w, c, backward=True)
    np.testing.assert_allclose(gx.cpu().numpy(), onn.pool2_adj(g.astype(np.float64)), rtol=1e-7)
    u = torch.empty((n, h, w, c), device="cuda")
    nn.up2(gd.data_ptr(), u.data_ptr(), n, h // 2, w // 2, c)
    np.testing.assert_array_equal(u.cpu().numpy(), onn.up2(g))
    ua = torch.empty((n, h // 2, w // 2, c), device="cuda")
    nn.up2(xd.data_ptr(), ua.data_ptr(), n, h // 2, w // 2, c, backward=True)
    np.testing.assert_allclose(ua.cpu().numpy(), onn.up2_adj(x.astype(np.float64)), rtol=1e-6, atol=1e-6)
    # ReLU adjoint, out of place and in place; add (m = 1000: float4 path, 999: scalar path)
    m = 1000 if c % 4 == 0 else 999
    yv = r.normal(0, 1, m).astype(np.float32)
    dy = r.normal(0, 1, m).astype(np.float32)
    dyd, yvd, out = _dev(dy), _dev(yv), torch.empty(m, device="cuda")
    nn.relu_bwd(dyd.data_ptr(), yvd.data_ptr(), out.data_ptr(), m)
    np.testing.assert_array_equal(out.cpu().numpy(), np.where(yv > 0, dy, 0.0))
    nn.relu_bwd(dyd.data_ptr(), yvd.data_ptr(), dyd.data_ptr(), m)
    np.testing.assert_array_equal(dyd.cpu().numpy(), np.where(yv > 0, dy, 0.0))
    a, b = _dev(dy), _dev(yv)
    nn.add(a.data_ptr(), a.data_ptr(), b.data_ptr(), -0.5, m)
    np.testing.assert_array_equal(a.cpu().numpy(), (dy + np.float32(-0.5) * yv).astype(np.float32))
    # network input
    phi0 = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    phi1 = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    ct = np.array([0.5, -0.25], np.float32)
    p0d, p1d, ctd = _dev(phi0), _dev(phi1), _dev(ct)
    xin = torch.full((n, h, w, 16), np.nan, device="cuda")
    nn.pack_input(p0d.data_ptr(), p1d.data_ptr(), ctd.data_ptr(), xin.data_ptr(), n, h, w)
    xi = xin.cpu().numpy()
    np.testing.assert_array_equal(xi[..., 0], phi0)
    np.testing.assert_array_equal(xi[..., 1], phi1)
    np.testing.assert_array_equal(xi[..., 2], np.broadcast_to(ct[:, None, None], (n, h, w)))
    assert np.all(xi[..., 3:] == 0)


def test_mse_adam_projection(nn):
    r = _rng(5)
    n, h, w, cp = 3, 20, 24, 32
    P = n * h * w
    out = r.normal(0, 0.2, (n, h, w, cp)).astype(np.float32)
    base = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    target = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    dout = torch.full((n, h, w, cp), np.nan, device="cuda")
    work = torch.empty(4096, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    outd, based, tgd = _dev(out), _dev(base), _dev(target)
    nn.mse_residual(outd.data_ptr(), cp, based.data_ptr(), tgd.data_ptr(), dout.data_ptr(), work.data_ptr(), 4096,
                    loss.data_ptr(), P)
    l_ref, d_ref = onn.mse_residual(out.astype(np.float64), base.astype(np.float64), target.astype(np.float64))
    assert abs(loss.item() - l_ref) <= 1e-6 * l_ref
    np.testing.assert_allclose(dout.cpu().numpy(), d_ref, rtol=1e-5, atol=1e-9)
    # three Adam steps against the reference update
    m0 = 5000
    wv = r.normal(0, 1, m0).astype(np.float32)
    wd, md, vd = _dev(wv), torch.zeros(m0, device="cuda"), torch.zeros(m0, device="cuda")
    wb = torch.empty(m0, dtype=torch.bfloat16, device="cuda")
    wr, mr, vr = wv.astype(np.float64), np.zeros(m0), np.zeros(m0)
    for t in range(1, 4):
        gv = r.normal(0, 1, m0).astype(np.float32)
        gvd = _dev(gv)
        nn.adam(wd.data_ptr(), md.data_ptr(), vd.data_ptr(), gvd.data_ptr(), wb.data_ptr(), m0, 1e-2, 0.9, 0.999, 1e-8,
                t)
        wr, mr, vr = onn.adam(wr, mr, vr, gv.astype(np.float64), 1e-2, 0.9, 0.999, 1e-8, t)
    np.testing.assert_allclose(wd.cpu().numpy(), wr, rtol=1e-6, atol=3e-7)
    np.testing.assert_allclose(md.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)
    assert np.array_equal(wb.float().cpu().numpy().astype(np.float64), onn.bf16_round(wd.cpu().numpy()))
    # projection onto [0, 1 - phi0] with the initial phase mass
    phi0 = np.clip(r.normal(0, 0.4, (n, h, w)), 0, 1).astype(np.float32)
    phi1 = np.clip(r.uniform(0, 1, (n, h, w)), 0, 1 - phi0).astype(np.float32)
    p0d, p1d = _dev(phi0), _dev(phi1)
    field = torch.empty((n, h, w), device="cuda")
    nn.project(outd.data_ptr(), cp, p0d.data_ptr(), p1d.data_ptr(), field.data_ptr(), work.data_ptr(), 4096, n, h, w)
    ref = onn.project(out[..., 0].astype(np.float64), phi0.astype(np.float64), phi1.astype(np.float64))
    got = field.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
    for i in range(n):
        assert abs(got[i].sum(dtype=np.float64) - phi1[i].sum(dtype=np.float64)) <= 1e-5 * phi1[i].sum()


@pytest.mark.parametrize("widths,n,h,w", [((32, 64), 2, 16, 24), ((32, 64, 128, 256), 1, 32, 40)])
def test_network_forward_backward(nn, widths, n, h, w):
    from paper_2311_05091_gb300.warmstart import WarmStartNet
    net = WarmStartNet(widths=widths, n=n, h=h, w=w, seed=3)
    r = _rng(6)
    for b in net.b:                                     # non-zero biases exercise the bias paths
        b.copy_(torch.tensor(r.normal(0, 0.05, b.numel()), dtype=torch.float32))
    net.refresh()
    phi0 = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    phi1 = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    target = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    ct = r.uniform(-1, 1, n).astype(np.float32)
    p0, p1, tg, cd = _dev(phi0), _dev(phi1), _dev(target), _dev(ct)
    x = net.pack(p0, p1, cd)
    out = net.forward(x)
    P = n * h * w
    nn.mse_residual(out.data_ptr(), 32, p1.data_ptr(), tg.data_ptr(), net.act["dout"].data_ptr(),
                    net.dwork.data_ptr(), net.dwork.numel(), net.loss.data_ptr(), P)
    net.backward(net.act["dout"])
    torch.cuda.synchronize()

    params = [(W.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)) for W, b in zip(net.W, net.b)]
    xr = x.cpu().numpy().astype(np.float64)

    def reference(prm):
        o, cache = onn.forward(xr, prm, list(widths), bf16=True)
        lo, do = onn.mse_residual(o, phi1.astype(np.float64), target.astype(np.float64))
        return o, lo, onn.backward(do, prm, list(widths), cache, bf16=True)

    out_ref, loss_ref, grads = reference(params)
    # The BF16 roundings make a network's output a discontinuous function of its
    # inputs: float32-sized differences in accumulation order flip a few
    # roundings, and the changed outputs flip more in the next layer.  Each
    # kernel is held to 1e-5 of the sum of absolute products by the tests
    # above; here the whole network (the wiring of every operation) is held to
    # 1e-3 on the output and every gradient, or to 4x the reference's own
    # change under a 1e-7 relative perturbation of the weights when that is
    # larger (15 convolutions: 2.5e-3).
    rp = np.random.default_rng(7)
    out_p, _, grads_p = reference([(W * (1 + 1e-7 * rp.normal(0, 1, W.shape)), b) for W, b in params])
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    bar_out = max(1e-3, 4 * rel(out_p, out_ref))
    assert rel(out.cpu().numpy(), out_ref) < bar_out
    assert abs(net.loss.item() - loss_ref) < bar_out * loss_ref
    for k, (dW, db) in enumerate(grads):
        assert rel(net.dW[k].cpu().numpy(), dW) < max(1e-3, 4 * rel(grads_p[k][0], dW)), k
        assert rel(net.db[k].cpu().numpy(), db) < max(1e-3, 4 * rel(grads_p[k][1], db)), k
