"""FP64 reference of the learned warm start network (not part of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A small U-Net with additive skips maps the input tensor x[n, y, x, 16]
(channels: phi0, phi1, cos theta, zeros) to a residual whose channel 0 is
added to phi1.  Every operation is written out plainly in float64:

* conv3x3: zero padding, stride 1, y = b + sum_tap shift(x, tap) W[tap]^T with
  W[tap] of shape (cout, cin), tap = 3 ky + kx.  With ``bf16=True`` the
  operands are first rounded to float32 and then to the nearest BF16 value
  (ties to even), the rounding the tensor-core kernels apply to their inputs.
* pool2 (2x2 mean), up2 (nearest), ReLU, MSE on the residual prediction.
* Architecture for widths C[0..L-1]: encoder level l (l > 0 after pool2):
  e_l = relu(conv(relu(conv(in)))); decoder level l = L-2 .. 0:
  s_l = relu(conv(up2(d_{l+1}))) + e_l, d_l = relu(conv(s_l)) with d_{L-1} =
  e_{L-1}; output o = conv(d_0) into ``cout_pad`` channels, prediction
  phi1 + o[..., 0].
* Backward by the chain rule, each adjoint written out next to its forward.
* Adam (Kingma and Ba) and the mass-preserving projection of the prediction.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Nearest BF16 value of float32(a) (round to nearest, ties to even), as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = a32.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, ky, kx):
    """x[n, y + ky - 1, x + kx - 1, c] with zeros outside."""
    n, h, w, c = x.shape
    p = np.zeros((n, h + 2, w + 2, c))
    p[:, 1:h + 1, 1:w + 1, :] = x
    return p[:, ky:ky + h, kx:kx + w, :]


def conv3x3(x, W, b=None, bf16=True):
    """y[n, y, x, co] = b[co] + sum_{ky, kx, ci} x[n, y+ky-1, x+kx-1, ci] W[3ky+kx, co, ci]."""
    if bf16:
        x, W = bf16_round(x), bf16_round(W)
    n, h, w, cin = x.shape
    cout = W.shape[1]
    y = np.zeros((n, h, w, cout))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        y += _shift(x, ky, kx).reshape(-1, cin).dot(W[tap].T).reshape(n, h, w, cout)
    if b is not None:
        y += b
    return y


def conv3x3_grads(x, W, dy, bf16=True):
    """Adjoints of conv3x3 before its activation: (dx, dW, db)."""
    xr, Wr, dyr = (bf16_round(x), bf16_round(W), bf16_round(dy)) if bf16 else (x, W, dy)
    n, h, w, cin = x.shape
    cout = W.shape[1]
    dW = np.zeros_like(W, dtype=np.float64)
    dx = np.zeros((n, h, w, cin))
    d2 = dyr.reshape(-1, cout)
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        dW[tap] = d2.T.dot(_shift(xr, ky, kx).reshape(-1, cin))
        # the input pixel q = p + shift receives dy[p] W[tap]: shift dy the other way
        dx += _shift((d2.dot(Wr[tap])).reshape(n, h, w, cin), 2 - ky, 2 - kx)
    db = np.asarray(dy, dtype=np.float64).reshape(-1, cout).sum(axis=0)
    return dx, dW, db


def pool2(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool2_adj(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_adj(dy):
    n, h, w, c = dy.shape
    return dy.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


def layer_shapes(widths, cin=16, cout_pad=32):
    """(cin, cout) of every convolution in forward order."""
    L = len(widths)
    shapes = []
    prev = cin
    for l in range(L):
        shapes += [(prev, widths[l]), (widths[l], widths[l])]
        prev = widths[l]
    for l in range(L - 2, -1, -1):
        shapes += [(widths[l + 1], widths[l]), (widths[l], widths[l])]
    shapes.append((widths[0], cout_pad))
    return shapes


def forward(x, params, widths, bf16=True):
    """Output tensor and the cache of every intermediate the backward pass needs."""
    L = len(widths)
    k = 0
    cache = {"x": x}
    e = []
    h = x
    for l in range(L):
        if l > 0:
            h = pool2(h)
        cache[f"enc_in{l}"] = h
        a = relu(conv3x3(h, *params[k], bf16=bf16))
        cache[f"enc_a{l}"] = a
        h = relu(conv3x3(a, *params[k + 1], bf16=bf16))
        cache[f"enc_e{l}"] = h
        e.append(h)
        k += 2
    d = e[L - 1]
    for l in range(L - 2, -1, -1):
        u = up2(d)
        cache[f"dec_u{l}"] = u
        r = relu(conv3x3(u, *params[k], bf16=bf16))
        cache[f"dec_r{l}"] = r
        s = r + e[l]
        cache[f"dec_s{l}"] = s
        d = relu(conv3x3(s, *params[k + 1], bf16=bf16))
        cache[f"dec_d{l}"] = d
        k += 2
    cache["d0"] = d
    out = conv3x3(d, *params[k], bf16=bf16)
    return out, cache


def backward(dout, params, widths, cache, bf16=True):
    """Gradients (dW, db) of every convolution, in forward order."""
    L = len(widths)
    nconv = len(params)
    grads = [None] * nconv
    k = nconv - 1
    dd, grads[k] = _conv_back(cache["d0"], params[k], dout, None, bf16)
    de = [None] * L
    for l in range(0, L - 1):
        k2 = 2 * L + 2 * (L - 2 - l)     # index of the first decoder conv of level l
        # d_l = relu(conv(s_l)), s_l = r_l + e_l, r_l = relu(conv(u_l))
        ds, grads[k2 + 1] = _conv_back(cache[f"dec_s{l}"], params[k2 + 1], dd, cache[f"dec_d{l}"], bf16)
        de[l] = ds
        du, grads[k2] = _conv_back(cache[f"dec_u{l}"], params[k2], ds, cache[f"dec_r{l}"], bf16)
        dd = up2_adj(du)
    # dd now is the gradient of d_{L-1} = e_{L-1}
    g = dd
    for l in range(L - 1, -1, -1):
        if de[l] is not None and l < L - 1:
            g = g + de[l]
        k = 2 * l
        da, grads[k + 1] = _conv_back(cache[f"enc_a{l}"], params[k + 1], g, cache[f"enc_e{l}"], bf16)
        dh, grads[k] = _conv_back(cache[f"enc_in{l}"], params[k], da, cache[f"enc_a{l}"], bf16)
        if l > 0:
            g = pool2_adj(dh)
    return grads


def _conv_back(x, param, dy_post, y_post, bf16):
    """Through relu (if y_post is given) and conv: (dx, (dW, db))."""
    dy = dy_post if y_post is None else dy_post * (y_post > 0)
    dx, dW, db = conv3x3_grads(x, param[0], dy, bf16)
    return dx, (dW, db)


def mse_residual(out, base, target):
    """Loss sum_p (base + out[..., 0] - target)^2 and its gradient with respect to out (mean scaling 2/P)."""
    pred = base + out[..., 0]
    d = pred - target
    P = d.size
    dout = np.zeros_like(out)
    dout[..., 0] = 2.0 * d / P
    return float(np.sum(d * d)), dout


def adam(w, m, v, g, lr, b1, b2, eps, t):
    """One Adam step with bias correction (Kingma and Ba): new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def project(out0, phi0, phi1, passes=3):
    """Warm-start field of images (leading axis n) from the network's channel 0.

    q = clamp(phi1 + out0, 0, hi) with hi = max(1 - phi0, 0); then ``passes``
    times per image q += lambda b(q) with b(q) = q (hi - q) / hi (0 where
    hi = 0) and lambda = clamp((sum phi1 - sum q) / sum b, -1, 1).  For
    |lambda| <= 1 the update is monotone in q with fixed points 0 and hi, so
    the field stays in [0, hi] while its mass moves to that of phi1.
    """
    hi = np.maximum(1.0 - phi0, 0.0)
    q = np.minimum(np.clip(phi1 + out0, 0.0, None), hi)
    safe = np.where(hi > 0, hi, 1.0)
    for i in range(q.shape[0]):
        for _ in range(passes):
            bump = np.where(hi[i] > 0, q[i] * (hi[i] - q[i]) / safe[i], 0.0)
            c = bump.sum()
            lam = float(np.clip((phi1[i].sum() - q[i].sum()) / c, -1.0, 1.0)) if c > 0 else 0.0
            q[i] = q[i] + lam * bump
    return q
