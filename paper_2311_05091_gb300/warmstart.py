"""Learned warm start: a small U-Net trained on solver runs, then plain lattice Boltzmann relaxation.

Not part of the paper.  The network maps (solid indicator phi0, initial phase
field phi1, cos theta) on a 2D lattice to a residual added to phi1; the
result, clamped to [0, 1 - phi0] and corrected to the initial phase mass
(``lbm_nn_project``), becomes the initial field of an ordinary run, whose
steps decide the final state.

Architecture for widths C[0..L-1] (default 32, 64, 128, 256: 15 convolutions,
1.76 M weights): encoder level l (after 2x2 average pooling for l > 0)
e_l = relu(conv(relu(conv(in)))); decoder level l = L-2 .. 0:
s_l = relu(conv(up2(d_{l+1}))) + e_l, d_l = relu(conv(s_l)), d_{L-1} = e_{L-1};
output conv(d_0) into 32 channels, channel 0 used.  Every operation is a
kernel of ``include/lbm_nn.h``; this module only orders the calls and owns
the buffers (PyTorch tensors used as device memory).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _nn

CIN, COUT_PAD = 16, 32


def layer_shapes(widths):
    L = len(widths)
    shapes, prev = [], CIN
    for l in range(L):
        shapes += [(prev, widths[l]), (widths[l], widths[l])]
        prev = widths[l]
    for l in range(L - 2, -1, -1):
        shapes += [(widths[l + 1], widths[l]), (widths[l], widths[l])]
    shapes.append((widths[0], COUT_PAD))
    return shapes


def _p(t):
    return t.data_ptr()


def forward_flops(widths, h, w):
    """Multiply-add FLOPs (2 per MAC) of the network's convolutions for one h x w image."""
    L = len(widths)
    fl = 0
    for k, (ci, co) in enumerate(layer_shapes(widths)):
        lv = k // 2 if k < 2 * L else (0 if k == 2 * L + 2 * (L - 1) else L - 2 - (k - 2 * L) // 2)
        fl += 2 * 9 * ci * co * (h >> lv) * (w >> lv)
    return fl


def train_flops(widths, h, w):
    """FLOPs of one training image: forward, data gradients (every convolution but the first) and weight gradients."""
    first = 2 * 9 * CIN * widths[0] * h * w
    f = forward_flops(widths, h, w)
    return 3 * f - first


class WarmStartNet:
    """Weights, optimiser state and activation buffers for n images of size h x w."""

    def __init__(self, widths=(32, 64, 128, 256), n=4, h=256, w=256, seed=0, device="cuda"):
        self.widths = tuple(widths)
        self.L = len(widths)
        self.n, self.h, self.w = n, h, w
        self.dev = device
        assert self.L >= 2 and h % (1 << (self.L - 1)) == 0 and w % (1 << (self.L - 1)) == 0
        rng = np.random.default_rng(seed)
        self.shapes = layer_shapes(self.widths)
        self.W, self.b = [], []
        for k, (ci, co) in enumerate(self.shapes):
            # He initialisation; the output layer starts small so the first prediction is close to phi1
            std = np.sqrt(2.0 / (9 * ci)) * (0.1 if k == len(self.shapes) - 1 else 1.0)
            self.W.append(torch.tensor(rng.normal(0.0, std, (9, co, ci)), dtype=torch.float32, device=device))
            self.b.append(torch.zeros(co, dtype=torch.float32, device=device))
        self._alloc_weights()
        self._alloc_acts(n)
        self.t = 0

    # -- buffers ---------------------------------------------------------------
    def _alloc_weights(self):
        z = lambda t: torch.zeros_like(t)
        self.Wb = [torch.empty(W.shape, dtype=torch.bfloat16, device=self.dev) for W in self.W]
        self.Wf = [torch.empty((9, W.shape[2], W.shape[1]), dtype=torch.bfloat16, device=self.dev) for W in self.W]
        self.dW = [z(W) for W in self.W]
        self.db = [z(b) for b in self.b]
        self.mW = [z(W) for W in self.W]
        self.vW = [z(W) for W in self.W]
        self.mb = [z(b) for b in self.b]
        self.vb = [z(b) for b in self.b]
        self.refresh()

    def refresh(self):
        """BF16 copies and the flipped, transposed copies used by the data gradient."""
        for k, (ci, co) in enumerate(self.shapes):
            _nn.to_bf16(_p(self.W[k]), _p(self.Wb[k]), self.W[k].numel())
            _nn.flip_transpose(_p(self.Wb[k]), _p(self.Wf[k]), ci, co)

    def _alloc_acts(self, n):
        self.n = n
        f = lambda h, w, c: torch.empty((n, h, w, c), dtype=torch.float32, device=self.dev)
        H, Wd = self.h, self.w
        self.act = {}
        for l in range(self.L):
            h, w, c = H >> l, Wd >> l, self.widths[l]
            if l > 0:
                self.act[f"in{l}"] = f(h, w, self.widths[l - 1])
            self.act[f"a{l}"] = f(h, w, c)
            self.act[f"e{l}"] = f(h, w, c)
            if l < self.L - 1:
                self.act[f"u{l}"] = f(h, w, self.widths[l + 1])
                self.act[f"r{l}"] = f(h, w, c)
                self.act[f"s{l}"] = f(h, w, c)
                self.act[f"d{l}"] = f(h, w, c)
                self.act[f"gu{l}"] = f(h, w, self.widths[l + 1])
            self.act[f"g{l}"] = f(h, w, c)      # gradient buffers of each level
            self.act[f"g2{l}"] = f(h, w, c)
            self.act[f"gs{l}"] = f(h, w, c)
        self.act["x"] = f(H, Wd, CIN)
        self.act["out"] = f(H, Wd, COUT_PAD)
        self.act["dout"] = f(H, Wd, COUT_PAD)
        ws = max(_nn.wgrad_workspace(n, H >> self._lvl(k), Wd >> self._lvl(k), ci, co)
                 for k, (ci, co) in enumerate(self.shapes))
        self.work = torch.empty(ws, dtype=torch.float32, device=self.dev)
        self.dwork = torch.empty(max(192 * n, (n * H * Wd + 127) // 128 + 8), dtype=torch.float64, device=self.dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)

    def _lvl(self, k):
        """Resolution level (0 finest) of convolution k."""
        L = self.L
        if k < 2 * L:
            return k // 2
        if k == len(self.shapes) - 1:
            return 0
        return L - 2 - (k - 2 * L) // 2

    # -- forward / backward ------------------------------------------------------
    def _conv(self, k, x, y, relu):
        ci, co = self.shapes[k]
        lv = self._lvl(k)
        _nn.conv3x3(_p(x), _p(self.Wb[k]), _p(self.b[k]), _p(y), self.n, self.h >> lv, self.w >> lv, ci, co, relu)

    def _back(self, k, x, dy, dx):
        """Gradients of conv k from dy (already through its ReLU); dx receives the data gradient (or None)."""
        ci, co = self.shapes[k]
        lv = self._lvl(k)
        n, h, w = self.n, self.h >> lv, self.w >> lv
        _nn.conv3x3_wgrad(_p(x), _p(dy), _p(self.dW[k]), _p(self.db[k]), _p(self.work), self.work.numel(),
                          n, h, w, ci, co)
        if dx is not None:
            _nn.conv3x3(_p(dy), _p(self.Wf[k]), 0, _p(dx), n, h, w, co, ci, 0)

    def forward(self, x):
        """x: (n, h, w, 16) float32 device tensor; returns the (n, h, w, 32) output buffer."""
        A, L = self.act, self.L
        k = 0
        h = x
        for l in range(L):
            if l > 0:
                c = self.widths[l - 1]
                _nn.pool2(_p(A[f"e{l - 1}"]), _p(A[f"in{l}"]), self.n, self.h >> (l - 1), self.w >> (l - 1), c)
                h = A[f"in{l}"]
            self._conv(k, h, A[f"a{l}"], True)
            self._conv(k + 1, A[f"a{l}"], A[f"e{l}"], True)
            k += 2
        d = A[f"e{L - 1}"]
        for l in range(L - 2, -1, -1):
            _nn.up2(_p(d), _p(A[f"u{l}"]), self.n, self.h >> (l + 1), self.w >> (l + 1), self.widths[l + 1])
            self._conv(k, A[f"u{l}"], A[f"r{l}"], True)
            _nn.add(_p(A[f"s{l}"]), _p(A[f"r{l}"]), _p(A[f"e{l}"]), 1.0, A[f"s{l}"].numel())
            self._conv(k + 1, A[f"s{l}"], A[f"d{l}"], True)
            d = A[f"d{l}"]
            k += 2
        self._conv(k, d, A["out"], False)
        return A["out"]

    def backward(self, dout):
        """Fills dW, db from the gradient of the (n, h, w, 32) output (forward must have run on this batch)."""
        A, L = self.act, self.L
        nconv = len(self.shapes)
        dd = A["g0"]
        self._back(nconv - 1, A["d0"], dout, dd)
        for l in range(0, L - 1):
            k2 = 2 * L + 2 * (L - 2 - l)       # first decoder convolution of level l
            # d_l = relu(conv(s_l)); the gradient of s_l goes to the skip (e_l) and to r_l
            _nn.relu_bwd(_p(dd), _p(A[f"d{l}"]), _p(dd), dd.numel())
            ds = A[f"gs{l}"]
            self._back(k2 + 1, A[f"s{l}"], dd, ds)
            dr = A[f"g2{l}"]
            _nn.relu_bwd(_p(ds), _p(A[f"r{l}"]), _p(dr), dr.numel())
            du = A[f"gu{l}"]
            self._back(k2, A[f"u{l}"], dr, du)
            nxt = A[f"g{l + 1}"]
            _nn.up2(_p(du), _p(nxt), self.n, self.h >> (l + 1), self.w >> (l + 1), self.widths[l + 1], backward=True)
            dd = nxt
        g = dd                                   # gradient of e_{L-1}
        for l in range(L - 1, -1, -1):
            if l < L - 1:
                _nn.add(_p(g), _p(g), _p(A[f"gs{l}"]), 1.0, g.numel())
            k = 2 * l
            _nn.relu_bwd(_p(g), _p(A[f"e{l}"]), _p(g), g.numel())
            da = A[f"g2{l}"]
            self._back(k + 1, A[f"a{l}"], g, da)
            _nn.relu_bwd(_p(da), _p(A[f"a{l}"]), _p(da), da.numel())
            if l > 0:
                dh = A[f"gu{l - 1}"]             # large enough for (n, h_l, w_l, C[l-1]); free at this point
                self._back(k, A[f"in{l}"], da, dh)
                g = A[f"g{l - 1}"]
                _nn.pool2(_p(dh), _p(g), self.n, self.h >> (l - 1), self.w >> (l - 1), self.widths[l - 1],
                          backward=True)
            else:
                self._back(k, A["x"], da, None)

    def step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        """Adam on every weight and bias, then the flipped copies for the next data gradients."""
        self.t += 1
        for k in range(len(self.shapes)):
            _nn.adam(_p(self.W[k]), _p(self.mW[k]), _p(self.vW[k]), _p(self.dW[k]), _p(self.Wb[k]),
                     self.W[k].numel(), lr, b1, b2, eps, self.t)
            _nn.adam(_p(self.b[k]), _p(self.mb[k]), _p(self.vb[k]), _p(self.db[k]), 0, self.b[k].numel(), lr, b1,
                     b2, eps, self.t)
        for k, (ci, co) in enumerate(self.shapes):
            _nn.flip_transpose(_p(self.Wb[k]), _p(self.Wf[k]), ci, co)

    # -- data in and out ---------------------------------------------------------
    def pack(self, phi0, phi1, costh):
        """phi0, phi1: (n, h, w) device tensors; costh: (n,) device tensor -> input buffer."""
        _nn.pack_input(_p(phi0), _p(phi1), _p(costh), _p(self.act["x"]), self.n, self.h, self.w)
        return self.act["x"]

    def train_step(self, phi0, phi1, costh, target, lr):
        """One Adam step on the batch; returns the device tensor holding the batch's summed squared error."""
        x = self.pack(phi0, phi1, costh)
        out = self.forward(x)
        P = self.n * self.h * self.w
        _nn.mse_residual(_p(out), COUT_PAD, _p(phi1), _p(target), _p(self.act["dout"]), _p(self.dwork),
                         self.dwork.numel(), _p(self.loss), P)
        self.backward(self.act["dout"])
        self.step(lr)
        return self.loss

    def predict(self, phi0, phi1, costh, field):
        """Warm-start field (n, h, w) device tensor: the projected residual prediction."""
        x = self.pack(phi0, phi1, costh)
        out = self.forward(x)
        _nn.project(_p(out), COUT_PAD, _p(phi0), _p(phi1), _p(field), _p(self.dwork), self.dwork.numel(),
                    self.n, self.h, self.w)
        return field

    def state(self):
        return {"widths": self.widths, "W": [W.cpu().numpy() for W in self.W], "b": [b.cpu().numpy() for b in self.b]}

    def load(self, st):
        for k in range(len(self.shapes)):
            self.W[k].copy_(torch.from_numpy(st["W"][k]))
            self.b[k].copy_(torch.from_numpy(st["b"][k]))
        self.refresh()


def fit(net, phi0, phi1, costh, target, iters, lr=2e-3, lr_end=1e-4, warmup=50, seed=0, log_every=50):
    """Train ``net`` on device tensors phi0, phi1, target (N, h, w) and costh (N,).

    Mini-batches of net.n samples are drawn without replacement per epoch
    (seeded), Adam with a linear warm-up of ``warmup`` iterations and then a
    cosine decay from lr to lr_end.  Returns [(iteration, mean squared error
    per pixel of the batch)] every ``log_every`` iterations."""
    N = phi0.shape[0]
    B = net.n
    assert N >= B
    rng = np.random.default_rng(seed)
    bufs = [torch.empty((B,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device) for t in (phi0, phi1, costh, target)]
    perm, pos, log = rng.permutation(N), 0, []
    P = B * net.h * net.w
    for it in range(iters):
        if pos + B > N:
            perm, pos = rng.permutation(N), 0
        idx = torch.from_numpy(perm[pos:pos + B]).to(phi0.device)
        pos += B
        for src, dst in zip((phi0, phi1, costh, target), bufs):
            torch.index_select(src, 0, idx, out=dst)
        if it < warmup:
            rate = lr * (it + 1) / warmup
        else:
            x = (it - warmup) / max(1, iters - warmup)
            rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + np.cos(np.pi * x))
        loss = net.train_step(bufs[0], bufs[1], bufs[2], bufs[3], rate)
        if (it + 1) % log_every == 0 or it == iters - 1:
            log.append((it + 1, loss.item() / P))
    return log


def predict_all(net, phi0, phi1, costh, out):
    """Warm-start fields for every sample, net.n at a time; out (N, h, w) device tensor, N >= net.n.

    A ragged tail is covered by the last net.n samples (the overlap is computed twice, with equal results)."""
    N, B = phi0.shape[0], net.n
    assert N >= B
    for lo in range(0, N, B):
        lo = min(lo, N - B)
        net.predict(phi0[lo:lo + B], phi1[lo:lo + B], costh[lo:lo + B], out[lo:lo + B])
    return out
