"""What the learned warm start gains over the method without it, on a small case.

A three-level network is trained on the GPU by the library's own kernels on
solver-generated labels (64^2 lattices of the batched distribution, labels
after T plain steps), then evaluated on held-out seeds: K plain steps from the
warm-start field against K plain steps from the initial field, both measured
against the T-step plain run (the method itself decides).  The warm
start must cut the error of the short run clearly, and the lattice Boltzmann
steps after it must keep the phase mass of the initial field."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

N_TRAIN, N_EVAL, SIDE, T, K = 160, 16, 64, 4000, 400


@pytest.fixture(scope="module")
def libs(lbm_lib):
    from paper_2311_05091_gb300 import _nn
    _nn.library()
    return lbm_lib


def _run(L, s, phase, steps):
    """Plain method from `phase` (host array or device tensor) for `steps` steps; phi1 afterwards (host)."""
    n, N = s["n"], len(s["params"])
    ctx = L.Context(L.LBM_D2Q9, n, n, 1, periodic=(True, True, False),
                    batch=[L.lbm_default_params(**p) for p in s["params"]])
    try:
        ctx.set_solid(s["phi0"])
        if isinstance(phase, torch.Tensor):
            ctx.set_phase_device(phase.data_ptr())
        else:
            ctx.set_phase(phase)
        ctx.step(steps)
        return ctx.get_fields()[0].reshape(N, n, n)
    finally:
        ctx.close()


def test_trained_warm_start_beats_the_plain_start(libs):
    from paper_2311_05091_gb300.warmstart import WarmStartNet, fit, predict_all
    from synthetic.workloads import warmstart_set
    L = libs
    train = warmstart_set(range(5000, 5000 + N_TRAIN), SIDE)
    ev = warmstart_set(range(9000, 9000 + N_EVAL), SIDE)
    target = _run(L, train, train["phi1"], T)
    assert np.isfinite(target).all()
    dev = torch.device("cuda", 0)
    todev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ct = lambda s: todev(np.cos(np.radians(s["theta_deg"])).astype(np.float32))
    net = WarmStartNet(widths=(32, 64, 128), n=16, h=SIDE, w=SIDE, seed=1)
    curve = fit(net, todev(train["phi0"]), todev(train["phi1"]), ct(train), todev(target), iters=600, lr=2e-3)
    assert curve[-1][1] < 0.5 * curve[0][1], curve

    e0, e1 = todev(ev["phi0"]), todev(ev["phi1"])
    warm = torch.empty_like(e1)
    predict_all(net, e0, e1, ct(ev), warm)
    ref = _run(L, ev, ev["phi1"], T)
    plain_K = _run(L, ev, ev["phi1"], K)
    warm_K = _run(L, ev, warm, K)
    err = lambda a: np.linalg.norm((a - ref).reshape(N_EVAL, -1), axis=1) / np.linalg.norm(ref.reshape(N_EVAL, -1),
                                                                                         axis=1)
    e_plain, e_warm, e_net = err(plain_K), err(warm_K), err(warm.cpu().numpy())
    msg = f"plain {e_plain.mean():.4f}, warm start {e_warm.mean():.4f}, network field {e_net.mean():.4f}"
    assert e_warm.mean() < 0.7 * e_plain.mean(), msg
    assert np.median(e_warm / e_plain) < 0.8, msg
    # the warm-start field carries the initial phase mass, and the steps after it keep it
    m0 = ev["phi1"].sum(axis=(1, 2), dtype=np.float64)
    np.testing.assert_allclose(warm.cpu().numpy().sum(axis=(1, 2), dtype=np.float64), m0, rtol=1e-5)
    np.testing.assert_allclose(warm_K.sum(axis=(1, 2), dtype=np.float64), m0, rtol=1e-4)
