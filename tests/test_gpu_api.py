"""Behaviour of the C ABI on the GPU: checkpoint / resume, graph replay, divergence
detection, error states, diagnostics, streams."""
import numpy as np
import pytest

from _parity import as_inputs, gpu_run
from synthetic import cylinder_droplet, wall_droplet

pytestmark = pytest.mark.gpu


def _ctx(L, geo, prm, periodic=(True, False, False)):
    ny, nx = geo.phi0.shape
    ctx = L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=periodic, params=L.lbm_default_params(**prm))
    phi0, phi1 = as_inputs(geo)
    ctx.set_solid(phi0)
    ctx.set_phase(phi1)
    return ctx


def test_checkpoint_resume_is_bitwise(lbm_lib):
    L = lbm_lib
    geo = wall_droplet(150, 48, 8, 16.0, 4.0)
    prm = dict(theta_deg=60.0, rho=(2.0, 2.0, 1.0), mu=(0.02, 0.02, 0.01))
    a = _ctx(L, geo, prm)
    a.step(100)
    image = a.get_state()
    a.step(100)
    fa, ga = a.get_populations()
    pa = a.get_fields()
    b = _ctx(L, geo, prm)
    b.set_state(image)
    b.step(100)
    fb, gb = b.get_populations()
    pb = b.get_fields()
    assert b.observables(0)["step"] == 200
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
    a.close()
    b.close()
    # an image of another shape is refused
    c = _ctx(L, wall_droplet(64, 48, 8, 10.0, 4.0), prm)
    with pytest.raises(L.LbmError) as e:
        c.set_state(image)
    assert e.value.status == -1
    c.close()


def test_graph_replay_matches_direct_launches(lbm_lib):
    L = lbm_lib
    geo = cylinder_droplet(n=128, Rs=20.0, R0=15.0, W=4.0)
    prm = dict(theta_deg=100.0, kappa=0.75, rho=(5.0, 5.0, 1.0), mu=(0.05, 0.05, 0.01))
    a = _ctx(L, geo, prm, (True, True, False))
    a.step(50)                      # 16-step graphs + direct tail
    b = _ctx(L, geo, prm, (True, True, False))
    b.set_profiling(True)           # direct launches only
    b.step(50)
    ms, n = b.kernel_time()
    assert n == 50 and ms > 0
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()


def test_divergence_is_reported_not_faulted(lbm_lib):
    L = lbm_lib
    geo = cylinder_droplet(n=64, Rs=10.0, R0=8.0, W=4.0)
    ctx = _ctx(L, geo, dict(theta_deg=90.0, kappa=0.8, body_force=(0.2, 0.0, 0.0)), (True, True, False))
    ctx.step(40)
    with pytest.raises(L.LbmError) as e:
        ctx.sync()
    assert e.value.status == -4
    ctx.close()


def test_state_errors(lbm_lib):
    L = lbm_lib
    ctx = L.Context(L.LBM_D2Q9, 32, 32, 1, periodic=(True, True, False), params=L.lbm_default_params())
    with pytest.raises(L.LbmError) as e:
        ctx.step(1)
    assert e.value.status == -6
    with pytest.raises(L.LbmError) as e:
        ctx.set_phase(np.zeros(32 * 32, np.float32))     # solid not set yet
    assert e.value.status == -6
    with pytest.raises(L.LbmError) as e:
        ctx.observables(0)
    assert e.value.status == -6
    ctx.set_solid(np.zeros(32 * 32, np.float32))
    ctx.set_phase(np.zeros(32 * 32, np.float32))
    with pytest.raises(L.LbmError) as e:
        ctx.step(-1)
    assert e.value.status == -1
    with pytest.raises(L.LbmError) as e:
        ctx.observables(3)
    assert e.value.status == -1
    ctx.close()


def test_observables_match_host_sums(lbm_lib):
    L = lbm_lib
    geo = wall_droplet(150, 48, 8, 16.0, 4.0)
    ctx = _ctx(L, geo, dict(theta_deg=60.0))
    ctx.step(300)
    obs = ctx.observables(0)
    phi1, u, p = ctx.get_fields()
    phi0 = geo.phi0.astype(np.float32).ravel()
    assert abs(obs["mass1"] - phi1[0].astype(np.float64).sum()) < 1e-12 * obs["mass1"]
    assert abs(obs["mass0"] - phi0.astype(np.float64).sum()) < 1e-12 * obs["mass0"]
    umag = np.sqrt((u[0].astype(np.float32) ** 2).sum(0))
    assert abs(obs["umax"] - umag.max()) < 1e-6 * umag.max()
    inside = phi1[0] >= 0.99
    outside = (1.0 - phi0 - phi1[0]) >= 0.99
    assert obs["n_in"] == inside.sum() and obs["n_out"] == outside.sum()
    dp = p[0][inside].astype(np.float64).mean() - p[0][outside].astype(np.float64).mean()
    assert abs(obs["dp"] - dp) < 1e-9 * abs(dp) + 1e-15
    ctx.close()


def test_caller_stream(lbm_lib):
    import torch
    L = lbm_lib
    geo = wall_droplet(96, 40, 6, 12.0, 4.0)
    a = _ctx(L, geo, dict(theta_deg=70.0))
    s = torch.cuda.Stream()
    a.set_stream(s.cuda_stream)
    a.step(40)
    a.sync()
    b = _ctx(L, geo, dict(theta_deg=70.0))
    b.step(40)
    assert np.array_equal(a.get_populations()[0], b.get_populations()[0])
    a.close()
    b.close()


def test_context_on_the_torch_caching_allocator(lbm_lib):
    """lbm_create_alloc with PyTorch's caching allocator and stream: the memory is accounted by PyTorch, returned
    at destruction, and the run is bitwise the run of a context that allocates for itself."""
    import torch
    L = lbm_lib
    from synthetic import free_drop
    geo = free_drop(48, 40, R=10.0)
    prm = L.lbm_default_params(sigma=0.01)
    ref = L.Context(L.LBM_D2Q9, 48, 40, 1, periodic=(True, True, False), params=prm)
    try:
        ref.set_solid(geo.phi0.astype(np.float32))
        ref.set_phase(geo.phi1.astype(np.float32))
        ref.step(120)
        want = ref.get_fields()
    finally:
        ref.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    stream = torch.cuda.Stream()
    alloc = L.TorchAllocator()
    ctx = L.Context(L.LBM_D2Q9, 48, 40, 1, periodic=(True, True, False), params=prm, allocator=alloc,
                    stream=stream.cuda_stream)
    try:
        # populations (2 x 2 x 9), history (2 x 5), phi0, p: 42 floats per node at least
        assert torch.cuda.memory_allocated() - before >= 42 * 4 * 48 * 40
        ctx.set_solid(geo.phi0.astype(np.float32))
        ctx.set_phase(geo.phi1.astype(np.float32))
        ctx.step(120)
        got = ctx.get_fields()
        ctx.tune(2)                                   # the autotuner's save area comes from the same allocator
    finally:
        ctx.close()
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    assert torch.cuda.memory_allocated() == before


def test_d3q19_context_on_the_torch_caching_allocator(lbm_lib):
    """The 3D pipelined kernel's tensor maps are built on the caller's memory: bitwise the default context's run."""
    import torch
    L = lbm_lib
    n = 24
    zc, yc, xc = np.mgrid[:n, :n, :n] + 0.5
    phi1 = (0.5 + 0.5 * np.tanh((6.0 - np.sqrt((xc - 12) ** 2 + (yc - 12) ** 2 + (zc - 12) ** 2)) / 2.0))
    prm = L.lbm_default_params(d0=1.0 / 3.0, sigma=0.01)
    out = []
    for alloc in (None, L.TorchAllocator()):
        ctx = L.Context(L.LBM_D3Q19, n, n, n, periodic=(True, True, True), params=prm, allocator=alloc)
        try:
            ctx.set_solid(np.zeros((n, n, n), np.float32))
            ctx.set_phase(phi1.astype(np.float32))
            ctx.step(60)
            out.append(ctx.get_fields())
        finally:
            ctx.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
