"""The allocation-free diagnostics entry point, for callers that cannot allocate
device memory when they ask for these numbers (their memory belongs to a host
application's pool, or a cudaMalloc would stall a latency-bound loop).

It must return what lbm_observables returns for the same fields, on two calls
in a row: the second call finds the first call's partial sums still in the
library's fixed record array and must not be affected by them.  This file is
collected last so that, should it fail, a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from synthetic import wall_droplet
from synthetic.workloads import disk_sweep

pytestmark = pytest.mark.gpu


def _context_fields(L, phi0, phi1, nx, ny, periodic, params, steps):
    ctx = L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=periodic, batch=params)
    ctx.set_solid(phi0)
    ctx.set_phase(phi1)
    ctx.step(steps)
    obs = [ctx.observables(b) for b in range(len(params))]
    fields = ctx.get_fields()
    ctx.close()
    return obs, fields


def _noalloc(L, phi0, phi1, u, p):
    import torch
    dev = torch.device("cuda", 0)
    n = phi1.size
    t0 = torch.from_numpy(np.ascontiguousarray(phi0.ravel())).to(dev)
    t1 = torch.from_numpy(np.ascontiguousarray(phi1.ravel())).to(dev)
    tu = torch.from_numpy(np.ascontiguousarray(u.reshape(-1))).to(dev)
    tp = torch.from_numpy(np.ascontiguousarray(p.ravel())).to(dev)
    out = torch.full((8,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = L.lbm_observables_noalloc(t0.data_ptr(), t1.data_ptr(), tu.data_ptr(), u.shape[0], tp.data_ptr(), n,
                                   out.data_ptr(), stream.cuda_stream)
    assert rc == 0, L.lbm_strerror(rc)
    stream.synchronize()
    return out.cpu().numpy(), (t0, t1, tu, tp, out, stream)


def _check(r, obs):
    assert abs(r[0] - obs["mass1"]) <= 1e-12 * abs(obs["mass1"])
    assert abs(r[1] - obs["mass0"]) <= 1e-12 * abs(obs["mass0"]) + 1e-300
    assert r[2] == obs["umax"]
    assert int(r[4]) == obs["n_in"] and int(r[6]) == obs["n_out"] and r[7] == 0
    dp = r[3] / r[4] - r[5] / r[6]
    assert abs(dp - obs["dp"]) <= 1e-9 * abs(obs["dp"]) + 1e-15


def test_noalloc_matches_observables_on_two_calls(lbm_lib):
    L = lbm_lib
    # call 1: one 1024^2 instance of the benchmark workload (1024 partial records)
    wl = disk_sweep(thetas=(60.0,))
    obs, (phi1, u, p) = _context_fields(L, wl["phi0"], wl["phi1"], 1024, 1024, (True, True, False),
                                        [L.lbm_default_params(**wl["params"][0])], 300)
    r1, _ = _noalloc(L, wl["phi0"][0], phi1[0], u[0], p[0])
    _check(r1, obs[0])
    # call 2: a small walled lattice (8 records) right after; stale records beyond 8 must not leak in
    geo = wall_droplet(150, 48, 8, 16.0, 4.0)
    phi0s = geo.phi0.astype(np.float32)
    obs2, (phi1s, us, ps) = _context_fields(L, phi0s[None], geo.phi1.astype(np.float32)[None], 150, 48,
                                            (True, False, False), [L.lbm_default_params(theta_deg=60.0)], 200)
    r2, keep = _noalloc(L, phi0s, phi1s[0], us[0], ps[0])
    _check(r2, obs2[0])
    # sizes beyond the fixed record array, and bad arguments, are refused before any launch
    t0, t1, tu, tp, out, stream = keep
    assert L.lbm_observables_noalloc(t0.data_ptr(), t1.data_ptr(), tu.data_ptr(), 2, tp.data_ptr(),
                                     16777217, out.data_ptr(), stream.cuda_stream) == -1
    assert L.lbm_observables_noalloc(t0.data_ptr(), t1.data_ptr(), tu.data_ptr(), 4, tp.data_ptr(),
                                     100, out.data_ptr(), stream.cuda_stream) == -1
    assert L.lbm_observables_noalloc(0, t1.data_ptr(), tu.data_ptr(), 2, tp.data_ptr(),
                                     100, out.data_ptr(), stream.cuda_stream) == -1


def test_noalloc_at_the_size_limit_in_3d(lbm_lib):
    # n = 16,777,216 nodes fills every one of the 16,384 records, with three velocity planes (a 256^3 field);
    # checked against float64 sums of the same float32 values on the host
    L = lbm_lib
    import torch
    n = 16_777_216
    rng = np.random.default_rng(7)
    phi0 = rng.random(n, dtype=np.float32) * 0.5
    phi1 = (rng.random(n, dtype=np.float32) * (1.0 - phi0)).astype(np.float32)
    phi1[::97] = 0.995                     # bulk fluid 1 ...
    phi0[::89] = 0.0
    phi1[::89] = 0.0                       # ... and bulk fluid 2
    u = (rng.standard_normal((3, n), dtype=np.float32) * 1e-3).astype(np.float32)
    p = rng.standard_normal(n, dtype=np.float32)
    for _ in range(2):
        r, _keep = _noalloc(L, phi0, phi1, u, p)
        del _keep
        torch.cuda.empty_cache()
        assert abs(r[0] - phi1.astype(np.float64).sum()) <= 1e-12 * phi1.astype(np.float64).sum()
        assert abs(r[1] - phi0.astype(np.float64).sum()) <= 1e-12 * phi0.astype(np.float64).sum()
        umax = float(np.sqrt((u.astype(np.float64) ** 2).sum(axis=0)).max())
        assert abs(r[2] - umax) <= 1e-6 * umax
        inside = phi1 >= np.float32(0.99)
        outside = (np.float32(1.0) - phi0 - phi1) >= np.float32(0.99)
        assert int(r[4]) == int(inside.sum()) > 0 and int(r[6]) == int(outside.sum()) > 0 and r[7] == 0
        ps = p.astype(np.float64)
        assert abs(r[3] - ps[inside].sum()) <= 1e-9 * np.abs(ps[inside]).sum()
        assert abs(r[5] - ps[outside].sum()) <= 1e-9 * np.abs(ps[outside]).sum()
