"""Relative-permeability diagnostic (lbm_phase_flux, Sec. 4.6, Eq. eq-Kp) on the GPU."""
import numpy as np
import pytest

from oracle import observables as ob
from synthetic.geometry import rsa_spheres, spheres_phi0

pytestmark = pytest.mark.gpu


def _channel(L, phi1, steps, nx=64, ny=24, mu=0.1, F=2e-6):
    prm = L.lbm_default_params(rho=(1.0, 1.0, 1.0), mu=(mu, mu, mu), d0=0.5, body_force=(F, 0.0, 0.0),
                               theta_deg=90.0)
    ctx = L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=(True, False, False), params=prm)
    try:
        ctx.set_solid(np.zeros((ny, nx), np.float32))
        ctx.set_phase(phi1.astype(np.float32))
        ctx.step(steps)
        flux = ctx.phase_flux(0, 0)
        phi, u, _ = ctx.get_fields()
    finally:
        ctx.close()
    return flux, phi[0].reshape(ny, nx), u[0].reshape(2, ny, nx)


def test_stratified_channel(lbm_lib):
    L = lbm_lib
    nx, ny = 64, 24
    y = np.arange(ny) + 0.5
    d = np.minimum(y, ny - y)
    phi1 = (0.5 + 0.5 * np.tanh((6 - d) / 2.0))[:, None] * np.ones((1, nx))
    steps = 6000
    two, phi, u = _channel(L, phi1, steps)
    one, _, _ = _channel(L, np.ones((ny, nx)), steps)
    zero, _, _ = _channel(L, np.zeros((ny, nx)), steps)
    # the library's reduction against the oracle's on the same float32 fields
    ref = ob.phase_flux(np.zeros((ny, nx)), phi.astype(np.float64), u.astype(np.float64))
    for k in ("q1", "q2", "q", "s1", "s2"):
        assert np.isclose(two[k], ref[k], rtol=1e-9, atol=0), k
    assert two["n_pore"] == ref["n_pore"] == nx * ny
    K1, K2 = L.relative_permeability(two, one, zero)
    assert abs(K1 + K2 - 1.0) < 1e-5
    ua = y * (ny - y)
    K1_exact = (phi1[:, 0] * ua).sum() / ua.sum()
    assert abs(K1 / K1_exact - 1.0) < 5e-3, (K1, K1_exact)


def test_porous_medium_fluxes(lbm_lib):
    """3D: spheres, the pore space counted with phi0 <= 1/2, fluxes equal to the oracle's sums of the same fields."""
    L = lbm_lib
    n = 32
    spheres = rsa_spheres(n=n, seed=3, rmin=4.0, rmax=6.0, target_solid=0.3)
    phi0 = spheres_phi0((n, n, n), spheres, W=4.0).astype(np.float32)
    zc = np.arange(n)[:, None, None] + 0.5
    phi1 = ((1 - phi0) * (0.5 + 0.5 * np.tanh((8.0 - np.abs(zc - n / 2)) / 2.0))).astype(np.float32)
    prm = L.lbm_default_params(d0=1.0 / 3.0, theta_deg=60.0, body_force=(1e-5, 0.0, 0.0))
    ctx = L.Context(L.LBM_D3Q19, n, n, n, periodic=(True, True, True), params=prm)
    try:
        ctx.set_solid(phi0)
        ctx.set_phase(phi1)
        ctx.step(300)
        fl = [ctx.phase_flux(0, a) for a in range(3)]
        ph, u, _ = ctx.get_fields()
    finally:
        ctx.close()
    ph = ph[0].reshape(n, n, n).astype(np.float64)
    u = u[0].reshape(3, n, n, n).astype(np.float64)
    for a in range(3):
        ref = ob.phase_flux(phi0.astype(np.float64), ph, u, axis=a)
        for k in ("q1", "q2", "q"):
            assert np.isclose(fl[a][k], ref[k], rtol=1e-9, atol=1e-12 * abs(ref["q"]) + 1e-300), (a, k)
        assert fl[a]["n_pore"] == ref["n_pore"]
    assert fl[0]["q"] > 0 and fl[0]["q1"] > 0 and fl[0]["q2"] > 0     # driven along +x
    assert 0.2 < fl[0]["s1"] < 0.8


def test_phase_flux_validation(lbm_lib):
    L = lbm_lib
    ctx = L.Context(L.LBM_D2Q9, 16, 8, 1, periodic=(True, True, False))
    try:
        ctx.set_solid(np.zeros((8, 16), np.float32))
        ctx.set_phase(np.ones((8, 16), np.float32))
        with pytest.raises(L.LbmError):
            ctx.phase_flux(0, 2)               # no z axis in 2D
        with pytest.raises(L.LbmError):
            ctx.phase_flux(1, 0)               # one instance
    finally:
        ctx.close()


def test_phase_flux_of_uneven_instances(lbm_lib):
    """lbm_phase_flux on a multi-size context reads each instance's own block."""
    L = lbm_lib
    sizes = [(32, 24), (48, 40)]
    def disk(nx, ny):
        y, x = np.mgrid[:ny, :nx] + 0.5
        return (0.5 + 0.5 * np.tanh((6.0 - np.hypot(x - nx / 3, y - ny / 2)) / 2.0)).astype(np.float32)
    phi0s = [disk(nx, ny) for nx, ny in sizes]
    phi1s = [((1 - p) * (0.5 + 0.5 * np.tanh((np.mgrid[:p.shape[0], :p.shape[1]][0] + 0.5 - p.shape[0] / 2) / 2.0)))
             .astype(np.float32) for p in phi0s]
    m = L.MultiContext(sizes, periodic=(True, True),
                       batch=[L.lbm_default_params(body_force=(1e-5, 0.0, 0.0)) for _ in sizes])
    try:
        m.set_solid(phi0s)
        m.set_phase(phi1s)
        m.step(50)
        fields = m.get_fields()
        for i, (nx, ny) in enumerate(sizes):
            fl = L.lbm_phase_flux(m.ctx, i, 0)
            ph, u = fields[i][0], fields[i][1]
            ref = ob.phase_flux(phi0s[i].astype(np.float64), ph.reshape(ny, nx).astype(np.float64),
                                u.reshape(2, ny, nx).astype(np.float64), axis=0)
            for k in ("q1", "q2", "q"):
                assert np.isclose(fl[k], ref[k], rtol=1e-9, atol=1e-15), (i, k)
            assert fl["n_pore"] == ref["n_pore"]
    finally:
        m.close()


def test_phase_flux_without_pore_space(lbm_lib):
    """A fully solid instance: no pore nodes, zero fluxes, undefined saturations (NaN), no error."""
    L = lbm_lib
    ctx = L.Context(L.LBM_D2Q9, 16, 8, 1, periodic=(True, True, False))
    try:
        ctx.set_solid(np.full((8, 16), 0.99, np.float32))
        ctx.set_phase(np.zeros((8, 16), np.float32))
        ctx.step(5)
        fl = ctx.phase_flux(0, 0)
    finally:
        ctx.close()
    assert fl["n_pore"] == 0 and fl["q"] == 0.0 and fl["q1"] == 0.0 and fl["q2"] == 0.0
    assert np.isnan(fl["s1"]) and np.isnan(fl["s2"])
