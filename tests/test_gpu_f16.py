"""FP16 storage of the NS populations (D2Q9): accuracy against the oracle and
against the float32 path.

The stored value is g * 2^12 rounded to the nearest FP16 number, a relative
error of at most 2^-12 per value per step; the CH populations, and with them
the conserved phase field, stay float32.  Bars:
* phi1 relative L2 <= 1e-5 after 1000 steps (the float32 bar: the phase field
  only feels the NS rounding through u);
* u and p within 2e-3 (relative L2; u against the run's peak velocity norm),
  eight times the per-value storage rounding 2^-11;
* the contact angle after 20000 steps within 0.5 deg of the float32 run
  (equal angle accuracy, the mixed-precision criterion) and a phase-mass
  drift of both runs within the float32 rate the full-size test allows
  (2e-6 per 400 steps, i.e. 1e-4 over 20000 steps);
* a checkpoint image of an FP16 context restores bitwise.
"""
import numpy as np
import pytest

from _parity import rel_l2
from oracle import lbm as olbm
from oracle import model as omodel
from synthetic import wall_droplet
from synthetic.workloads import flat_wall

pytestmark = pytest.mark.gpu


def _ctx(L, nx, ny, prm, periodic, flags):
    return L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=periodic, params=L.lbm_default_params(**prm), flags=flags)


def test_f16_storage_against_oracle_1000_steps(lbm_lib):
    L = lbm_lib
    geo = wall_droplet(152, 48, 8, 16.0, 4.0, xc=76.0)
    phi0, phi1 = geo.phi0.astype(np.float32), geo.phi1.astype(np.float32)
    prm = dict(theta_deg=60.0, sigma=0.01, d0=0.5)
    ctx = _ctx(L, 152, 48, prm, (True, False, False), L.LBM_STORE_G_F16)
    try:
        ctx.set_solid(phi0)
        ctx.set_phase(phi1)
        ctx.step(1000)
        g_phi1, g_u, g_p = ctx.get_fields()
        g_f, _ = ctx.get_populations()
    finally:
        ctx.close()
    st = olbm.init_state("D2Q9", phi0.astype(np.float64), phi1.astype(np.float64), omodel.Params(**prm),
                         (True, False))
    peak = 0.0
    for _ in range(10):
        olbm.step(st, nsteps=100)
        peak = max(peak, float(np.linalg.norm(st.macro["u"])))
    e_phi = rel_l2(g_phi1[0], st.macro["phi1"])
    e_u = float(np.linalg.norm(g_u[0] - st.macro["u"].reshape(2, -1))) / peak
    e_p = rel_l2(g_p[0], st.macro["p"])
    e_f = rel_l2(g_f[0], st.f.reshape(9, -1))
    print("f16 parity", e_phi, e_u, e_p, e_f)
    assert e_phi <= 1e-5 and e_f <= 1e-5, (e_phi, e_f)
    assert e_u <= 2e-3 and e_p <= 2e-3, (e_u, e_p)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_f16_storage_keeps_the_contact_angle(lbm_lib, theta):
    L = lbm_lib
    wl = flat_wall(theta=theta)
    out = {}
    for flags in (0, L.LBM_STORE_G_F16):
        ctx = _ctx(L, wl["nx"], wl["ny"], wl["params"][0], (True, False, False), flags)
        try:
            ctx.set_solid(wl["phi0"])
            ctx.set_phase(wl["phi1"])
            ctx.step(20000)
            th, _ = ctx.contact_angle(0, 0, wl["nx"] // 2)
            out[flags] = (th, ctx.observables(0)["mass1"])
        finally:
            ctx.close()
    (t32, m32), (t16, m16) = out[0], out[L.LBM_STORE_G_F16]
    m0 = float(np.sum(wl["phi1"].astype(np.float64)))
    print("theta f32 / f16", t32, t16, "mass drift f32 / f16", m32 / m0 - 1.0, m16 / m0 - 1.0)
    assert abs(t16 - t32) < 0.5, (t16, t32)
    assert abs(m16 / m0 - 1.0) < 1e-4 and abs(m32 / m0 - 1.0) < 1e-4, (m0, m32, m16)


def test_f16_checkpoint_restores_bitwise(lbm_lib):
    L = lbm_lib
    wl = flat_wall(theta=60.0)
    a = _ctx(L, wl["nx"], wl["ny"], wl["params"][0], (True, False, False), L.LBM_STORE_G_F16)
    b = _ctx(L, wl["nx"], wl["ny"], wl["params"][0], (True, False, False), L.LBM_STORE_G_F16)
    c = _ctx(L, wl["nx"], wl["ny"], wl["params"][0], (True, False, False), 0)
    try:
        for ctx in (a, b, c):
            ctx.set_solid(wl["phi0"])
        a.set_phase(wl["phi1"])
        a.step(300)
        img = a.get_state()
        b.set_state(img)
        a.step(200)
        b.step(200)
        for x, y in zip(a.get_populations() + a.get_fields(), b.get_populations() + b.get_fields()):
            assert np.array_equal(x, y)
        with pytest.raises(L.LbmError):
            c.set_state(img)          # a float32 context refuses an FP16 image
    finally:
        a.close()
        b.close()
        c.close()


def test_f16_storage_d3q19_against_oracle(lbm_lib):
    from synthetic import sphere_box_droplet
    # nx = 40 (a multiple of 8): TMA tiles of FP16 g in the pipelined kernel
    geo = sphere_box_droplet(40, 20, 18, [(20.0, 6.0, 5.0, 4.5), (30.0, 15.0, 12.0, 5.0)], slab=12.0)
    prm = dict(theta_deg=120.0, sigma=0.01, d0=1.0 / 3.0, body_force=(1e-5, 0.0, 0.0))
    L = lbm_lib
    phi0, phi1 = geo.phi0.astype(np.float32), geo.phi1.astype(np.float32)
    out = {}
    for depth in (1, 2):
        ctx = L.Context(L.LBM_D3Q19, 40, 20, 18, periodic=(True, True, True), params=L.lbm_default_params(**prm),
                        flags=L.LBM_STORE_G_F16)
        try:
            ctx.set_launch(6, depth)
            ctx.set_solid(phi0)
            ctx.set_phase(phi1)
            ctx.step(500)
            out[depth] = ctx.get_fields() + ctx.get_populations()
        finally:
            ctx.close()
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(a, b)          # generic and pipelined kernels agree bitwise
    g_phi1, g_u, g_p, g_f, _ = out[2]
    st = olbm.init_state("D3Q19", phi0.astype(np.float64), phi1.astype(np.float64), omodel.Params(**prm),
                         (True, True, True))
    peak = 0.0
    for _ in range(5):
        olbm.step(st, nsteps=100)
        peak = max(peak, float(np.linalg.norm(st.macro["u"])))
    e_phi = rel_l2(g_phi1[0], st.macro["phi1"])
    e_u = float(np.linalg.norm(g_u[0] - st.macro["u"].reshape(3, -1))) / peak
    e_p = rel_l2(g_p[0], st.macro["p"])
    e_f = rel_l2(g_f[0], st.f.reshape(19, -1))
    print("f16 d3q19 parity", e_phi, e_u, e_p, e_f)
    assert e_phi <= 1e-5 and e_f <= 1e-5, (e_phi, e_f)
    assert e_u <= 2e-3 and e_p <= 2e-3, (e_u, e_p)
