"""Velocity inlet / pressure outlet (lbm_set_inout) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import lbm as olbm
from oracle import model as omodel
from _parity import rel_l2

pytestmark = pytest.mark.gpu


def _run_both(L, lattice, phi0, phi1, prm, periodic, u_in, phi_in, p_out, mode, steps, flags=0):
    d = 2 if lattice == "D2Q9" else 3
    shape = phi0.shape
    nx, ny = shape[-1], shape[-2]
    nz = 1 if d == 2 else shape[0]
    lat = {"D2Q9": L.LBM_D2Q9, "D3Q19": L.LBM_D3Q19, "D3Q15": L.LBM_D3Q15}[lattice]
    per = tuple(periodic) + (False,) * (3 - len(periodic))
    ctx = L.Context(lat, nx, ny, nz, periodic=per, params=L.lbm_default_params(**prm), flags=flags)
    try:
        ctx.set_solid(phi0)
        ctx.set_phase(phi1)
        ctx.set_inout(mode, u_in, -1.0 if phi_in is None else phi_in, 0.0 if p_out is None else p_out)
        ctx.step(steps)
        g_phi1, g_u, g_p = ctx.get_fields()
    finally:
        ctx.close()
    st = olbm.init_state(lattice, phi0.astype(np.float64), phi1.astype(np.float64), omodel.Params(**prm),
                         tuple(periodic))
    st.inout = olbm.InOut(u_in=None if not mode & 1 else u_in.astype(np.float64),
                          phi_in=phi_in, p_out=p_out if mode & 2 else None)
    olbm.step(st, nsteps=steps)
    n = phi0.size
    o_u = st.macro["u"].reshape(d, n)
    errs = dict(phi1=rel_l2(g_phi1[0], st.macro["phi1"]),
                u=float(np.linalg.norm(g_u[0].astype(np.float64) - o_u) / np.linalg.norm(o_u)),
                p=rel_l2(g_p[0], st.macro["p"]))
    return errs, (g_phi1[0], g_u[0], g_p[0]), st


def test_d2q9_poiseuille_channel(lbm_lib):
    nx, ny, U = 64, 16, 0.02
    prm = dict(rho=(1.0, 1.0, 1.0), mu=(0.1, 0.1, 0.1), d0=0.5)
    y = np.arange(ny) + 0.5
    prof = 1.5 * U * (1.0 - ((y - ny / 2) / (ny / 2)) ** 2)
    u_in = np.stack([prof, 0 * prof]).astype(np.float32)
    errs, _, _ = _run_both(lbm_lib, "D2Q9", np.zeros((ny, nx), np.float32), np.ones((ny, nx), np.float32), prm,
                           (False, False), u_in, 1.0, 0.0, 3, 500)
    print("parity", errs)
    assert errs["phi1"] <= 1e-6 and errs["u"] <= 1e-5 and errs["p"] <= 1e-4, errs


def test_d2q9_droplet_carried_through_an_open_channel(lbm_lib):
    """Two phases with density ratio 2: fluid 2 enters at x = 0 and carries a fluid-1 droplet to the outlet."""
    nx, ny = 96, 32
    yy, xx = np.mgrid[:ny, :nx] + 0.5
    phi1 = (0.5 + 0.5 * np.tanh((8.0 - np.hypot(xx - 30, yy - 16)) / 2.0)).astype(np.float32)
    phi0 = np.zeros((ny, nx), np.float32)
    prm = dict(rho=(1.0, 2.0, 1.0), mu=(0.05, 0.05, 0.05), d0=0.5, theta_deg=90.0)
    u_in = np.stack([np.full(ny, 0.01), np.zeros(ny)]).astype(np.float32)
    errs, (phi_g, u_g, _), st = _run_both(lbm_lib, "D2Q9", phi0, phi1, prm, (False, False), u_in, 0.0, 0.0, 3, 400)
    print("parity", errs)
    assert errs["phi1"] <= 1e-5 and errs["u"] <= 1e-5, errs
    # the droplet moved downstream
    xc0 = (phi1 * xx).sum() / phi1.sum()
    ph = phi_g.reshape(ny, nx)
    assert (ph * xx).sum() / ph.sum() > xc0 + 1.0


def test_d2q9_inlet_only_and_outlet_only(lbm_lib):
    nx, ny = 40, 12
    prm = dict(rho=(1.0, 1.0, 1.0), mu=(0.1, 0.1, 0.1), d0=0.5)
    phi1 = np.ones((ny, nx), np.float32)
    phi0 = np.zeros((ny, nx), np.float32)
    u_in = np.stack([np.full(ny, 0.005), np.full(ny, 0.001)]).astype(np.float32)
    e1, _, _ = _run_both(lbm_lib, "D2Q9", phi0, phi1, prm, (False, True), u_in, None, None, 1, 200)
    # outlet only, on a lattice pushed by a body force against the wall at x = 0
    prm2 = dict(prm, body_force=(-1e-5, 0.0, 0.0))
    e2, _, _ = _run_both(lbm_lib, "D2Q9", phi0, phi1, prm2, (False, True), None, None, 0.001, 2, 200)
    print("parity", e1, e2)
    assert e1["phi1"] <= 1e-6 and e1["u"] <= 1e-5, e1
    assert e2["phi1"] <= 1e-6 and e2["u"] <= 1e-5, e2


@pytest.mark.parametrize("lattice", ["D3Q19", "D3Q15"])
def test_3d_duct(lbm_lib, lattice):
    nx, ny, nz = 24, 10, 8
    prm = dict(rho=(1.0, 1.0, 1.0), mu=(0.1, 0.1, 0.1), d0=1.0 / 3.0,
               eta_hat=0.05 if lattice == "D3Q15" else 0.1)
    zz, yy = np.mgrid[:nz, :ny] + 0.5
    prof = 0.02 * (1 - ((yy - ny / 2) / (ny / 2)) ** 2) * (1 - ((zz - nz / 2) / (nz / 2)) ** 2)
    u_in = np.stack([prof, 0 * prof, 0 * prof]).astype(np.float32)
    zc, yc, xc = np.mgrid[:nz, :ny, :nx] + 0.5
    phi1 = (0.5 + 0.5 * np.tanh((3.5 - np.sqrt((xc - 8) ** 2 + (yc - 5) ** 2 + (zc - 4) ** 2)) / 2.0))
    errs, _, _ = _run_both(lbm_lib, lattice, np.zeros((nz, ny, nx), np.float32), phi1.astype(np.float32), prm,
                           (False, False, False), u_in, 0.0, 0.0, 3, 150)
    print("parity", errs)
    assert errs["phi1"] <= 1e-5 and errs["u"] <= 1e-5, errs


def test_inout_with_fp16_storage_matches_float32(lbm_lib):
    """FP16 NS populations go through the same boundary arithmetic (loads and stores scaled)."""
    L = lbm_lib
    nx, ny = 64, 16
    prm = L.lbm_default_params(rho=(1.0, 1.0, 1.0), mu=(0.1, 0.1, 0.1), d0=0.5)
    y = np.arange(ny) + 0.5
    prof = 0.03 * (1.0 - ((y - ny / 2) / (ny / 2)) ** 2)
    u_in = np.stack([prof, 0 * prof]).astype(np.float32)
    out = []
    for flags in (0, L.LBM_STORE_G_F16):
        ctx = L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=(False, False, False), params=prm, flags=flags)
        try:
            ctx.set_solid(np.zeros((ny, nx), np.float32))
            ctx.set_phase(np.ones((ny, nx), np.float32))
            ctx.set_inout(3, u_in, 1.0, 0.0)
            ctx.step(1000)
            out.append(ctx.get_fields()[1][0].copy())
        finally:
            ctx.close()
    assert rel_l2(out[1], out[0]) < 2e-3


def test_set_inout_validation(lbm_lib):
    L = lbm_lib
    ctx = L.Context(L.LBM_D2Q9, 16, 8, 1, periodic=(True, False, False))
    try:
        with pytest.raises(L.LbmError):            # periodic x
            ctx.set_inout(1, np.zeros((2, 8), np.float32), 1.0, 0.0)
        ctx.set_inout(0)                          # turning it off is always allowed
    finally:
        ctx.close()
    ctx = L.Context(L.LBM_D2Q9, 16, 8, 1, periodic=(False, False, False))
    try:
        with pytest.raises(L.LbmError):            # too fast
            ctx.set_inout(1, np.full((2, 8), 0.7, np.float32), 1.0, 0.0)
        with pytest.raises(L.LbmError):
            ctx.set_inout(4)
    finally:
        ctx.close()
    ctx = L.Context(L.LBM_D2Q9, 3, 8, 1, periodic=(False, False, False))
    try:
        with pytest.raises(L.LbmError):            # inlet and outlet columns need nx >= 4
            ctx.set_inout(2, None, -1.0, 0.0)
    finally:
        ctx.close()


def test_inout_batch_equals_single_runs(lbm_lib):
    """The boundary kernel walks every instance of a batch with its own constants: bitwise the single runs."""
    L = lbm_lib
    nx, ny = 48, 16
    yy, xx = np.mgrid[:ny, :nx] + 0.5
    phi1 = (0.5 + 0.5 * np.tanh((6.0 - np.hypot(xx - 16, yy - 8)) / 2.0)).astype(np.float32)
    phi0 = np.zeros((ny, nx), np.float32)
    prms = [L.lbm_default_params(rho=(1.0, r, 1.0), mu=(0.05, 0.05, 0.05), d0=0.5) for r in (1.0, 3.0)]
    u_in = np.stack([np.full(ny, 0.01), np.zeros(ny)]).astype(np.float32)

    def run(batch):
        ctx = L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=(False, False, False), batch=batch)
        try:
            ctx.set_solid(np.broadcast_to(phi0, (len(batch), ny, nx)).copy())
            ctx.set_phase(np.broadcast_to(phi1, (len(batch), ny, nx)).copy())
            ctx.set_inout(3, u_in, 0.0, 0.0)
            ctx.step(300)
            return ctx.get_fields()
        finally:
            ctx.close()
    both = run(prms)
    for b in range(2):
        one = run([prms[b]])
        for a, c in zip(both, one):
            np.testing.assert_array_equal(a[b], c[0])


def test_inout_d3q19_fp16_matches_float32(lbm_lib):
    """FP16 NS populations on a 3D lattice go through the same boundary arithmetic (scaled loads and stores)."""
    L = lbm_lib
    nx, ny, nz = 32, 10, 8
    prm = L.lbm_default_params(rho=(1.0, 1.0, 1.0), mu=(0.1, 0.1, 0.1), d0=1.0 / 3.0)
    zz, yy = np.mgrid[:nz, :ny] + 0.5
    prof = 0.03 * (1 - ((yy - ny / 2) / (ny / 2)) ** 2) * (1 - ((zz - nz / 2) / (nz / 2)) ** 2)
    u_in = np.stack([prof, 0 * prof, 0 * prof]).astype(np.float32)
    out = []
    for flags in (0, L.LBM_STORE_G_F16):
        ctx = L.Context(L.LBM_D3Q19, nx, ny, nz, periodic=(False, False, False), params=prm, flags=flags)
        try:
            ctx.set_solid(np.zeros((nz, ny, nx), np.float32))
            ctx.set_phase(np.ones((nz, ny, nx), np.float32))
            ctx.set_inout(3, u_in, 1.0, 0.0)
            ctx.step(400)
            out.append(ctx.get_fields()[1][0].copy())
        finally:
            ctx.close()
    assert rel_l2(out[1], out[0]) < 2e-3
