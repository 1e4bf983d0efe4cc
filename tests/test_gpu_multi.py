"""Instances of different sizes in one persistent launch (lbm_create_multi).

Every instance must come out bitwise equal to the same instance run alone in
a single-instance context (same kernel body, same arithmetic), before and
after the autotuner (which saves and restores the state), and one instance
is checked against the oracle directly.
"""
import numpy as np
import pytest

from _parity import rel_l2
from oracle import lbm as olbm
from oracle import model as omodel
from synthetic import random_disks_droplet

pytestmark = pytest.mark.gpu

# sizes: ragged column tiles (200, 72), several strips, a 1-tile instance, non-square lattices
SIZES = [(64, 64), (200, 96), (128, 128), (72, 40), (256, 160), (48, 112)]


def _instances():
    out = []
    for k, (nx, ny) in enumerate(SIZES):
        geo, theta = random_disks_droplet(n=nx, seed=100 + k, W=4.0, ny=ny)
        prm = dict(theta_deg=theta, kappa=geo.kappa, sigma=0.01, d0=0.5, rho=(2.0, 2.0, 1.0), mu=(0.05, 0.05, 0.02))
        out.append((geo.phi0.astype(np.float32), geo.phi1.astype(np.float32), prm))
    return out


def _single(L, phi0, phi1, prm, steps):
    ny, nx = phi0.shape
    ctx = L.Context(L.LBM_D2Q9, nx, ny, 1, periodic=(True, True, False), params=L.lbm_default_params(**prm))
    try:
        ctx.set_solid(phi0)
        ctx.set_phase(phi1)
        ctx.step(steps)
        return ctx.get_fields(), ctx.get_populations(), ctx.observables(0)
    finally:
        ctx.close()


def test_multi_size_batch_equals_single_runs(lbm_lib):
    L = lbm_lib
    inst = _instances()
    m = L.MultiContext(SIZES, batch=[L.lbm_default_params(**p) for _, _, p in inst])
    try:
        m.set_solid([a for a, _, _ in inst])
        m.set_phase([b for _, b, _ in inst])
        m.step(150)
        img = m.get_state()
        strips = m.tune(5)
        assert m.get_state() == img            # the tuner restores the state bitwise
        candidates = (4, 8, 12, 16, 18, 20, 24, 32, 48, 64)   # the autotuner's strips (include/lbm.h)
        assert len(strips) == len(SIZES)
        assert all(s in candidates or s == ny for s, (_, ny) in zip(strips, SIZES))
        m.step(150)
        fields = m.get_fields()
        pops = m.get_populations()
        obs = [m.observables(k) for k in range(len(SIZES))]
    finally:
        m.close()
    for k, (phi0, phi1, prm) in enumerate(inst):
        (s_phi1, s_u, s_p), (s_f, s_g), s_obs = _single(L, phi0, phi1, prm, 300)
        nx, ny = SIZES[k]
        assert np.array_equal(fields[k][0].ravel(), s_phi1[0]), k
        assert np.array_equal(fields[k][1].reshape(2, -1), s_u[0]), k
        assert np.array_equal(fields[k][2].ravel(), s_p[0]), k
        assert np.array_equal(pops[k][0].reshape(9, -1), s_f[0]), k
        assert np.array_equal(pops[k][1].reshape(9, -1), s_g[0]), k
        for key in ("mass1", "umax", "dp", "n_in", "n_out"):
            a, b = obs[k][key], s_obs[key]
            assert a == b or (np.isnan(a) and np.isnan(b)), (k, key, a, b)


def test_multi_size_instance_against_oracle(lbm_lib):
    L = lbm_lib
    inst = _instances()[:4]
    sizes = SIZES[:4]
    m = L.MultiContext(sizes, batch=[L.lbm_default_params(**p) for _, _, p in inst])
    try:
        m.set_solid([a for a, _, _ in inst])
        m.set_phase([b for _, b, _ in inst])
        m.step(200)
        phi1, u, _ = m.get_fields()[3]
    finally:
        m.close()
    phi0, phi1_in, prm = inst[3]
    st = olbm.init_state("D2Q9", phi0.astype(np.float64), phi1_in.astype(np.float64), omodel.Params(**prm),
                         (True, True))
    olbm.step(st, nsteps=200)
    e_phi1, e_u = rel_l2(phi1, st.macro["phi1"]), rel_l2(u, st.macro["u"])
    print("parity multi", e_phi1, e_u)
    assert e_phi1 <= 1e-5 and e_u <= 1e-5, (e_phi1, e_u)


def test_multi_size_checkpoint_restores_bitwise(lbm_lib):
    L = lbm_lib
    inst = _instances()
    params = [L.lbm_default_params(**p) for _, _, p in inst]
    a = L.MultiContext(SIZES, batch=params)
    b = L.MultiContext(SIZES, batch=params)
    try:
        for ctx in (a, b):
            ctx.set_solid([x for x, _, _ in inst])
        a.set_phase([y for _, y, _ in inst])
        a.step(100)
        b.set_state(a.get_state())
        a.step(64)
        b.step(64)
        for (pa, ua, qa), (pb, ub, qb) in zip(a.get_fields(), b.get_fields()):
            assert np.array_equal(pa, pb) and np.array_equal(ua, ub) and np.array_equal(qa, qb)
    finally:
        a.close()
        b.close()
