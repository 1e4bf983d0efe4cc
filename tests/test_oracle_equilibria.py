"""Pins of the equilibria, sources and pressure formula through their moments (Sec. 3)."""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import lbm as olbm

LATS = [("D2Q9", 0.5), ("D2Q9", 1.0 / 3.0), ("D2Q9", 0.4), ("D3Q19", 1.0 / 3.0), ("D3Q19", 0.3),
        ("D3Q15", 1.0 / 3.0), ("D3Q15", 0.3)]


def _mom(lat, h):
    c = lat.c.astype(float)
    m0 = h.sum(0)
    m1 = np.stack([np.tensordot(c[:, a], h, 1) for a in range(lat.d)])
    m2 = np.stack([np.stack([np.tensordot(c[:, a] * c[:, b], h, 1) for b in range(lat.d)]) for a in range(lat.d)])
    return m0, m1, m2


def _rand(lat, rng, n=7):
    shp = (n,)
    u = 0.05 * rng.standard_normal((lat.d,) + shp)
    S = 0.01 * rng.standard_normal((lat.d,) + shp)
    return shp, u, S


@pytest.mark.parametrize("name,d0", LATS)
def test_ch_equilibrium_moments(name, d0):
    lat = L.make(name, d0)
    rng = np.random.default_rng(1)
    shp, u, _ = _rand(lat, rng)
    phi = rng.uniform(0, 1, shp)
    mub = 0.01 * rng.standard_normal(shp)
    eta = 7.0
    feq = olbm.f_equilibrium(lat, phi, mub, u, eta)
    m0, m1, m2 = _mom(lat, feq)
    assert np.allclose(m0, phi, atol=1e-14)
    assert np.allclose(m1, phi * u, atol=1e-14)
    for a in range(lat.d):
        for b in range(lat.d):
            assert np.allclose(m2[a, b], (d0 * eta * mub) if a == b else 0.0, atol=1e-14)


@pytest.mark.parametrize("name,d0", LATS)
def test_ns_equilibrium_moments(name, d0):
    lat = L.make(name, d0)
    rng = np.random.default_rng(2)
    shp, u, S = _rand(lat, rng)
    rho = rng.uniform(1, 10, shp)
    p = 1e-3 * rng.standard_normal(shp)
    rho_ref = 2.5
    geq = olbm.g_equilibrium(lat, p, rho, u, S, rho_ref)
    m0, m1, m2 = _mom(lat, geq)
    assert np.allclose(m0, rho_ref, atol=1e-13)
    assert np.allclose(m1, rho * u, atol=1e-14)
    for a in range(lat.d):
        for b in range(lat.d):
            expect = rho * u[a] * u[b] - 0.5 * (S[a] * u[b] + u[a] * S[b]) + (p if a == b else 0.0)
            assert np.allclose(m2[a, b], expect, atol=1e-14)


@pytest.mark.parametrize("name,d0", LATS)
def test_ns_forcing_moments(name, d0):
    lat = L.make(name, d0)
    rng = np.random.default_rng(5)
    shp, u, _ = _rand(lat, rng)
    gr = 0.1 * rng.standard_normal((lat.d,) + shp)
    Ft = 1e-3 * rng.standard_normal((lat.d,) + shp)
    M2F = [[1e-4 * rng.standard_normal(shp) for _ in range(lat.d)] for _ in range(lat.d)]
    for a in range(lat.d):
        for b in range(a):
            M2F[a][b] = M2F[b][a]
    Fi = olbm.ns_forcing(lat, u, gr, Ft, M2F)
    m0, m1, m2 = _mom(lat, Fi)
    udg = sum(u[a] * gr[a] for a in range(lat.d))
    assert np.allclose(m0, udg, atol=1e-15)
    assert np.allclose(m1, Ft, atol=1e-15)
    for a in range(lat.d):
        for b in range(lat.d):
            assert np.allclose(m2[a, b], M2F[a][b] + (d0 * udg if a == b else 0.0), atol=1e-15)


@pytest.mark.parametrize("name,d0", [x for x in LATS if x[0] == "D2Q9"])
def test_pressure_formula_recovers_equilibrium_pressure(name, d0):
    # with g = g^eq and no u.grad rho or time-derivative terms, the pressure formula returns p
    lat = L.make(name, d0)
    rng = np.random.default_rng(6)
    shp, u, S = _rand(lat, rng)
    rho = rng.uniform(1, 3, shp)
    p = 1e-3 * rng.standard_normal(shp)
    geq = olbm.g_equilibrium(lat, p, rho, u, S, 1.0)
    w0, cs2 = lat.w[0], d0
    q = sum((rho * u[a] - S[a]) * u[a] for a in range(lat.d))
    p_rec = cs2 / (1 - w0) * (geq[1:].sum(0) - w0 * q / (1 - cs2))
    assert np.allclose(p_rec, p, atol=1e-15)


@pytest.mark.parametrize("name,d0", LATS)
def test_ch_source_moments(name, d0):
    # R_i = w_i [c_i.d_t(phi u)/cs2 + corr c_i.eta grad mubar]: zero sum, first moment
    # d_t(phi u) + cs2 corr eta grad mubar, zero second moment
    lat = L.make(name, d0)
    rng = np.random.default_rng(7)
    shp = (5,)
    dt_phiu = 1e-3 * rng.standard_normal((lat.d,) + shp)
    gm = 1e-4 * rng.standard_normal((lat.d,) + shp)
    corr, eta = 0.7, 3.0
    R = np.stack([lat.w[i] * (sum(ci[a] * dt_phiu[a] for a in range(lat.d)) / d0
                              + corr * eta * sum(ci[a] * gm[a] for a in range(lat.d)))
                  for i, ci in enumerate(lat.c)])
    m0, m1, m2 = _mom(lat, R)
    assert np.allclose(m0, 0, atol=1e-16)
    assert np.allclose(m1, dt_phiu + d0 * corr * eta * gm, atol=1e-16)
    assert np.allclose(m2, 0, atol=1e-16)
