"""Pins of the spreading coefficients and the Lagrange multiplier (Sec. 2)."""
import math

import numpy as np
import pytest

from oracle import lbm as olbm
from oracle import model as M

THETAS = [15.0, 30.0, 45.0, 60.0, 75.0, 90.0, 105.0, 120.0, 135.0, 150.0, 165.0]


@pytest.mark.parametrize("theta_deg", THETAS)
@pytest.mark.parametrize("kappa", [0.0, 0.75, 2.0])
def test_k_closure_trigonometric_identity(theta_deg, kappa):
    # 1 - 2 sin^2 x = cos 2x: k = 9 cos(pi/2 cos t)/(1+kappa) below 90 deg, 9(2 - cos(.))/(1+kappa) above
    t = math.radians(theta_deg)
    k = M.k_closure(t, kappa)
    c = math.cos(math.pi / 2 * math.cos(t))
    expect = 9 / (1 + kappa) * (c if theta_deg < 90 else (2 - c if theta_deg > 90 else 1.0))
    assert abs(k - expect) < 1e-13


@pytest.mark.parametrize("theta_deg", THETAS)
def test_gamma_closed_forms_and_young(theta_deg):
    t = math.radians(theta_deg)
    sigma = 0.013
    k, (g0, g1, g2) = M.spreading(t, 0.4, sigma)
    # printed closed forms (Sec. 2.2)
    assert abs(g0 - (2 * k + math.cos(t) - 1) * sigma) < 1e-15
    assert abs(g1 - (1 - math.cos(t)) * sigma) < 1e-15
    assert abs(g2 - (1 + math.cos(t)) * sigma) < 1e-15
    # pairwise tensions back from the gammas: s_pq = (g_p + g_q)/2
    s01, s02, s12 = (g0 + g1) / 2, (g0 + g2) / 2, (g1 + g2) / 2
    assert abs(s12 - sigma) < 1e-15                    # gamma_1 + gamma_2 = 2 sigma
    assert abs(s01 - k * sigma) < 1e-15                # s01 = k s12
    assert abs((s02 - s01) / s12 - math.cos(t)) < 1e-12  # Young's law


def test_lagrange_multiplier_keeps_volume():
    # mubar_p = mu_p + L with L = -gT/3 sum_q mu_q / gamma_q makes sum_p mubar_p / gamma_p = 0,
    # which is what keeps phi0 + phi1 + phi2 = 1 under the three CH equations (Eq. sumCH)
    rng = np.random.default_rng(3)
    gam = np.array([0.21, 0.005, 0.015])
    gT = 3 / np.sum(1 / gam)
    for _ in range(20):
        mu = rng.standard_normal(3)
        L_ = -gT / 3 * np.sum(mu / gam)
        mubar = mu + L_
        assert abs(np.sum(mubar / gam)) < 1e-12
        # the second form of Eq. CHmodel
        for p in range(3):
            alt = gT / 3 * sum((mu[p] - mu[q]) / gam[q] for q in range(3) if q != p)
            assert abs(alt - mubar[p]) < 1e-12


def test_oracle_mubar_uses_the_lagrange_form():
    rng = np.random.default_rng(4)
    prm = M.Params(theta_deg=70.0)
    c = M.constants(prm)
    phi0 = rng.uniform(0, 0.3, (12, 10))
    phi1 = rng.uniform(0, 0.6, (12, 10))
    cp = olbm.chemical_potentials(phi0, phi1, (True, True), c, prm.W)
    mu = cp["mu"]
    L_ = -c.gammaT / 3 * sum(m / g for m, g in zip(mu, c.gamma))
    assert np.allclose(cp["mubar1"], mu[1] + L_, atol=1e-15)


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.5])
def test_ch_rate_relation(d0):
    prm = M.Params(d0=d0, M_deg=0.07, M_cst=0.01, eta_hat=0.2, theta_deg=50.0)
    c = M.constants(prm)
    s1 = c.s_ch["s1"]
    # (M_cst + M_deg)/gamma_1 = (1/s1 - 1/2) eta_1 cs2 (Sec. 3)
    assert abs((prm.M_cst + prm.M_deg) / c.gamma[1] - (1 / s1 - 0.5) * c.eta * d0) < 1e-14
