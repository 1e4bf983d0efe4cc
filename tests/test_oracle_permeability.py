"""Pins of the relative-permeability diagnostic (Sec. 4.6, Eq. eq-Kp)."""
import numpy as np

from oracle import lbm, model
from oracle import observables as ob


def test_phase_flux_closed_form():
    r = np.random.default_rng(0)
    phi0 = np.where(r.uniform(size=(6, 9)) < 0.3, 1.0, 0.0)
    phi0[0, 0] = 0.5                                   # the pore space includes phi0 = 1/2
    phi1 = 0.25 * (1.0 - phi0)
    u = np.stack([np.full((6, 9), 0.02), np.full((6, 9), -0.01)])
    f = ob.phase_flux(phi0, phi1, u, axis=0)
    pore = phi0 <= 0.5
    n = int(pore.sum())
    assert f["n_pore"] == n
    assert np.isclose(f["q"], 0.02 * n)
    assert np.isclose(f["q1"], 0.02 * phi1[pore].sum())
    assert np.isclose(f["q2"], 0.02 * (1 - phi0 - phi1)[pore].sum())
    assert np.isclose(f["s1"] + f["s2"], 1.0)
    assert np.isclose(ob.phase_flux(phi0, phi1, u, axis=1)["q"], -0.01 * n)


def _channel(phi1, steps, nx=4, ny=24, mu=0.1, F=2e-6):
    prm = model.Params(rho=(1.0, 1.0, 1.0), mu=(mu, mu, mu), d0=0.5, body_force=(F, 0.0, 0.0), theta_deg=90.0)
    st = lbm.init_state("D2Q9", np.zeros((ny, nx)), phi1, prm, (True, False))
    lbm.step(st, model.constants(prm), nsteps=steps)
    return ob.phase_flux(st.phi0, st.macro["phi1"], st.macro["u"])


def test_stratified_channel_relative_permeabilities():
    """Layers of fluid 1 along both walls, fluid 2 in the core, equal densities and viscosities: the flow is the
    single-phase one, so K1 + K2 = 1, and K1 is the Poiseuille-weighted share of fluid 1."""
    nx, ny = 4, 24
    y = np.arange(ny) + 0.5
    d = np.minimum(y, ny - y)
    phi1 = (0.5 + 0.5 * np.tanh((6 - d) / 2.0))[:, None] * np.ones((1, nx))
    steps = 2000
    K1, K2 = ob.relative_permeability(_channel(phi1, steps), _channel(np.ones((ny, nx)), steps),
                                      _channel(np.zeros((ny, nx)), steps))
    assert abs(K1 + K2 - 1.0) < 1e-7
    ua = y * (ny - y)
    K1_exact = (phi1[:, 0] * ua).sum() / ua.sum()
    assert abs(K1 / K1_exact - 1.0) < 5e-3, (K1, K1_exact)
