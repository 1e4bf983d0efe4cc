"""3D physics pins of the FP64 oracle (D3Q19 and D3Q15).

The viscosity relation of Sec. 3 fixes how a small shear wave decays: at
nu k^2 whatever its orientation.  A wave with u_x varying along y relaxes
through the off-diagonal second-order moment (rate s2b); a wave along the xy
face diagonal relaxes through the traceless diagonal moments (rate s2a).  Both
rates act on the lattice's second-order Hermite rows through the rate groups
of the 3D collision, so a wrong second-order row of the D3Q19 Gram-Schmidt
basis, a wrong group in K, or a wrong 3D viscosity constant decays the wave at
the wrong rate.  Also in 3D: sum phi1 conserved to round-off in a closed box
with a solid sphere and a drop, and the flat-interface tanh profile of width W.
"""
import math

import numpy as np
import pytest

from oracle import lbm, model
from synthetic.geometry import Geometry


def _shear_rate_3d(lattice, d0, diagonal, nu=0.02, n=48, t1=100, t2=400):
    """Measured decay rate of a small shear wave in a periodic box, and nu k^2."""
    shape = (1, n, n) if diagonal else (2, n, 2)       # (nz, ny, nx)
    z, y, x = np.meshgrid(*(np.arange(s, dtype=float) for s in shape), indexing="ij")
    k = 2 * math.pi / n
    prm = model.Params(d0=d0, mu=(nu, nu, nu))
    geo = Geometry(np.zeros(shape), np.zeros(shape), (True, True, True))
    st = lbm.init_state(lattice, geo.phi0, geo.phi1, prm, geo.periodic)
    U = 1e-4
    if diagonal:
        ux, uy = U * np.sin(k * (x + y)), -U * np.sin(k * (x + y))
        k2 = 2 * k * k
    else:
        ux, uy = U * np.sin(k * y), 0 * y
        k2 = k * k
    uz = 0 * y
    # first-order velocity perturbation of the NS populations: g_i += w_i c_i . (rho u) / cs2
    for i, ci in enumerate(st.lat.c):
        st.g[i] += st.lat.w[i] * (ci[0] * ux + ci[1] * uy + ci[2] * uz) / st.lat.cs2
    st.hist_u = np.stack([ux, uy, uz])
    amps = []
    for t in (t1, t2 - t1):
        lbm.step(st, nsteps=t)
        u = st.macro["u"]
        amps.append(np.sum(u[0] * ux) / np.sum(ux * ux))
        # the wave stays a pure shear: no velocity along z appears
        assert np.abs(u[2]).max() < 1e-12
    return -math.log(amps[1] / amps[0]) / (t2 - t1), nu * k2


@pytest.mark.parametrize("lattice,d0", [("D3Q19", 1.0 / 3.0), ("D3Q19", 0.4), ("D3Q15", 1.0 / 3.0)])
@pytest.mark.parametrize("diagonal", [False, True])
def test_viscosity_relation_shear_wave_3d(lattice, d0, diagonal):
    rate, expect = _shear_rate_3d(lattice, d0, diagonal)
    assert abs(rate / expect - 1.0) < 1e-2, (rate, expect)


def test_shear_wave_3d_sees_a_wrong_viscosity():
    # the pin has teeth: the same wave measured against a viscosity 5 % off fails the 1 % bar
    rate, expect = _shear_rate_3d("D3Q19", 1.0 / 3.0, True)
    assert abs(rate / (1.05 * expect) - 1.0) > 2e-2


@pytest.mark.parametrize("lattice,eta_hat", [("D3Q19", 0.1), ("D3Q15", 0.05)])
def test_mass_conservation_closed_box_3d(lattice, eta_hat):
    # walls on every axis, a solid sphere and a drop touching it: sum phi1 is conserved to round-off (Sec. 3:
    # zeroth moments of f^eq and R; streaming and half-way bounce-back move populations without loss)
    from synthetic.geometry import sphere_box_droplet
    geo = sphere_box_droplet(15, 13, 11, [(7.0, 6.0, 3.0, 3.0)], drop=(7.0, 6.0, 7.0, 3.5),
                             periodic=(False, False, False))
    prm = model.Params(theta_deg=70.0, sigma=0.01, d0=1.0 / 3.0, eta_hat=eta_hat, rho=(2.0, 2.0, 1.0),
                       mu=(0.05, 0.05, 0.02))
    st = lbm.init_state(lattice, geo.phi0, geo.phi1, prm, (False, False, False))
    m0 = st.f.sum()
    lbm.step(st, nsteps=200)
    assert abs(st.f.sum() - m0) / m0 < 1e-12
    assert abs(st.macro["phi1"].sum() - m0) / m0 < 1e-12


@pytest.mark.parametrize("lattice,eta_hat", [("D3Q19", 0.1), ("D3Q15", 0.05)])
def test_flat_interface_tanh_profile_3d(lattice, eta_hat):
    # a slab of fluid 1 along z relaxes to the profile 1/2 + 1/2 tanh(2z/W) of the free energy of Sec. 2.1
    nz, W = 64, 4.0
    z = np.arange(nz, dtype=float)
    phi1 = (0.5 + 0.5 * np.tanh(2 * (z - 16) / W)) * (0.5 + 0.5 * np.tanh(2 * (48 - z) / W))
    geo = Geometry(np.zeros((nz, 1, 1)), phi1[:, None, None], (True, True, True))
    prm = model.Params(W=W, sigma=0.01, mu=(0.1, 0.1, 0.1), d0=1.0 / 3.0, eta_hat=eta_hat)
    st = lbm.init_state(lattice, geo.phi0, geo.phi1, prm, geo.periodic)
    lbm.step(st, nsteps=600)
    prof = 0.5 + 0.5 * np.tanh(2 * (z - 16) / W)
    lower = slice(4, 32)
    got = st.macro["phi1"][lower, 0, 0]
    assert np.abs(got - prof[lower]).max() < 1e-2
    wrong = 0.5 + 0.5 * np.tanh(2 * (z - 16) / (1.3 * W))
    assert np.abs(got - wrong[lower]).max() > 3e-2
