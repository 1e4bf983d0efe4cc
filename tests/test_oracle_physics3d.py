"""3D physics pins of the FP64 oracle (D3Q19 and D3Q15).

The viscosity relation of Sec. 3 fixes how a small shear wave decays: at
nu k^2 whatever its orientation.  A wave with u_x varying along y relaxes
through the off-diagonal second-order moment (rate s2b); a wave along the xy
face diagonal relaxes through the traceless diagonal moments (rate s2a).  Both
rates act on the lattice's second-order Hermite rows through the rate groups
of the 3D collision, so a wrong second-order row of the D3Q19 Gram-Schmidt
basis, a wrong group in K, or a wrong 3D viscosity constant decays the wave at
the wrong rate.
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
