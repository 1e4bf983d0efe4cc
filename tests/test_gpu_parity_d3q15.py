"""D3Q15 (the paper's 3D lattice, Appendix A weights and matrices): CUDA
library versus the FP64 oracle on the same float32 inputs.

Same bars as D3Q19: relative L2 <= 1e-5 on phi1 and on the final velocity
field, 1e-4 on populations and pressure, with one exception: the driven porous
box, whose velocity is held to 1.5e-5.  There the float32 velocity floor is
reached: u comes from the first moment of NS populations whose pressure part
w_i p / cs2 is about ten times the momentum part, so storing them in float32
costs about eps p / (rho u) ~ 6e-7 of u per step (measured 5.9e-7 after one
step, 6.8e-6 after 100, 1.04e-5 after 1000; the D3Q19 box, same geometry,
lands at 8.2e-6).  The CH parameter is
eta_hat = 0.05 where d0 = 1/3: with the default 0.1 the D3Q15 CH populations
blow up on the porous box within 60 steps in the oracle itself (the explicit
fourth-order term of the CH equilibrium), while 0.05 runs stably.
"""
import numpy as np
import pytest

from _parity import as_inputs, compare_run
from synthetic import sphere_box_droplet, wall_drop_3d

pytestmark = pytest.mark.gpu

POROUS_PRM = dict(theta_deg=120.0, sigma=0.01, d0=1.0 / 3.0, eta_hat=0.05, body_force=(1e-5, 0.0, 0.0))


def porous_box():
    return sphere_box_droplet(36, 20, 18, [(20.0, 6.0, 5.0, 4.5), (28.0, 15.0, 12.0, 5.0), (8.0, 14.0, 13.0, 3.5)],
                              slab=12.0)


def test_d3q15_porous_periodic_1000_steps(lbm_lib):
    compare_run(lbm_lib, "D3Q15", porous_box(), POROUS_PRM, (True, True, True), 1000, tol_u=1.5e-5)


def test_d3q15_wall_drop_density_ratio_10(lbm_lib):
    geo = wall_drop_3d(28, 26, 20, 4, 7.0)
    prm = dict(theta_deg=60.0, sigma=0.01, d0=0.25, rho=(10.0, 10.0, 1.0), mu=(0.1, 0.1, 0.01))
    compare_run(lbm_lib, "D3Q15", geo, prm, (True, True, False), 500, strip=6)


def test_d3q15_closed_box_general_rates(lbm_lib):
    # 21 x 13 x 9: odd node count (scalar moment pass) and nx % 4 != 0 (generic kernel)
    geo = sphere_box_droplet(21, 13, 9, [(10.0, 6.0, 4.0, 3.0)], drop=(5.0, 6.0, 4.0, 3.5),
                             periodic=(False, False, False))
    prm = dict(theta_deg=45.0, sigma=0.01, d0=0.3, eta_hat=0.05, rho=(1.0, 2.0, 1.0), mu=(0.05, 0.05, 0.02),
               s_free_ch=0.8, s_free_ns=1.2)
    compare_run(lbm_lib, "D3Q15", geo, prm, (False, False, False), 500, strip=4)


def test_d3q15_pipelined_and_generic_kernels_agree_bitwise(lbm_lib):
    L = lbm_lib
    phi0, phi1 = as_inputs(porous_box())
    nz, ny, nx = phi0.shape
    out = []
    for depth in (1, 2):
        ctx = L.Context(L.LBM_D3Q15, nx, ny, nz, periodic=(True, True, True),
                        params=L.lbm_default_params(**POROUS_PRM))
        try:
            ctx.set_launch(5, depth)
            ctx.set_solid(phi0)
            ctx.set_phase(phi1)
            ctx.step(60)
            out.append(ctx.get_populations() + ctx.get_fields())
        finally:
            ctx.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
