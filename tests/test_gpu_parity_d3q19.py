"""D3Q19: CUDA library versus the FP64 oracle on the same float32 inputs.

Same bars as the D2Q9 parity tests: relative L2 <= 1e-5 on phi1 and u (u
normalised by the largest velocity norm of the oracle run), 1e-4 on the
populations and the pressure.

Cases cover what the 3D kernels add over D2Q9: the moment pass (vectorised
and scalar paths, chosen by nodes mod 4), the z sweep with its rings and
strip seams, column tiles with ragged right and top edges, bounce-back on
each axis including edges and corners of a closed box, the general CH
collision (free rates != 1) and the closed-form third-order group.
"""
import numpy as np
import pytest

from _parity import as_inputs, gpu_run, oracle_run, rel_l2
from _parity import compare_run
from oracle import lbm as olbm
from oracle import model as omodel
from synthetic import sphere_box_droplet, wall_drop_3d

pytestmark = pytest.mark.gpu

# porous configuration parameters (contact angle 120, ratios 1, d0 = 1/3) with
# a body force raised to 1e-5 so that the short run carries a visible flow
POROUS_PRM = dict(theta_deg=120.0, sigma=0.01, d0=1.0 / 3.0, body_force=(1e-5, 0.0, 0.0))


def porous_box():
    # 36 x 20 x 18: two column tiles in x (32 + 4), three in y (8 + 8 + 4)
    return sphere_box_droplet(36, 20, 18, [(20.0, 6.0, 5.0, 4.5), (28.0, 15.0, 12.0, 5.0), (8.0, 14.0, 13.0, 3.5)],
                              slab=12.0)


def closed_box():
    # 21 x 13 x 9 = 2457 nodes (odd: scalar moment pass), walls on every axis
    return sphere_box_droplet(21, 13, 9, [(10.0, 6.0, 4.0, 3.0)], drop=(5.0, 6.0, 4.0, 3.5),
                              periodic=(False, False, False))


def test_porous_periodic_1000_steps(lbm_lib):
    compare_run(lbm_lib, "D3Q19", porous_box(), POROUS_PRM, (True, True, True), 1000)


def test_porous_periodic_short_strips(lbm_lib):
    # strips of 5 planes: four strips, the last one ragged (3 planes)
    compare_run(lbm_lib, "D3Q19", porous_box(), POROUS_PRM, (True, True, True), 200, strip=5)


def test_wall_drop_density_ratio_10(lbm_lib):
    geo = wall_drop_3d(28, 26, 20, 4, 7.0)
    prm = dict(theta_deg=60.0, sigma=0.01, d0=0.25, rho=(10.0, 10.0, 1.0), mu=(0.1, 0.1, 0.01))
    compare_run(lbm_lib, "D3Q19", geo, prm, (True, True, False), 500)


def test_closed_box_general_ch_rates(lbm_lib):
    prm = dict(theta_deg=45.0, sigma=0.01, d0=0.3, rho=(1.0, 2.0, 1.0), mu=(0.05, 0.05, 0.02), s_free_ch=0.8,
               s_free_ns=1.2)
    compare_run(lbm_lib, "D3Q19", closed_box(), prm, (False, False, False), 1000, strip=4)


def test_strip_choice_is_bitwise_neutral(lbm_lib):
    phi0, phi1 = as_inputs(porous_box())
    out = []
    for strip in (None, 7, 1):
        ctx = gpu_run(lbm_lib, "D3Q19", phi0, phi1, POROUS_PRM, (True, True, True), 40, strip)
        try:
            out.append(ctx.get_populations() + ctx.get_fields())
        finally:
            ctx.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def test_zero_steps_is_initial_state(lbm_lib):
    geo = porous_box()
    phi0, phi1 = as_inputs(geo)
    ctx = gpu_run(lbm_lib, "D3Q19", phi0, phi1, POROUS_PRM, (True, True, True), 0)
    try:
        g_f, g_g = ctx.get_populations()
        g_phi1, g_u, _ = ctx.get_fields()
    finally:
        ctx.close()
    st = olbm.init_state("D3Q19", phi0.astype(np.float64), phi1.astype(np.float64), omodel.Params(**POROUS_PRM),
                         (True, True, True))
    assert rel_l2(g_f[0], st.f.reshape(19, -1)) < 1e-6
    assert np.all(g_g == 0.0)
    assert np.array_equal(g_phi1[0], phi1.ravel()) and np.all(g_u == 0.0)


def test_batch_instances_are_independent(lbm_lib):
    L = lbm_lib
    phi0, phi1 = as_inputs(porous_box())
    prms = [dict(POROUS_PRM, theta_deg=t) for t in (60.0, 120.0)]
    nz, ny, nx = phi0.shape
    ctx = L.Context(L.LBM_D3Q19, nx, ny, nz, periodic=(True, True, True),
                    batch=[L.lbm_default_params(**p) for p in prms])
    try:
        ctx.set_solid(np.stack([phi0] * 2))
        ctx.set_phase(np.stack([phi1] * 2))
        ctx.step(100)
        b_phi1, b_u, _ = ctx.get_fields()
    finally:
        ctx.close()
    for i, prm in enumerate(prms):
        single = gpu_run(L, "D3Q19", phi0, phi1, prm, (True, True, True), 100)
        try:
            s_phi1, s_u, _ = single.get_fields()
        finally:
            single.close()
        assert np.array_equal(b_phi1[i], s_phi1[0]) and np.array_equal(b_u[i], s_u[0])
    st = oracle_run("D3Q19", phi0, phi1, prms[0], (True, True, True), 100)
    assert rel_l2(b_phi1[0], st.macro["phi1"]) < 1e-5


def test_pipelined_and_generic_kernels_agree_bitwise(lbm_lib):
    # depth 1 selects the generic fused kernel, depth 2 the pipelined (TMA) one
    phi0, phi1 = as_inputs(porous_box())
    L = lbm_lib
    nz, ny, nx = phi0.shape
    out = []
    for depth in (1, 2):
        ctx = L.Context(L.LBM_D3Q19, nx, ny, nz, periodic=(True, True, True),
                        params=L.lbm_default_params(**POROUS_PRM))
        try:
            ctx.set_launch(6, depth)
            ctx.set_solid(phi0)
            ctx.set_phase(phi1)
            ctx.step(60)
            out.append(ctx.get_populations() + ctx.get_fields())
        finally:
            ctx.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_pipelined_kernel_walls_and_ragged_tiles(lbm_lib):
    # nx % 4 == 0 with mirror ghosts on x and y: the reversed 4-byte halo chunks
    geo = sphere_box_droplet(40, 13, 11, [(20.0, 6.0, 5.0, 3.0)], drop=(8.0, 6.0, 5.0, 3.5),
                             periodic=(False, False, True))
    prm = dict(theta_deg=70.0, sigma=0.01, d0=0.3, rho=(1.0, 2.0, 1.0), mu=(0.05, 0.05, 0.02))
    compare_run(lbm_lib, "D3Q19", geo, prm, (False, False, True), 400, strip=4)
