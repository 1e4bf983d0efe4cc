"""The relaxed contact angle does not depend on where the drop starts (flat-wall configuration, GPU).

128 x 64, 8 solid rows, sigma 0.01, densities 1, viscosities 0.01, mobility
0.1, d0 = 1/2, contact angle 60 deg: caps of equal area drawn at 40 deg and
80 deg and the half-disk (90 deg) relax for 120000 steps in one batched
context.  An equilibrium of the method is reached from both sides: the three
angles end within 0.5 deg of each other, and the 40 deg start rises while the
others fall.  The common angle, 58-59 deg, is the method's at R0/D = 6.25
(the flat-wall study of the bench's wetting workload).
"""
import numpy as np
import pytest

from synthetic import wall_cap, wall_droplet

pytestmark = pytest.mark.gpu


def test_relaxed_angle_is_reached_from_both_sides(lbm_lib):
    L = lbm_lib
    geos = [wall_cap(128, 64, 8, 25.0, 40.0, 4.0), wall_cap(128, 64, 8, 25.0, 80.0, 4.0),
            wall_droplet(128, 64, 8, 25.0, 4.0)]
    prm = L.lbm_default_params(theta_deg=60.0, sigma=0.01, mu=(0.01, 0.01, 0.01), M_deg=0.1, d0=0.5)
    ctx = L.Context(L.LBM_D2Q9, 128, 64, 1, periodic=(True, False, False), batch=[prm] * 3)
    try:
        ctx.set_solid(np.stack([g.phi0.astype(np.float32) for g in geos]))
        ctx.set_phase(np.stack([g.phi1.astype(np.float32) for g in geos]))
        start = [ctx.contact_angle(i, 0, 64)[0] for i in range(3)]
        ctx.step(120000)
        end = [ctx.contact_angle(i, 0, 64)[0] for i in range(3)]
    finally:
        ctx.close()
    print("paths: start", start, "end", end)
    assert end[0] > start[0] + 5.0 and end[1] < start[1] - 5.0 and end[2] < start[2] - 5.0
    assert max(end) - min(end) < 0.5, end
    assert 55.0 < float(np.mean(end)) < 61.0, end
