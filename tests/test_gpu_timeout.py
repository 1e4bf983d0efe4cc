"""Failure detection of the bounded device waits (lbm_set_wait_limit).

The pipelined 3D kernel waits on an mbarrier for the TMA tile load of each z
plane, with a poll limit.  A limit of 0 makes every such wait give up at
once: the kernel stops the step, drains the load still in flight, and raises
a flag that the next synchronising call reports as LBM_ETIMEOUT.  Nothing
faults or hangs; the context stays usable, and once the limit is restored and
the state set again it runs bitwise like a fresh context.
"""
import numpy as np
import pytest

from synthetic.geometry import wall_drop_3d

pytestmark = pytest.mark.gpu

NX, NY, NZ = 64, 32, 40   # nx % 4 == 0: the pipelined (TMA) kernel runs


def _ctx(L, geo, prm):
    ctx = L.Context(L.LBM_D3Q19, NX, NY, NZ, periodic=(True, True, False), params=prm)
    ctx.set_solid(geo.phi0.astype(np.float32))
    ctx.set_phase(geo.phi1.astype(np.float32))
    return ctx


def test_wait_limit_zero_reports_timeout_and_the_context_recovers(lbm_lib):
    L = lbm_lib
    geo = wall_drop_3d(NX, NY, NZ, 6, 10.0)
    prm = L.lbm_default_params(theta_deg=75.0, sigma=0.01, d0=1.0 / 3.0)
    ref = _ctx(L, geo, prm)
    try:
        ref.step(50)
        f_ref, g_ref = ref.get_populations()
    finally:
        ref.close()

    ctx = _ctx(L, geo, prm)
    try:
        ctx.set_wait_limit(0)
        ctx.step(3)
        with pytest.raises(L.LbmError) as err:
            ctx.sync()
        assert err.value.status == -5           # LBM_ETIMEOUT
        ctx.sync()                              # the flag was consumed; the context is not marked failed
        ctx.set_wait_limit(-1)                  # default limit
        ctx.set_phase(geo.phi1.astype(np.float32))
        ctx.step(50)
        f, g = ctx.get_populations()
    finally:
        ctx.close()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)
