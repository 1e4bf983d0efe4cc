"""Helpers that run the CUDA library and the FP64 oracle on the same float32 inputs."""
from __future__ import annotations

import numpy as np

from oracle import lbm as olbm
from oracle import model as omodel


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def as_inputs(geo):
    """float32 fields as the GPU receives them; the oracle gets the same values in float64."""
    return geo.phi0.astype(np.float32), geo.phi1.astype(np.float32)


def oracle_run(lattice, phi0, phi1, prm: dict, periodic, steps):
    st = olbm.init_state(lattice, phi0.astype(np.float64), phi1.astype(np.float64), omodel.Params(**prm),
                         tuple(periodic))
    olbm.step(st, nsteps=steps)
    return st


def gpu_run(L, lattice, phi0, phi1, prm: dict, periodic, steps, strip=None):
    shape = phi0.shape
    if lattice == "D2Q9":
        ny, nx = shape
        nz = 1
        lat = L.LBM_D2Q9
        per = (periodic[0], periodic[1], False)
    else:
        nz, ny, nx = shape
        lat = L.LBM_D3Q19
        per = tuple(periodic)
    ctx = L.Context(lat, nx, ny, nz, periodic=per, params=L.lbm_default_params(**prm))
    if strip is not None:
        ctx.set_launch(strip)
    ctx.set_solid(phi0)
    ctx.set_phase(phi1)
    ctx.step(steps)
    return ctx
