"""Named workloads of the benchmark and the tests (geometry recipe + parameters).

Each entry returns plain data: float32 solid / phase fields, periodicity and a
list of per-instance parameter dictionaries (keys of ``lbm_params``).  No
method arithmetic lives here.
"""
from __future__ import annotations

import numpy as np

from .geometry import cylinder_droplet, wall_droplet

# Disk + droplet on a 1024^2 periodic lattice, contact angle swept over five
# values, density and viscosity ratio 10 (fluid 1 heavier and more viscous;
# the solid takes fluid 1's density and viscosity), scale factor 1/2.
DISK_SWEEP_THETAS = (30.0, 60.0, 90.0, 120.0, 150.0)


def disk_sweep(n=1024, Rs=160.0, R0=120.0, W=4.0, thetas=DISK_SWEEP_THETAS):
    geo = cylinder_droplet(n=n, Rs=Rs, R0=R0, W=W)
    phi0 = np.broadcast_to(geo.phi0.astype(np.float32), (len(thetas),) + geo.phi0.shape).copy()
    phi1 = np.broadcast_to(geo.phi1.astype(np.float32), (len(thetas),) + geo.phi1.shape).copy()
    params = [dict(W=W, M_deg=0.1, theta_deg=t, kappa=R0 / Rs, sigma=0.01, rho=(10.0, 10.0, 1.0),
                   mu=(0.1, 0.1, 0.01), d0=0.5) for t in thetas]
    return dict(name=f"D2Q9 disk+droplet {n}x{n} x{len(thetas)} angles (Rs={Rs}, R0={R0}, rho/mu ratio 10)",
                lattice="D2Q9", nx=n, ny=n, nz=1, periodic=(True, True, False), phi0=phi0, phi1=phi1,
                params=params, geometry=geo)


def flat_wall(nx=128, ny=64, wall_rows=8, R=25.0, W=4.0, theta=60.0, d0=0.5):
    geo = wall_droplet(nx, ny, wall_rows, R, W)
    params = [dict(W=W, M_deg=0.1, theta_deg=theta, kappa=0.0, sigma=0.01, d0=d0)]
    return dict(name=f"D2Q9 flat wall {nx}x{ny}, R={R}, theta={theta}", lattice="D2Q9", nx=nx, ny=ny, nz=1,
                periodic=(True, False, False), phi0=geo.phi0.astype(np.float32)[None],
                phi1=geo.phi1.astype(np.float32)[None], params=params, geometry=geo)
