"""Named workloads of the benchmark and the tests (geometry recipe + parameters).

Each entry returns plain data: float32 solid / phase fields, periodicity and a
list of per-instance parameter dictionaries (keys of ``lbm_params``).  No
method arithmetic lives here.
"""
from __future__ import annotations

import numpy as np

from .geometry import cylinder_droplet, porous_inlet_slab, random_disks_droplet, splitmix64, wall_droplet

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


def porous_slab(n=256, seed=0, W=4.0, slab=32.0, rmin=10.0, rmax=20.0, target_solid=0.4, body_force=1e-6):
    """3D porous run: RSA spheres (radii uniform in [rmin, rmax], sharp solid
    fraction ``target_solid``) on an n^3 periodic D3Q19 lattice, the
    non-wetting fluid 1 filling the inlet slab x < ``slab``, contact angle
    120 deg, body force along x, density and viscosity ratio 1, d0 = 1/3."""
    geo = porous_inlet_slab(n=n, seed=seed, W=W, slab=slab, rmin=rmin, rmax=rmax, target_solid=target_solid)
    params = [dict(W=W, M_deg=0.1, theta_deg=120.0, kappa=0.0, sigma=0.01, d0=1.0 / 3.0,
                   body_force=(body_force, 0.0, 0.0))]
    return dict(name=f"D3Q19 porous {n}^3 ({geo.note}), inlet slab x<{slab:g}, theta=120, body force "
                     f"{body_force:g} x, ratios 1, d0=1/3",
                lattice="D3Q19", nx=n, ny=n, nz=n, periodic=(True, True, True),
                phi0=geo.phi0.astype(np.float32)[None], phi1=geo.phi1.astype(np.float32)[None],
                params=params, geometry=geo)


BATCH_SIDES = (64, 128, 256, 512)


def batch_uneven(n_inst=64, seed=0, W=4.0):
    """Many independent D2Q9 geometries of uneven size: each instance is a
    square lattice with side drawn uniformly from 64 / 128 / 256 / 512, 1-6
    seeded random disks (radii 8-40), one droplet (radius 10-60) on the
    largest disk, contact angle uniform in 30-150 deg, kappa = R0 / max R_s;
    density / viscosity ratio 1, d0 = 1/2, all sides periodic."""
    u = splitmix64(seed * 31 + 5)
    inst = []
    for k in range(n_inst):
        side = BATCH_SIDES[min(int(u() * len(BATCH_SIDES)), len(BATCH_SIDES) - 1)]
        geo, theta = random_disks_droplet(n=side, seed=seed * 1000 + k, W=W)
        prm = dict(W=W, M_deg=0.1, theta_deg=theta, kappa=geo.kappa, sigma=0.01, d0=0.5)
        inst.append(dict(nx=side, ny=side, phi0=geo.phi0.astype(np.float32), phi1=geo.phi1.astype(np.float32),
                         params=prm, geometry=geo))
    nodes = sum(i["nx"] * i["ny"] for i in inst)
    return dict(name=f"D2Q9 batch of {n_inst} instances, sides in {BATCH_SIDES}, 1-6 disks, droplet, "
                     f"theta in 30-150 deg (seed {seed}), {nodes} nodes",
                lattice="D2Q9", instances=inst, nodes=nodes, periodic=(True, True))


def warmstart_set(seeds, n=256, W=4.0):
    """Samples of the learned warm start: the distribution of ``batch_uneven``
    (1-6 disks of radii 8-40, one droplet of radius 10-60 on the largest disk,
    theta uniform in 30-150 deg, d0 = 1/2, ratios 1) at one side n.  Each
    sample is rolled by whole nodes (an exact symmetry of the periodic
    lattice) so that the droplet's initial centre sits at (n/2, n/2) and its
    disk right below it, which keeps the droplet away from the image border
    that the network's zero padding sees.

    Returns phi0, phi1 (N, n, n) float32, theta_deg (N,), the rolled disk
    (N, 3: cx, cy, Rs) and the per-instance parameter dictionaries."""
    N = len(seeds)
    phi0 = np.empty((N, n, n), np.float32)
    phi1 = np.empty((N, n, n), np.float32)
    theta = np.empty(N)
    disk = np.empty((N, 3))
    params = []
    for i, s in enumerate(seeds):
        geo, th = random_disks_droplet(n=n, seed=int(s), W=W)
        cx, cy = geo.disk_center
        Rs = geo.disk_radius
        sx = int(round(n / 2 - cx))
        sy = int(round(n / 2 - (cy + Rs)))
        phi0[i] = np.roll(geo.phi0, (sy, sx), axis=(0, 1))
        phi1[i] = np.roll(geo.phi1, (sy, sx), axis=(0, 1))
        theta[i] = th
        disk[i] = ((cx + sx) % n, (cy + sy) % n, Rs)
        params.append(dict(W=W, M_deg=0.1, theta_deg=th, kappa=geo.kappa, sigma=0.01, d0=0.5))
    return dict(phi0=phi0, phi1=phi1, theta_deg=theta, disk=disk, params=params, n=n)
