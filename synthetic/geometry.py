"""Seeded geometry generators for the ternary (two fluids + one solid) LB workloads.

Every array is float64, C order, indexed ``[y, x]`` in 2D and ``[z, y, x]`` in
3D (x fastest).  Node ``(x, y)`` sits at integer coordinates; a half-way
bounce-back wall lies half a spacing outside the first and last node.

Diffuse profiles follow the paper's initial conditions (Sec. 4.1-4.3, 4.6):
a phase indicator across an interface at signed distance ``d`` (positive
inside) of width ``W`` is ``1/2 + 1/2 tanh(2 d / W)``.  The solid indicator is
``phi0`` and the droplet / driving fluid is ``phi1 = (1 - phi0) * indicator``.

Nothing here is part of the method; it only produces inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "diffuse",
    "Geometry",
    "wall_droplet",
    "wall_cap",
    "cylinder_droplet",
    "free_drop",
    "flat_layer",
    "capillary_slug",
    "random_disks_droplet",
    "rsa_spheres",
    "porous_inlet_slab",
    "spheres_phi0",
    "sphere_box_droplet",
    "wall_drop_3d",
    "splitmix64",
    "splitmix64_block",
]


def diffuse(signed_distance, W):
    """``1/2 + 1/2 tanh(2 d / W)``: 1 well inside (d > 0), 0 well outside."""
    return 0.5 + 0.5 * np.tanh(2.0 * np.asarray(signed_distance, dtype=np.float64) / W)


@dataclasses.dataclass
class Geometry:
    """A lattice workload: fields plus the descriptors the diagnostics need."""

    phi0: np.ndarray
    phi1: np.ndarray
    periodic: tuple
    # probe line used for the droplet height: origin node coordinates and axis
    probe_origin: tuple = (0.0, 0.0)
    probe_axis: int = 1
    # wall level (flat wall, in node coordinates) or solid disk radius/centre
    wall_level: float | None = None
    disk_center: tuple | None = None
    disk_radius: float | None = None
    droplet_radius: float | None = None
    kappa: float = 0.0
    note: str = ""

    @property
    def shape(self):
        return self.phi0.shape


def _grid2(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def wall_droplet(nx=128, ny=64, wall_rows=8, R=25.0, W=4.0, xc=None):
    """Half-disk droplet resting on a flat solid wall (Sec. 4.2 set-up).

    The bottom ``wall_rows`` rows are solid: the wall surface lies at
    ``y_w = wall_rows - 1/2``.  The droplet of radius ``R`` is centred on the
    wall at ``(xc, y_w)``; x is periodic, y has no-flux walls.
    """
    x, y = _grid2(nx, ny)
    yw = wall_rows - 0.5
    xc = nx / 2.0 if xc is None else xc
    phi0 = diffuse(yw - y, W)
    r = np.hypot(x - xc, y - yw)
    phi1 = (1.0 - phi0) * diffuse(R - r, W)
    return Geometry(phi0, phi1, (True, False), probe_origin=(xc, 0.0), probe_axis=1,
                    wall_level=yw, droplet_radius=R, kappa=0.0,
                    note=f"flat wall, {nx}x{ny}, wall rows {wall_rows}, R={R}, W={W}")


def wall_cap(nx=64, ny=40, wall_rows=8, R0=15.0, theta_deg=60.0, W=4.0, xc=None):
    """Circular cap resting on a flat wall with apparent contact angle ``theta_deg``.

    The cap holds the area of a half-disk of radius ``R0`` (pi R0^2 / 2), so
    its circle radius is R = R0 sqrt((pi/2)/(t - sin t cos t)) and its centre
    sits R cos(t) below the wall surface (Sec. 4.2 geometry).  x periodic,
    y walls.
    """
    x, y = _grid2(nx, ny)
    yw = wall_rows - 0.5
    xc = nx / 2.0 if xc is None else xc
    t = math.radians(theta_deg)
    R = R0 * math.sqrt((math.pi / 2.0) / (t - math.sin(t) * math.cos(t)))
    yc = yw - R * math.cos(t)
    phi0 = diffuse(yw - y, W)
    phi1 = (1.0 - phi0) * diffuse(R - np.hypot(x - xc, y - yc), W)
    return Geometry(phi0, phi1, (True, False), probe_origin=(xc, 0.0), probe_axis=1,
                    wall_level=yw, droplet_radius=R0, kappa=0.0,
                    note=f"cap theta={theta_deg} on flat wall, {nx}x{ny}, R0={R0}, W={W}")


def cylinder_droplet(n=1024, Rs=160.0, R0=120.0, W=4.0, ny=None):
    """Droplet of radius ``R0`` centred on the top of a solid disk (Sec. 4.3 set-up).

    The disk of radius ``Rs`` is centred at ``(n/2, ny/2)``; all sides periodic.
    The dimensionless curvature is ``kappa = R0 / Rs`` as in Sec. 4.3.
    """
    nx = n
    ny = n if ny is None else ny
    x, y = _grid2(nx, ny)
    xc, yc = nx / 2.0, ny / 2.0
    phi0 = diffuse(Rs - np.hypot(x - xc, y - yc), W)
    phi1 = (1.0 - phi0) * diffuse(R0 - np.hypot(x - xc, y - (yc + Rs)), W)
    return Geometry(phi0, phi1, (True, True), probe_origin=(xc, yc), probe_axis=1,
                    disk_center=(xc, yc), disk_radius=Rs, droplet_radius=R0, kappa=R0 / Rs,
                    note=f"disk Rs={Rs}, droplet R0={R0}, {nx}x{ny}, W={W}")


def free_drop(nx=96, ny=96, R=24.0, W=4.0):
    """Circular drop of fluid 1 in fluid 2, no solid, all periodic (Laplace test)."""
    x, y = _grid2(nx, ny)
    phi0 = np.zeros((ny, nx))
    phi1 = diffuse(R - np.hypot(x - nx / 2.0, y - ny / 2.0), W)
    return Geometry(phi0, phi1, (True, True), probe_origin=(nx / 2.0, ny / 2.0), probe_axis=1,
                    droplet_radius=R, note=f"free drop R={R}, {nx}x{ny}, W={W}")


def flat_layer(nx=4, ny=128, W=4.0, y_lo=None, y_hi=None):
    """Slab of fluid 1 between two flat interfaces, no solid, all periodic."""
    x, y = _grid2(nx, ny)
    y_lo = ny / 4.0 if y_lo is None else y_lo
    y_hi = 3.0 * ny / 4.0 if y_hi is None else y_hi
    phi0 = np.zeros((ny, nx))
    # slab [y_lo, y_hi] as the intersection of two half-planes
    phi1 = diffuse(y - y_lo, W) * diffuse(y_hi - y, W)
    return Geometry(phi0, phi1, (True, True), probe_origin=(0.0, 0.0), probe_axis=1,
                    note=f"flat slab {nx}x{ny}, interfaces at {y_lo},{y_hi}, W={W}")


# --- seeded random geometry ---------------------------------------------------

def capillary_slug(nx=64, ny=40, wall_rows=6, W=4.0):
    """A slug of fluid 1 filling a channel between two flat solid walls, with flat menisci.

    The bottom and top ``wall_rows`` rows are solid; the wall surfaces lie at
    ``y = wall_rows - 1/2`` and ``y = ny - wall_rows - 1/2``, so the channel is
    ``ny - 2 wall_rows`` lattice units wide.  Fluid 1 fills ``nx/4 <= x <
    3 nx/4`` of the channel with two straight interfaces normal to the walls
    (a 90 deg start); x is periodic, y has no-flux walls.
    """
    x, y = _grid2(nx, ny)
    ylo, yhi = wall_rows - 0.5, ny - wall_rows - 0.5
    phi0 = diffuse(ylo - y, W) + diffuse(y - yhi, W)
    x0, x1 = nx / 4.0, 3.0 * nx / 4.0
    phi1 = (1.0 - phi0) * diffuse(np.minimum(x - x0, x1 - x), W)
    return Geometry(phi0, phi1, (True, False), probe_origin=(nx / 2.0, 0.0), probe_axis=1, wall_level=ylo,
                    note=f"capillary slug, {nx}x{ny}, walls {wall_rows} rows, channel {yhi - ylo:g}, W={W}")


def splitmix64(seed):
    """A tiny seeded uniform generator (SplitMix64), returned as a closure on [0, 1)."""
    state = [seed & 0xFFFFFFFFFFFFFFFF]

    def nxt():
        state[0] = (state[0] + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = state[0]
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        z ^= z >> 31
        return (z >> 11) / float(1 << 53)

    return nxt


def random_disks_droplet(n=256, seed=0, W=4.0, ny=None):
    """1-6 non-overlapping solid disks (radii 8-40) plus one droplet (radius 10-60).

    The droplet is placed on top of the largest disk; kappa = R0 / max(Rs)
    (minimum curvature of the solid is that of its largest disk).  All sides
    periodic.  Returns the geometry and the drawn contact angle in degrees
    (uniform in 30-150).
    """
    u = splitmix64(seed * 7919 + 17)
    nx = n
    ny = n if ny is None else ny
    ndisk = 1 + int(u() * 6)
    disks = []
    tries = 0
    while len(disks) < ndisk and tries < 10000:
        tries += 1
        r = 8.0 + 32.0 * u()
        r = min(r, 0.2 * min(nx, ny))
        cx, cy = nx * u(), ny * u()
        ok = True
        for (qx, qy, qr) in disks:
            dx = min(abs(cx - qx), nx - abs(cx - qx))
            dy = min(abs(cy - qy), ny - abs(cy - qy))
            if math.hypot(dx, dy) < r + qr + 2.0 * W:
                ok = False
                break
        if ok:
            disks.append((cx, cy, r))
    x, y = _grid2(nx, ny)
    phi0 = np.zeros((ny, nx))
    for (cx, cy, r) in disks:
        dx = np.abs(x - cx)
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - cy)
        dy = np.minimum(dy, ny - dy)
        phi0 = np.maximum(phi0, diffuse(r - np.hypot(dx, dy), W))
    big = max(disks, key=lambda d: d[2])
    R0 = 10.0 + 50.0 * u()
    R0 = min(R0, 0.2 * min(nx, ny))
    cx, cy = big[0], big[1] + big[2]
    dx = np.abs(x - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - cy)
    dy = np.minimum(dy, ny - dy)
    phi1 = (1.0 - phi0) * diffuse(R0 - np.hypot(dx, dy), W)
    theta = 30.0 + 120.0 * u()
    g = Geometry(phi0, phi1, (True, True), probe_origin=(big[0], big[1]), probe_axis=1,
                 disk_center=(big[0], big[1]), disk_radius=big[2], droplet_radius=R0,
                 kappa=R0 / big[2], note=f"{len(disks)} disks, seed {seed}")
    return g, theta


def splitmix64_block(seed, start, count):
    """Draws ``start + 1 .. start + count`` of ``splitmix64(seed)`` as one array.

    The k-th draw of the generator mixes the state ``seed + k * gamma`` (mod
    2^64), so a block of draws is a vectorised evaluation with the same values.
    """
    k = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) / float(1 << 53)


def rsa_spheres(n=256, seed=0, rmin=10.0, rmax=20.0, target_solid=0.4, max_fail=1_000_000):
    """Random sequential addition of non-overlapping spheres with periodic images.

    Radii uniform in ``[rmin, rmax]``; stops when the sharp solid fraction
    reaches ``target_solid`` or after ``max_fail`` consecutive rejections.
    Candidates are drawn in sequence (radius, then x, y, z centre) from
    ``splitmix64``; blocks of candidates are tested together, which gives the
    same accepted list as testing them one at a time.
    Returns the list ``[(cx, cy, cz, r), ...]``.
    """
    gen_seed = seed * 104729 + 3
    L = float(n)
    # cell lists: a candidate can only overlap spheres whose centre lies in its
    # own or one of the 26 neighbouring cells (cell side >= 2 rmax)
    nc = max(1, int(L // (2.0 * rmax)))
    use_cells = nc >= 3
    if not use_cells:
        nc = 1
    h = L / nc
    members = [[] for _ in range(nc ** 3)]
    spheres = []
    cen = np.empty((0, 3))
    rad = np.empty(0)

    def cell_of(p):
        q = np.minimum((p // h).astype(np.int64), nc - 1)
        return (q[..., 2] * nc + q[..., 1]) * nc + q[..., 0]

    def neighbour_table():
        if not use_cells:
            return np.arange(len(rad))[None, :]
        lists = []
        for cid in range(nc ** 3):
            ix, iy, iz = cid % nc, (cid // nc) % nc, cid // (nc * nc)
            idx = []
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        idx += members[(((iz + dz) % nc) * nc + (iy + dy) % nc) * nc + (ix + dx) % nc]
            lists.append(idx)
        width = max(1, max(len(x) for x in lists))
        tab = np.full((nc ** 3, width), -1, dtype=np.int64)
        for cid, idx in enumerate(lists):
            tab[cid, :len(idx)] = idx
        return tab

    def clear_of(c, r, tab):
        rows = tab[cell_of(c)] if use_cells else np.broadcast_to(tab, (len(r), tab.shape[1]))
        if rows.shape[1] == 0:
            return np.ones(len(r), dtype=bool)
        valid = rows >= 0
        safe = np.where(valid, rows, 0)
        d = np.abs(c[:, None, :] - cen[safe])
        d = np.minimum(d, L - d)
        d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        hit = (d2 < (r[:, None] + rad[safe]) ** 2) & valid
        return ~np.any(hit, axis=1)

    vol = 0.0
    fails = 0
    drawn = 0
    B = 8192
    tab = neighbour_table()
    while vol / L ** 3 < target_solid and fails < max_fail:
        u = splitmix64_block(gen_seed, drawn, 4 * B).reshape(B, 4)
        drawn += 4 * B
        r = rmin + (rmax - rmin) * u[:, 0]
        c = L * u[:, 1:]
        ok = clear_of(c, r, tab) if len(rad) else np.ones(B, dtype=bool)
        pos = 0
        while pos < B:
            nxt = np.flatnonzero(ok[pos:])
            if nxt.size == 0:
                if fails + (B - pos) >= max_fail:
                    return spheres
                fails += B - pos
                break
            j = pos + int(nxt[0])
            if fails + (j - pos) >= max_fail:
                return spheres
            fails = 0
            spheres.append((float(c[j, 0]), float(c[j, 1]), float(c[j, 2]), float(r[j])))
            cen = np.vstack([cen, c[j][None]])
            rad = np.append(rad, r[j])
            members[int(cell_of(c[j][None])[0]) if use_cells else 0].append(len(rad) - 1)
            tab = neighbour_table()
            vol += 4.0 / 3.0 * math.pi * r[j] ** 3
            if vol / L ** 3 >= target_solid:
                return spheres
            pos = j + 1
            if pos < B:
                # later candidates of the block against the new sphere only
                d = np.abs(c[pos:] - c[j])
                d = np.minimum(d, L - d)
                d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
                ok[pos:] &= ~(d2 < (r[pos:] + r[j]) ** 2)
    return spheres


def porous_inlet_slab(n=256, seed=0, W=4.0, slab=32.0, rmin=10.0, rmax=20.0, target_solid=0.4,
                      spheres=None):
    """3D porous workload: RSA spheres (tanh phi0) with fluid 1 filling the slab x < ``slab``.

    All sides periodic.  Returns the geometry; ``note`` records the achieved
    diffuse porosity ``1 - mean(phi0)``.
    """
    if spheres is None:
        spheres = rsa_spheres(n, seed, rmin, rmax, target_solid)
    phi0 = spheres_phi0((n, n, n), spheres, W)
    x = np.arange(n, dtype=np.float64)[None, None, :]
    phi1 = (1.0 - phi0) * diffuse(slab - x, W)
    phi1 = np.broadcast_to(phi1, phi0.shape).copy()
    poro = 1.0 - phi0.mean()
    return Geometry(phi0, phi1, (True, True, True), probe_origin=(0.0, 0.0, 0.0), probe_axis=0,
                    note=f"{len(spheres)} RSA spheres r in [{rmin},{rmax}], seed {seed}, porosity {poro:.4f}")


def spheres_phi0(shape, spheres, W=4.0):
    """Diffuse solid indicator of (possibly overlapping) spheres on a periodic box.

    ``shape`` is ``(nz, ny, nx)``; ``spheres`` lists ``(cx, cy, cz, r)``.  Each
    sphere is drawn with its periodic images and the union takes the maximum.
    """
    nz, ny, nx = shape
    phi0 = np.zeros(shape)
    for (cx, cy, cz, r) in spheres:
        lo = [int(math.floor(c - r - 2 * W)) for c in (cz, cy, cx)]
        hi = [int(math.ceil(c + r + 2 * W)) + 1 for c in (cz, cy, cx)]
        rng = []
        for lo_a, hi_a, n_a, c in zip(lo, hi, shape, (cz, cy, cx)):
            if hi_a - lo_a >= n_a:
                # nearest periodic image of every node along this axis
                idx = np.arange(n_a)
                d = idx - c
                d = d - n_a * np.round(d / n_a)
                rng.append((idx, d))
            else:
                k = np.arange(lo_a, hi_a)
                rng.append((k % n_a, k - c))
        (iz, dz), (iy, dy), (ix, dx) = rng
        d = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        blk = diffuse(r - d, W)
        sub = phi0[np.ix_(iz, iy, ix)]
        phi0[np.ix_(iz, iy, ix)] = np.maximum(sub, blk)
    return phi0


def sphere_box_droplet(nx, ny, nz, spheres, slab=None, drop=None, W=4.0, periodic=(True, True, True)):
    """Spheres in a box with fluid 1 either filling ``x < slab`` or as a drop.

    ``drop`` is ``(cx, cy, cz, R)``.  ``phi1 = (1 - phi0) * indicator``.
    """
    phi0 = spheres_phi0((nz, ny, nx), spheres, W)
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    if drop is not None:
        cx, cy, cz, R = drop
        ind = diffuse(R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2), W)
    else:
        ind = diffuse(slab - x, W)
    phi1 = (1.0 - phi0) * ind
    return Geometry(phi0, phi1, tuple(periodic), probe_origin=(0.0, 0.0, 0.0), probe_axis=0,
                    note=f"{len(spheres)} spheres")


def wall_drop_3d(nx, ny, nz, wall_layers, R, W=4.0, xc=None, yc=None):
    """Flat solid layer at the bottom (z) with a spherical drop resting on it.

    Periodic in x and y, half-way walls in z.  The drop centre sits on the
    solid surface ``z = wall_layers - 1/2``.
    """
    xc = (nx - 1) / 2.0 if xc is None else xc
    yc = (ny - 1) / 2.0 if yc is None else yc
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    zw = wall_layers - 0.5
    phi0 = diffuse(zw - z, W)
    ind = diffuse(R - np.sqrt((x - xc) ** 2 + (y - yc) ** 2 + (z - zw) ** 2), W)
    phi1 = (1.0 - phi0) * ind
    return Geometry(phi0, phi1, (True, True, False), probe_origin=(xc, yc, 0.0), probe_axis=2,
                    wall_level=zw, droplet_radius=R, note="drop on a flat wall (3D)")
