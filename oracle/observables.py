"""Diagnostics of the 2f1s runs (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Mass: sum of phi1 (and of the CH populations).
* Laplace pressure: mean p over nodes with phi1 >= 0.99 minus mean p over
  nodes with phi2 >= 0.99 (the bulk of each fluid).
* Droplet height on a probe column: position of the outermost phi1 = 1/2
  crossing, linearly interpolated between nodes (Sec. 4.2 measures the height
  of the equilibrium shape; Sec. 4.3 the maximum height).
* Flat wall (Sec. 4.2): H = R - R cos(theta), R = R0 sqrt((pi/2)/(theta -
  sin theta cos theta)), with R0 from the conserved area A = sum phi1 =
  pi R0^2 / 2.  The contact angle is the theta solving H/R0 = h(theta).
  The tests check h against the table "normalized droplet heights".
* Disk (Sec. 4.3): H_max = r + k_s with k_s^2 = r^2 + Rs^2 - 2 r Rs cos(theta)
  and the drop area outside the disk S_0.  The printed area equation lacks the
  square of the half-chord term under the last root; the standard two-circle
  lens area is used: pi r^2 - r^2 acos((k^2 + r^2 - Rs^2)/(2 k r))
  - Rs^2 acos((k^2 - r^2 + Rs^2)/(2 k Rs)) + k sqrt(Rs^2 - ((k^2 - r^2 + Rs^2)/(2k))^2).
* Relative permeability (Sec. 4.6, Eq. eq-Kp): K_p = integral over the pore
  space (phi0 <= 1/2) of u_{x,p} over the same integral of u'_{x,p} of a
  single-phase run.  Reading: u_{x,p} = phi_p u_x, the part of the x velocity
  carried by fluid p, and u'_{x,p} = u_x of the run with the pore space full
  of fluid p under the same driving.
"""
from __future__ import annotations

import math

import numpy as np


def mass(field):
    return float(np.sum(field, dtype=np.float64))


def laplace_dp(phi0, phi1, p, thresh=0.99):
    phi2 = 1.0 - phi0 - phi1
    inside = phi1 >= thresh
    outside = phi2 >= thresh
    if not inside.any() or not outside.any():
        return float("nan")
    return float(p[inside].mean() - p[outside].mean())


def column_crossing(values, level=0.5):
    """Outermost (largest index) position where a 1D profile falls through ``level``."""
    v = np.asarray(values, dtype=np.float64)
    for k in range(len(v) - 2, -1, -1):
        if v[k] >= level > v[k + 1]:
            return k + (v[k] - level) / (v[k] - v[k + 1])
    return float("nan")


def rising_crossing(values, level=0.5):
    """First position (from index 0 upward) where a profile falls through ``level``."""
    v = np.asarray(values, dtype=np.float64)
    for k in range(len(v) - 1):
        if v[k] >= level > v[k + 1]:
            return k + (v[k] - level) / (v[k] - v[k + 1])
    return float("nan")


def flat_height_ratio(theta):
    """h(theta) = H/R0 = (1 - cos theta) sqrt((pi/2) / (theta - sin theta cos theta))."""
    return (1.0 - math.cos(theta)) * math.sqrt((math.pi / 2.0) / (theta - math.sin(theta) * math.cos(theta)))


def _bisect(fn, lo, hi, target, it=200):
    flo = fn(lo) - target
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        fm = fn(mid) - target
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def flat_wall_angle(phi0, phi1, column):
    """Contact angle (degrees) of a 2D droplet on a flat bottom wall, measured on ``column``."""
    A = mass(phi1)
    R0 = math.sqrt(2.0 * A / math.pi)
    y_top = column_crossing(phi1[:, column])
    y_wall = rising_crossing(phi0[:, column])
    H = y_top - y_wall
    th = _bisect(flat_height_ratio, 1e-6, math.pi - 1e-6, H / R0)
    return math.degrees(th), H, R0


def lens_area_outside(r, Rs, k):
    """Area of a circle (radius r, centre at distance k from the disk centre) outside the disk Rs."""
    a = (k * k - r * r + Rs * Rs) / (2.0 * k)
    h2 = max(Rs * Rs - a * a, 0.0)
    c1 = np.clip((k * k + r * r - Rs * Rs) / (2.0 * k * r), -1.0, 1.0)
    c2 = np.clip((k * k - r * r + Rs * Rs) / (2.0 * k * Rs), -1.0, 1.0)
    return math.pi * r * r - r * r * math.acos(c1) - Rs * Rs * math.acos(c2) + k * math.sqrt(h2)


def disk_hmax(theta, Rs, S0):
    """H_max(theta) for a drop of outside area S0 on a disk of radius Rs (Sec. 4.3)."""
    def area(r):
        k = math.sqrt(r * r + Rs * Rs - 2.0 * r * Rs * math.cos(theta))
        return lens_area_outside(r, Rs, k)
    r = _bisect(area, 1e-6, 10.0 * (Rs + math.sqrt(S0)), S0)
    k = math.sqrt(r * r + Rs * Rs - 2.0 * r * Rs * math.cos(theta))
    return r + k


def disk_angle(phi0, phi1, center, Rs):
    """Contact angle (degrees) from the maximum height above the disk centre."""
    xc, yc = int(round(center[0])), center[1]
    y_top = column_crossing(phi1[:, xc])
    Hmax = y_top - yc
    S0 = mass(phi1)
    th = _bisect(lambda t: disk_hmax(t, Rs, S0), 1e-3, math.pi - 1e-3, Hmax)
    return math.degrees(th), Hmax, S0


def phase_flux(phi0, phi1, u, axis=0):
    """Pore-space sums (Eq. eq-Kp): q1 = sum phi1 u_a, q2 = sum phi2 u_a, q = sum u_a, saturations."""
    pore = phi0 <= 0.5
    phi2 = 1.0 - phi0 - phi1
    ua = u[axis]
    s1, s2 = float(phi1[pore].sum()), float(phi2[pore].sum())
    return dict(q1=float((phi1 * ua)[pore].sum()), q2=float((phi2 * ua)[pore].sum()), q=float(ua[pore].sum()),
                s1=s1 / (s1 + s2), s2=s2 / (s1 + s2), n_pore=int(pore.sum()))


def relative_permeability(two_phase, single_1, single_2):
    """(K_1, K_2) from phase_flux records of the two-phase run and of single-phase runs of each fluid."""
    return two_phase["q1"] / single_1["q"], two_phase["q2"] / single_2["q"]
