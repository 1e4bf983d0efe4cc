"""Pins of the diagnostics against the paper's table and closed-form limits (Sec. 4.2, 4.3)."""
import math
import os

import numpy as np
import pytest

from oracle import observables as ob
from synthetic import wall_cap

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table():
    rows = []
    for line in open(os.path.join(GOLD, "paper_table_heights.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_closed_form_reproduces_printed_row():
    tab = _table()
    for th, row_a, row_n, err in tab:
        h = ob.flat_height_ratio(math.radians(th))
        assert abs(h - row_n) < 5e-5, (th, h, row_n)       # the closed form is the row printed "Numerical"
        # the printed errors compare the other row with this one
        assert abs(100 * abs(row_a - row_n) / row_n - err) < 0.01 + 1e-9


def test_flat_height_ratio_limits():
    assert abs(ob.flat_height_ratio(math.pi / 2) - 1.0) < 1e-15   # half disk: H = R0
    # monotone in theta
    ts = np.linspace(0.1, 3.0, 50)
    hs = [ob.flat_height_ratio(t) for t in ts]
    assert np.all(np.diff(hs) > 0)


@pytest.mark.parametrize("theta", [45.0, 90.0, 135.0])
def test_flat_wall_angle_recovers_a_drawn_cap(theta):
    geo = wall_cap(256, 120, 8, 40.0, theta, 4.0)
    th, H, R0 = ob.flat_wall_angle(geo.phi0, geo.phi1, 128)
    assert abs(R0 - 40.0) < 0.3
    assert abs(th - theta) < 0.6, th


def test_disk_hmax_limits():
    Rs, S0 = 30.0, math.pi * 20.0 ** 2
    # non-wetting limit: the drop touches the disk at one point, H_max = Rs + 2 r with pi r^2 = S0
    r = math.sqrt(S0 / math.pi)
    assert abs(ob.disk_hmax(math.pi - 1e-6, Rs, S0) - (Rs + 2 * r)) < 1e-3
    # theta = 90 deg: the circles meet at right angles, k^2 = r^2 + Rs^2
    h90 = ob.disk_hmax(math.pi / 2, Rs, S0)
    lo, hi = 1e-6, 200.0
    for _ in range(200):   # independent solve of the right-angle lens
        mid = 0.5 * (lo + hi)
        k = math.hypot(mid, Rs)
        area = math.pi * mid ** 2 - mid ** 2 * math.atan2(Rs, mid) - Rs ** 2 * math.atan2(mid, Rs) + mid * Rs
        lo, hi = (mid, hi) if area < S0 else (lo, mid)
    assert abs(h90 - (lo + math.hypot(lo, Rs))) < 1e-6
    # monotone in the contact angle
    hs = [ob.disk_hmax(t, Rs, S0) for t in np.linspace(0.2, 3.0, 20)]
    assert np.all(np.diff(hs) > 0)


def test_laplace_dp_bulk_means():
    phi1 = np.zeros((10, 10))
    phi1[3:7, 3:7] = 1.0
    phi0 = np.zeros_like(phi1)
    p = np.where(phi1 > 0.5, 2.0, -1.0)
    assert ob.laplace_dp(phi0, phi1, p) == 3.0
