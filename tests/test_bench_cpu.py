"""Host-side logic of bench.py: the time-to-equilibrium criterion and the contact-angle readings (CPU)."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from synthetic import wall_cap, wall_droplet  # noqa: E402


def test_settle_against_a_reference():
    th = [80.0, 70.0, 64.0, 60.6, 60.3, 59.8, 60.1]
    assert bench._settle(th, 60.0, 100, 0.5) == 500          # from the fifth sample on, within 0.5 deg of 60
    assert bench._settle(th, 50.0, 100, 0.5) is None          # never there
    assert bench._settle([61.0, 60.9, 60.8], 60.0, 100, 0.5) is None


def test_settle_against_its_own_end_needs_a_run_of_samples():
    th = [80.0, 70.0, 64.0, 62.0]
    # the last sample always matches itself: one matching sample is no evidence of equilibrium
    assert bench._settle(th, th[-1], 100, 0.5, min_run=5) is None
    th = [80.0, 70.0, 60.4, 60.2, 60.1, 60.0, 60.0, 60.0]
    assert bench._settle(th, th[-1], 100, 0.5, min_run=5) == 300


@pytest.mark.parametrize("theta", [45.0, 90.0, 135.0])
def test_wall_angle_readings_of_a_drawn_cap(theta):
    # a circular cap drawn at theta on a flat diffuse wall: all three readings return theta
    geo = wall_cap(256, 128, 16, 40.0, theta, 4.0) if theta != 90.0 else wall_droplet(256, 128, 16, 40.0, 4.0)
    m = bench._wall_angles(geo.phi0, geo.phi1, 15.5)
    for key in ("height", "cap", "circle"):
        assert abs(m[key] - theta) < 0.3, (key, m)
    assert m["phi2_min"] >= -1e-12


def test_wall_angle_readings_see_a_wrong_angle():
    geo = wall_cap(256, 128, 16, 40.0, 70.0, 4.0)
    m = bench._wall_angles(geo.phi0, geo.phi1, 15.5)
    assert all(abs(m[k] - 60.0) > 5.0 for k in ("height", "cap", "circle"))
    assert math.isfinite(m["phi1_in_solid"])
