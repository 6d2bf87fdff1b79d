"""Host measurements of the learned warm start (bulk densities, interface
width, contact angle by the spherical-cap formulas of Sec. V) against
synthetic circular caps of known angle, width and area: geometry fixes
the answer, no simulation involved."""
import math

import numpy as np
import pytest

from paper_1611_00907_gb300 import observables as obs
from paper_1611_00907_gb300 import warmstart as ws

CASE = dict(area=0.1, rho_l=2.0, rho_v=0.05)


def cap(theta, W, nx=512, ny=256):
    return ws.warm_field(CASE, dict(theta=theta, rho_l=2.0, rho_v=0.05,
                                    width=W), nx, ny)


@pytest.mark.parametrize("theta", [20, 45, 90, 120, 150])
@pytest.mark.parametrize("W", [2.0, 5.0])
def test_contact_angle_of_a_known_cap(theta, W):
    m = obs.measure(cap(theta, W))
    assert abs(m["theta"] - theta) < 0.1
    assert abs(m["rho_l"] - 2.0) < 4e-3
    assert abs(m["rho_v"] - 0.05) < 1e-6
    assert abs(m["width"] - W) < 0.2 * W


def test_nearly_non_wetting_cap():
    # the chord's linear extrapolation to the wall plane loses accuracy as
    # the base closes up
    assert abs(obs.contact_angle(cap(165, 2.0)) - 165) < 0.5


def test_lifted_drop_and_no_liquid():
    nx, ny = 256, 128
    yy, xx = np.mgrid[0:ny, 0:nx]
    d = 20.0 - np.hypot(xx - 128, yy - 60)           # disc clear of the wall
    rho = np.where(d > 0, 2.0, 0.05)
    assert obs.contact_angle(rho) == 180.0
    assert math.isnan(obs.contact_angle(np.full((ny, nx), 0.05)))


def test_warm_field_keeps_the_area():
    nx, ny = 384, 192
    for theta in (30, 90, 140):
        rho = cap(theta, 1.0, nx, ny)
        inside = (rho[1:-1] > 0.5 * (2.0 + 0.05)).sum()
        assert abs(inside / (CASE["area"] * nx * (ny - 2)) - 1) < 0.02


def test_drop_column_tracks_the_centre():
    rho = cap(60, 2.0)
    rho = np.roll(rho, 37, axis=1)
    assert abs(obs.drop_column(rho) - (256 + 37)) <= 1
