"""Host measurements of the learned warm start (bulk densities, interface
width, contact angle by the spherical-cap formulas of Sec. V) against
synthetic circular caps of known angle, width and area: geometry fixes
the answer, no simulation involved."""
import math

import numpy as np
import pytest

from paper_1611_00907_gb300 import inputs
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


def test_equimolar_radius_and_jump_of_a_disc():
    n = 256
    yy, xx = np.mgrid[0:n, 0:n]
    for R in (20.0, 45.0):
        d = R - np.hypot(xx - n / 2 + 0.5, yy - n / 2 + 0.5)
        rho = inputs.tanh_profile(d, 0.3, 0.02, 4.0)
        rin, rout = obs.periodic_drop_bulk(rho)
        # the centre of a disc of radius >= 20 is bulk to tanh(10) = 1 - 4e-9
        assert abs(rin - 0.3) < 1e-8 and abs(rout - 0.02) < 1e-9
        # a symmetric tanh profile puts the excess mass's edge at d = 0 up
        # to a curvature correction of order W^2 / R
        assert abs(obs.equimolar_radius(rho, rin, rout) - R) < 3.0 / R
        dp, r = obs.laplace_jump(rho, lambda v: 2.0 * v)
        assert abs(dp - 2.0 * (rin - rout)) < 1e-12 and abs(r - R) < 3.0 / R


def test_line_fit_recovers_a_line():
    x = np.linspace(0.01, 0.1, 8)
    s, c, r2 = obs.line_fit(x, 3.0 * x - 0.5)
    assert abs(s - 3.0) < 1e-12 and abs(c + 0.5) < 1e-12 and r2 == pytest.approx(1.0)


def test_slab_bulk_reads_the_plateaus():
    rho = inputs.slab(16, 256, 0.3, 0.02, 4.0)
    l, v = obs.slab_bulk(rho)
    assert abs(l - 0.3) < 1e-9 and abs(v - 0.02) < 1e-9


def test_film_over_the_wall_is_complete_wetting():
    nx, ny = 128, 64
    yy = np.mgrid[0:ny, 0:nx][0]
    rho = np.where(yy < 10, 2.0, 0.05)
    assert obs.contact_angle(rho) == 0.0


def test_centre_density_follows_a_drifted_drop():
    n = 128
    yy, xx = np.mgrid[0:n, 0:n]
    # a drop whose centre sits across the periodic corner
    d = 20.0 - np.hypot((xx + 10) % n - 10.3, (yy + 10) % n - 7.6)
    rho = inputs.tanh_profile(d, 0.3, 0.02, 4.0)
    rin, rout = obs.periodic_drop_bulk(rho)
    assert abs(rin - 0.3) < 1e-8 and abs(rout - 0.02) < 1e-9


@pytest.mark.parametrize("Tr", [0.7, 0.85, 0.9])
def test_surface_tension_from_the_bulk_pressure_matches_the_oracle(Tr):
    """The product's sigma (bulk pressure only, through the library's EOS)
    against the oracle's (the printed psi, Eq. 1)."""
    from oracle import thermo
    from paper_1611_00907_gb300 import eos_coexistence, eos_pressure
    rv, rl, _ = eos_coexistence("cs", 1.0, 4.0, 1.0, Tr)
    got = obs.surface_tension(
        lambda v: eos_pressure("cs", 1.0, 4.0, 1.0, Tr, 0.344, v), rv, rl, 0.5)
    want = thermo.surface_tension(thermo.make_eos("cs", 1.0, 4.0, 1.0, Tr), 0.5)
    assert got == pytest.approx(want, rel=1e-7)


@pytest.mark.parametrize("theta", [30, 90, 150])
def test_warm_cap_holds_the_requested_mass(theta):
    """The mass-matched warm cap carries exactly the total density asked for
    (the cold start's), whatever its angle and densities, and without a
    target keeps the case's area."""
    nx, ny = 256, 128
    case = dict(CASE, area=0.1)
    cold = inputs.wall_drop(nx, ny, math.sqrt(2 * 0.1 * nx * (ny - 2) / math.pi),
                            2.0, 0.05, 4.0)
    M = ws.fluid_mass(cold)
    pred = dict(theta=theta, rho_l=1.97, rho_v=0.058, width=3.0)
    rho = ws.warm_field(case, pred, nx, ny, mass=M)
    assert abs(ws.fluid_mass(rho) / M - 1) < 1e-6
    # the cap grows when the case's area at these densities holds too little
    # mass, and shrinks when it holds too much
    plain = ws.warm_field(case, pred, nx, ny)
    grew = (rho[1:-1] > 1.0).sum() > (plain[1:-1] > 1.0).sum()
    assert grew == (ws.fluid_mass(plain) < M)
    assert abs(ws.fluid_mass(ws.warm_field(case, pred, nx, ny, mass=1.05 * M)) / (1.05 * M) - 1) < 1e-6
