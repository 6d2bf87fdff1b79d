"""Pins of the oracle's step pieces against closed forms and invariants.

* Gradient and Laplacian: exact Fourier symbols of the isotropic D2Q9
  stencils on periodic plane waves, and exactness on low-order polynomials.
* Eq. 28 solid-row density: its weights read back from a delta row.
* Wall chemical potential: the surface value on the bottom row (Sec. IV),
  the copied neighbour on the top row (Sec. V).
* Equilibrium (Eq. 14): zeroth, first and second moments of the D2Q9
  Maxwellian.
* Collision (Eq. 13 with u_eq = u + tau F / rho): mass kept, momentum raised
  by exactly F, equilibrium left unchanged when F = 0.
* Streaming: a permutation of populations; halfway bounce-back returns each
  population that would enter a solid row reversed at its own node.
* Whole step: a uniform state moving at any uniform velocity is a fixed
  point; mass is conserved to round-off, periodic and walled.
"""
import numpy as np
import pytest

import oracle
from oracle import EX, EY, OPP, W, thermo
from paper_1611_00907_gb300 import inputs


def _lat(nx=24, ny=20, walls=False, **kw):
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    return oracle.Lattice(nx, ny, e, kw.pop("tau", 1.0), kw.pop("kappa", 0.5),
                          walls=walls, **kw)


@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 2), (3, 1), (5, 4)])
def test_stencil_fourier_symbols(kx, ky):
    nx, ny = 24, 20
    L = _lat(nx, ny)
    yy, xx = np.mgrid[0:ny, 0:nx]
    qx, qy = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    phase = qx * xx + qy * yy
    phi = np.sin(phase)
    lap = L.laplacian(phi)
    sym = (4 * (2 * np.cos(qx) + 2 * np.cos(qy)) + 4 * np.cos(qx) * np.cos(qy)
           - 20) / 6
    assert np.max(np.abs(lap - sym * phi)) < 1e-13
    gx, gy = L.gradient(phi)
    assert np.max(np.abs(gx - np.sin(qx) * (2 + np.cos(qy)) / 3 *
                         np.cos(phase))) < 1e-13
    assert np.max(np.abs(gy - np.sin(qy) * (2 + np.cos(qx)) / 3 *
                         np.cos(phase))) < 1e-13


def test_stencils_exact_on_polynomials_in_interior():
    nx, ny = 16, 16
    L = _lat(nx, ny)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    lin = 0.3 * xx - 0.7 * yy + 2.0
    quad = 1.5 * xx ** 2 - 0.5 * xx * yy + 0.25 * yy ** 2 + xx
    gx, gy = L.gradient(lin)
    lap = L.laplacian(quad)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    assert np.allclose(gx[inner], 0.3, atol=1e-13)
    assert np.allclose(gy[inner], -0.7, atol=1e-13)
    assert np.allclose(lap[inner], 2 * 1.5 + 2 * 0.25, atol=1e-12)


def test_wall_density_eq28_weights():
    nx, ny = 10, 8
    L = _lat(nx, ny, walls=True)
    rho = np.zeros((ny, nx))
    rho[1, 4] = 1.0          # delta on the first fluid row
    rho[ny - 2, 0] = 6.0     # delta on the last fluid row, at the x seam
    out = L.wall_density(rho)
    expect0 = np.zeros(nx)
    expect0[[3, 4, 5]] = [1 / 6, 2 / 3, 1 / 6]
    expectN = np.zeros(nx)
    expectN[[nx - 1, 0, 1]] = [1.0, 4.0, 1.0]
    assert np.allclose(out[0], expect0, atol=1e-15)
    assert np.allclose(out[ny - 1], expectN, atol=1e-15)
    assert np.array_equal(out[1:ny - 1], rho[1:ny - 1])


def test_wall_chemical_potential_rows():
    nx, ny = 12, 9
    L = _lat(nx, ny, walls=True, mu_bottom=-0.0125)
    rng = np.random.default_rng(3)
    rho = L.wall_density(0.15 + 0.05 * rng.uniform(-1, 1, (ny, nx)))
    mu = L.chem_potential(rho)
    assert np.all(mu[0] == -0.0125)
    assert np.array_equal(mu[ny - 1], mu[ny - 2])
    # fluid rows: psi'(rho) - kappa lap(rho), lap using the Eq. 28 rows
    lap = L.laplacian(rho)
    fl = slice(1, ny - 1)
    assert np.allclose(mu[fl], L.eos.mu(rho[fl]) - 0.5 * lap[fl], atol=1e-15,
                       rtol=1e-14)
    L2 = _lat(nx, ny, walls=True, mu_bottom=0.0, top_mode=1, mu_top=0.03)
    assert np.all(L2.chem_potential(rho)[ny - 1] == 0.03)


@pytest.mark.parametrize("u", [(0.0, 0.0), (0.05, -0.02), (-0.1, 0.07)])
def test_equilibrium_moments(u):
    rho = 0.37
    f = oracle.equilibrium(rho, *u)
    ux, uy = u
    assert f.sum() == pytest.approx(rho, rel=1e-15)
    assert (f * EX).sum() == pytest.approx(rho * ux, abs=1e-16)
    assert (f * EY).sum() == pytest.approx(rho * uy, abs=1e-16)
    cs2 = 1 / 3
    assert (f * EX * EX).sum() == pytest.approx(rho * (cs2 + ux * ux), 1e-14)
    assert (f * EY * EY).sum() == pytest.approx(rho * (cs2 + uy * uy), 1e-14)
    assert (f * EX * EY).sum() == pytest.approx(rho * ux * uy, abs=1e-16)
    assert np.allclose(oracle.equilibrium(rho, 0, 0), rho * W, rtol=1e-15)


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.3])
def test_collision_mass_and_momentum(tau):
    rng = np.random.default_rng(11)
    f = oracle.equilibrium(0.2, 0.03, -0.01) * (1 + 0.1 * rng.uniform(-1, 1, 9))
    Fx, Fy = 1.3e-3, -2.1e-3
    out = oracle.collide_node(f, Fx, Fy, tau)
    assert out.sum() == pytest.approx(f.sum(), rel=1e-15)
    assert (out * EX).sum() == pytest.approx((f * EX).sum() + Fx, abs=1e-16)
    assert (out * EY).sum() == pytest.approx((f * EY).sum() + Fy, abs=1e-16)
    feq = oracle.equilibrium(0.25, -0.04, 0.02)
    assert np.allclose(oracle.collide_node(feq, 0.0, 0.0, tau), feq,
                       rtol=1e-14, atol=0)


def test_collision_relaxes_to_shifted_equilibrium_at_tau_one():
    f = oracle.equilibrium(0.3, 0.0, 0.0) * np.linspace(0.9, 1.1, 9)
    Fx, Fy = 2e-3, 1e-3
    rho = f.sum()
    ux, uy = (f * EX).sum() / rho, (f * EY).sum() / rho
    out = oracle.collide_node(f, Fx, Fy, 1.0)
    expect = oracle.equilibrium(rho, ux + Fx / rho, uy + Fy / rho)
    assert np.allclose(out, expect, rtol=1e-14, atol=1e-17)


def test_streaming_periodic_is_a_shift():
    nx, ny = 7, 6
    L = _lat(nx, ny)
    for i in range(9):
        fpost = np.zeros((9, ny, nx))
        fpost[i, 2, 3] = 1.0
        out = L.stream(fpost)
        assert out.sum() == 1.0
        assert out[i, (2 + EY[i]) % ny, (3 + EX[i]) % nx] == 1.0


def test_streaming_bounce_back_on_both_walls():
    nx, ny = 7, 6
    L = _lat(nx, ny, walls=True)
    for y in (1, ny - 2):
        for i in range(9):
            fpost = np.zeros((9, ny, nx))
            fpost[i, y, 0] = 1.0
            out = L.stream(fpost)
            yt = y + EY[i]
            if yt in (0, ny - 1):
                assert out[OPP[i], y, 0] == 1.0
            else:
                assert out[i, yt, (0 + EX[i]) % nx] == 1.0
            assert out.sum() == 1.0


@pytest.mark.parametrize("walls", [False, True])
def test_uniform_moving_state_is_a_fixed_point(walls):
    nx, ny = 12, 10
    L = _lat(nx, ny, walls=walls)
    ux = 0.0 if walls else 0.04
    rho = np.full((ny, nx), 0.2)
    L.init_equilibrium(rho, np.full((ny, nx), ux), np.full((ny, nx), -0.02 *
                                                          (not walls)))
    f0 = L.f.copy()
    L.mu_bottom = float(L.eos.mu(0.2))
    L.step(10)
    assert np.max(np.abs(L.f - f0)) < 1e-15


@pytest.mark.parametrize("walls", [False, True])
def test_mass_conservation(walls, oracle_threads):
    nx, ny = 40, 30
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    rv, rl, mc, _ = thermo.maxwell(e)
    L = oracle.Lattice(nx, ny, e, 1.0, 0.5, walls=walls, mu_bottom=mc + 0.01)
    rho = (inputs.wall_drop(nx, ny, 12, rl, rv) if walls
           else inputs.drop(nx, ny, 10, rl, rv))
    L.init_equilibrium(rho)
    fl = L.fluid_rows()
    m0 = L.density()[fl].sum()
    L.step(300)
    m1 = L.density()[fl].sum()
    assert abs(m1 - m0) / m0 < 1e-13
