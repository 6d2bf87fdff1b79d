"""Pins of the oracle's pressure-tensor force (Eq. 5 with Eq. 9), the form
the chemical-potential method replaces.

The paper's identity div(P) = rho grad(mu) (Eq. 11) makes the two forces
equal in the continuum; on the lattice they differ by the discretisation,
which must shrink at second order as the field gets smoother.  A uniform
state feels no force, and a step with this force conserves mass.
"""
import numpy as np
import pytest

import oracle
from oracle import thermo


def _lat(n, kappa=0.5):
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    return oracle.Lattice(n, n, e, 1.0, kappa)


@pytest.mark.parametrize("kappa", [0.5, 0.0])
def test_pressure_tensor_force_converges_to_chemical_potential_force(kappa):
    errs = []
    for n in (32, 64, 128):
        L = _lat(n, kappa)
        yy, xx = np.mgrid[0:n, 0:n]
        rho = 0.15 + 0.05 * np.sin(2 * np.pi * xx / n) * np.cos(
            2 * np.pi * 2 * yy / n)
        fx_pt, fy_pt = L.force_pressure_tensor(rho)
        mu = L.chem_potential(rho)
        fx_cp, fy_cp = L.force(rho, mu)
        scale = np.abs(fx_cp).max() + np.abs(fy_cp).max()
        errs.append((np.abs(fx_pt - fx_cp).max() + np.abs(fy_pt - fy_cp).max())
                    / scale)
    # halving the grid spacing relative to the wave cuts the gap ~4x
    assert errs[0] / errs[1] > 3.2 and errs[1] / errs[2] > 3.5
    assert errs[2] < 2e-3


def test_uniform_state_feels_no_pressure_tensor_force():
    L = _lat(16)
    fx, fy = L.force_pressure_tensor(np.full((16, 16), 0.2))
    assert np.abs(fx).max() < 1e-15 and np.abs(fy).max() < 1e-15


def test_pressure_tensor_step_conserves_mass_and_rejects_walls():
    n = 40
    L = _lat(n)
    yy, xx = np.mgrid[0:n, 0:n]
    rho = 0.15 + 0.1 * np.exp(-((xx - 20) ** 2 + (yy - 20) ** 2) / 50.0)
    L.init_equilibrium(rho)
    m0 = L.density().sum()
    L.step_pressure_tensor(200)
    assert abs(L.density().sum() - m0) / m0 < 1e-13
    W = oracle.Lattice(n, n, L.eos, 1.0, 0.5, walls=True)
    W.init_equilibrium(rho)
    with pytest.raises(ValueError):
        W.step_pressure_tensor(1)
