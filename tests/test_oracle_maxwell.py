"""Pins of the oracle's coexistence and surface-tension helpers.

* Maxwell's equal-area rule itself (Sec. III): integral of p0 dv between the
  coexisting specific volumes equals p_sat (v_v - v_l).  It is checked by
  quadrature of the printed p0 alone, independent of psi and mu, which the
  solver uses.
* Mean-field critical scaling with the van der Waals closed form
  (rho_l - rho_v) / rho_c -> 4 sqrt(1 - T_r).
* Law of corresponding states: reduced coexistence densities do not depend
  on a, b, R.
* Square-gradient tension near T_c against the quartic (Landau) double well:
  sigma -> sqrt(2 kappa c4) (rho_l - rho_v)^3 / 6, c4 = psi''''(rho_c) / 24.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import thermo

CASES = [("vdw", 9 / 49, 2 / 21), ("cs", 1.0, 4.0), ("pr", 2 / 49, 2 / 21),
         ("rks", 2 / 49, 2 / 21)]


@pytest.mark.parametrize("kind,a,b", CASES)
@pytest.mark.parametrize("Tr", [0.6, 0.8, 0.95])
def test_equal_area_rule(kind, a, b, Tr):
    e = thermo.make_eos(kind, a, b, 1.0, Tr, 0.344)
    rv, rl, mu_c, p_c = thermo.maxwell(e)
    assert rv < rl
    vl, vv = 1 / rl, 1 / rv
    area, _ = integrate.quad(lambda v: float(e.p0(1 / v)), vl, vv,
                             epsabs=0, epsrel=1e-12, limit=500)
    assert area == pytest.approx(p_c * (vv - vl), rel=1e-9,
                                 abs=1e-12 * abs(e.T * (vv - vl) / vl))
    assert float(e.p0(rv)) == pytest.approx(float(e.p0(rl)), rel=1e-10,
                                            abs=1e-14)


def test_vdw_critical_scaling():
    a, b = 9 / 49, 2 / 21
    _, rc = thermo.critical_point("vdw", a, b)
    for t in (1e-4, 4e-4):
        e = thermo.make_eos("vdw", a, b, 1.0, 1 - t)
        rv, rl, _, _ = thermo.maxwell(e)
        assert (rl - rv) / rc == pytest.approx(4 * math.sqrt(t), rel=2e-3)


@pytest.mark.parametrize("kind", ["vdw", "cs", "pr", "rks"])
def test_corresponding_states(kind):
    e1 = thermo.make_eos(kind, 1.0, 1.0, 1.0, 0.8, 0.344)
    e2 = thermo.make_eos(kind, 3.0, 0.25, 0.5, 0.8, 0.344)
    r1 = np.array(thermo.maxwell(e1)[:2]) / thermo.critical_point(
        kind, 1.0, 1.0, 1.0)[1]
    r2 = np.array(thermo.maxwell(e2)[:2]) / thermo.critical_point(
        kind, 3.0, 0.25, 0.5)[1]
    assert np.allclose(r1, r2, rtol=1e-10)


def test_surface_tension_near_critical_landau_limit():
    a, b, kappa = 9 / 49, 2 / 21, 0.3
    Tc, rc = thermo.critical_point("vdw", a, b)
    ec = oracle.Eos("vdw", a, b, 1.0, Tc)
    h = 2e-2 * rc
    p = [float(ec.p0(rc + k * h)) for k in (-2, -1, 1, 2)]
    p3 = (-p[0] + 2 * p[1] - 2 * p[2] + p[3]) / (2 * h ** 3)
    c4 = p3 / rc / 24.0
    e = thermo.make_eos("vdw", a, b, 1.0, 1 - 1e-4)
    rv, rl, _, _ = thermo.maxwell(e)
    landau = math.sqrt(2 * kappa * c4) * (rl - rv) ** 3 / 6
    assert thermo.surface_tension(e, kappa) == pytest.approx(landau, rel=2e-2)


def test_surface_tension_scales_as_sqrt_kappa():
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    s1 = thermo.surface_tension(e, 0.5)
    s2 = thermo.surface_tension(e, 2.0)
    assert s2 == pytest.approx(2 * s1, rel=1e-9)


def test_no_coexistence_above_critical():
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 1.05)
    with pytest.raises(ValueError):
        thermo.spinodal(e)
