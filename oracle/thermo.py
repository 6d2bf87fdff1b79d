"""EOS-level helpers of the oracle: temperature function alpha(T), critical
point, spinodal, Maxwell equal-area coexistence and square-gradient surface
tension.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Every EOS of the paper splits as p0(rho, T) = T A(rho) - alpha B(rho)
(Eqs. 16, 19, 22, 25).  The critical point is where dp0/drho and
d2p0/drho2 both vanish with alpha = 1 (alpha(T_c) = 1 by its definition under
Eq. 19 and Eq. 22): eliminating T gives B' A'' - B'' A' = 0 for rho_c and then
T_c = B'(rho_c) / A'(rho_c).  The derivatives below are worked out by hand
from the printed p0 and are pinned by the tests against finite differences,
the closed-form van der Waals point and the textbook cubic-EOS constants.
"""
import math

import numpy as np
from scipy import integrate, optimize

from . import EOS_CS, EOS_NAMES, EOS_PR, EOS_RKS, EOS_VDW, Eos


def _kind(kind):
    return EOS_NAMES[kind] if isinstance(kind, str) else int(kind)


def rho_max(kind, b):
    """Upper end of the physical density range (repulsive pole)."""
    return 4.0 / b if _kind(kind) == EOS_CS else 1.0 / b


def alpha_of(kind, Tr, omega):
    """alpha(T) of RKS (text under Eq. 19) and PR (text under Eq. 22);
    1 for vdW and CS.  Tr = T / T_c."""
    k = _kind(kind)
    if k == EOS_PR:
        m = 0.37464 + 1.54226 * omega - 0.26992 * omega ** 2
    elif k == EOS_RKS:
        m = 0.480 + 1.574 * omega - 0.176 * omega ** 2
    else:
        return 1.0
    return (1.0 + m * (1.0 - math.sqrt(Tr))) ** 2


def _AB_derivs(kind, a, b, R, rho):
    """(A', A'', B', B'') of p0 = T A - alpha B at density rho."""
    k = _kind(kind)
    if k == EOS_CS:
        h = b * rho / 4.0
        A1 = R * (1 + 4 * h + 4 * h * h - 4 * h ** 3 + h ** 4) / (1 - h) ** 4
        A2 = R * (b / 4.0) * (8 + 20 * h - 4 * h * h) / (1 - h) ** 5
    else:
        A1 = R / (1 - b * rho) ** 2
        A2 = 2 * R * b / (1 - b * rho) ** 3
    if k in (EOS_VDW, EOS_CS):
        B1, B2 = 2 * a * rho, 2 * a
    elif k == EOS_RKS:
        B1 = a * rho * (2 + b * rho) / (1 + b * rho) ** 2
        B2 = 2 * a / (1 + b * rho) ** 3
    else:  # PR
        D = 1 + 2 * b * rho - (b * rho) ** 2
        B1 = 2 * a * rho * (1 + b * rho) / D ** 2
        B2 = 2 * a * (1 + 3 * (b * rho) ** 2 + 2 * (b * rho) ** 3) / D ** 3
    return A1, A2, B1, B2


def dp0_drho(kind, a, b, R, T, alpha, rho):
    A1, _, B1, _ = _AB_derivs(kind, a, b, R, rho)
    return T * A1 - alpha * B1


def critical_point(kind, a, b, R=1.0):
    """(T_c, rho_c) with alpha = 1."""

    def g(r):
        A1, A2, B1, B2 = _AB_derivs(kind, a, b, R, r)
        return B1 * A2 - B2 * A1

    top = rho_max(kind, b)
    rc = optimize.brentq(g, 1e-9 * top, (1 - 1e-9) * top, xtol=1e-300,
                         rtol=4 * np.finfo(float).eps, maxiter=500)
    A1, _, B1, _ = _AB_derivs(kind, a, b, R, rc)
    return B1 / A1, rc


def make_eos(kind, a, b, R=1.0, Tr=0.85, omega=0.344):
    """The paper's EOS at reduced temperature Tr = T / T_c."""
    Tc, _ = critical_point(kind, a, b, R)
    return Eos(kind, a, b, R, Tr * Tc, alpha_of(kind, Tr, omega))


def spinodal(eos: Eos):
    """(rho_s1, rho_s2): the two roots of dp0/drho = 0 around rho_c."""
    _, rc = critical_point(eos.kind, eos.a, eos.b, eos.R)
    top = rho_max(eos.kind, eos.b)

    def d(r):
        return dp0_drho(eos.kind, eos.a, eos.b, eos.R, eos.T, eos.alpha, r)

    if d(rc) >= 0:
        raise ValueError("no spinodal: temperature at or above critical")
    lo = optimize.brentq(d, 1e-12 * top, rc, xtol=1e-300, rtol=1e-15)
    hi = optimize.brentq(d, rc, (1 - 1e-12) * top, xtol=1e-300, rtol=1e-15)
    return lo, hi


def maxwell(eos: Eos):
    """Coexisting (rho_v, rho_l, mu_coex, p_coex) from the Maxwell equal-area
    construction (Sec. III): equal pressure and equal chemical potential."""
    s1, s2 = spinodal(eos)
    top = rho_max(eos.kind, eos.b)
    p_s1, p_s2 = float(eos.p0(s1)), float(eos.p0(s2))

    def roots(p):
        rv = optimize.brentq(lambda r: float(eos.p0(r)) - p, 1e-300, s1,
                             xtol=1e-300, rtol=1e-15)
        rl = optimize.brentq(lambda r: float(eos.p0(r)) - p, s2,
                             (1 - 1e-14) * top, xtol=1e-300, rtol=1e-15)
        return rv, rl

    def dmu(p):
        rv, rl = roots(p)
        return float(eos.mu(rv)) - float(eos.mu(rl))

    lo = max(p_s2, 0.0) + 1e-14 * abs(p_s1)
    hi = p_s1 * (1 - 1e-12)
    p = optimize.brentq(dmu, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    rv, rl = roots(p)
    # Newton polish on (rho_v, rho_l): mu_v - mu_l = 0, p_v - p_l = 0.
    for _ in range(4):
        _, mv, pv = (float(x) for x in eos.eval(rv))
        _, ml, pl = (float(x) for x in eos.eval(rl))
        dv = dp0_drho(eos.kind, eos.a, eos.b, eos.R, eos.T, eos.alpha, rv)
        dl = dp0_drho(eos.kind, eos.a, eos.b, eos.R, eos.T, eos.alpha, rl)
        J = np.array([[dv / rv, -dl / rl], [dv, -dl]])
        step = np.linalg.solve(J, -np.array([mv - ml, pv - pl]))
        rv, rl = rv + step[0], rl + step[1]
    mu_c = 0.5 * (float(eos.mu(rv)) + float(eos.mu(rl)))
    p_c = 0.5 * (float(eos.p0(rv)) + float(eos.p0(rl)))
    return rv, rl, mu_c, p_c


def surface_tension(eos: Eos, kappa: float):
    """Flat-interface tension of the square-gradient free energy (Eq. 1):
    sigma = integral over [rho_v, rho_l] of sqrt(2 kappa (psi - mu_c rho + p_c)),
    the excess grand potential density being psi - mu_c rho + p_c >= 0."""
    rv, rl, mu_c, p_c = maxwell(eos)

    def integrand(r):
        w = float(eos.psi(r)) - mu_c * r + p_c
        return math.sqrt(2.0 * kappa * max(w, 0.0))

    val, _ = integrate.quad(integrand, rv, rl, epsabs=0, epsrel=1e-10,
                            limit=400)
    return val
