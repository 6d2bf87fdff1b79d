"""Post-processing of density fields: bulk densities, Laplace pressure jump
and contact angle.  TEST INFRASTRUCTURE ONLY (see the package docstring).

These are measurements on a field, not part of the step.  Readings of the
paper's measurement conventions (Sec. V gives the spherical-cap formulas but
not how L and H are taken off the lattice):

* the interface is the rho_m = (rho_l + rho_v) / 2 contour, located by linear
  interpolation between nodes;
* with halfway bounce-back the wall plane lies at y = 0.5, half a node below
  the first fluid row y = 1;
* the base L is the contour's chord on row y = 1 and the height H is the apex
  of the contour above the wall plane along the drop's centre column;
* R = (4 H^2 + L^2) / (8 H) and tan(theta) = L / (2 (R - H)) (Sec. V), taken
  with atan2 so that theta > 90 degrees when R < H;
* a drop with no liquid left on the first fluid row has lifted off the wall
  and counts as 180 degrees (the paper's superhydrophobic end, Fig. 2f).
"""
import math

import numpy as np


def _crossing(vals, level):
    """Fractional index positions where a 1-D sequence crosses `level`."""
    out = []
    for k in range(len(vals) - 1):
        a, b = vals[k] - level, vals[k + 1] - level
        if a == 0.0:
            out.append(float(k))
        elif a * b < 0.0:
            out.append(k + a / (a - b))
    return out


def equimolar_radius(rho, rho_in, rho_out):
    """Radius of the disc holding the same excess mass as the field: the
    Gibbs equimolar radius sqrt(A / pi), A = sum (rho - rho_out) /
    (rho_in - rho_out)."""
    A = float(((rho - rho_out) / (rho_in - rho_out)).sum())
    return math.sqrt(A / math.pi)


def laplace_jump(eos, rho, centre=None, far=(0, 0)):
    """(Delta p, r_eq) of a periodic drop: Delta p = p0(rho at the centre) -
    p0(rho far away) (Eq. 3; gradients vanish in both bulks)."""
    ny, nx = rho.shape
    cy, cx = centre if centre is not None else (ny // 2, nx // 2)
    rin, rout = float(rho[cy, cx]), float(rho[far])
    dp = float(eos.p0(rin)) - float(eos.p0(rout))
    return dp, equimolar_radius(rho, rin, rout)


def contact_angle(rho, rho_l, rho_v, wall_row=0):
    """Contact angle in degrees of a drop sitting on the solid row `wall_row`
    (0: bottom wall; the drop's liquid touches row 1).  Returns
    (theta_deg, L, H)."""
    level = 0.5 * (rho_l + rho_v)
    base = rho[wall_row + 1]
    xs = _crossing(base, level)
    liquid = base > level
    if not liquid.any():
        # no liquid on the wall: a drop that has lifted off is fully
        # non-wetting (180 degrees); no liquid at all has no angle
        return (180.0 if (rho > level).any() else float("nan")), 0.0, 0.0
    if len(xs) < 2:
        return float("nan"), float("nan"), float("nan")
    # The chord is the liquid run around the densest node of the base row.
    peak = int(np.argmax(base))
    left = max([x for x in xs if x <= peak], default=None)
    right = min([x for x in xs if x >= peak], default=None)
    if left is None or right is None:
        return float("nan"), float("nan"), float("nan")
    L = right - left
    # Centre column: mass-weighted centroid of the liquid excess.
    ex = np.clip(rho - rho_v, 0.0, None)
    cx = float((ex.sum(axis=0) * np.arange(rho.shape[1])).sum() / ex.sum())
    col = int(round(cx))
    ys = _crossing(rho[wall_row + 1:, col], level)
    if not ys:
        return float("nan"), float("nan"), float("nan")
    H = (wall_row + 1 + max(ys)) - (wall_row + 0.5)
    R = (4.0 * H * H + L * L) / (8.0 * H)
    theta = math.degrees(math.atan2(L / 2.0, R - H))
    return theta, L, H


def slab_bulk(rho, axis=0):
    """(max, min) of the row- (or column-) averaged density of a slab."""
    prof = rho.mean(axis=1 - axis)
    return float(prof.max()), float(prof.min())
