"""Measurements on converged density fields: for a wall droplet the bulk
liquid and vapour densities, interface width and contact angle (Sec. V's
spherical-cap formulas); for a free droplet in a periodic box the Laplace
pressure jump and equimolar radius (Sec. III).  Used by the learned warm
start and the physics reports; plain NumPy on host arrays [ny, nx].

Conventions: rows 0 and ny - 1 are solid; the wall plane of the halfway
bounce-back lies half a node above row 0; the interface is the level set
rho_m = (rho_l + rho_v) / 2, located by linear interpolation.
"""
import math

import numpy as np


def bulk_densities(rho):
    """(rho_l, rho_v): mean of the liquid plateau (within 2 % of the largest
    density) and median of the top quarter of the fluid rows."""
    fluid = rho[1:-1]
    top = fluid.max()
    rho_l = float(fluid[fluid >= top - 0.02 * abs(top)].mean())
    q = max(1, fluid.shape[0] // 4)
    rho_v = float(np.median(fluid[-q:]))
    return rho_l, rho_v


def _level_crossings(v, level):
    """Fractional positions where the sequence v crosses `level`."""
    s = v - level
    i = np.nonzero(s[:-1] * s[1:] < 0)[0]
    return i + s[i] / (s[i] - s[i + 1])


def drop_column(rho):
    """Column through the drop's mass centre (excess over the vapour)."""
    _, rho_v = bulk_densities(rho)
    w = np.clip(rho[1:-1] - rho_v, 0.0, None).sum(axis=0)
    if w.sum() <= 0:
        return rho.shape[1] // 2
    return int(round(float((w * np.arange(rho.shape[1])).sum() / w.sum())))


def interface_width(rho):
    """10-90 % thickness of the drop's top interface along its centre
    column, converted to the width W of a tanh(2 d / W) profile."""
    rho_l, rho_v = bulk_densities(rho)
    col = rho[1:-1, drop_column(rho)]
    lo = _level_crossings(col, rho_v + 0.1 * (rho_l - rho_v))
    hi = _level_crossings(col, rho_v + 0.9 * (rho_l - rho_v))
    if len(lo) == 0 or len(hi) == 0:
        return float("nan")
    return float((lo.max() - hi.max()) / math.atanh(0.8))


def contact_angle(rho):
    """Contact angle in degrees from the base chord L on the wall plane
    (extrapolated from the first two fluid rows) and the apex height H
    above it (Sec. V):
    R = (4 H^2 + L^2) / (8 H), tan(theta) = L / (2 (R - H)).  A drop no
    longer touching the wall gives 180, liquid covering the whole wall 0."""
    rho_l, rho_v = bulk_densities(rho)
    mid = 0.5 * (rho_l + rho_v)
    if not (rho[1] > mid).any():
        return 180.0 if (rho[1:-1] > mid).any() else float("nan")
    if (rho[1] > mid).all():
        return 0.0                     # a film over the whole wall
    cx = drop_column(rho)
    chords = []
    for row in (rho[1], rho[2]):
        xs = _level_crossings(row, mid)
        left, right = xs[xs <= cx], xs[xs >= cx]
        if len(left) == 0 or len(right) == 0:
            return float("nan")
        chords.append(float(right.min() - left.max()))
    # rows 1 and 2 sit 0.5 and 1.5 above the wall plane: extrapolate the
    # chord linearly down to the plane
    L = 1.5 * chords[0] - 0.5 * chords[1]
    ys = _level_crossings(rho[1:-1, cx], mid)
    if len(ys) == 0:
        return float("nan")
    H = float(ys.max()) + 0.5          # fluid row 1 is 0.5 above the wall
    R = (4 * H * H + L * L) / (8 * H)
    return math.degrees(math.atan2(L / 2, R - H))


def measure(rho):
    """dict of rho_l, rho_v, width, theta for a wall-droplet field."""
    rho_l, rho_v = bulk_densities(rho)
    return dict(rho_l=rho_l, rho_v=rho_v, width=interface_width(rho),
                theta=contact_angle(rho))


def periodic_drop_bulk(rho):
    """(rho_in, rho_out) of a static drop in a periodic box: the density at
    the drop's centre - the mean of the 3 x 3 nodes around the density
    maximum, where the bulk pressure of a static drop peaks and its profile
    is flat - and the median of the box's edge rows and columns, the points
    farthest from a centred drop.  (A mean over a band of the largest
    densities takes in the top of the interface profile and biases rho_in
    low; the pressure jump of a large drop is too small to afford that.)"""
    ny, nx = rho.shape
    jy, jx = np.unravel_index(int(np.argmax(rho)), rho.shape)
    rows = (np.arange(-1, 2) + jy) % ny
    cols = (np.arange(-1, 2) + jx) % nx
    rho_in = float(rho[np.ix_(rows, cols)].mean())
    edge = np.concatenate([rho[0], rho[-1], rho[:, 0], rho[:, -1]])
    return rho_in, float(np.median(edge))


def equimolar_radius(rho, rho_in, rho_out):
    """Radius of the disc that holds the drop's excess mass at the bulk
    densities: A = sum(rho - rho_out) / (rho_in - rho_out), R = sqrt(A / pi)."""
    area = float((rho - rho_out).sum()) / (rho_in - rho_out)
    return math.sqrt(max(area, 0.0) / math.pi)


def laplace_jump(rho, pressure):
    """(Delta p, R) of a static periodic drop: the bulk pressure p0 of the
    interior density minus that of the far field, and the equimolar radius.
    pressure maps an array of densities to p0 (the library's EOS)."""
    rho_in, rho_out = periodic_drop_bulk(rho)
    p_in, p_out = pressure(np.array([rho_in, rho_out]))
    return float(p_in - p_out), equimolar_radius(rho, rho_in, rho_out)


def surface_tension(pressure, rho_v, rho_l, kappa, nodes=64):
    """Tension of a flat interface in the square-gradient theory of Eq. 1:
    sigma = integral over [rho_v, rho_l] of sqrt(2 kappa w(rho)), w the
    excess grand-potential density.  With psi from the bulk pressure (Eq. 15)
    and Eq. 3, d(w / rho) / drho = (p0(rho) - p_c) / rho^2 and w(rho_v) = 0,
    so w(rho) = rho * integral from rho_v to rho of (p0(s) - p_c) / s^2 ds,
    p_c = p0(rho_v): only the bulk pressure is needed.  pressure maps an
    array of densities to p0 (the library's EOS); rho_v, rho_l are the
    coexisting densities.  Gauss-Legendre quadrature of `nodes` points,
    inner and outer."""
    x, wq = np.polynomial.legendre.leggauss(nodes)
    p_c = float(np.asarray(pressure(np.array([rho_v])))[0])

    def w_of(r):
        s = rho_v + (r - rho_v) * 0.5 * (x + 1.0)
        g = (np.asarray(pressure(s)) - p_c) / (s * s)
        return r * 0.5 * (r - rho_v) * float((wq * g).sum())

    r_out = rho_v + (rho_l - rho_v) * 0.5 * (x + 1.0)
    vals = np.array([math.sqrt(2.0 * kappa * max(w_of(r), 0.0)) for r in r_out])
    return 0.5 * (rho_l - rho_v) * float((wq * vals).sum())


def line_fit(x, y):
    """Least-squares y = slope x + intercept: (slope, intercept, r^2)."""
    x, y = np.asarray(x, float), np.asarray(y, float)
    slope, icpt = np.polyfit(x, y, 1)
    res = y - (slope * x + icpt)
    tot = ((y - y.mean()) ** 2).sum()
    return float(slope), float(icpt), float(1 - (res ** 2).sum() / tot) if tot > 0 else 1.0


def slab_bulk(rho):
    """(rho_l, rho_v) of a liquid slab centred in a periodic box along y:
    medians of the x-averaged profile over the central quarter of the rows
    and over the quarter farthest from the slab (the box edges)."""
    prof = rho.mean(axis=1)
    n = prof.size
    mid = prof[3 * n // 8:5 * n // 8]
    far = np.concatenate([prof[:n // 8], prof[n - n // 8:]])
    return float(np.median(mid)), float(np.median(far))
