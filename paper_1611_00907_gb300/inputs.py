"""Seeded synthetic initial states shared by the tests, the benchmark and the
oracle's callers.

This module holds geometry and random numbers only, none of the method's
arithmetic: every density it needs (coexistence densities, critical density)
is an argument supplied by the caller.  Profiles are smoothed steps
rho = (rho_l + rho_v) / 2 + (rho_l - rho_v) / 2 * tanh(2 d / width), where d
is the signed distance to the interface, positive inside the liquid.  Fields
are float64 arrays of shape [ny, nx], row-major; node (x, y) sits at integer
coordinates.
"""
import numpy as np


def tanh_profile(d, rho_l, rho_v, width):
    return 0.5 * (rho_l + rho_v) + 0.5 * (rho_l - rho_v) * np.tanh(
        2.0 * np.asarray(d, dtype=np.float64) / width)


def _grid(nx, ny):
    yy, xx = np.mgrid[0:ny, 0:nx]
    return xx.astype(np.float64), yy.astype(np.float64)


def slab(nx, ny, rho_l, rho_v, width=4.0, half_thickness=None, axis="y"):
    """Liquid layer centred in the domain, normal along `axis`, periodic.

    The liquid occupies |c - centre| < half_thickness (default: a quarter of
    the domain along the normal), centre = n / 2 between nodes."""
    xx, yy = _grid(nx, ny)
    c, n = (yy, ny) if axis == "y" else (xx, nx)
    h = n / 4.0 if half_thickness is None else half_thickness
    d = h - np.abs(c + 0.5 - n / 2.0)
    return tanh_profile(d, rho_l, rho_v, width)


def drop(nx, ny, radius, rho_l, rho_v, width=4.0, centre=None):
    """Circular liquid drop (periodic domain), centred between nodes."""
    xx, yy = _grid(nx, ny)
    cx, cy = centre if centre is not None else (nx / 2.0 - 0.5, ny / 2.0 - 0.5)
    d = radius - np.hypot(xx - cx, yy - cy)
    return tanh_profile(d, rho_l, rho_v, width)


def wall_drop(nx, ny, radius, rho_l, rho_v, width=4.0, centre_x=None):
    """Half disc of liquid resting on the bottom wall.

    The solid rows are y = 0 and y = ny - 1; with halfway bounce-back the
    wall plane is y = 0.5, where the disc is centred.  Solid-row values are
    returned too but never used as state."""
    xx, yy = _grid(nx, ny)
    cx = nx / 2.0 - 0.5 if centre_x is None else centre_x
    d = radius - np.hypot(xx - cx, yy - 0.5)
    return tanh_profile(d, rho_l, rho_v, width)


def spinodal_noise(nx, ny, rho_mean, amplitude=0.01, seed=1):
    """rho = rho_mean (1 + amplitude xi), xi ~ U[-1, 1) i.i.d., numpy PCG64."""
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, size=(ny, nx))
    return rho_mean * (1.0 + amplitude * xi)


def perturbed(nx, ny, rho_mean, amplitude, seed, velocity_amplitude=0.0):
    """Random smooth-free test state (rho, ux, uy) for parity checks."""
    rng = np.random.default_rng(seed)
    rho = rho_mean * (1.0 + amplitude * rng.uniform(-1.0, 1.0, (ny, nx)))
    ux = velocity_amplitude * rng.uniform(-1.0, 1.0, (ny, nx))
    uy = velocity_amplitude * rng.uniform(-1.0, 1.0, (ny, nx))
    return rho, ux, uy


def uneven_sides(count, lo=64, hi=1024, seed=161100907):
    """Square sides drawn log-uniformly in [lo, hi]: round(lo (hi/lo)^U)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, count)
    return np.rint(lo * (hi / lo) ** u).astype(np.int64)


# The paper's parameter sets (Sec. III), with the vdW set of the wetting
# sweep; kappa is chosen per EOS so the scheme stays stable across its
# density range (0.5 for Carnahan-Starling, 0.01 for the cubic EOS whose
# liquid densities are ~20x larger, as the paper's Sec. V run uses).
EOS_SETS = {
    "vdw": dict(a=9 / 49, b=2 / 21, kappa=0.01),
    "cs": dict(a=1.0, b=4.0, kappa=0.5),
    "pr": dict(a=2 / 49, b=2 / 21, kappa=0.01, omega=0.344),
}


def uneven_batch(count=256, seed=161100907, lo=64, hi=1024):
    """Specs of a batch of uneven independent lattices: square sides
    round(lo (hi/lo)^U), EOS uniform over vdW / CS / PR, T_r ~ U[0.6, 0.95],
    tau ~ U[0.6, 1.2], a drop (radius ~ U[0.1, 0.3] side) or a slab with
    probability 1/2 each, all from numpy PCG64 with `seed`."""
    rng = np.random.default_rng(seed)
    sides = np.rint(lo * (hi / lo) ** rng.uniform(0.0, 1.0, count))
    kinds = rng.choice(["vdw", "cs", "pr"], size=count)
    Tr = rng.uniform(0.6, 0.95, count)
    tau = rng.uniform(0.6, 1.2, count)
    geom = rng.choice(["drop", "slab"], size=count)
    rfrac = rng.uniform(0.1, 0.3, count)
    specs = []
    for k in range(count):
        e = dict(EOS_SETS[kinds[k]])
        kappa = e.pop("kappa")
        specs.append(dict(nx=int(sides[k]), ny=int(sides[k]), eos=str(kinds[k]),
                          Tr=float(Tr[k]), tau=float(tau[k]), kappa=kappa,
                          geometry=str(geom[k]), radius_fraction=float(rfrac[k]),
                          **e))
    return specs


def wetting_sweep(count=32, nx=512, ny=256, mu_coex=0.0, mu_span=0.3):
    """Specs of the wall-wetting sweep: vdW (a = 9/49, b = 2/21) at
    T_r = 0.85 on nx x ny lattices with solid rows at the bottom and top, the
    bottom wall's chemical potential evenly spaced over mu_coex +- mu_span/2."""
    e = dict(EOS_SETS["vdw"])
    kappa = e.pop("kappa")
    mus = half_open_linspace(mu_coex - mu_span / 2, mu_coex + mu_span / 2, count)
    return [dict(nx=nx, ny=ny, eos="vdw", Tr=0.85, tau=1.0, kappa=kappa,
                 walls=True, mu_bottom=m, geometry="wall_drop", radius=60.0, **e)
            for m in mus]


def initial_density(spec, rho_v, rho_l):
    """Initial field of one spec of uneven_batch / wetting_sweep."""
    nx, ny = spec["nx"], spec["ny"]
    width = 4.0 if spec["kappa"] >= 0.1 else 2.0
    g = spec.get("geometry", "drop")
    if g == "slab":
        return slab(nx, ny, rho_l, rho_v, width)
    if g == "wall_drop":
        return wall_drop(nx, ny, spec["radius"], rho_l, rho_v, width)
    r = spec.get("radius", spec.get("radius_fraction", 0.25) * min(nx, ny))
    return drop(nx, ny, r, rho_l, rho_v, width)


def ring_radii(lo, hi, count):
    """Evenly spaced radii from lo to hi, rounded to integers."""
    return [int(round(lo + (hi - lo) * k / (count - 1))) for k in range(count)]


def half_open_linspace(lo, hi, count):
    return [lo + (hi - lo) * k / (count - 1) for k in range(count)] \
        if count > 1 else [lo]


__all__ = ["tanh_profile", "slab", "drop", "wall_drop", "spinodal_noise",
           "perturbed", "uneven_sides", "ring_radii", "half_open_linspace",
           "EOS_SETS", "uneven_batch", "wetting_sweep", "initial_density"]
