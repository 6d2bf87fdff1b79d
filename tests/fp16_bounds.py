"""Error bounds of the FP16-offset storage against the FP64 oracle, from the
half-precision unit roundoff u (round to nearest).

Every step stores each moving population once, as g_i = f_i - w_i rho_ref
in half: an error of at most u |g_i| <= u w_i A, A = max |f_i / w_i -
rho_ref| over the run.  A node's density sums eight such values, sum w_i =
5/9: one step adds at most (5/9) u A.  The roundings of successive steps are
independent, and density and momentum are conserved, so each step's error
spreads over the lattice (over ~t nodes after t steps) instead of piling up
at one node: a node collects sum_t 1/t ~ 1 + ln n of one step's variance,
K(n) = sqrt(1 + ln n), and
    d_rho <= (5/9) u A K(n).
mu = psi'(rho) - kappa lap(rho) (Eq. 8): the spread error passes through
psi'', the last step's fresh error through the Laplacian's stencil, whose
weights sum to 40/6 in magnitude:
    d_mu <= max|psi''| d_rho + kappa (40/6) (5/9) u A.
v = (sum_i f_i e_i)/rho + F/(2 rho), F = -rho grad mu + c_s^2 grad rho
(Eq. 12, Sec. II): the momentum takes sum_i w_i |e_ix| u A = u A / 3 per
step, spread as the density's; grad mu / 2 takes d_mu; c_s^2 grad rho /
(2 rho) takes d_rho / (3 rho):
    d_v <= (u A K(n) / 3 + d_rho / 3) / rho_min + d_mu.
The tests allow twice these, for the propagation through collision and
streaming.  The velocity bound grows with A / rho_min: with rho_ref between
the phases, a vapour node stores offsets of half the density range, large
against its own density, so for density ratios near 30 (the RKS and PR
lattices here) FP16-offset storage resolves vapour velocities only to a
sizeable fraction of the largest velocity, and the bound says so."""
import numpy as np

import oracle
from oracle import thermo

EPS_HALF = 2.0 ** -11


def run_with_bounds(ref, rho, steps, rho_ref, eos, kappa):
    """Step the oracle lattice `ref` from the equilibrium of `rho` for
    `steps` steps; returns its moments and the bound of each field."""
    ref.init_equilibrium(rho)
    A = 0.0
    for n in range(steps + 1):
        if n:
            ref.step(1)
        A = max(A, float(np.abs(ref.f[1:] / oracle.W[1:, None, None] - rho_ref).max()))
    want = ref.moments()
    fluid = want["rho"][ref.fluid_rows()]
    grid = np.linspace(fluid.min(), fluid.max(), 2001)
    psi2 = np.abs(thermo.dp0_drho(eos.kind, eos.a, eos.b, eos.R, eos.T, eos.alpha,
                                  grid) / grid).max()
    K = np.sqrt(1 + np.log(steps))
    d_rho = (5 / 9) * EPS_HALF * A * K
    d_mu = psi2 * d_rho + kappa * (40 / 6) * (5 / 9) * EPS_HALF * A
    d_v = (EPS_HALF * A * K / 3 + d_rho / 3) / fluid.min() + d_mu
    return want, {"rho": d_rho, "mu": d_mu, "vx": d_v, "vy": d_v}


def check(got, want, bounds, label="", meaningful=("rho", "mu", "vx", "vy")):
    """Every field within twice its bound, and the bounds of the fields in
    `meaningful` well below the field's own size (so that the check means
    something there)."""
    for key, bound in bounds.items():
        err = np.abs(got[key] - want[key]).max()
        assert err <= 2 * bound, (label, key, err, bound)
        if key in meaningful:
            assert 2 * bound < 0.2 * np.abs(want[key]).max(), (label, key, bound)
