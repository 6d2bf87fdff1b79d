"""Learned warm start for wall-droplet runs.

A BF16 MLP (mlp.py) maps a case's parameters - EOS (one-hot vdW / CS /
PR), T/T_c, kappa, tau, the wall's surface chemical potential (relative to
coexistence) and the drop's area fraction - to its converged observables:
liquid and vapour densities, interface width and contact angle.  It is
trained on converged runs of the method itself (batched lattices), and a
new case then starts from a circular-cap drop with the predicted angle,
densities and width instead of the plain half-disc at the Maxwell
densities.  The plain cold start stays the fallback and the measure of
the warm start's error: both are run to convergence and their
observables compared.
"""
import json
import math

import numpy as np

from . import Batch, eos_coexistence, eos_critical, inputs
from . import observables as obs

KINDS = ("vdw", "cs", "pr")
# parameter ranges kept inside the scheme's stable region
RANGES = {
    "vdw": dict(Tr=(0.78, 0.95), kappa=(0.008, 0.016), tau=(0.9, 1.3), dmu=0.15),
    "cs": dict(Tr=(0.78, 0.95), kappa=(0.4, 0.6), tau=(0.9, 1.3), dmu=0.05),
    "pr": dict(Tr=(0.8, 0.95), kappa=(0.008, 0.016), tau=(1.0, 1.3), dmu=0.15),
}
NFEAT, NTARG = 8, 4


def sample_cases(n, seed):
    """n random wall-droplet cases: EOS, T_r, kappa, tau, mu_s - mu_coex,
    drop area fraction."""
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        kind = KINDS[rng.integers(3)]
        r = RANGES[kind]
        e = dict(inputs.EOS_SETS[kind])
        e.pop("kappa")
        Tr = rng.uniform(*r["Tr"])
        rv, rl, mc = eos_coexistence(kind, e["a"], e["b"], 1.0, Tr,
                                     e.get("omega", 0.344))
        dmu = rng.uniform(-r["dmu"], r["dmu"])
        cases.append(dict(eos=kind, Tr=Tr, kappa=rng.uniform(*r["kappa"]),
                          tau=rng.uniform(*r["tau"]), dmu=dmu,
                          mu_bottom=mc + dmu, area=rng.uniform(0.05, 0.15),
                          rho_v=rv, rho_l=rl, **e))
    return cases


def features(cases):
    X = np.zeros((len(cases), NFEAT), dtype=np.float32)
    for i, c in enumerate(cases):
        X[i, KINDS.index(c["eos"])] = 1.0
        X[i, 3:] = (c["Tr"], math.log(c["kappa"]), c["tau"],
                    c["dmu"] / RANGES[c["eos"]]["dmu"], c["area"])
    return X


def targets(cases, measured):
    """Observables scaled to O(1): rho_l / rho_c, log(rho_v / rho_c),
    width, theta / 180."""
    Y = np.zeros((len(cases), NTARG), dtype=np.float32)
    for i, (c, m) in enumerate(zip(cases, measured)):
        _, rc = eos_critical(c["eos"], c["a"], c["b"], 1.0)
        Y[i] = (m["rho_l"] / rc, math.log(max(m["rho_v"], 1e-12) / rc),
                m["width"], m["theta"] / 180.0)
    return Y


def untarget(case, y):
    _, rc = eos_critical(case["eos"], case["a"], case["b"], 1.0)
    return dict(rho_l=float(y[0]) * rc, rho_v=math.exp(float(y[1])) * rc,
                width=float(y[2]), theta=float(y[3]) * 180.0)


def _spec(case, nx, ny):
    return dict(nx=nx, ny=ny, walls=True, tau=case["tau"], kappa=case["kappa"],
                eos=case["eos"], a=case["a"], b=case["b"], Tr=case["Tr"],
                omega=case.get("omega", 0.344), mu_bottom=case["mu_bottom"])


def cold_field(case, nx, ny):
    """The plain start: a half disc of the requested area at the Maxwell
    densities, on the wall plane."""
    area = case["area"] * nx * (ny - 2)
    r = math.sqrt(2 * area / math.pi)
    width = 4.0 if case["kappa"] > 0.1 else 2.0
    return inputs.wall_drop(nx, ny, r, case["rho_l"], case["rho_v"], width)


def warm_field(case, pred, nx, ny, mass=None):
    """A circular cap meeting the wall at the predicted angle, with the
    predicted bulk densities and interface width: of the case's area, or,
    with `mass`, of the area that gives the fluid rows that total density
    (mass_matched_area)."""
    th = math.radians(min(max(pred["theta"], 5.0), 175.0))
    if mass is not None:
        case = dict(case, area=mass_matched_area(case, pred, nx, ny, mass))
    area = case["area"] * nx * (ny - 2)
    R = math.sqrt(area / (th - math.sin(th) * math.cos(th)))
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cx, cy = nx / 2.0 - 0.5, 0.5 - R * math.cos(th)   # centre below/above wall
    d = R - np.hypot(xx - cx, yy - cy)   # row 0 (solid) is ignored
    rl = pred["rho_l"] if pred["rho_l"] > pred["rho_v"] else case["rho_l"]
    rv = max(pred["rho_v"], 1e-6)
    W = min(max(pred["width"], 1.0), 12.0)
    return inputs.tanh_profile(d, rl, rv, W)


def fluid_mass(rho):
    """Total density of the fluid rows (rows 0 and ny - 1 are solid)."""
    return float(np.asarray(rho)[1:-1].sum())


def mass_matched_area(case, pred, nx, ny, mass, iters=4):
    """Area fraction of the warm cap whose fluid rows hold `mass` (the cold
    start's): the same system, with the same total mass, as the cold start,
    so that both relax to one equilibrium.  Mass grows with the cap's area at
    the rate rho_l - rho_v per node; a few corrections settle the tanh
    profile's share."""
    rl = pred["rho_l"] if pred["rho_l"] > pred["rho_v"] else case["rho_l"]
    rv = max(pred["rho_v"], 1e-6)
    c = dict(case)
    for _ in range(iters):
        m = fluid_mass(warm_field(c, pred, nx, ny))
        c["area"] += (mass - m) / ((rl - rv) * nx * (ny - 2))
    return c["area"]


# A settled drop (the convergence test of the sweep comparison): between two
# checks its contact angle moves by less than theta_deg and its bulk
# densities by less than the relative rho_l, rho_v, `repeats` checks in a
# row.  A film over the wall (0 degrees) or a drop that left it (180) counts
# on its densities alone.
SETTLE = dict(theta_deg=0.05, rho_l=1e-5, rho_v=1e-4, repeats=2)


def _settled(prev, cur, settle):
    if prev is None:
        return False
    th0, th1 = prev["theta"], cur["theta"]
    if np.isfinite(th0) and np.isfinite(th1):
        if abs(th1 - th0) >= settle["theta_deg"]:
            return False
    elif np.isfinite(th0) != np.isfinite(th1):
        return False
    return (abs(cur["rho_l"] / prev["rho_l"] - 1) < settle["rho_l"] and
            abs(cur["rho_v"] / prev["rho_v"] - 1) < settle["rho_v"])


def run_batch(cases, fields, nx, ny, max_steps, check_every=200, tol=1e-6,
              precision="f32", stream=None, settle=None):
    """Run every case from its field until it has converged, or max_steps;
    a case that has converged (or gone non-finite) leaves the batched launch.
    Convergence: with settle None, max |rho change| over check_every steps
    (even) below tol * rho_l (the library's FP64 reduction); with a settle
    dict (SETTLE), the drop has settled: its contact angle and bulk
    densities, measured on the density read back every check_every steps,
    stop moving (_settled).  Returns the per-case convergence step (max_steps
    if never), the final fields, the device milliseconds of stepping until
    the last case converged (the host's checks between the blocks of steps
    not included), and the steps run."""
    import torch
    specs = [_spec(c, nx, ny) for c in cases]
    conv = np.full(len(cases), max_steps, dtype=np.int64)
    done = np.zeros(len(cases), dtype=bool)
    prev = [None] * len(cases)
    calm = np.zeros(len(cases), dtype=np.int64)
    steps = 0
    ms = 0.0
    st = stream if stream else torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Batch(specs, precision=precision,
               stream=stream.cuda_stream if stream else None) as b:
        for k, f in enumerate(fields):
            b.init(k, f)
        for k in range(len(cases)):
            b.reduce(k)
        torch.cuda.synchronize()
        while steps < max_steps and not done.all():
            ev0.record(st)
            b.step(check_every)
            ev1.record(st)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            steps += check_every
            for k in range(len(cases)):
                if done[k]:
                    continue
                try:
                    d = b.reduce(k)[3]
                except Exception:
                    done[k] = True            # non-finite: never converges
                    b.set_active(k, False)
                    continue
                if settle is None:
                    ok = d < tol * cases[k]["rho_l"]
                else:
                    m = obs.measure(b.moments(k, fields=("rho",))["rho"])
                    calm[k] = calm[k] + 1 if _settled(prev[k], m, settle) else 0
                    prev[k] = m
                    ok = calm[k] >= settle["repeats"]
                if ok:
                    done[k] = True
                    conv[k] = steps
                    b.set_active(k, False)
        final = [b.moments(k, fields=("rho",))["rho"] for k in range(len(cases))]
    return conv, final, ms, steps


def build_dataset(n, nx, ny, steps, seed, stream=None):
    """Converged runs of n random cases from the cold start: features and
    targets of the finite ones with a measurable angle."""
    cases = sample_cases(n, seed)
    fields = [cold_field(c, nx, ny) for c in cases]
    _, final, _, _ = run_batch(cases, fields, nx, ny, steps, check_every=steps,
                               tol=0.0, stream=stream)
    keep, meas = [], []
    for c, rho in zip(cases, final):
        if not np.isfinite(rho).all():
            continue
        m = obs.measure(rho)
        # caps only: no film (0) and no drop that left the wall (180)
        if all(np.isfinite(v) for v in m.values()) and 0.0 < m["theta"] < 179.0:
            keep.append(c)
            meas.append(m)
    return keep, features(keep), targets(keep, meas)


class Model:
    """The trained network with its input / output standardisation."""

    def __init__(self, X, Y, iters=3000, lr=2e-3, seed=0):
        import torch
        from .mlp import Mlp
        self.xm, self.xs = X.mean(0), X.std(0) + 1e-6
        self.ym, self.ys = Y.mean(0), Y.std(0) + 1e-6
        Xd = torch.tensor((X - self.xm) / self.xs, device="cuda")
        Yd = torch.tensor((Y - self.ym) / self.ys, device="cuda")
        self.net = Mlp(seed=seed)
        self.loss = self.net.train(Xd, Yd, iters, lr)

    def predict(self, cases):
        import torch
        X = (features(cases) - self.xm) / self.xs
        Y = self.net.predict(torch.tensor(X, device="cuda"), NTARG).cpu().numpy()
        Y = Y * self.ys + self.ym
        return [untarget(c, y) for c, y in zip(cases, Y)]

    def close(self):
        self.net.close()


def _stat(values, fn):
    return float(fn(np.asarray(values))) if len(values) else float("nan")


def compare(model, cases, nx, ny, max_steps, check_every=200, tol=1e-6,
            stream=None, settle=None):
    """Cold and warm starts of the same cases run to convergence (run_batch's
    test, by tol or by settle): step counts, device time of stepping to the
    last converged case, and, over the cases both starts converged on, the
    warm start's observable errors against the cold start's result."""
    preds = model.predict(cases)
    cold = run_batch(cases, [cold_field(c, nx, ny) for c in cases], nx, ny,
                     max_steps, check_every, tol, stream=stream, settle=settle)
    # the warm cap holds the cold start's mass: the same system
    warm = run_batch(cases, [warm_field(c, p, nx, ny, mass=fluid_mass(cold_field(c, nx, ny)))
                             for c, p in zip(cases, preds)], nx, ny, max_steps,
                     check_every, tol, stream=stream, settle=settle)
    both = (cold[0] < max_steps) & (warm[0] < max_steps)
    err = {"rho_l": [], "rho_v": [], "theta": []}
    for k, (rc, rw) in enumerate(zip(cold[1], warm[1])):
        if not both[k]:
            continue
        mc, mw = obs.measure(rc), obs.measure(rw)
        err["rho_l"].append(abs(mw["rho_l"] - mc["rho_l"]) / mc["rho_l"])
        err["rho_v"].append(abs(mw["rho_v"] - mc["rho_v"]) / mc["rho_v"])
        err["theta"].append(abs(mw["theta"] - mc["theta"]))
    pred_err = []
    for p, rc in zip(preds, cold[1]):
        if np.isfinite(rc).all():
            t = obs.measure(rc)["theta"]
            if np.isfinite(t):
                pred_err.append(abs(p["theta"] - t))
    return dict(
        cases=len(cases), nx=nx, ny=ny, check_every=check_every,
        convergence=("settled drop: " + json.dumps(settle)) if settle else
        "max |rho change| over check_every steps < %g rho_l" % tol,
        max_steps=max_steps,
        capped_cold=int((cold[0] >= max_steps).sum()),
        capped_warm=int((warm[0] >= max_steps).sum()),
        cold_steps_mean=float(cold[0].mean()), warm_steps_mean=float(warm[0].mean()),
        both_converged=int(both.sum()),
        cold_steps_median_both=float(np.median(cold[0][both])) if both.any() else None,
        warm_steps_median_both=float(np.median(warm[0][both])) if both.any() else None,
        step_ratio_median_both=float(np.median(warm[0][both] / cold[0][both]))
        if both.any() else None,
        # lattice-steps to convergence summed over the cases both starts
        # converged on: the work the warm start saves there
        cold_steps_sum_both=int(cold[0][both].sum()),
        warm_steps_sum_both=int(warm[0][both].sum()),
        cold_ms=cold[2], warm_ms=warm[2],
        cold_converged=float((cold[0] < max_steps).mean()),
        warm_converged=float((warm[0] < max_steps).mean()),
        max_rel_err_rho_l=_stat(err["rho_l"], np.max),
        max_rel_err_rho_v=_stat(err["rho_v"], np.max),
        max_abs_err_theta_deg=_stat(err["theta"], np.max),
        median_rel_err_rho_l=_stat(err["rho_l"], np.median),
        median_rel_err_rho_v=_stat(err["rho_v"], np.median),
        median_abs_err_theta_deg=_stat(err["theta"], np.median),
        p90_rel_err_rho_v=_stat(err["rho_v"], lambda v: np.percentile(v, 90)),
        p90_abs_err_theta_deg=_stat(err["theta"], lambda v: np.percentile(v, 90)),
        mlp_theta_err_deg_median=float(np.median(pred_err)) if pred_err else None)
