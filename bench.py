"""Throughput benchmark of the fused chemical-potential LBM step.

Workload: a 4096 x 4096 periodic D2Q9 lattice, Carnahan-Starling EOS (a = 1,
b = 4, R = 1) at T_r = 0.85, kappa = 0.5, tau = 1, spinodal decomposition
from rho_c (1 + 0.01 xi), xi ~ U[-1, 1) with seed 1.  The FP32 state is
0.6 GB, far above the 129 MB L2, so no flush is needed between steps.

One line of JSON on stdout (rank 0).  `value` is MLUPS (million lattice
updates per second) of the FP32 step over all ranks; `roofline` relates the
step kernel's algorithmic bytes (9 populations read and written: 72 B per
update in FP32) to the measured HBM copy bandwidth.  `fp64` repeats the
measurement with FP64 storage and arithmetic.  `e2e` runs the same steps
through the public API from host memory (initial field uploaded, a global
FP64 reduction read back every `check_every` steps, final density read back).
`cpu_baseline` times the CPU oracle on a bounded sample of the same workload.

--impl reference times the CPU oracle (FP64, all host cores) on the same
workload and metric.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SIDE = 4096
EOS_ARGS = dict(eos="cs", a=1.0, b=4.0, R=1.0, Tr=0.85, tau=1.0, kappa=0.5)
BYTES_PER_LU = {"f64": 144, "f32": 72, "f32_offset": 72, "f16_offset": 36}
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1611_00907_gb300/csrc/step_impl.cuh",
                  "paper_1611_00907_gb300/csrc/device_common.cuh",
                  "paper_1611_00907_gb300/csrc/cplbm_internal.h"]


def workload_config(n=N_SIDE, ny=None, walls=False):
    if walls:
        ny = ny or n
        return {"workload": "cs_wall_drop_%dx%d" % (n, ny), "nx": n, "ny": ny,
                "eos": "carnahan-starling a=1 b=4 R=1", "T_over_Tc": 0.85,
                "kappa": 0.5, "tau": 1.0,
                "init": "half disc r = min(nx, ny)/4 on the bottom wall, Maxwell "
                        "densities, tanh width 4; mu_s = mu_coex + 0.01",
                "boundary": "solid rows y=0 and y=ny-1, x periodic",
                "l2": "working set > L2 (no flush)" if n * ny > 4 * 1024 * 1024
                      else "working set in L2"}
    return {"workload": "cs_spinodal_%dx%d" % (n, n), "nx": n, "ny": n,
            "eos": "carnahan-starling a=1 b=4 R=1", "T_over_Tc": 0.85,
            "kappa": 0.5, "tau": 1.0, "init": "rho_c(1+0.01*U[-1,1)), seed 1",
            "boundary": "periodic", "l2": "working set > L2 (no flush)"}


def initial_rho(n=N_SIDE, ny=None, walls=False):
    """The bench lattice: the spinodal workload, or (walls) a drop on the
    bottom wall of an n x ny lattice with solid bottom and top rows."""
    from paper_1611_00907_gb300 import eos_coexistence, eos_critical, inputs
    if walls:
        ny = ny or n
        rv, rl, _ = eos_coexistence("cs", 1.0, 4.0, 1.0, 0.85)
        return inputs.wall_drop(n, ny, min(n, ny) / 4, rl, rv, 4.0)
    _, rc = eos_critical("cs", 1.0, 4.0, 1.0)
    return inputs.spinodal_noise(n, n, rc, 0.01, seed=1)


def wall_mu():
    """Surface chemical potential of the walled bench lattice."""
    from paper_1611_00907_gb300 import eos_coexistence
    return eos_coexistence("cs", 1.0, 4.0, 1.0, 0.85)[2] + 0.01


# ---------------------------------------------------------------------------
# Peaks, traffic record, clocks
# ---------------------------------------------------------------------------
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_code(text):
    """Source text without comments and with whitespace collapsed: what the
    compiler sees of the kernel, so that editing a comment does not void
    counters measured on the code."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel)) as fh:
            h.update(kernel_code(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(precision, n_side=N_SIDE):
    """DRAM bytes per step-kernel launch from the committed ncu summary,
    scaled to the bench lattice, or None when the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "step_kernel_%s.md" % precision)
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_node:\s*([0-9.eE+-]+)", text)
    hm = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not hm or hm.group(1) != kernel_hash():
        return None
    return float(m.group(1)) * n_side * n_side


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU measurement
# ---------------------------------------------------------------------------
def time_steps(sim, steps, warmup):
    """Device time (ms) of `steps` launches of the step kernel, measured with
    CUDA events on the library's stream, after `warmup` steps."""
    import torch
    stream = torch.cuda.current_stream()
    sim.step(warmup)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    sim.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1)


def measure_gpu(precision, steps, warmup, rho, tile=None, no_tma=False,
                force_model=None, walls=False):
    import torch
    from paper_1611_00907_gb300 import Simulation
    ny, nx = rho.shape
    rho_dev = torch.tensor(rho, device="cuda")
    old = os.environ.get("CPLBM_NO_TMA")
    if no_tma:
        os.environ["CPLBM_NO_TMA"] = "1"
    try:
        wall_args = dict(walls=True, mu_bottom=wall_mu()) if walls else {}
        sim = Simulation(nx, ny, precision=precision,
                         rho_ref=0.15 if "offset" in precision else 0.0,
                         **EOS_ARGS, **wall_args)
    finally:
        if no_tma:
            if old is None:
                os.environ.pop("CPLBM_NO_TMA")
            else:
                os.environ["CPLBM_NO_TMA"] = old
    with sim:
        if force_model:
            sim.set_force_model(force_model)
        if tile:
            sim.set_tile(*tile)
        sim.init(rho_dev)
        del rho_dev
        ms = time_steps(sim, steps, warmup)
    return ms


def measure_e2e(precision, steps, warmup, rho, check_every):
    """Same steps through the public API with host buffers."""
    import numpy as np
    import torch
    from paper_1611_00907_gb300 import Simulation
    n = rho.shape[0]
    host_rho = torch.from_numpy(np.ascontiguousarray(rho)).pin_memory()
    out = torch.empty((n, n), dtype=torch.float64).pin_memory()
    sim = Simulation(n, n, precision=precision, **EOS_ARGS)
    with sim:
        sim.init(host_rho.numpy()).step(warmup)
        sim.reduce()
        sim.moments(fields=("rho",), out={"rho": out.numpy()})  # staging before timing
        torch.cuda.synchronize()
        t = time.perf_counter()
        sim.init(host_rho.numpy())
        reads = 0
        for k in range(0, steps, check_every):
            sim.step(min(check_every, steps - k))
            sim.reduce()
            reads += 1
        sim.moments(fields=("rho",), out={"rho": out.numpy()})  # into pinned memory
        dt = time.perf_counter() - t
    field = n * n * 8
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": field / steps,
            "d2h_bytes_per_step": (field + 32 * reads) / steps,
            "seconds": dt, "check_every": check_every}


def batch_specs(which):
    """Specs and initial densities of a batched workload (library
    coexistence densities)."""
    from paper_1611_00907_gb300 import eos_coexistence, inputs
    if which == "uneven":
        specs = inputs.uneven_batch(256)
    else:
        # mu_s over mu_coex +- 0.25: the contact angle from about 0 to 180 deg
        _, _, mc = eos_coexistence("vdw", 9 / 49, 2 / 21, 1.0, 0.85)
        specs = inputs.wetting_sweep(32, mu_coex=mc, mu_span=0.5)
    fields = []
    for sp in specs:
        rv, rl, _ = eos_coexistence(sp["eos"], sp["a"], sp["b"], 1.0, sp["Tr"],
                                    sp.get("omega", 0.344))
        fields.append(inputs.initial_density(sp, rv, rl))
        sp["rho_ref"] = 0.5 * (rv + rl)   # used by the offset storages only
    keep = ("nx", "ny", "walls", "tau", "kappa", "eos", "a", "b", "Tr",
            "omega", "mu_bottom", "rho_ref")
    return [{k: v for k, v in sp.items() if k in keep} for sp in specs], fields


def measure_batch(which, precision, steps, warmup, sequential=True, config=None):
    """One launch per step over every lattice's tiles (graph-replayed),
    and the same lattices stepped one by one, each its own launch."""
    import math
    import torch
    from paper_1611_00907_gb300 import Batch, LbmError, Simulation
    specs, fields = batch_specs(which)
    stream = torch.cuda.Stream()
    nodes = sum(sp["nx"] * sp["ny"] for sp in specs)
    out = {"instances": len(specs), "nodes": nodes, "steps": steps,
           "precision": precision, "unit": "MLUPS"}
    with torch.cuda.stream(stream):
        with Batch(specs, precision=precision,
                   stream=stream.cuda_stream) as b:
            for k, f in enumerate(fields):
                b.init(k, f)
            if config is None:
                out["tile"] = list(b.autotune(6))
            else:  # a fixed configuration (profiling runs)
                b.set_tile(*config[0])
                b.items_per_cta = config[1]
                out["tile"] = list(config[0])
                out["autotuned"] = False
            out["items_per_cta"] = b.items_per_cta
            b.step(warmup)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            b.step(steps)
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            out["value"] = nodes * steps / (ms * 1e-3) / 1e6
            out["ms_per_step"] = ms / steps
            def finite_flags():
                flags = []
                for k in range(len(specs)):
                    try:
                        flags.append(math.isfinite(b.reduce(k)[0]))
                    except LbmError:   # non-finite values on that lattice
                        flags.append(False)
                return flags

            ok = finite_flags()
            out["finite_fraction"] = sum(ok) / len(specs)
            if not all(ok):
                # A sweep drops the lattices its parameters cannot hold:
                # take them out of the launch (the batch has run an even
                # number of steps) and time the ones that stay finite.
                if (warmup + steps) % 2:
                    b.step(1)
                for k, good in enumerate(ok):
                    if not good:
                        b.set_active(k, False)
                live = sum(sp["nx"] * sp["ny"] for sp, good in zip(specs, ok) if good)
                torch.cuda.synchronize()
                t0.record(stream)
                b.step(steps)
                t1.record(stream)
                torch.cuda.synchronize()
                ms2 = t0.elapsed_time(t1)
                still = finite_flags()
                out["finite_only"] = {
                    "value": live * steps / (ms2 * 1e-3) / 1e6,
                    "instances": sum(ok), "nodes": live,
                    "ms_per_step": ms2 / steps,
                    "still_finite": sum(s and g for s, g in zip(still, ok)) / max(1, sum(ok))}
        if sequential:
            sims = []
            for sp, f in zip(specs, fields):
                kw = {k: v for k, v in sp.items() if k not in ("nx", "ny")}
                sim = Simulation(sp["nx"], sp["ny"], precision=precision,
                                 stream=stream.cuda_stream, **kw)
                sims.append(sim.init(f))
            for sim in sims:
                sim.step(warmup)
            torch.cuda.synchronize()
            t0.record(stream)
            for _ in range(steps):
                for sim in sims:
                    sim.step(1)
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            out["sequential_value"] = nodes * steps / (ms * 1e-3) / 1e6
            for sim in sims:
                sim.close()
    return out


def _run_batch(specs, fields, precision, steps):
    """Run a batch `steps` steps from its fields: (device ms, final
    densities, finite flags)."""
    import math
    import torch
    from paper_1611_00907_gb300 import Batch, LbmError
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with Batch(specs, precision=precision, stream=stream.cuda_stream) as b:
            for k, f in enumerate(fields):
                b.init(k, f)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            b.step(steps)
            t1.record(stream)
            torch.cuda.synchronize()
            rhos, finite = [], []
            for k in range(len(specs)):
                try:
                    ok = math.isfinite(b.reduce(k)[0])
                except LbmError:
                    ok = False
                finite.append(ok)
                rhos.append(b.moments(k)["rho"] if ok else None)
    return t0.elapsed_time(t1), rhos, finite


# (T/T_c, tau) of the Laplace study: at T/T_c = 0.7 the CS drop with
# kappa = 0.5 holds only with tau = 1.5 (tau = 1 diverges, in the oracle too)
LAPLACE_T = ((0.7, 1.5), (0.8, 1.0), (0.9, 1.0))


def measure_laplace(steps):
    """Static CS drops (a 1, b 4, kappa 0.5) of radii 16 .. 80 in 256^2
    periodic boxes at three temperatures, one batch per storage (FP32 offset,
    FP64): Laplace pressure jump against 1 / R per temperature, its slope
    against the flat-interface tension sigma of Eq. 1."""
    from paper_1611_00907_gb300 import eos_coexistence, eos_pressure, inputs
    from paper_1611_00907_gb300 import observables as obs
    radii = inputs.ring_radii(16, 80, 8)
    specs, fields = [], []
    for Tr, tau in LAPLACE_T:
        rv, rl, _ = eos_coexistence("cs", 1.0, 4.0, 1.0, Tr)
        for r in radii:
            specs.append(dict(nx=256, ny=256, eos="cs", a=1.0, b=4.0, Tr=Tr,
                              tau=tau, kappa=0.5, rho_ref=0.5 * (rv + rl)))
            fields.append(inputs.drop(256, 256, r, rl, rv, 4.0))
    out = {"lattice": [256, 256], "steps": steps, "radii": radii,
           "eos": "carnahan-starling a=1 b=4", "kappa": 0.5,
           "T_over_Tc_tau": [list(v) for v in LAPLACE_T]}
    for prec in ("f32_offset", "f64"):
        ms, rhos, finite = _run_batch(specs, fields, prec, steps)
        res = {"seconds": ms * 1e-3,
               "mlups": len(specs) * 256 * 256 * steps / (ms * 1e-3) / 1e6,
               "finite_fraction": sum(finite) / len(finite)}
        for j, (Tr, _) in enumerate(LAPLACE_T):
            rv, rl, _ = eos_coexistence("cs", 1.0, 4.0, 1.0, Tr)
            pts, gone = [], []
            for k in range(j * len(radii), (j + 1) * len(radii)):
                if rhos[k] is None:
                    continue
                rin, rout = obs.periodic_drop_bulk(rhos[k])
                if rin - rout < 0.5 * (rl - rv):   # the drop evaporated
                    gone.append(radii[k - j * len(radii)])
                    continue
                dp, R = obs.laplace_jump(
                    rhos[k], lambda v: eos_pressure("cs", 1.0, 4.0, 1.0, Tr, 0.344, v))
                pts.append((1.0 / R, dp))
            fit = obs.line_fit(*zip(*pts)) if len(pts) >= 3 else (None,) * 3
            # the 2-D Laplace law: slope = sigma of square-gradient theory
            sigma = obs.surface_tension(
                lambda v: eos_pressure("cs", 1.0, 4.0, 1.0, Tr, 0.344, v), rv, rl, 0.5)
            res["T%.1f" % Tr] = {"slope": fit[0], "intercept": fit[1],
                                 "r2": fit[2], "sigma": sigma,
                                 "slope_over_sigma": (fit[0] / sigma
                                                      if fit[0] is not None else None),
                                 "inv_R_dp": pts,
                                 "evaporated_initial_radii": gone}
        out[prec] = res
    out["slope_rel_diff_f32_offset_vs_f64"] = {
        key: (abs(out["f32_offset"][key]["slope"] / out["f64"][key]["slope"] - 1)
              if out["f32_offset"][key]["slope"] and out["f64"][key]["slope"]
              else None)
        for key in ("T%.1f" % Tr for Tr, _ in LAPLACE_T)}
    return out


def measure_wetting_angles(steps):
    """The wetting sweep run to `steps` steps in FP32 and in FP16 offset
    storage: contact angle against the wall's surface chemical potential."""
    from paper_1611_00907_gb300 import eos_coexistence
    from paper_1611_00907_gb300 import observables as obs
    specs, fields = batch_specs("wetting")
    _, _, mc = eos_coexistence("vdw", 9 / 49, 2 / 21, 1.0, 0.85)
    out = {"instances": len(specs), "lattice": [specs[0]["nx"], specs[0]["ny"]],
           "steps": steps,
           "mu_s_minus_mu_coex": [sp["mu_bottom"] - mc for sp in specs]}
    for prec in ("f32", "f16_offset"):
        ms, rhos, finite = _run_batch(specs, fields, prec, steps)
        th = [obs.contact_angle(r) if r is not None else float("nan") for r in rhos]
        pts = [(m, t) for m, t in zip(out["mu_s_minus_mu_coex"], th)
               if 0.0 < t < 180.0]
        fit = obs.line_fit(*zip(*pts)) if len(pts) >= 3 else (None,) * 3
        out[prec] = {"seconds": ms * 1e-3, "theta_deg": th,
                     "finite_fraction": sum(finite) / len(finite),
                     "dtheta_dmu_s": fit[0], "theta_at_mu_coex": fit[1],
                     "r2": fit[2]}
    d = [abs(a - b) for a, b in zip(out["f32"]["theta_deg"], out["f16_offset"]["theta_deg"])
         if a == a and b == b]
    out["max_abs_theta_diff_f16_vs_f32_deg"] = max(d) if d else None
    return out


def measure_slab64(steps):
    """The flat CS slab of the plain method (64 x 64 periodic, T/T_c 0.85,
    kappa 0.5, tau 1, tanh width 4 at the Maxwell densities, FP64): bulk
    densities after `steps` steps against the Maxwell construction."""
    from paper_1611_00907_gb300 import eos_coexistence, inputs
    from paper_1611_00907_gb300 import observables as obs
    rv, rl, _ = eos_coexistence("cs", 1.0, 4.0, 1.0, 0.85)
    spec = dict(nx=64, ny=64, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0, kappa=0.5)
    ms, rhos, finite = _run_batch([spec], [inputs.slab(64, 64, rl, rv, 4.0)], "f64", steps)
    l, v = obs.slab_bulk(rhos[0]) if finite[0] else (float("nan"),) * 2
    return {"lattice": [64, 64], "steps": steps, "precision": "f64",
            "rho_l": l, "rho_v": v, "maxwell": [rv, rl],
            "rel_err_vs_maxwell": [v / rv - 1, l / rl - 1]}


# Fig. 2 (Sec. V): the paper's printed (surface chemical potential, contact
# angle) pairs for RKS at T/T_c 0.8, kappa 0.01, tau 1.3
FIG2 = ((-0.23, 30.0), (-0.13, 60.0), (0.0, 105.0), (0.09, 135.0),
        (0.15, 160.0), (0.18, 180.0))


def measure_fig2(steps):
    """Fig. 2 at the paper's size (500 x 200, walls, drop radius 50 on the
    bottom wall), one FP64 batch of the six surface chemical potentials:
    measured contact angle beside the printed one."""
    from paper_1611_00907_gb300 import eos_coexistence, inputs
    from paper_1611_00907_gb300 import observables as obs
    a, b = 2 / 49, 2 / 21
    rv, rl, _ = eos_coexistence("rks", a, b, 1.0, 0.8, 0.344)
    specs = [dict(nx=500, ny=200, walls=True, eos="rks", a=a, b=b, Tr=0.8,
                  omega=0.344, tau=1.3, kappa=0.01, mu_bottom=cp) for cp, _ in FIG2]
    fields = [inputs.wall_drop(500, 200, 50, rl, rv, 2.0) for _ in FIG2]
    ms, rhos, finite = _run_batch(specs, fields, "f64", steps)
    rows = []
    for (cp, printed), rho in zip(FIG2, rhos):
        th = obs.contact_angle(rho) if rho is not None else float("nan")
        rows.append({"mu_s": cp, "theta_printed": printed, "theta": th,
                     "diff": th - printed})
    return {"lattice": [500, 200], "steps": steps, "precision": "f64",
            "seconds": ms * 1e-3, "rows": rows}


# Fig. 1: coexistence curves of flat interfaces against the Maxwell
# construction (Sec. III, V): (label, EOS, a, b, omega, kappa, tau)
FIG1_EOS = (("pr_water", "pr", 2 / 49, 2 / 21, 0.344, 0.01, 1.3),
            ("pr_methane", "pr", 2 / 49, 2 / 21, 0.011, 0.01, 1.3),
            ("rks_water", "rks", 2 / 49, 2 / 21, 0.344, 0.01, 1.3),
            ("cs", "cs", 1.0, 4.0, 0.344, 0.5, 1.0))
FIG1_TR = (0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95)


def measure_coexistence_curves(steps):
    """Flat liquid slabs (32 x 256 periodic, FP64) of every Fig. 1 EOS over
    a range of temperatures, one batch: bulk densities against the Maxwell
    construction."""
    from paper_1611_00907_gb300 import eos_coexistence, inputs
    from paper_1611_00907_gb300 import observables as obs
    specs, fields, meta = [], [], []
    for label, kind, a, b, om, kappa, tau in FIG1_EOS:
        for Tr in FIG1_TR:
            rv, rl, _ = eos_coexistence(kind, a, b, 1.0, Tr, om)
            specs.append(dict(nx=32, ny=256, eos=kind, a=a, b=b, Tr=Tr,
                              omega=om, kappa=kappa, tau=tau))
            fields.append(inputs.slab(32, 256, rl, rv, 4.0 if kappa > 0.1 else 2.0))
            meta.append((label, Tr, rv, rl))
    ms, rhos, finite = _run_batch(specs, fields, "f64", steps)
    out = {"lattice": [32, 256], "steps": steps, "precision": "f64",
           "seconds": ms * 1e-3, "finite_fraction": sum(finite) / len(finite)}
    for (label, Tr, rv, rl), rho in zip(meta, rhos):
        row = {"T_over_Tc": Tr, "maxwell": [rv, rl]}
        if rho is not None:
            l, v = obs.slab_bulk(rho)
            row.update(sim=[v, l], rel_err=[v / rv - 1, l / rl - 1])
        out.setdefault(label, []).append(row)
    return out


def measure_warmstart(full):
    """Sweep time-to-converge, learned warm start against the plain
    half-disc start.  Small: 64 wall drops of 256x128 after training on
    1024 runs of 128x64; full: 256 drops of 512x256 after 4096 runs."""
    import torch
    from paper_1611_00907_gb300 import warmstart as ws
    ntrain, neval, nx, ny, max_steps = ((4096, 256, 512, 256, 40000) if full
                                        else (1024, 64, 256, 128, 20000))
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        cases, X, Y = ws.build_dataset(ntrain, 128, 64, 6000, seed=1,
                                       stream=stream)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    model = ws.Model(X, Y, iters=3000, lr=2e-3)
    t_train = time.perf_counter() - t0
    try:
        with torch.cuda.stream(stream):
            # convergence: the drop has settled (contact angle and bulk
            # densities steady between checks), read every 500 (250) steps
            r = ws.compare(model, ws.sample_cases(neval, seed=99), nx, ny,
                           max_steps, check_every=500 if full else 250,
                           stream=stream, settle=ws.SETTLE)
    finally:
        model.close()
    r.update(training_runs=ntrain, training_kept=len(cases),
             training_lattice=[128, 64], training_steps=6000,
             dataset_s=round(t_data, 2), train_s=round(t_train, 2),
             final_loss=model.loss)
    return r


def cpu_baseline(budget_s=15.0):
    """The oracle as it stands (FP64 C) on a 512 x 512 sample of the same
    workload, all host cores."""
    import oracle
    from oracle import thermo
    from paper_1611_00907_gb300 import inputs
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = 512
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    _, rc = thermo.critical_point("cs", 1.0, 4.0)
    L = oracle.Lattice(n, n, e, 1.0, 0.5)
    L.init_equilibrium(inputs.spinodal_noise(n, n, rc, 0.01, seed=1))
    L.step(2)
    steps, t = 0, time.perf_counter()
    while time.perf_counter() - t < budget_s:
        L.step(5)
        steps += 5
    dt = time.perf_counter() - t
    # the same oracle on one core, a shorter sample
    oracle.set_threads(1)
    m = 128
    L1 = oracle.Lattice(m, m, e, 1.0, 0.5)
    L1.init_equilibrium(inputs.spinodal_noise(m, m, rc, 0.01, seed=1))
    s1, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < budget_s / 5:
        L1.step(5)
        s1 += 5
    dt1 = time.perf_counter() - t1
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS",
            "cores": cores, "kind": "oracle",
            "sample": "%dx%d CS spinodal, %d steps, FP64 C oracle" % (
                n, n, steps),
            "single_core_value": m * m * s1 / dt1 / 1e6,
            "single_core_sample": "%dx%d, %d steps, 1 thread" % (m, m, s1)}


def roofline(precision, ms_per_step, n_nodes, n_side=N_SIDE, walls=False):
    peak, src = hbm_peak()
    achieved = BYTES_PER_LU[precision] * n_nodes / (ms_per_step * 1e-3) / 1e9
    # the recorded counters are of the periodic spinodal workload
    traffic = None if walls else recorded_traffic(precision, n_side)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "peak_source": src,
            "bytes_per_update": BYTES_PER_LU[precision]}


# GB300's FP64 pipe: 2 thread instructions per SM per clock (ncu's sustained
# peak of the pipe, 304 per clock over the GPU) x 152 SMs x 2.07 GHz.
FP64_PIPE_GINST = 2 * 152 * 2.07


def recorded_fp64_ops():
    """FP64-pipe thread instructions per lattice update from the committed
    ncu summary of the FP64 step, or None when the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "step_kernel_f64.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"fp64_pipe_inst_per_node:\s*([0-9.eE+-]+)", text)
    hm = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not hm or hm.group(1) != kernel_hash():
        return None
    return float(m.group(1))


def roofline_fp64(ms_per_step, n_nodes, n_side=N_SIDE):
    """The FP64 step is bound by the FP64 pipe: its instructions per update
    (ncu) over the launch time against the pipe's peak; the HBM figures
    beside it for reference."""
    ops = recorded_fp64_ops()
    hbm = roofline("f64", ms_per_step, n_nodes, n_side)
    if ops is None:
        return dict(hbm, bound="alu", achieved=None,
                    peak=round(FP64_PIPE_GINST, 1), unit="G FP64-pipe inst/s",
                    frac=None, peak_source="derived", hbm_frac=hbm["frac"])
    achieved = ops * n_nodes / (ms_per_step * 1e-3) / 1e9
    return {"bound": "alu", "achieved": round(achieved, 1),
            "peak": round(FP64_PIPE_GINST, 1), "unit": "G FP64-pipe inst/s",
            "frac": round(achieved / FP64_PIPE_GINST, 4),
            "fp64_inst_per_update": ops, "peak_source": "derived",
            "traffic": hbm["traffic"], "hbm_achieved_gbs": hbm["achieved"],
            "hbm_frac": hbm["frac"]}


# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    return rank, world


def max_over_ranks(value, world):
    """Largest value over all ranks (the job's wall time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands (FP64 C, all host cores),
    W untimed and K timed steps on a sample of the bench workload, the
    sample's side halved from 512 until the K steps fit in about 90 s.
    Under torchrun only rank 0 runs it."""
    if rank != 0:
        return 0
    import oracle
    from oracle import thermo
    from paper_1611_00907_gb300 import inputs
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    _, rc = thermo.critical_point("cs", 1.0, 4.0)
    n = 512
    while True:
        L = oracle.Lattice(n, n, e, 1.0, 0.5)
        L.init_equilibrium(inputs.spinodal_noise(n, n, rc, 0.01, seed=1))
        t = time.perf_counter()
        L.step(args.warmup)
        rate = n * n * args.warmup / max(time.perf_counter() - t, 1e-9)
        if n <= 64 or args.steps * n * n / rate <= 90.0:
            break
        n //= 2
    t = time.perf_counter()
    L.step(args.steps)
    dt = time.perf_counter() - t
    oracle.set_threads(1)
    value = n * n * args.steps / dt / 1e6
    base = {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%dx%d CS spinodal (T_r 0.85, kappa 0.5, tau 1), %d "
                      "steps after %d warm-up, FP64 C oracle" % (
                          n, n, args.steps, args.warmup)}
    line = {"impl": "reference", "metric": "MLUPS", "value": value,
            "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "cpu_baseline": base,
            "e2e": {"value": value, "unit": "MLUPS",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--precision", default="f32",
                    choices=["f32", "f32_offset", "f16_offset", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=200)
    ap.add_argument("--fp16-steps", type=int, default=500,
                    help="steps of the FP16-storage leg (0: skip)")
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=N_SIDE,
                    help="lattice side (profiling runs use smaller cases)")
    ap.add_argument("--walls", action="store_true",
                    help="time a walled lattice (a drop on the bottom wall) "
                         "instead of the spinodal workload")
    ap.add_argument("--ny", type=int, default=None,
                    help="lattice height with --walls, solid rows included "
                         "(default: --n)")
    ap.add_argument("--batches", default="uneven,wetting,wetting_f16",
                    help="batched workloads to time (comma list)")
    ap.add_argument("--tile", default=None,
                    help="step tile shape TXxTY (default: the library's)")
    ap.add_argument("--batch-config", default=None,
                    help="TXxTY:SCHEDULE for the batched legs instead of "
                         "the autotuner (profiling runs), e.g. 64x32:0")
    ap.add_argument("--batch-steps", type=int, default=100,
                    help="steps of the batched workloads (0: skip them)")
    ap.add_argument("--pt-steps", type=int, default=200,
                    help="steps of the pressure-tensor comparison (0: skip)")
    ap.add_argument("--warmstart", default="small",
                    choices=["small", "full", "off"],
                    help="learned warm-start sweep (full: 256 x 512x256)")
    ap.add_argument("--physics-steps", type=int, default=20000,
                    help="steps of the Laplace study; the wetting sweep runs "
                         "1.5x as many (0: skip both)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.walls:
        # the end-to-end and pressure-tensor legs are defined on the periodic
        # spinodal workload
        args.no_e2e, args.pt_steps = True, 0
    rank, world = dist_setup()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    import __graft_entry__
    __graft_entry__.build()
    rho = initial_rho(args.n, args.ny, args.walls)
    n_nodes = rho.size
    tile = tuple(int(v) for v in args.tile.split("x")) if args.tile else None

    barrier(world)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        ms = measure_gpu(args.precision, args.steps, args.warmup, rho, tile,
                         walls=args.walls)
    ms = max_over_ranks(ms, world)
    ms_step = ms / args.steps
    value = world * n_nodes * args.steps / (ms * 1e-3) / 1e6

    fp64 = None
    if args.fp64_steps > 0:
        fp64_ms = measure_gpu("f64", args.fp64_steps, 3, rho,
                              walls=args.walls) / args.fp64_steps
        fp64_ms = max_over_ranks(fp64_ms, world)
        fp64 = {"value": world * n_nodes / (fp64_ms * 1e-3) / 1e6,
                "unit": "MLUPS", "ms_per_step": fp64_ms,
                "steps": args.fp64_steps,
                "roofline": roofline_fp64(fp64_ms, n_nodes, args.n)}

    # the FP16-storage variant (FP32 arithmetic, 36 B per update) on the same
    # lattice
    fp16 = None
    if args.fp16_steps > 0:
        f16_ms = measure_gpu("f16_offset", args.fp16_steps, 3, rho,
                             walls=args.walls) / args.fp16_steps
        f16_ms = max_over_ranks(f16_ms, world)
        fp16 = {"value": world * n_nodes / (f16_ms * 1e-3) / 1e6,
                "unit": "MLUPS", "ms_per_step": f16_ms,
                "steps": args.fp16_steps,
                "roofline": roofline("f16_offset", f16_ms, n_nodes, args.n, args.walls)}

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args.precision, args.steps, args.warmup, rho,
                          args.check_every)
        e2e["value"] = world * e2e["value"]

    # The paper's efficiency claim (Sec. II, VI): the chemical-potential force
    # against the pressure-tensor force it replaces, same lattice and tile,
    # on the TMA tile paths the product runs and on the general paths: FP32
    # at the default tile (two nodes per lane) and at 32 x 32, FP64 at 32 x 16.
    pt = None
    if args.pt_steps > 0:
        pt = {}
        for key, prec, tile in (("f32", "f32", (64, 16)), ("f32_32x32", "f32", (32, 32)),
                                ("f64", "f64", (32, 16))):
            k = args.pt_steps if prec == "f32" else max(2, args.pt_steps // 10)
            pt[key] = {"tile": list(tile), "steps": k}
            for path, no_tma in (("tma", False), ("general", True)):
                cp_ms = measure_gpu(prec, k, 3, rho, tile, no_tma=no_tma) / k
                pt_ms = measure_gpu(prec, k, 3, rho, tile, no_tma=no_tma,
                                    force_model="pressure_tensor") / k
                pt[key][path] = {
                    "chemical_potential_mlups": n_nodes / (cp_ms * 1e-3) / 1e6,
                    "pressure_tensor_mlups": n_nodes / (pt_ms * 1e-3) / 1e6,
                    "speedup": pt_ms / cp_ms}

    batches = {}
    legs = set(args.batches.split(",")) if args.batch_steps > 0 else set()
    bcfg = None
    if args.batch_config:
        shape, sched = args.batch_config.split(":")
        bcfg = (tuple(int(v) for v in shape.split("x")), int(sched))
    if "uneven" in legs:
        batches["batch_uneven"] = measure_batch("uneven", "f32",
                                                args.batch_steps, 4, config=bcfg)
    if "wetting" in legs:
        batches["batch_wetting"] = measure_batch("wetting", "f32",
                                                 args.batch_steps, 4, config=bcfg)
    if "wetting_f16" in legs:
        batches["batch_wetting_f16"] = measure_batch(
            "wetting", "f16_offset", args.batch_steps, 4, sequential=False,
            config=bcfg)

    warm = None
    if args.warmstart != "off" and rank == 0:
        warm = measure_warmstart(args.warmstart == "full")

    physics = {}
    if args.physics_steps > 0 and rank == 0:
        physics["laplace"] = measure_laplace(args.physics_steps)
        physics["wetting_angles"] = measure_wetting_angles(
            3 * args.physics_steps // 2)
        physics["coexistence_curves"] = measure_coexistence_curves(
            args.physics_steps)
        physics["slab_64"] = measure_slab64(args.physics_steps // 4)
        physics["fig2_contact_angles"] = measure_fig2(args.physics_steps)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    if rank == 0:
        line = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic",
                "config": workload_config(args.n, args.ny, args.walls),
                "roofline": roofline(args.precision, ms_step, n_nodes, args.n,
                                     args.walls),
                "fp64": fp64, "fp16_offset": fp16, "e2e": e2e,
                "cpu_baseline": base,
                "gpu_launches": args.steps, "clocks": clocks.summary()}
        line.update(batches)
        if pt:
            line["pressure_tensor_vs_chemical_potential"] = pt
        if warm:
            line["warm_start"] = warm
        line.update(physics)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
