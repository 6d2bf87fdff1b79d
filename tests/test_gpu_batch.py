"""Batched lattices (one launch per step over every lattice's
tiles, blocks of steps from a CUDA graph) against the FP64 oracle and the
single-lattice path, lattice by lattice."""
import numpy as np
import pytest

import oracle
from oracle import thermo
from fp16_bounds import check, run_with_bounds
from paper_1611_00907_gb300 import Batch, LbmError, Simulation, inputs

pytestmark = pytest.mark.gpu

# heterogeneous lattices: sizes with ragged tiles, walls, every EOS, taus
SPECS = [
    dict(nx=70, ny=21, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0, kappa=0.5),
    dict(nx=131, ny=100, eos="cs", a=1.0, b=4.0, Tr=0.9, tau=0.9, kappa=0.5,
         walls=True, mu_delta=0.02),
    dict(nx=97, ny=40, eos="rks", a=2 / 49, b=2 / 21, Tr=0.8, tau=1.3,
         kappa=0.01, walls=True, mu_delta=-0.05),
    dict(nx=64, ny=64, eos="pr", a=2 / 49, b=2 / 21, Tr=0.85, tau=1.3,
         kappa=0.01),
    dict(nx=230, ny=140, eos="vdw", a=9 / 49, b=2 / 21, Tr=0.85, tau=1.0,
         kappa=0.01, walls=True),
    # 3 x 3 tiles of 32 x 32: every tile but the centre wraps around an edge
    dict(nx=96, ny=96, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0, kappa=0.5),
]


def _instances(specs=None):
    out = []
    for s in (SPECS if specs is None else specs):
        e = thermo.make_eos(s["eos"], s["a"], s["b"], 1.0, s["Tr"], 0.344)
        rv, rl, mc, _ = thermo.maxwell(e)
        d = {k: v for k, v in s.items() if k != "mu_delta"}
        d["mu_bottom"] = mc + s.get("mu_delta", 0.0)
        width = 4.0 if s["eos"] == "cs" else 2.0
        r = max(2.0, min(s["nx"], s["ny"]) / 4)
        rho = (inputs.wall_drop(s["nx"], s["ny"], r, rl, rv, width)
               if s.get("walls") else inputs.drop(s["nx"], s["ny"], r, rl, rv,
                                                  width))
        out.append((d, e, rho))
    return out


def _rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("steps", [37, 1])
@pytest.mark.parametrize("per_cta", [1, 3])
def test_batch_matches_oracle_per_lattice(steps, per_cta, oracle_threads):
    inst = _instances()
    with Batch([d for d, _, _ in inst], precision="f64") as b:
        b.items_per_cta = per_cta          # CTAs spanning lattice boundaries
        assert b.items_per_cta == per_cta
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(steps)          # odd: graph blocks of 16 plus single steps
        assert b.info()["steps"] == steps
        for k, (d, e, rho) in enumerate(inst):
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(steps)
            got, want = b.moments(k), ref.moments()
            for key in ("rho", "mu", "vx", "vy"):
                assert _rel(got[key], want[key]) < 1e-12, (k, key)
            fg = b.populations(k)
            for i in range(9):
                assert _rel(fg[i], ref.f[i]) < 1e-12, (k, i)


def test_batch_matches_single_lattice_runs():
    inst = _instances()
    with Batch([d for d, _, _ in inst], precision="f32") as b:
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(50)
        for k, (d, _, rho) in enumerate(inst):
            kw = {x: d[x] for x in ("eos", "a", "b", "tau", "kappa", "walls",
                                    "mu_bottom") if x in d}
            with Simulation(d["nx"], d["ny"], Tr=d["Tr"], precision="f32",
                            **kw) as sim:
                sim.set_tile(*b.info()["tile"])
                sim.init(rho).step(50)
                one = sim.moments()
            got = b.moments(k)
            assert _rel(got["rho"], one["rho"]) < 1e-5


def test_batch_autotune_keeps_state_and_reduce_conserves_mass():
    inst = _instances()
    with Batch([d for d, _, _ in inst], precision="f64") as b:
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(4)
        m0 = [b.reduce(k)[0] for k in range(len(inst))]
        before = [b.populations(k) for k in range(len(inst))]
        shape = b.autotune(4)
        assert shape == b.info()["tile"]
        assert b.info()["steps"] == 4
        for k in range(len(inst)):
            assert np.array_equal(b.populations(k), before[k])
        b.step(40)
        for k in range(len(inst)):
            assert abs(b.reduce(k)[0] - m0[k]) / m0[k] < 1e-13


def test_batch_schedule_arguments():
    inst = _instances()
    with Batch([d for d, _, _ in inst], precision="f32") as b:
        assert b.items_per_cta == 0
        b.items_per_cta = 64
        for bad in (65, -2):
            with pytest.raises(LbmError):
                b.items_per_cta = bad
        assert b.items_per_cta == 64
        b.items_per_cta = 0
        assert b.items_per_cta == 0


def test_batch_rejects_init_at_odd_step_and_bad_index():
    inst = _instances()[:2]
    with Batch([d for d, _, _ in inst], precision="f32") as b:
        with pytest.raises(LbmError):
            b.step(1)                     # not initialised
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(1)
        with pytest.raises(LbmError):
            b.init(0, inst[0][2])         # odd step count
        with pytest.raises(IndexError):
            b.moments(5)
        # the C ABI checks the index itself
        assert b._lib.lbm_batch_reduce(b._b, 5, None) == -1
        b.step(1)
        b.init(0, inst[0][2])             # even again: allowed


def test_inactive_lattices_keep_their_state(oracle_threads):
    # a lattice that leaves the launch is frozen; the others go on; back in
    # the launch it continues from where it stopped
    inst = _instances()[:3]
    with Batch([d for d, _, _ in inst], precision="f64") as b:
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(10)
        frozen = b.populations(1)
        b.set_active(1, False)
        b.step(20)
        assert np.array_equal(b.populations(1), frozen)
        b.set_active(0, False)
        b.set_active(2, False)
        b.step(6)                          # nothing in the launch
        b.set_active(1, True)
        b.set_active(2, True)
        b.step(1)
        with pytest.raises(LbmError):
            b.set_active(0, True)          # odd batch step count
        b.step(9)
        for k, steps in ((0, 30), (1, 20), (2, 40)):
            d, e, rho = inst[k]
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(steps)
            got = b.moments(k)
            for key in ("rho", "mu", "vx", "vy"):
                assert _rel(got[key], ref.moments()[key]) < 1e-12, (k, key)


# Lattices whose 64-wide tiles include interior, periodic-seam and wall tiles
# (three or more full 64-wide tiles across), plus the heterogeneous set.
PAIR_SPECS = [
    dict(nx=192, ny=66, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0, kappa=0.5,
         walls=True, mu_delta=0.01),
    dict(nx=256, ny=128, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0, kappa=0.5),
    dict(nx=200, ny=100, eos="rks", a=2 / 49, b=2 / 21, Tr=0.8, tau=1.3,
         kappa=0.01, walls=True, mu_delta=-0.05),
]


@pytest.mark.parametrize("tile", [(32, 16), (32, 24), (32, 32), (64, 16), (64, 32)])
@pytest.mark.parametrize("precision", ["f32", "f32_offset", "f16_offset"])
@pytest.mark.parametrize("per_cta", [1, 4])
def test_batch_tile_shapes_reduced_precision(tile, precision, per_cta):
    """Every tile shape of the batched kernel in FP32 arithmetic (the
    64-wide shapes on the two-nodes-per-lane TMA path, edge tiles
    included): each lattice against the FP64 oracle and against its own
    single-lattice run at the same shape."""
    inst = _instances(SPECS + PAIR_SPECS)
    for d, e, rho in inst:
        rv, rl, _, _ = thermo.maxwell(e)
        d["rho_ref"] = 0.5 * (rv + rl) if precision != "f32" else 0.0
    with Batch([d for d, _, _ in inst], precision=precision) as b:
        b.set_tile(*tile)
        b.items_per_cta = per_cta
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(40)
        for k, (d, e, rho) in enumerate(inst):
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(40)
            kw = {x: d[x] for x in ("eos", "a", "b", "tau", "kappa", "walls",
                                    "mu_bottom", "rho_ref") if x in d}
            with Simulation(d["nx"], d["ny"], Tr=d["Tr"], precision=precision,
                            **kw) as sim:
                sim.set_tile(*tile)
                sim.init(rho).step(40)
                one = sim.moments()
            got, want = b.moments(k), ref.moments()
            if precision == "f16_offset":
                # half-precision populations: every field within the bounds
                # of the half unit roundoff (tests/fp16_bounds.py)
                want, bounds = run_with_bounds(ref, rho, 40, d["rho_ref"], e, d["kappa"])
                check(got, want, bounds, (k, tile), meaningful=("rho", "mu"))
                assert _rel(got["rho"], one["rho"]) < 2e-3, (k, "rho")
                continue
            # the velocity is a small difference of populations of size rho/9:
            # its FP32 rounding relative to max |v| reaches ~1e-4 on the RKS
            # lattice (density ratio ~30)
            for key, tol in (("rho", 1e-4), ("mu", 1e-4), ("vx", 3e-4), ("vy", 3e-4)):
                assert _rel(got[key], want[key]) < tol, (k, key)
            assert _rel(got["rho"], one["rho"]) < 1e-5, k


# Lattices whose tiles all take a TMA path (full tiles, periodic seams or
# walls, at least three 64-wide tiles across): the batched kernel is then
# launched without its general tile path.
TMA_SPECS = [
    PAIR_SPECS[0], PAIR_SPECS[1],
    dict(nx=192, ny=98, eos="rks", a=2 / 49, b=2 / 21, Tr=0.8, tau=1.3,
         kappa=0.01, walls=True, mu_delta=-0.05),
    dict(nx=192, ny=96, eos="pr", a=2 / 49, b=2 / 21, Tr=0.85, tau=1.3,
         kappa=0.01),
]


@pytest.mark.parametrize("tile", [(32, 16), (32, 32), (64, 16), (64, 32)])
@pytest.mark.parametrize("precision", ["f64", "f32", "f16_offset"])
@pytest.mark.parametrize("per_cta", [1, 3])
def test_batch_tma_only_work_list(tile, precision, per_cta):
    """A work list without general tiles (the kernel variant compiled
    without the general path) against the FP64 oracle, lattice by lattice,
    over both in-place parities."""
    from paper_1611_00907_gb300 import tile_kinds
    if precision == "f64" and tile[0] == 64:
        pytest.skip("FP64 64-wide tiles have no TMA path")
    inst = _instances(TMA_SPECS)
    for d, e, rho in inst:
        assert (np.asarray(tile_kinds(d["nx"], d["ny"], d.get("walls", False),
                                      tile, True)) > 0).all()
        rv, rl, _, _ = thermo.maxwell(e)
        d["rho_ref"] = 0.5 * (rv + rl) if precision == "f16_offset" else 0.0
    with Batch([d for d, _, _ in inst], precision=precision) as b:
        b.set_tile(*tile)
        b.items_per_cta = per_cta
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(21)
        for k, (d, e, rho) in enumerate(inst):
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(21)
            got, want = b.moments(k), ref.moments()
            if precision == "f16_offset":
                want, bounds = run_with_bounds(ref, rho, 21, d["rho_ref"], e, d["kappa"])
                check(got, want, bounds, (k, tile), meaningful=("rho", "mu"))
                continue
            tols = ((("rho", 1e-12), ("mu", 1e-12), ("vx", 1e-12), ("vy", 1e-12))
                    if precision == "f64" else
                    (("rho", 1e-4), ("mu", 1e-4), ("vx", 3e-4), ("vy", 3e-4)))
            for key, tol in tols:
                assert _rel(got[key], want[key]) < tol, (k, key)


def test_batch_of_more_lattices_than_one_launch_takes():
    """A batch larger than one launch's group of lattices (their tensor maps
    travel as a kernel parameter): the groups run as separate launches, on
    parallel branches of the captured graph, and every lattice still
    follows the oracle."""
    base = dict(nx=64, ny=32, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0, kappa=0.5)
    specs = [dict(base, tau=0.8 + 0.004 * k) for k in range(70)]
    specs[3] = dict(specs[3], nx=70, ny=21)          # ragged: general tiles
    specs[66] = dict(specs[66], walls=True, ny=34, mu_delta=0.02)
    inst = _instances(specs)
    with Batch([d for d, _, _ in inst], precision="f64") as b:
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(17)
        for k in (0, 3, 63, 64, 66, 69):
            d, e, rho = inst[k]
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(17)
            got, want = b.moments(k), ref.moments()
            for key in ("rho", "mu", "vx", "vy"):
                assert _rel(got[key], want[key]) < 1e-12, (k, key)


# Sweeps on one geometry (the wetting study's shape): the grid-per-lattice
# launch, physics differing lattice by lattice.
SWEEPS = {
    "walls": [dict(nx=192, ny=66, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=tau,
                   kappa=0.5, walls=True, mu_delta=md)
              for tau, md in ((1.0, -0.02), (0.9, 0.0), (1.2, 0.015), (1.0, 0.03))],
    "periodic": [dict(nx=256, ny=128, eos="cs", a=1.0, b=4.0, Tr=tr, tau=1.0,
                      kappa=0.5) for tr in (0.8, 0.85, 0.9)],
}


@pytest.mark.parametrize("sweep", ["walls", "periodic"])
@pytest.mark.parametrize("tile", [(32, 16), (32, 32), (64, 16), (64, 32)])
@pytest.mark.parametrize("precision", ["f64", "f32", "f16_offset"])
def test_batch_grid_per_lattice_on_one_geometry(sweep, tile, precision):
    """The grid-per-lattice launch (descriptors as a kernel parameter)
    against the FP64 oracle, lattice by lattice, over both in-place
    parities; a lattice taken out of the launch half-way keeps its state
    and the grid rows of the others move up."""
    if precision == "f64" and tile[0] == 64:
        pytest.skip("FP64 64-wide tiles have no TMA path")
    inst = _instances(SWEEPS[sweep])
    for d, e, rho in inst:
        rv, rl, _, _ = thermo.maxwell(e)
        d["rho_ref"] = 0.5 * (rv + rl) if precision == "f16_offset" else 0.0
    with Batch([d for d, _, _ in inst], precision=precision) as b:
        b.set_tile(*tile)
        b.items_per_cta = 0
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(6)
        b.set_active(1, False)
        b.step(17)
        for k, (d, e, rho) in enumerate(inst):
            n = 6 if k == 1 else 23
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(n)
            got, want = b.moments(k), ref.moments()
            if precision == "f16_offset":
                want, bounds = run_with_bounds(ref, rho, n, d["rho_ref"], e, d["kappa"])
                check(got, want, bounds, (k, tile), meaningful=("rho", "mu"))
                continue
            tols = ((("rho", 1e-12), ("mu", 1e-12), ("vx", 1e-12), ("vy", 1e-12))
                    if precision == "f64" else
                    (("rho", 1e-4), ("mu", 1e-4), ("vx", 3e-4), ("vy", 3e-4)))
            for key, tol in tols:
                assert _rel(got[key], want[key]) < tol, (k, key)


def test_batch_with_no_lattice_in_the_launch_and_zero_steps():
    """Degenerate schedules: zero steps change nothing; with every lattice
    out of the launch a step launches nothing and only counts; back in, the
    lattices continue from where they stopped."""
    inst = _instances(SPECS[:3])
    with Batch([d for d, _, _ in inst], precision="f64") as b:
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(0)
        b.step(4)
        before = [b.populations(k) for k in range(len(inst))]
        for k in range(len(inst)):
            b.set_active(k, False)
        b.step(6)
        b.step(0)
        assert b.info()["steps"] == 10
        for k in range(len(inst)):
            assert np.array_equal(b.populations(k), before[k])
            b.set_active(k, True)
        b.step(3)
        for k, (d, e, rho) in enumerate(inst):
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=d.get("walls", False),
                                 mu_bottom=d["mu_bottom"])
            ref.init_equilibrium(rho).step(7)
            got = b.moments(k)
            for key in ("rho", "mu", "vx", "vy"):
                assert _rel(got[key], ref.moments()[key]) < 1e-12, (k, key)


@pytest.mark.parametrize("precision", ["f32", "f16_offset"])
def test_autotune_over_both_schedules_keeps_the_state(precision):
    """A batch of one geometry: the autotuner times the grid-per-lattice
    launch beside the work list at every tile shape, keeps the fastest and
    leaves every lattice's state and step count as they were; the batch then
    follows the oracle."""
    inst = _instances(SWEEPS["walls"])
    for d, e, rho in inst:
        rv, rl, _, _ = thermo.maxwell(e)
        d["rho_ref"] = 0.5 * (rv + rl)
    with Batch([d for d, _, _ in inst], precision=precision) as b:
        for k, (_, _, rho) in enumerate(inst):
            b.init(k, rho)
        b.step(6)
        before = [b.populations(k) for k in range(len(inst))]
        shape = b.autotune(4)
        assert shape == b.info()["tile"] and b.info()["steps"] == 6
        assert b.items_per_cta in (0, 1, 2, 4)
        for k in range(len(inst)):
            assert np.array_equal(b.populations(k), before[k])
        b.step(17)
        for k, (d, e, rho) in enumerate(inst):
            ref = oracle.Lattice(d["nx"], d["ny"], e, d["tau"], d["kappa"],
                                 walls=True, mu_bottom=d["mu_bottom"])
            got = b.moments(k)
            if precision == "f16_offset":
                want, bounds = run_with_bounds(ref, rho, 23, d["rho_ref"], e, d["kappa"])
                check(got, want, bounds, (k, shape), meaningful=("rho", "mu"))
            else:
                want = ref.init_equilibrium(rho).step(23).moments()
                for key, tol in (("rho", 1e-4), ("mu", 1e-4), ("vx", 3e-4), ("vy", 3e-4)):
                    assert _rel(got[key], want[key]) < tol, (k, key)
