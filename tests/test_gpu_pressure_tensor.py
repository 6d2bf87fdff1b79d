"""The pressure-tensor baseline (Eq. 5 with Eq. 9) on the GPU against the
oracle's pressure-tensor step, and its argument checks.  Interior and
periodic-seam tiles take the TMA tile paths, as in the chemical-potential
step: the 32-wide path (FP64 at 32 x 16, FP32 at 32 x 32; 224 x 165 and
96 x 96 have both kinds, and general tiles in the first) and the
two-nodes-per-lane path of FP32 at 64 x 16 (192 x 96: every tile on it,
seams included; 224 x 165: with general tiles on the ragged edges)."""
import numpy as np
import pytest

import oracle
from oracle import thermo
from paper_1611_00907_gb300 import LbmError, Simulation, inputs

pytestmark = pytest.mark.gpu


def _case(nx, ny, precision):
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    rv, rl, _, _ = thermo.maxwell(e)
    rho = inputs.drop(nx, ny, min(nx, ny) / 4, rl, rv, 4.0)
    sim = Simulation(nx, ny, "cs", 1.0, 4.0, 1.0, 0.85, tau=1.0, kappa=0.5,
                     precision=precision)
    ref = oracle.Lattice(nx, ny, e, 1.0, 0.5)
    return sim, ref, rho


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("size", [(70, 21), (224, 165), (96, 96), (5, 5)])
@pytest.mark.parametrize("steps", [1, 2, 200])
def test_pressure_tensor_step_matches_oracle_fp64(size, steps, oracle_threads):
    sim, ref, rho = _case(*size, "f64")
    with sim:
        sim.set_force_model("pressure_tensor")
        sim.init(rho).step(steps)
        ref.init_equilibrium(rho).step_pressure_tensor(steps)
        f = sim.populations()
        for i in range(9):
            assert _rel(f[i], ref.f[i]) < 1e-12, i


@pytest.mark.parametrize("size,tile", [((224, 165), (32, 32)), ((96, 96), (32, 32)),
                                       ((192, 96), (64, 16)), ((224, 165), (64, 16))])
@pytest.mark.parametrize("steps", [49, 50])
def test_pressure_tensor_fp32(size, tile, steps, oracle_threads, monkeypatch):
    # against the oracle, and against the same lattice on the general path;
    # an odd step count ends on the odd-step kernel
    runs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("CPLBM_NO_TMA", "1")
        sim, ref, rho = _case(*size, "f32")
        with sim:
            sim.set_force_model("pressure_tensor").set_tile(*tile)
            assert sim.tile == tile
            sim.init(rho).step(steps)
            runs.append(sim.moments()["rho"])
    ref.init_equilibrium(rho).step_pressure_tensor(steps)
    want = ref.moments()["rho"]
    assert _rel(runs[0], want) < 1e-5
    assert _rel(runs[0], runs[1]) < 1e-5


def test_pressure_tensor_arguments():
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    rv, rl, _, _ = thermo.maxwell(e)
    with Simulation(70, 21, walls=True) as sim:
        with pytest.raises(LbmError):
            sim.set_force_model("pressure_tensor")
    with Simulation(70, 21, precision="f16_offset", rho_ref=0.15) as sim:
        with pytest.raises(LbmError):
            sim.set_force_model("pressure_tensor")
    with Simulation(70, 21, precision="f64") as sim:
        sim.set_force_model("pressure_tensor")
        assert sim.tile == (32, 16)
        with pytest.raises(LbmError):
            sim.set_tile(64, 16)
        sim.init(inputs.drop(70, 21, 5, rl, rv)).step(3)
        sim.set_force_model("chemical_potential")
        sim.step(3)
    # FP32: the default tile, 32 x 32 too, no other; autotune keeps to them
    with Simulation(192, 96, precision="f32") as sim:
        sim.set_force_model("pressure_tensor")
        assert sim.tile == (64, 16)
        sim.set_tile(32, 32)
        for shape in ((32, 16), (32, 24), (64, 32)):
            with pytest.raises(LbmError):
                sim.set_tile(*shape)
        assert sim.tile == (32, 32)
        sim.init(inputs.drop(192, 96, 20, rl, rv)).step(2)
        assert sim.autotune(4) in ((64, 16), (32, 32))
        sim.step(2)
