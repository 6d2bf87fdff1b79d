"""Failure paths of the library, driven from the host: nothing here faults,
traps or hangs the GPU.

* A bounded wait that runs out: the step kernels' first wait for a tile's
  staged data is given a limit of zero cycles (lbm_test_set_wait_cycles), so
  it gives up at its first unsuccessful poll.  The tile then drains its
  copies with the long limit and leaves its nodes untouched; the next
  synchronising call reports the timeout, and the context, re-initialised,
  steps correctly again.
* Device allocations that fail: lbm_test_fail_device_alloc makes the n-th
  allocation report out-of-memory.  Every create call returns LBM_ERR_OOM
  for every n and holds no device memory afterwards; a failed staging
  buffer leaves the context usable.
* A lattice that diverges returns LBM_ERR_NUMERIC from the reduction
  (test_gpu_parity.py::test_diverging_lattice_reports_numeric_error).
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle import thermo
from paper_1611_00907_gb300 import Batch, LbmError, Simulation, _lib, inputs
from paper_1611_00907_gb300 import mlp as mlp_mod

pytestmark = pytest.mark.gpu


def _cs_drop(nx, ny):
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    rv, rl, _, _ = thermo.maxwell(e)
    return e, inputs.drop(nx, ny, min(nx, ny) / 4, rl, rv)


@pytest.mark.parametrize("precision,tile", [("f64", (32, 32)),
                                            ("f32", (64, 16))])
def test_wait_timeout_is_reported_and_the_context_recovers(precision, tile):
    # 192 x 96 with these tiles: every tile is interior or a periodic seam,
    # so every tile takes a TMA path and waits on its mbarriers
    nx, ny = 192, 96
    kinds = np.asarray(_kinds(nx, ny, tile))
    assert (kinds > 0).all()
    e, rho = _cs_drop(nx, ny)
    lib = _lib.load()
    with Simulation(nx, ny, "cs", 1.0, 4.0, 1.0, 0.85, tau=1.0, kappa=0.5,
                    precision=precision) as sim:
        sim.set_tile(*tile)
        assert lib.lbm_test_set_wait_cycles(sim._ctx, 0) == _lib.LBM_OK
        sim.init(rho)
        f0 = sim.populations()
        sim.step(2)
        with pytest.raises(LbmError) as ei:
            sim.moments()
        assert ei.value.status == _lib.LBM_ERR_CUDA
        assert "timed out" in str(ei.value)
        # the flag is cleared once reported; every tile gave up at once and
        # left its nodes as they were, so two steps changed nothing
        got = sim.populations()
        assert np.array_equal(got, f0)
        # default limit again: the re-initialised lattice follows the oracle
        assert lib.lbm_test_set_wait_cycles(sim._ctx, -1) == _lib.LBM_OK
        sim.init(rho).step(3)
        got = sim.populations()
    ref = oracle.Lattice(nx, ny, e, 1.0, 0.5).init_equilibrium(rho).step(3)
    # populations: FP64 round-off, or FP32 storage rounding
    tol = 1e-13 if precision == "f64" else 1e-6
    for i in range(9):
        scale = np.abs(ref.f[i]).max()
        assert np.abs(got[i] - ref.f[i]).max() <= tol * scale, i


def _kinds(nx, ny, tile):
    from paper_1611_00907_gb300 import tile_kinds
    return tile_kinds(nx, ny, False, tile)


def _create_raw(nx, ny, walls=0, precision=0):
    lib = _lib.load()
    cfg = _lib.LbmConfig(nx, ny, walls, 1.0, 0.5, 0.0, precision, None, 0)
    ctx = C.c_void_p()
    return lib.lbm_create(C.byref(cfg), C.byref(ctx)), ctx


@pytest.fixture
def disarm():
    yield
    _lib.load().lbm_test_fail_device_alloc(-1)


def test_failed_allocation_in_create_leaks_nothing(disarm):
    lib = _lib.load()
    base = lib.lbm_test_device_allocs()
    st, ctx = _create_raw(70, 21, walls=1)
    assert st == _lib.LBM_OK
    n_allocs = lib.lbm_test_device_allocs() - base
    assert n_allocs >= 20          # populations, densities, 16 rings, ...
    lib.lbm_destroy(ctx)
    assert lib.lbm_test_device_allocs() == base
    for n in range(n_allocs):
        lib.lbm_test_fail_device_alloc(n)
        st, ctx = _create_raw(70, 21, walls=1)
        assert st == _lib.LBM_ERR_OOM, n
        assert not ctx.value
        assert b"out of memory" in lib.lbm_last_error(None)
        assert lib.lbm_test_device_allocs() == base, n
    lib.lbm_test_fail_device_alloc(-1)
    st, ctx = _create_raw(70, 21, walls=1)
    assert st == _lib.LBM_OK
    lib.lbm_destroy(ctx)
    assert lib.lbm_test_device_allocs() == base


def test_failed_staging_buffer_leaves_the_context_usable(disarm):
    lib = _lib.load()
    e, rho = _cs_drop(70, 21)
    with Simulation(70, 21, "cs", 1.0, 4.0, 1.0, 0.85, tau=1.0,
                    kappa=0.5) as sim:
        sim.init(rho).step(4)
        held = lib.lbm_test_device_allocs()
        lib.lbm_test_fail_device_alloc(0)
        # host outputs of all four fields need a larger staging buffer than
        # lbm_init's three: the reallocation fails
        with pytest.raises(LbmError) as ei:
            sim.moments()
        assert ei.value.status == _lib.LBM_ERR_OOM
        assert lib.lbm_test_device_allocs() == held - 1   # old buffer freed
        got = sim.moments()
    want = oracle.Lattice(70, 21, e, 1.0, 0.5).init_equilibrium(rho).step(4)
    assert np.abs(got["rho"] - want.moments()["rho"]).max() < 1e-13


def test_failed_allocation_in_batch_and_network_create(disarm):
    lib = _lib.load()
    base = lib.lbm_test_device_allocs()
    inst = [dict(nx=70, ny=21), dict(nx=40, ny=33, walls=True)]
    b = Batch(inst, precision="f64")
    n_allocs = lib.lbm_test_device_allocs() - base
    b.close()
    assert lib.lbm_test_device_allocs() == base
    for n in range(n_allocs):
        lib.lbm_test_fail_device_alloc(n)
        with pytest.raises(LbmError) as ei:
            Batch(inst, precision="f64")
        assert ei.value.status == _lib.LBM_ERR_OOM, n
        assert lib.lbm_test_device_allocs() == base, n
    lib.lbm_test_fail_device_alloc(-1)
    net = mlp_mod.Mlp(seed=0)
    n_net = lib.lbm_test_device_allocs() - base
    net.close()
    assert n_net == 7 and lib.lbm_test_device_allocs() == base
    for n in range(n_net):
        lib.lbm_test_fail_device_alloc(n)
        with pytest.raises(LbmError) as ei:
            mlp_mod.Mlp(seed=0)
        assert ei.value.status == _lib.LBM_ERR_OOM, n
        assert lib.lbm_test_device_allocs() == base, n
