"""The allocation-free step, lbm_step_noalloc, against the context-based step.

lbm_step_noalloc serves callers that may not allocate device memory (for
example an application whose own allocator owns the GPU): the caller passes
its population array, and the library works in a fixed device array it
holds for the life of the process.  Through the C ABI, two calls in a row
must reproduce what lbm_create / lbm_init / lbm_step give for the same
steps, to the FP64 step tolerance of the parity tests (1e-13 relative per
population).  This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import thermo
from paper_1611_00907_gb300 import Simulation, _lib, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _config(nx, ny, walls, stream, tau=1.0, kappa=0.5):
    return _lib.LbmConfig(nx, ny, int(walls), tau, kappa, 0.0, 0,
                          C.c_void_p(stream), 0)


@pytest.mark.parametrize("walls,size", [(False, (70, 21)), (True, (131, 37)),
                                        (True, (512, 384)), (False, (702, 702))])
def test_noalloc_matches_context_step_on_two_calls(walls, size):
    torch = pytest.importorskip("torch")
    nx, ny = size
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    rv, rl, mc, _ = thermo.maxwell(e)
    rho = (inputs.wall_drop(nx, ny, 12, rl, rv) if walls
           else inputs.drop(nx, ny, 7, rl, rv))
    mu_s = mc + 0.01
    with Simulation(nx, ny, "cs", 1.0, 4.0, 1.0, 0.85, tau=1.0, kappa=0.5,
                    walls=walls, precision="f64", mu_bottom=mu_s) as sim:
        sim.init(rho)
        f0 = sim.populations()
        sim.step(10)
        want10 = sim.populations()
        sim.step(12)
        want22 = sim.populations()

    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    cfg = _config(nx, ny, walls, stream)
    f = torch.tensor(f0, device="cuda")
    for steps, want in ((10, want10), (12, want22)):
        st = lib.lbm_step_noalloc(C.byref(cfg), 1, 1.0, 4.0, 1.0, 0.85, 0.344,
                                  mu_s, 0, 0.0, f.data_ptr(), steps)
        assert st == _lib.LBM_OK, lib.lbm_last_error(None)
        torch.cuda.synchronize()
        got = f.cpu().numpy()
        fl = slice(1, ny - 1) if walls else slice(0, ny)
        for i in range(9):
            scale = np.abs(want[i, fl]).max()
            err = np.abs(got[i, fl] - want[i, fl]).max() / scale
            assert err < TOL, (steps, i, err)


def test_noalloc_rejects_oversized_and_odd_requests():
    lib = _lib.load()
    # 702 x 702 periodic is the largest square the fixed array holds
    cfg = _config(703, 703, False, None)
    dummy = C.c_void_p(16)   # never dereferenced: checks come first
    st = lib.lbm_step_noalloc(C.byref(cfg), 1, 1.0, 4.0, 1.0, 0.85, 0.344,
                              0.0, 0, 0.0, dummy, 2)
    assert st == _lib.LBM_ERR_ARG
    assert b"LBM_NOALLOC_SCRATCH_BYTES" in lib.lbm_last_error(None)
    cfg = _config(64, 64, False, None)
    st = lib.lbm_step_noalloc(C.byref(cfg), 1, 1.0, 4.0, 1.0, 0.85, 0.344,
                              0.0, 0, 0.0, dummy, 3)
    assert st == _lib.LBM_ERR_ARG
    assert b"even" in lib.lbm_last_error(None)
