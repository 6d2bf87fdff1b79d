"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/cplbm.h declares; argument validation and the host-side
critical-point helper work without touching a device."""
import ctypes as C
import math

import numpy as np
import subprocess

import pytest

from paper_1611_00907_gb300 import _build, _lib


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _lib.header_symbols()
    for must in ("lbm_create", "lbm_set_eos", "lbm_set_wall_mu", "lbm_init",
                 "lbm_step", "lbm_moments", "lbm_reduce", "lbm_get_state",
                 "lbm_set_state", "lbm_destroy", "lbm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _lib.header_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(_lib.header_symbols()) <= exported


def test_bindings_cover_the_header():
    assert set(_lib.SIGNATURES) == set(_lib.header_symbols())


def _cfg(**kw):
    base = dict(nx=32, ny=32, walls=0, tau=1.0, kappa=0.5, rho_ref=0.0,
                precision=0, stream=None, device=0)
    base.update(kw)
    return _lib.LbmConfig(**base)


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(tau=float("nan")),
                                 dict(tau=float("inf")), dict(nx=4), dict(ny=3),
                                 dict(walls=2), dict(kappa=-1.0),
                                 dict(kappa=float("nan")), dict(precision=7),
                                 dict(precision=-1), dict(walls=1, ny=6),
                                 dict(rho_ref=float("inf")),
                                 # the largest lattice: 2^31 nodes
                                 dict(nx=65536, ny=32769)])
def test_create_rejects_invalid_configuration(lib, bad):
    ctx = C.c_void_p()
    cfg = _cfg(**bad)
    st = lib.lbm_create(C.byref(cfg), C.byref(ctx))
    assert st == _lib.LBM_ERR_ARG
    assert ctx.value is None
    assert lib.lbm_last_error(None)


def test_batch_create_rejects_empty_and_bad_precision(lib):
    b = C.c_void_p()
    inst = (_lib.LbmInstance * 1)()
    assert lib.lbm_batch_create(inst, 0, 1, None, 0, C.byref(b)) == _lib.LBM_ERR_ARG
    assert lib.lbm_batch_create(inst, 1, 9, None, 0, C.byref(b)) == _lib.LBM_ERR_ARG
    assert lib.lbm_batch_create(None, 1, 1, None, 0, C.byref(b)) == _lib.LBM_ERR_ARG
    assert b.value is None
    assert lib.lbm_batch_last_error(None)
    assert lib.lbm_batch_step(None, 1) == _lib.LBM_ERR_ARG
    assert lib.lbm_batch_schedule(None, 1, None) == _lib.LBM_ERR_ARG
    lib.lbm_batch_destroy(None)


def test_null_arguments_are_errors_not_crashes(lib):
    assert lib.lbm_create(None, None) == _lib.LBM_ERR_ARG
    assert lib.lbm_step(None, 1) == _lib.LBM_ERR_ARG
    assert lib.lbm_init(None, None, None, None, 0) == _lib.LBM_ERR_ARG
    assert lib.lbm_state_size(None) == 0
    lib.lbm_destroy(None)


@pytest.mark.parametrize("eos,a,b", [(0, 9 / 49, 2 / 21), (1, 1.0, 4.0),
                                     (2, 2 / 49, 2 / 21), (3, 2 / 49, 2 / 21)])
def test_library_critical_point_matches_closed_forms(lib, eos, a, b):
    Tc, rc = C.c_double(), C.c_double()
    assert lib.lbm_eos_critical(eos, a, b, 1.0, C.byref(Tc), C.byref(rc)) == 0
    if eos == 0:
        assert Tc.value == pytest.approx(8 * a / (27 * b), rel=1e-14)
        assert rc.value == pytest.approx(1 / (3 * b), rel=1e-13)
    if eos == 3:
        assert b * rc.value == pytest.approx(2 ** (1 / 3) - 1, rel=1e-13)
    if eos == 2:   # Peng-Robinson textbook ratio Omega_b / Omega_a
        assert Tc.value * b / a == pytest.approx(0.07780 / 0.45724, rel=2e-4)
    assert math.isfinite(Tc.value) and Tc.value > 0


def test_library_and_oracle_critical_points_agree(lib):
    from oracle import thermo
    for eos, kind, a, b in [(1, "cs", 1.0, 4.0), (2, "pr", 2 / 49, 2 / 21),
                            (3, "rks", 2 / 49, 2 / 21)]:
        Tc, rc = C.c_double(), C.c_double()
        lib.lbm_eos_critical(eos, a, b, 1.0, C.byref(Tc), C.byref(rc))
        T2, r2 = thermo.critical_point(kind, a, b)
        assert Tc.value == pytest.approx(T2, rel=1e-13)
        assert rc.value == pytest.approx(r2, rel=1e-9)


def test_critical_rejects_bad_eos(lib):
    Tc, rc = C.c_double(), C.c_double()
    assert lib.lbm_eos_critical(9, 1, 1, 1, C.byref(Tc), C.byref(rc)) == \
        _lib.LBM_ERR_ARG
    assert lib.lbm_eos_critical(1, -1, 1, 1, C.byref(Tc), C.byref(rc)) == \
        _lib.LBM_ERR_ARG


@pytest.mark.parametrize("kind,eos,a,b", [("vdw", 0, 9 / 49, 2 / 21),
                                          ("cs", 1, 1.0, 4.0),
                                          ("pr", 2, 2 / 49, 2 / 21),
                                          ("rks", 3, 2 / 49, 2 / 21)])
@pytest.mark.parametrize("Tr", [0.6, 0.85, 0.95])
def test_library_coexistence_matches_oracle(lib, kind, eos, a, b, Tr):
    from oracle import thermo
    v, l, m = C.c_double(), C.c_double(), C.c_double()
    assert lib.lbm_eos_coexistence(eos, a, b, 1.0, Tr, 0.344, C.byref(v),
                                   C.byref(l), C.byref(m)) == 0
    rv, rl, mc, _ = thermo.maxwell(thermo.make_eos(kind, a, b, 1.0, Tr, 0.344))
    assert v.value == pytest.approx(rv, rel=1e-9)
    assert l.value == pytest.approx(rl, rel=1e-9)
    assert m.value == pytest.approx(mc, rel=1e-9, abs=1e-12)


def test_library_coexistence_rejects_supercritical(lib):
    v, l = C.c_double(), C.c_double()
    assert lib.lbm_eos_coexistence(1, 1.0, 4.0, 1.0, 1.02, 0.3, C.byref(v),
                                   C.byref(l), None) == _lib.LBM_ERR_ARG


@pytest.mark.parametrize("kind,a,b,Tr", [("vdw", 9 / 49, 2 / 21, 0.85),
                                         ("cs", 1.0, 4.0, 0.85),
                                         ("pr", 2 / 49, 2 / 21, 0.8),
                                         ("rks", 2 / 49, 2 / 21, 0.8)])
def test_library_pressure_matches_oracle(kind, a, b, Tr):
    from oracle import thermo
    from paper_1611_00907_gb300 import LbmError, eos_pressure
    e = thermo.make_eos(kind, a, b, 1.0, Tr, 0.344)
    rv, rl, _, _ = thermo.maxwell(e)
    rho = np.linspace(0.5 * rv, 1.2 * rl, 41)
    got = eos_pressure(kind, a, b, 1.0, Tr, 0.344, rho)
    want = e.p0(rho)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    with pytest.raises(LbmError):
        eos_pressure(kind, a, b, 1.0, Tr, 0.344, [-0.1])


def test_default_device_follows_torch():
    # an explicit device wins; otherwise PyTorch's current CUDA device (so
    # each torchrun rank uses its own GPU), 0 without CUDA
    from paper_1611_00907_gb300 import _default_device
    assert _default_device(3) == 3
    torch = pytest.importorskip("torch")
    want = torch.cuda.current_device() if torch.cuda.is_available() else 0
    assert _default_device(None) == want
