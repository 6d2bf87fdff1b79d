"""The FP64 logarithm and reciprocal of the FP64 step (device_common.cuh:
log_tab after Tang's table-driven method, rcp_nr a Newton-refined
reciprocal) against the host's log and IEEE division, in units in the last
place, through the lbm_test_fp64_math hook.

Error budget of log_tab: the rounded 1/F and the product f * (1/F) move r by
at most 2^-60 absolutely; the series through r^7 leaves less than 2^-59 of r;
ln F and the final two additions round three times, each by at most half an
ulp of the result: 2 ulp in all.  The host's log adds up to one ulp of its
own, so the two agree within 3.  rcp_nr: once the Newton steps have
converged, only the last step's rounding remains, and it starts from a value
within an ulp, so the result is within one ulp of the correctly rounded
1/x."""
import numpy as np
import pytest

from paper_1611_00907_gb300 import _lib

pytestmark = pytest.mark.gpu


def _run(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    lg, rc = np.empty_like(x), np.empty_like(x)
    lib = _lib.load()
    st = lib.lbm_test_fp64_math(x.ctypes.data, x.size, lg.ctypes.data, rc.ctypes.data)
    assert st == _lib.LBM_OK
    return lg, rc


def _ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def _inputs():
    rng = np.random.default_rng(1611_00907)
    parts = [
        np.exp(rng.uniform(np.log(2.0 ** -1020), np.log(2.0 ** 1020), 200_000)),
        rng.uniform(1e-3, 10.0, 200_000),                  # the lattice densities
        1.0 + np.arange(-4096, 4097) * 2.0 ** -52,          # around 1
        1.0 - np.arange(1, 4097) * 2.0 ** -21,              # the branch just below 1
        np.ldexp(1.0, np.arange(-1020, 1021)),              # powers of two
    ]
    F = 1.0 + np.arange(129) / 128.0
    for d in (-3, -1, 0, 1, 3):                             # around every breakpoint
        for e in (-5, 0, 7):
            parts.append(np.ldexp(F + d * 2.0 ** -52, e))
    half = 1.0 + (np.arange(128) + 0.5) / 128.0             # midway between them
    parts.append(half)
    parts.append(np.nextafter(half, 0.0))
    x = np.concatenate(parts)
    return x[(x > 2.0 ** -1021) & (x < 2.0 ** 1021)]


def test_log_within_three_ulp():
    x = _inputs()
    lg, _ = _run(x)
    want = np.log(x)
    nz = want != 0.0
    assert np.all(lg[~nz] == 0.0)
    err = _ulps(lg[nz], want[nz])
    assert err.max() <= 3.0, (err.max(), x[nz][np.argmax(err)])
    # and typically within one
    assert np.mean(err <= 1.0) > 0.99


def test_reciprocal_within_one_ulp():
    x = _inputs()
    x = np.concatenate([x, -x])
    _, rc = _run(x)
    err = _ulps(rc, 1.0 / x)
    assert err.max() <= 1.0, (err.max(), x[np.argmax(err)])


def test_special_values():
    x = np.array([0.0, -1.0, np.inf, np.nan, 5e-324, 2.0 ** -1060, -np.inf])
    lg, rc = _run(x)
    with np.errstate(divide="ignore", invalid="ignore"):
        want = np.log(x)
    # non-positive, subnormal, infinite and NaN arguments go to log()
    assert np.array_equal(lg, want, equal_nan=True)
    # zero, infinite and NaN arguments of the reciprocal give NaN
    assert np.isnan(rc[[0, 2, 3, 6]]).all()
    assert rc[1] == -1.0
