"""ctypes declarations of the C ABI in include/cplbm.h.

Loading fails loudly when libcplbm.so has not been built: there is no CPU
fallback anywhere in this package.  CPLBM_LIBRARY_VARIANT=checked in the
environment loads the bounds-checked debug build (libcplbm_checked.so,
`python -m paper_1611_00907_gb300._build --checked`) instead.
"""
import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
_VARIANT = os.environ.get("CPLBM_LIBRARY_VARIANT", "")
if _VARIANT not in ("", "checked"):
    raise ImportError("CPLBM_LIBRARY_VARIANT must be unset or 'checked'")
LIB_PATH = os.path.join(HERE, "libcplbm_checked.so" if _VARIANT else "libcplbm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cplbm.h")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_NUMERIC, \
    LBM_ERR_STATE = 0, -1, -2, -3, -4, -5
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA",
                -3: "LBM_ERR_OOM", -4: "LBM_ERR_NUMERIC", -5: "LBM_ERR_STATE"}

EOS = {"vdw": 0, "cs": 1, "pr": 2, "rks": 3}
PRECISION = {"f64": 0, "f32": 1, "f32_offset": 2, "f16_offset": 3}


class LbmConfig(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("walls", C.c_int),
                ("tau", C.c_double), ("kappa", C.c_double),
                ("rho_ref", C.c_double), ("precision", C.c_int),
                ("stream", C.c_void_p), ("device", C.c_int)]


class LbmInstance(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("walls", C.c_int),
                ("tau", C.c_double), ("kappa", C.c_double),
                ("rho_ref", C.c_double), ("eos", C.c_int), ("a", C.c_double),
                ("b", C.c_double), ("R", C.c_double),
                ("T_over_Tc", C.c_double), ("omega", C.c_double),
                ("mu_bottom", C.c_double), ("top_mode", C.c_int),
                ("mu_top", C.c_double)]


_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_ctx = C.c_void_p

SIGNATURES = {
    "lbm_create": ([C.POINTER(LbmConfig), C.POINTER(_ctx)], C.c_int),
    "lbm_set_eos": ([_ctx, C.c_int, C.c_double, C.c_double, C.c_double,
                     C.c_double, C.c_double], C.c_int),
    "lbm_set_wall_mu": ([_ctx, C.c_double, C.c_int, C.c_double], C.c_int),
    "lbm_init": ([_ctx, _vp, _vp, _vp, C.c_int], C.c_int),
    "lbm_set_tile": ([_ctx, C.c_int, C.c_int], C.c_int),
    "lbm_set_force_model": ([_ctx, C.c_int], C.c_int),
    "lbm_get_tile": ([_ctx, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "lbm_autotune": ([_ctx, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)],
                     C.c_int),
    "lbm_step": ([_ctx, C.c_int], C.c_int),
    "lbm_moments": ([_ctx, _vp, _vp, _vp, _vp, C.c_int], C.c_int),
    "lbm_get_populations": ([_ctx, _vp, C.c_int], C.c_int),
    "lbm_reduce": ([_ctx, _dp], C.c_int),
    "lbm_state_size": ([_ctx], C.c_size_t),
    "lbm_get_state": ([_ctx, _vp, C.c_size_t], C.c_int),
    "lbm_set_state": ([_ctx, _vp, C.c_size_t], C.c_int),
    "lbm_step_count": ([_ctx], C.c_longlong),
    "lbm_eos_info": ([_ctx, _dp, _dp, _dp, _dp], C.c_int),
    "lbm_eos_critical": ([C.c_int, C.c_double, C.c_double, C.c_double, _dp,
                          _dp], C.c_int),
    "lbm_eos_coexistence": ([C.c_int, C.c_double, C.c_double, C.c_double,
                             C.c_double, C.c_double, _dp, _dp, _dp], C.c_int),
    "lbm_eos_pressure": ([C.c_int, C.c_double, C.c_double, C.c_double,
                          C.c_double, C.c_double, _vp, _vp, C.c_size_t], C.c_int),
    "lbm_tile_kinds": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                        _vp, C.c_size_t], C.c_int),
    "lbm_test_set_wait_cycles": ([_ctx, C.c_longlong], C.c_int),
    "lbm_test_fail_device_alloc": ([C.c_int], None),
    "lbm_test_device_allocs": ([], C.c_longlong),
    "lbm_test_fp64_math": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "lbm_test_shrink_bounds": ([_ctx, C.c_longlong], C.c_int),
    "lbm_step_noalloc": ([C.POINTER(LbmConfig), C.c_int, C.c_double,
                          C.c_double, C.c_double, C.c_double, C.c_double,
                          C.c_double, C.c_int, C.c_double, _vp, C.c_int],
                         C.c_int),
    "lbm_batch_create": ([C.POINTER(LbmInstance), C.c_int, C.c_int, _vp,
                          C.c_int, C.POINTER(_ctx)], C.c_int),
    "lbm_batch_init": ([_ctx, C.c_int, _vp, _vp, _vp, C.c_int], C.c_int),
    "lbm_batch_step": ([_ctx, C.c_int], C.c_int),
    "lbm_batch_set_active": ([_ctx, C.c_int, C.c_int], C.c_int),
    "lbm_batch_moments": ([_ctx, C.c_int, _vp, _vp, _vp, _vp, C.c_int],
                          C.c_int),
    "lbm_batch_populations": ([_ctx, C.c_int, _vp, C.c_int], C.c_int),
    "lbm_batch_reduce": ([_ctx, C.c_int, _dp], C.c_int),
    "lbm_batch_set_tile": ([_ctx, C.c_int, C.c_int], C.c_int),
    "lbm_batch_autotune": ([_ctx, C.c_int, C.POINTER(C.c_int),
                            C.POINTER(C.c_int)], C.c_int),
    "lbm_batch_schedule": ([_ctx, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "lbm_batch_info": ([_ctx, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                        C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                        C.POINTER(C.c_int)], C.c_int),
    "lbm_batch_destroy": ([_ctx], None),
    "lbm_batch_last_error": ([_ctx], C.c_char_p),
    "lbm_mlp_param_count": ([], C.c_int),
    "lbm_mlp_create": ([C.c_int, _vp, C.POINTER(_ctx)], C.c_int),
    "lbm_mlp_train": ([_ctx, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int,
                       C.c_float, C.POINTER(C.c_float)], C.c_int),
    "lbm_mlp_predict": ([_ctx, _vp, C.c_int, _vp, C.c_int, C.c_int], C.c_int),
    "lbm_mlp_gradient": ([_ctx, _vp, C.c_int, _vp, C.c_int, C.c_int, _vp,
                          C.POINTER(C.c_float)], C.c_int),
    "lbm_mlp_get_params": ([_ctx, _vp], C.c_int),
    "lbm_mlp_destroy": ([_ctx], None),
    "lbm_mlp_last_error": ([_ctx], C.c_char_p),
    "lbm_destroy": ([_ctx], None),
    "lbm_last_error": ([_ctx], C.c_char_p),
}

_lib = None


def header_symbols():
    """Function names declared in include/cplbm.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def load():
    """The loaded library with argument and result types declared."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "%s is not built (expected at %s); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`%s"
                % (os.path.basename(LIB_PATH), LIB_PATH,
                   " and `python -m paper_1611_00907_gb300._build --checked`"
                   if _VARIANT else ""))
        lib = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def check(status, ctx=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(ctx)
        raise LbmError(status, msg.decode() if msg else "")
    return status


def check_mlp(status, mlp=None):
    if status != LBM_OK:
        msg = load().lbm_mlp_last_error(mlp)
        raise LbmError(status, msg.decode() if msg else "")
    return status


def check_batch(status, batch=None):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error(batch)
        raise LbmError(status, msg.decode() if msg else "")
    return status
