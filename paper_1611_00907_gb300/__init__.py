"""GB300 implementation of the chemical-potential lattice Boltzmann method
for nonideal fluids (Wen et al., arXiv 1611.00907).

The numerical work runs in libcplbm.so (CUDA, sm_103a) behind the C ABI of
include/cplbm.h; this module only marshals arguments.  PyTorch is used for
device buffers and the CUDA stream when the caller passes CUDA tensors.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import EOS, PRECISION, LbmError, check

__all__ = ["Simulation", "Batch", "LbmError", "eos_critical",
           "eos_coexistence", "eos_pressure", "tile_kinds", "EOS", "PRECISION"]


def eos_critical(eos, a, b, R=1.0):
    """(T_c, rho_c) of an EOS with alpha = 1, from the library."""
    lib = _lib.load()
    Tc, rc = C.c_double(), C.c_double()
    check(lib.lbm_eos_critical(EOS[eos] if isinstance(eos, str) else int(eos),
                               float(a), float(b), float(R), C.byref(Tc),
                               C.byref(rc)))
    return Tc.value, rc.value


def eos_coexistence(eos, a, b, R=1.0, Tr=0.85, omega=0.344):
    """(rho_v, rho_l, mu_coex) of the Maxwell construction, from the library."""
    lib = _lib.load()
    v, l, m = C.c_double(), C.c_double(), C.c_double()
    check(lib.lbm_eos_coexistence(EOS[eos] if isinstance(eos, str) else int(eos),
                                  float(a), float(b), float(R), float(Tr),
                                  float(omega), C.byref(v), C.byref(l),
                                  C.byref(m)))
    return v.value, l.value, m.value


def eos_pressure(eos, a, b, R=1.0, Tr=0.85, omega=0.344, rho=None):
    """Bulk pressure p0(rho) of the EOS (array in, array out), from the
    library."""
    lib = _lib.load()
    r = np.ascontiguousarray(rho, dtype=np.float64)
    p = np.empty_like(r)
    check(lib.lbm_eos_pressure(EOS[eos] if isinstance(eos, str) else int(eos),
                               float(a), float(b), float(R), float(Tr),
                               float(omega), r.ctypes.data, p.ctypes.data,
                               r.size))
    return p


def tile_kinds(nx, ny, walls=False, tile=(32, 32), seams=True):
    """Path class of every tile of the fused step, [nty][ntx]: 2 interior,
    1 seam (halo wraps a periodic edge; TMA paths), 0 general.  seams=False
    gives a batch's classes.  From the library; no device work."""
    lib = _lib.load()
    tx, ty = tile
    nyf = ny - 2 if walls else ny
    ntx, nty = -(-nx // tx), -(-nyf // ty)
    out = np.zeros((max(nty, 1), max(ntx, 1)), dtype=np.int32)
    check(lib.lbm_tile_kinds(int(nx), int(ny), int(bool(walls)), int(tx), int(ty),
                             int(bool(seams)), out.ctypes.data, out.size))
    return out


def _default_device(device):
    """device, or PyTorch's current CUDA device when None (0 without
    PyTorch or CUDA): under torchrun each rank's set_device is followed."""
    if device is not None:
        return int(device)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_device()
    except ImportError:
        pass
    return 0


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arg(x, n):
    """(pointer, on_device, keepalive) for a [ny][nx] float64 field."""
    if x is None:
        return None, None, None
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != n:
            raise ValueError("device fields must be contiguous float64 [ny, nx]")
        return x.data_ptr(), 1 if x.is_cuda else 0, x
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.size != n:
        raise ValueError("field has %d values, expected %d" % (a.size, n))
    return a.ctypes.data, 0, a


class Simulation:
    """One D2Q9 lattice on one GPU.

    Parameters follow the paper: eos in {'vdw', 'cs', 'pr', 'rks'} with a, b,
    R (Sec. III), reduced temperature Tr = T / T_c, acentric factor omega
    (PR, RKS), relaxation time tau (Eq. 13), kappa (Eq. 8).  walls=True puts
    solid rows at y = 0 and y = ny - 1 with surface chemical potential
    mu_bottom (top: copies its neighbour, top_mode=0, or mu_top, top_mode=1).
    precision in {'f64', 'f32', 'f32_offset', 'f16_offset'}; rho_ref is the
    reference density of the offset storages.
    """

    def __init__(self, nx, ny, eos="cs", a=1.0, b=4.0, R=1.0, Tr=0.85,
                 omega=0.344, tau=1.0, kappa=0.5, walls=False,
                 precision="f64", rho_ref=0.0, mu_bottom=0.0, top_mode=0,
                 mu_top=0.0, device=None, stream=None):
        self._lib = _lib.load()
        self.nx, self.ny, self.walls = int(nx), int(ny), bool(walls)
        self.precision = precision
        self.device = _default_device(device)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(self.device).cuda_stream
            except ImportError:
                stream = None
        cfg = _lib.LbmConfig(self.nx, self.ny, int(self.walls), float(tau),
                             float(kappa), float(rho_ref), PRECISION[precision],
                             C.c_void_p(stream) if stream else None,
                             self.device)
        ctx = C.c_void_p()
        check(self._lib.lbm_create(C.byref(cfg), C.byref(ctx)))
        self._ctx = ctx
        try:
            check(self._lib.lbm_set_eos(ctx, EOS[eos], float(a), float(b),
                                        float(R), float(Tr), float(omega)),
                  ctx)
            check(self._lib.lbm_set_wall_mu(ctx, float(mu_bottom),
                                            int(top_mode), float(mu_top)), ctx)
        except Exception:
            self.close()
            raise

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.lbm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n(self):
        return self.nx * self.ny

    def _check(self, status):
        return check(status, self._ctx)

    # ------------------------------------------------------------------
    def set_wall_mu(self, mu_bottom, top_mode=0, mu_top=0.0):
        self._check(self._lib.lbm_set_wall_mu(self._ctx, float(mu_bottom),
                                              int(top_mode), float(mu_top)))

    def set_force_model(self, model):
        """'chemical_potential' (Eq. 12, default) or 'pressure_tensor' (the
        Eq. 5 baseline: periodic, f32 / f64)."""
        m = {"chemical_potential": 0, "pressure_tensor": 1}[model]
        self._check(self._lib.lbm_set_force_model(self._ctx, m))
        return self

    def set_tile(self, tx, ty):
        """Tile shape of the step kernel (speed only; results unchanged)."""
        self._check(self._lib.lbm_set_tile(self._ctx, int(tx), int(ty)))
        return self

    def autotune(self, nsteps=20):
        """Time every tile shape on this lattice, keep the fastest; the state
        is left unchanged.  Returns the shape."""
        tx, ty = C.c_int(), C.c_int()
        self._check(self._lib.lbm_autotune(self._ctx, int(nsteps), C.byref(tx),
                                           C.byref(ty)))
        return tx.value, ty.value

    @property
    def tile(self):
        tx, ty = C.c_int(), C.c_int()
        self._check(self._lib.lbm_get_tile(self._ctx, C.byref(tx), C.byref(ty)))
        return tx.value, ty.value

    def init(self, rho, ux=None, uy=None):
        """Equilibrium state (Eq. 14) from [ny, nx] float64 fields given as
        numpy arrays (host) or CUDA tensors (device)."""
        pr, dr, kr = _arg(rho, self.n)
        px, dx, kx = _arg(ux, self.n)
        py, dy, ky = _arg(uy, self.n)
        kinds = {d for d in (dr, dx, dy) if d is not None}
        if len(kinds) != 1:
            raise ValueError("rho, ux, uy must all be host or all device")
        self._check(self._lib.lbm_init(self._ctx, pr, px, py, dr))
        del kr, kx, ky
        return self

    def step(self, n=1):
        self._check(self._lib.lbm_step(self._ctx, int(n)))
        return self

    @property
    def step_count(self):
        return int(self._lib.lbm_step_count(self._ctx))

    def eos_info(self):
        """dict(T, alpha, Tc, rhoc) of the selected EOS."""
        v = [C.c_double() for _ in range(4)]
        self._check(self._lib.lbm_eos_info(self._ctx, *[C.byref(x) for x in v]))
        return dict(zip(("T", "alpha", "Tc", "rhoc"), (x.value for x in v)))

    def moments(self, device=False, fields=("rho", "vx", "vy", "mu"), out=None):
        """dict of the requested fields among rho, vx, vy, mu [ny, nx] float64:
        numpy arrays, or CUDA tensors when device=True.  Only the requested
        fields are computed and copied.  out: optional dict of C-contiguous
        float64 arrays [ny, nx] to write into (host arrays, e.g. views of
        pinned memory, for device=False; CUDA tensors for device=True)."""
        names = ("rho", "vx", "vy", "mu")
        if any(k not in names for k in fields):
            raise ValueError("fields must be among %s" % (names,))
        out = dict(out or {})
        ptr = []
        for k in names:
            if k not in fields:
                ptr.append(None)
                continue
            a = out.get(k)
            if a is None:
                if device:
                    import torch
                    a = torch.empty((self.ny, self.nx), dtype=torch.float64,
                                    device="cuda:%d" % self.device)
                else:
                    a = np.empty((self.ny, self.nx))
                out[k] = a
            if device:
                ok = (tuple(a.shape) == (self.ny, self.nx) and a.is_cuda and
                      a.is_contiguous() and str(a.dtype) == "torch.float64")
                ptr.append(a.data_ptr() if ok else None)
            else:
                ok = (a.shape == (self.ny, self.nx) and a.dtype == np.float64
                      and a.flags["C_CONTIGUOUS"] and a.flags["WRITEABLE"])
                ptr.append(a.ctypes.data if ok else None)
            if not ok:
                raise ValueError("out[%r] must be a contiguous float64 [ny, nx] "
                                 "%s array" % (k, "CUDA" if device else "host"))
        self._check(self._lib.lbm_moments(self._ctx, *ptr, 1 if device else 0))
        return {k: out[k] for k in names if k in fields}

    def populations(self):
        """Natural-order FP64 distributions [9, ny, nx] (numpy)."""
        f = np.empty((9, self.ny, self.nx))
        self._check(self._lib.lbm_get_populations(self._ctx, f.ctypes.data, 0))
        return f

    def reduce(self):
        """(mass, momentum x, momentum y, max |rho - rho at last call|)."""
        out = (C.c_double * 4)()
        self._check(self._lib.lbm_reduce(self._ctx, out))
        return tuple(out)

    def get_state(self):
        n = self._lib.lbm_state_size(self._ctx)
        buf = np.empty(n, dtype=np.uint8)
        self._check(self._lib.lbm_get_state(self._ctx, buf.ctypes.data, n))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self._lib.lbm_set_state(self._ctx, buf.ctypes.data,
                                            buf.size))
        return self


class Batch:
    """Many independent lattices advanced together (one kernel launch per
    step over all their tiles, blocks of steps replayed from a CUDA graph).

    instances: list of dicts with keys nx, ny and optionally walls, tau,
    kappa, rho_ref, eos, a, b, R, Tr, omega, mu_bottom, top_mode, mu_top
    (defaults as for Simulation).  All share one precision.
    """

    DEFAULTS = dict(walls=False, tau=1.0, kappa=0.5, rho_ref=0.0, eos="cs",
                    a=1.0, b=4.0, R=1.0, Tr=0.85, omega=0.344, mu_bottom=0.0,
                    top_mode=0, mu_top=0.0)

    def __init__(self, instances, precision="f32", device=None, stream=None):
        self._lib = _lib.load()
        self.device = _default_device(device)
        self.specs = []
        arr = (_lib.LbmInstance * len(instances))()
        for k, spec in enumerate(instances):
            d = dict(self.DEFAULTS)
            d.update(spec)
            self.specs.append(d)
            arr[k] = _lib.LbmInstance(
                int(d["nx"]), int(d["ny"]), int(bool(d["walls"])),
                float(d["tau"]), float(d["kappa"]), float(d["rho_ref"]),
                EOS[d["eos"]] if isinstance(d["eos"], str) else int(d["eos"]),
                float(d["a"]), float(d["b"]), float(d["R"]), float(d["Tr"]),
                float(d["omega"]), float(d["mu_bottom"]), int(d["top_mode"]),
                float(d["mu_top"]))
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    s = torch.cuda.current_stream(self.device).cuda_stream
                    stream = s if s else None
            except ImportError:
                stream = None
        handle = C.c_void_p()
        _lib.check_batch(self._lib.lbm_batch_create(
            arr, len(instances), PRECISION[precision],
            C.c_void_p(stream) if stream else None, self.device,
            C.byref(handle)))
        self._b = handle
        self.precision = precision

    def close(self):
        if getattr(self, "_b", None):
            self._lib.lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.specs)

    def _check(self, status):
        return _lib.check_batch(status, self._b)

    def init(self, index, rho, ux=None, uy=None):
        d = self.specs[index]
        n = int(d["nx"]) * int(d["ny"])
        pr, dr, kr = _arg(rho, n)
        px, _, kx = _arg(ux, n)
        py, _, ky = _arg(uy, n)
        self._check(self._lib.lbm_batch_init(self._b, int(index), pr, px, py, dr))
        del kr, kx, ky
        return self

    def step(self, n=1):
        self._check(self._lib.lbm_batch_step(self._b, int(n)))
        return self

    def set_active(self, index, active=True):
        """Take a lattice out of the launch (or put it back); after an even
        number of batch steps."""
        self._check(self._lib.lbm_batch_set_active(self._b, int(index),
                                                   1 if active else 0))
        return self

    def moments(self, index, fields=("rho", "vx", "vy", "mu")):
        """dict of the requested fields among rho, vx, vy, mu of lattice
        `index` (numpy [ny, nx]); only those are computed and copied."""
        d = self.specs[index]
        shape = (int(d["ny"]), int(d["nx"]))
        names = ("rho", "vx", "vy", "mu")
        if any(k not in names for k in fields):
            raise ValueError("fields must be among %s" % (names,))
        out = {k: np.empty(shape) for k in names if k in fields}
        ptr = [out[k].ctypes.data if k in out else None for k in names]
        self._check(self._lib.lbm_batch_moments(self._b, int(index), *ptr, 0))
        return out

    def populations(self, index):
        d = self.specs[index]
        f = np.empty((9, int(d["ny"]), int(d["nx"])))
        self._check(self._lib.lbm_batch_populations(self._b, int(index),
                                                    f.ctypes.data, 0))
        return f

    def reduce(self, index):
        out = (C.c_double * 4)()
        self._check(self._lib.lbm_batch_reduce(self._b, int(index), out))
        return tuple(out)

    def set_tile(self, tx, ty):
        self._check(self._lib.lbm_batch_set_tile(self._b, int(tx), int(ty)))
        return self

    @property
    def items_per_cta(self):
        """Work items (tiles) each CTA of the batched kernel takes; 0: one
        grid row per lattice for groups of one geometry (lbm_batch_schedule)."""
        cur = C.c_int()
        self._check(self._lib.lbm_batch_schedule(self._b, -1, C.byref(cur)))
        return cur.value

    @items_per_cta.setter
    def items_per_cta(self, k):
        self._check(self._lib.lbm_batch_schedule(self._b, int(k), None))

    def autotune(self, nsteps=10):
        tx, ty = C.c_int(), C.c_int()
        self._check(self._lib.lbm_batch_autotune(self._b, int(nsteps),
                                                 C.byref(tx), C.byref(ty)))
        return tx.value, ty.value

    def info(self):
        cnt, nodes, steps = C.c_int(), C.c_longlong(), C.c_longlong()
        tx, ty = C.c_int(), C.c_int()
        self._check(self._lib.lbm_batch_info(self._b, C.byref(cnt),
                                             C.byref(nodes), C.byref(steps),
                                             C.byref(tx), C.byref(ty)))
        return dict(count=cnt.value, nodes=nodes.value, steps=steps.value,
                    tile=(tx.value, ty.value))
