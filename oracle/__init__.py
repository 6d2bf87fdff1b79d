"""Plain FP64 CPU oracle of the chemical-potential lattice Boltzmann method
(Wen et al., arXiv 1611.00907).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this package; the CUDA library never
does, and this package imports nothing from it.

``cplbm_oracle.c`` holds one time step written out in the paper's order:
density, Eq. 28 wall density, Eq. 8 chemical potential, Eq. 12 force, Eq. 13-14
BGK collision with the velocity-shift forcing of Sec. II, push streaming with
halfway bounce-back (Sec. IV).  ``thermo`` holds the EOS-level helpers
(critical point, Maxwell construction, surface tension) and ``observables``
the post-processing of fields (bulk densities, Laplace pressure jump, contact
angle).
"""
import ctypes as C

import numpy as np

from . import build as _build

EOS_VDW, EOS_CS, EOS_PR, EOS_RKS = 0, 1, 2, 3
EOS_NAMES = {"vdw": EOS_VDW, "cs": EOS_CS, "pr": EOS_PR, "rks": EOS_RKS}

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


class _Eos(C.Structure):
    _fields_ = [("eos", C.c_int), ("a", C.c_double), ("b", C.c_double),
                ("R", C.c_double), ("T", C.c_double), ("alpha", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("walls", C.c_int),
                ("tau", C.c_double), ("kappa", C.c_double), ("eos", _Eos),
                ("mu_bottom", C.c_double), ("top_mode", C.c_int),
                ("mu_top", C.c_double)]


_lib = None


def lib():
    """The oracle's shared library, compiled on first use."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        pe, pp = C.POINTER(_Eos), C.POINTER(_Params)
        for name, args, res in [
            ("orc_psi", [pe, C.c_double], C.c_double),
            ("orc_mu_bulk", [pe, C.c_double], C.c_double),
            ("orc_p0", [pe, C.c_double], C.c_double),
            ("orc_eos_eval", [pe, dp, C.c_long, dp, dp, dp], None),
            ("orc_density", [pp, dp, dp], None),
            ("orc_wall_density", [pp, dp], None),
            ("orc_laplacian", [pp, dp, dp], None),
            ("orc_gradient", [pp, dp, dp, dp], None),
            ("orc_chem_potential", [pp, dp, dp], None),
            ("orc_force", [pp, dp, dp, dp, dp], None),
            ("orc_equilibrium", [C.c_double, C.c_double, C.c_double, dp],
             None),
            ("orc_collide_node", [dp, C.c_double, C.c_double, C.c_double, dp],
             None),
            ("orc_stream", [pp, dp, dp], None),
            ("orc_step", [pp, dp, C.c_int], C.c_int),
            ("orc_step_pressure_tensor", [pp, dp, C.c_int], C.c_int),
            ("orc_force_pressure_tensor", [pp, dp, dp, dp], None),
            ("orc_moments", [pp, dp, dp, dp, dp, dp, dp, dp], C.c_int),
            ("orc_init_equilibrium", [pp, dp, dp, dp, dp], None),
            ("orc_set_threads", [C.c_int], None),
            ("orc_get_threads", [], C.c_int),
        ]:
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n: int) -> None:
    """Threads used by the oracle's row loops (default 1)."""
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------------------
# Equation of state
# ---------------------------------------------------------------------------
class Eos:
    """One of the paper's EOS with absolute temperature T and alpha(T).

    Use ``oracle.thermo.make_eos`` to build one from a reduced temperature.
    """

    def __init__(self, kind, a, b, R, T, alpha=1.0):
        self.kind = EOS_NAMES[kind] if isinstance(kind, str) else int(kind)
        self.a, self.b, self.R, self.T, self.alpha = (
            float(a), float(b), float(R), float(T), float(alpha))

    def _c(self):
        return _Eos(self.kind, self.a, self.b, self.R, self.T, self.alpha)

    def eval(self, rho):
        """(psi, psi', p0) at the densities rho (printed Eqs. 16-27)."""
        r = np.ascontiguousarray(np.atleast_1d(rho), dtype=np.float64)
        psi, mu, p0 = (np.empty_like(r) for _ in range(3))
        e = self._c()
        lib().orc_eos_eval(C.byref(e), _ptr(r), r.size, _ptr(psi), _ptr(mu),
                           _ptr(p0))
        shape = np.shape(rho)
        return psi.reshape(shape), mu.reshape(shape), p0.reshape(shape)

    def psi(self, rho):
        return self.eval(rho)[0]

    def mu(self, rho):
        return self.eval(rho)[1]

    def p0(self, rho):
        return self.eval(rho)[2]


# ---------------------------------------------------------------------------
# Lattice state and the step
# ---------------------------------------------------------------------------
class Lattice:
    """An nx x ny D2Q9 domain with the oracle's FP64 state f[9, ny, nx].

    walls=False: fully periodic.  walls=True: rows 0 and ny-1 are solid with
    surface chemical potentials (mu_bottom; top copies its neighbour when
    top_mode == 0, else mu_top), x periodic.
    """

    def __init__(self, nx, ny, eos, tau, kappa, walls=False, mu_bottom=0.0,
                 top_mode=0, mu_top=0.0):
        self.nx, self.ny, self.eos = int(nx), int(ny), eos
        self.tau, self.kappa, self.walls = float(tau), float(kappa), bool(walls)
        self.mu_bottom, self.top_mode, self.mu_top = (
            float(mu_bottom), int(top_mode), float(mu_top))
        self.f = np.zeros((9, self.ny, self.nx))

    def params(self):
        return _Params(self.nx, self.ny, int(self.walls), self.tau, self.kappa,
                       self.eos._c(), self.mu_bottom, self.top_mode,
                       self.mu_top)

    def fluid_rows(self):
        return slice(1, self.ny - 1) if self.walls else slice(0, self.ny)

    def field(self):
        return np.zeros((self.ny, self.nx))

    # --- state --------------------------------------------------------------
    def init_equilibrium(self, rho, ux=None, uy=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        ux = None if ux is None else np.ascontiguousarray(ux, np.float64)
        uy = None if uy is None else np.ascontiguousarray(uy, np.float64)
        p = self.params()
        lib().orc_init_equilibrium(C.byref(p), _ptr(rho), _ptr(ux), _ptr(uy),
                                   _ptr(self.f))
        return self

    def step(self, n=1):
        p = self.params()
        rc = lib().orc_step(C.byref(p), _ptr(self.f), int(n))
        if rc != 0:
            raise MemoryError("oracle step: allocation failed")
        return self

    def step_pressure_tensor(self, n=1):
        """n steps with the pressure-tensor force of Eq. 5 (periodic only)."""
        p = self.params()
        rc = lib().orc_step_pressure_tensor(C.byref(p), _ptr(self.f), int(n))
        if rc == -2:
            raise ValueError("the pressure-tensor form has no wall rule")
        if rc != 0:
            raise MemoryError("oracle step: allocation failed")
        return self

    def force_pressure_tensor(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        Fx, Fy = self.field(), self.field()
        p = self.params()
        lib().orc_force_pressure_tensor(C.byref(p), _ptr(rho), _ptr(Fx),
                                        _ptr(Fy))
        return Fx, Fy

    def moments(self):
        """dict of rho, vx, vy, mu, Fx, Fy ([ny, nx] each)."""
        out = {k: self.field() for k in ("rho", "vx", "vy", "mu", "Fx", "Fy")}
        p = self.params()
        rc = lib().orc_moments(C.byref(p), _ptr(self.f), _ptr(out["rho"]),
                               _ptr(out["vx"]), _ptr(out["vy"]),
                               _ptr(out["mu"]), _ptr(out["Fx"]),
                               _ptr(out["Fy"]))
        if rc != 0:
            raise MemoryError("oracle moments: allocation failed")
        return out

    # --- pieces, for pinning each step of the method separately ------------
    def density(self, f=None):
        out = self.field()
        p = self.params()
        f = self.f if f is None else np.ascontiguousarray(f)
        lib().orc_density(C.byref(p), _ptr(f), _ptr(out))
        return out

    def wall_density(self, rho):
        rho = np.array(rho, dtype=np.float64, order="C")
        p = self.params()
        lib().orc_wall_density(C.byref(p), _ptr(rho))
        return rho

    def laplacian(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        out = self.field()
        p = self.params()
        lib().orc_laplacian(C.byref(p), _ptr(phi), _ptr(out))
        return out

    def gradient(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        gx, gy = self.field(), self.field()
        p = self.params()
        lib().orc_gradient(C.byref(p), _ptr(phi), _ptr(gx), _ptr(gy))
        return gx, gy

    def chem_potential(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        out = self.field()
        p = self.params()
        lib().orc_chem_potential(C.byref(p), _ptr(rho), _ptr(out))
        return out

    def force(self, rho, mu):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        Fx, Fy = self.field(), self.field()
        p = self.params()
        lib().orc_force(C.byref(p), _ptr(rho), _ptr(mu), _ptr(Fx), _ptr(Fy))
        return Fx, Fy

    def stream(self, fpost):
        fpost = np.ascontiguousarray(fpost, dtype=np.float64)
        out = np.zeros_like(self.f)
        p = self.params()
        lib().orc_stream(C.byref(p), _ptr(fpost), _ptr(out))
        return out


def equilibrium(rho, ux, uy):
    """Eq. 14 populations (9,) for one node."""
    out = np.empty(9)
    lib().orc_equilibrium(float(rho), float(ux), float(uy), _ptr(out))
    return out


def collide_node(f, Fx, Fy, tau):
    """Post-collision populations (9,) of one node (Eq. 13, velocity shift)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty(9)
    lib().orc_collide_node(_ptr(f), float(Fx), float(Fy), float(tau),
                           _ptr(out))
    return out
