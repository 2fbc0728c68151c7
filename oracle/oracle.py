"""ctypes binding of the FP64 CPU oracle (``lb_oracle.c``).  Test infrastructure only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "liblboracle.so")
_lock = threading.Lock()
_lib = None

GRID_FIELDS = [("nx", C.c_int), ("ny", C.c_int), ("bc_bottom", C.c_int), ("bc_top", C.c_int),
               ("T_bottom", C.c_double), ("T_top", C.c_double), ("T_bottom_amp", C.c_double),
               ("T_bottom_modes", C.c_int), ("cos_theta_bottom", C.c_double), ("cos_theta_top", C.c_double)]
PARAM_FIELDS = [(k, C.c_double) for k in (
    "rho_l", "rho_s", "rho_g", "mu_l", "mu_s", "mu_g", "lam_l", "lam_s", "lam_g",
    "cp_l", "cp_s", "cp_g", "latent", "T_sol", "T_liq", "k_p", "D_l", "D_s", "eps", "mobility",
    "sigma0", "sigma_T", "sigma_c", "T_ref", "c_ref", "gx", "gy")] + [
    ("fs_modulated_st", C.c_int), ("phase_change_on", C.c_int), ("divu_mode", C.c_int), ("lattice_fl", C.c_int),
    ("rhocp_rule", C.c_int)]


class _Grid(C.Structure):
    _fields_ = GRID_FIELDS


class _Params(C.Structure):
    _fields_ = PARAM_FIELDS


_dp = C.POINTER(C.c_double)


def build_oracle(force: bool = False) -> str:
    """Compile lb_oracle.c into liblboracle.so (gcc, -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lb_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            L = C.CDLL(_LIB)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(_Grid), C.POINTER(_Params), _dp, _dp, _dp, _dp, _dp]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_fields.argtypes = [C.c_void_p] + [_dp] * 8
            L.orc_reduce.argtypes = [C.c_void_p, _dp]
            L.orc_step_count.restype = C.c_long
            L.orc_step_count.argtypes = [C.c_void_p]
            L.orc_get_populations.argtypes = [C.c_void_p, C.c_int, _dp]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            L.orc_zeta.restype = C.c_double
            L.orc_zeta.argtypes = [C.c_double] * 5
            L.orc_enthalpy_invert.argtypes = [C.POINTER(_Params), C.c_double, C.c_double, _dp, _dp]
            L.orc_enthalpy_forward.restype = C.c_double
            L.orc_enthalpy_forward.argtypes = [C.POINTER(_Params), C.c_double, C.c_double]
            L.orc_equilibria.argtypes = [C.POINTER(_Params)] + [C.c_double] * 9 + [_dp] * 4
            L.orc_sources.argtypes = [C.c_double] * 21 + [_dp] * 4
            L.orc_stencil_field.argtypes = [C.POINTER(_Grid), _dp, C.c_int, _dp, _dp, _dp]
            _lib = L
    return _lib


def _grid(g: dict) -> _Grid:
    s = _Grid()
    for k, _ in GRID_FIELDS:
        setattr(s, k, g.get(k, 0))
    return s


def _params(p: dict) -> _Params:
    s = _Params()
    for k, _ in PARAM_FIELDS:
        setattr(s, k, p.get(k, 0) if k in ("divu_mode", "lattice_fl", "rhocp_rule") else p[k])
    return s


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError("field has %d values, expected %d" % (a.size, n))
    return a


class Oracle:
    """Whole-lattice FP64 LB state.  ``fields`` holds phi, T, C and optionally ux, uy,
    each ny*nx (row-major, x fastest)."""

    def __init__(self, grid: dict, params: dict, fields: dict):
        L = lib()
        self.nx, self.ny = int(grid["nx"]), int(grid["ny"])
        n = self.nx * self.ny
        self._g, self._p = _grid(grid), _params(params)
        arrs = [_f64(fields[k], n) for k in ("phi", "T", "C")]
        ux = _f64(fields["ux"], n) if fields.get("ux") is not None else np.zeros(n)
        uy = _f64(fields["uy"], n) if fields.get("uy") is not None else np.zeros(n)
        self._keep = arrs + [ux, uy]
        h = L.orc_create(C.byref(self._g), C.byref(self._p), *[_ptr(a) for a in self._keep])
        if not h:
            raise ValueError("oracle rejected the grid")
        self._h = C.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(lib().orc_step_count(self._h))

    def fields(self) -> dict:
        n = self.nx * self.ny
        out = {k: np.empty(n) for k in ("phi", "T", "fs", "C", "ux", "uy", "p", "rhoH")}
        lib().orc_fields(self._h, *[_ptr(out[k]) for k in ("phi", "T", "fs", "C", "ux", "uy", "p", "rhoH")])
        return {k: v.reshape(self.ny, self.nx) for k, v in out.items()}

    def reduce(self) -> np.ndarray:
        out = np.empty(8)
        lib().orc_reduce(self._h, _ptr(out))
        return out

    def populations(self, which: int) -> np.ndarray:
        """Populations of set 0..3 (f, g, h, l) as (9, ny, nx)."""
        out = np.empty(9 * self.nx * self.ny)
        lib().orc_get_populations(self._h, int(which), _ptr(out))
        return out.reshape(9, self.ny, self.nx)


def set_threads(k: int):
    lib().orc_set_num_threads(int(k))


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---- building blocks (for the invariant pins) -------------------------------------------

def zeta(phi, fs, zl, zs, zg) -> float:
    return lib().orc_zeta(phi, fs, zl, zs, zg)


def enthalpy_invert(params: dict, e: float, chi: float):
    T, fs = C.c_double(), C.c_double()
    p = _params(params)
    lib().orc_enthalpy_invert(C.byref(p), e, chi, C.byref(T), C.byref(fs))
    return T.value, fs.value


def enthalpy_forward(params: dict, T: float, chi: float) -> float:
    p = _params(params)
    return lib().orc_enthalpy_forward(C.byref(p), T, chi)


def equilibria(params: dict, phi, Cc, rhoH, T, pr, ux, uy, rho, rhocp):
    out = [np.empty(9) for _ in range(4)]
    p = _params(params)
    lib().orc_equilibria(C.byref(p), phi, Cc, rhoH, T, pr, ux, uy, rho, rhocp, *[_ptr(a) for a in out])
    return tuple(out)


def sources(**kw):
    names = ["dphiux", "dphiuy", "nx", "ny", "phi", "eps", "mdot", "S", "Fx", "Fy", "rfx", "rfy",
             "Ftx", "Fty", "ux", "uy", "Q", "dCux", "dCuy", "Rx", "Ry"]
    out = [np.empty(9) for _ in range(4)]
    lib().orc_sources(*[float(kw.get(k, 0.0)) for k in names], *[_ptr(a) for a in out])
    return tuple(out)


def stencil_field(grid: dict, v: np.ndarray, kind: int):
    """Gradient and Laplacian of a (ny, nx) field with the oracle's wall ghosts;
    kind 0 mirror, 1 temperature (Dirichlet walls extrapolate)."""
    g = _grid(grid)
    v = np.ascontiguousarray(v, dtype=np.float64)
    gx, gy, lap = (np.empty_like(v) for _ in range(3))
    lib().orc_stencil_field(C.byref(g), _ptr(v), int(kind), _ptr(gx), _ptr(gy), _ptr(lap))
    return gx, gy, lap
