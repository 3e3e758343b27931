"""FP64 CPU oracle of the MRT-Smagorinsky LBM step (TEST INFRASTRUCTURE ONLY).

This package is the parity oracle for the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA library
(``paper_2512_23116_gb300``) and never imports it.

* ``lbm_oracle.c``   -- the time step, plain C in FP64 (collide in moment space,
  push-stream on two lattices), each function citing the equation it follows;
* ``diagnostics.py`` -- energy spectrum, structure functions / flatness, the
  domain statistics of the turbulent Knudsen number and the derived scales,
  in numpy FP64;
* ``params.py``      -- the parameter chain of Secs. 3.1 and 4
  (nu0 from Re, F0 from Cf and U0, the bare shear rate).

Every function has a pin in ``tests/test_oracle_*.py`` (closed forms,
invariants, brute force on tiny inputs, the paper's worked numbers in
``tests/golden/``); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

FORCE_NONE, FORCE_PAPER_SIN, FORCE_CONST, FORCE_KOLMOGOROV = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c with gcc (FP64, OpenMP) into liblbm_oracle.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(ctypes.c_double)
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, D]
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_init_equilibrium.argtypes = [ctypes.c_void_p, D, D]
        lib.orc_set_populations.argtypes = [ctypes.c_void_p, D]
        lib.orc_get_populations.argtypes = [ctypes.c_void_p, D]
        lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.orc_fields.argtypes = [ctypes.c_void_p, D, D, D, D, ctypes.c_int]
        lib.orc_set_fixed_rate.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_time.restype = ctypes.c_int64
        lib.orc_time.argtypes = [ctypes.c_void_p]
        lib.orc_force_at.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, D]
        lib.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), D]
        lib.orc_moment_matrix.argtypes = [D]
        lib.orc_invert.argtypes = [D, D, ctypes.c_int]
        lib.orc_relaxation_rates.argtypes = [ctypes.c_double, D]
        lib.orc_meq.argtypes = [ctypes.c_double, D, D]
        lib.orc_force_moments_printed.argtypes = [D, D, D]
        lib.orc_guo_source.argtypes = [D, D, D]
        lib.orc_feq_poly.argtypes = [ctypes.c_double, D, D]
        lib.orc_strain.argtypes = [D, ctypes.c_double, ctypes.c_double, D]
        lib.orc_strain_norm.restype = ctypes.c_double
        lib.orc_strain_norm.argtypes = [D]
        lib.orc_collide_one.argtypes = [D, D, ctypes.c_double, ctypes.c_double, ctypes.c_int, D, D]
        lib.orc_strain_norm_selfconsistent.restype = ctypes.c_double
        lib.orc_strain_norm_selfconsistent.argtypes = [D, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_set_strain_mode.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_tau_e.restype = ctypes.c_double
        lib.orc_tau_e.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


# ---- scalar building blocks (App. A, App. B) --------------------------------

def lattice():
    """D3Q19 velocities (19, 3) int and weights (19,) in the paper's order."""
    lib = _load()
    c = (ctypes.c_int * 57)()
    w = np.zeros(19)
    lib.orc_lattice(ctypes.cast(c, ctypes.POINTER(ctypes.c_int)), _dp(w))
    return np.array(list(c), dtype=np.int64).reshape(19, 3), w


def moment_matrix() -> np.ndarray:
    """M of Eq. (moment-matrix), 19 x 19."""
    M = np.zeros(361)
    _load().orc_moment_matrix(_dp(M))
    return M.reshape(19, 19)


def invert(A: np.ndarray) -> np.ndarray:
    """The oracle's own Gauss-Jordan inverse."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    out = np.zeros_like(A)
    if _load().orc_invert(_dp(A), _dp(out), n) != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def relaxation_rates(s_nu: float) -> np.ndarray:
    out = np.zeros(19)
    _load().orc_relaxation_rates(float(s_nu), _dp(out))
    return out


def meq(drho: float, u) -> np.ndarray:
    out = np.zeros(19)
    _load().orc_meq(float(drho), _dp(_vec(u, 3)), _dp(out))
    return out


def force_moments_printed(u, F) -> np.ndarray:
    out = np.zeros(19)
    _load().orc_force_moments_printed(_dp(_vec(u, 3)), _dp(_vec(F, 3)), _dp(out))
    return out


def guo_source(u, F) -> np.ndarray:
    out = np.zeros(19)
    _load().orc_guo_source(_dp(_vec(u, 3)), _dp(_vec(F, 3)), _dp(out))
    return out


def feq_poly(rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    _load().orc_feq_poly(float(rho), _dp(_vec(u, 3)), _dp(out))
    return out


def strain(mneq, s1: float, s9: float) -> np.ndarray:
    """(Sxx, Syy, Szz, Sxy, Sxz, Syz) of Eq. (yu_strain)."""
    out = np.zeros(6)
    _load().orc_strain(_dp(_vec(mneq, 19)), float(s1), float(s9), _dp(out))
    return out


def strain_norm(S) -> float:
    return float(_load().orc_strain_norm(_dp(_vec(S, 6))))


def tau_e(nu0: float, C: float, S_norm: float) -> float:
    return float(_load().orc_tau_e(float(nu0), float(C), float(S_norm)))


def strain_norm_selfconsistent(mneq, s1: float, nu0: float, C: float) -> float:
    """|S| with the local shear rate s_nu(|S|) in Eq. (yu_strain) (fixed point)."""
    return float(_load().orc_strain_norm_selfconsistent(_dp(_vec(mneq, 19)), float(s1), float(nu0), float(C)))


def collide_one(fp, F, nu0: float, C: float, fixed_rate: bool = False):
    """Post-collision f'* (19,) and theta of one cell (Eq. mrt_les_guo)."""
    out = np.zeros(19)
    th = np.zeros(1)
    _load().orc_collide_one(_dp(_vec(fp, 19)), _dp(_vec(F, 3)), float(nu0), float(C),
                            1 if fixed_rate else 0, _dp(out), _dp(th))
    return out, float(th[0])


# ---- the lattice ------------------------------------------------------------

class OracleLBM:
    """Two-lattice FP64 LBM state of shape (nz, ny, nx).

    Arrays exchanged with this class: populations (19, nz, ny, nx) as
    weight-shifted f' = f - w; vectors (3, nz, ny, nx); scalars (nz, ny, nx).
    """

    def __init__(self, nx: int, ny: int, nz: int, nu0: float, C: float,
                 force_mode: int = FORCE_NONE, F0: float = 0.0, body=(0.0, 0.0, 0.0)):
        self._lib = _load()
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nu0, self.C, self.F0 = float(nu0), float(C), float(F0)
        self.force_mode = int(force_mode)
        b = _vec(body, 3)
        self._h = self._lib.orc_create(nx, ny, nz, float(nu0), float(C), int(force_mode),
                                       float(F0), _dp(b))
        if not self._h:
            raise ValueError("orc_create rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def time(self) -> int:
        return int(self._lib.orc_time(self._h))

    def set_fixed_rate(self, fixed: bool) -> None:
        self._lib.orc_set_fixed_rate(self._h, 1 if fixed else 0)

    def set_strain_mode(self, mode: int) -> None:
        """0: explicit (bare s_nu0 in Eq. yu_strain); 1: self-consistent s_nu(|S|)."""
        self._lib.orc_set_strain_mode(self._h, int(mode))

    def init_equilibrium(self, u: np.ndarray, drho: np.ndarray | None = None) -> None:
        """f' = M^-1 m^eq(drho, u) in every cell (initial condition)."""
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, *self.shape)
        d = None if drho is None else _dp(np.ascontiguousarray(drho, dtype=np.float64).reshape(self.shape))
        self._lib.orc_init_equilibrium(self._h, d, _dp(u))

    def set_populations(self, fprime: np.ndarray) -> None:
        f = np.ascontiguousarray(fprime, dtype=np.float64).reshape(19, *self.shape)
        self._lib.orc_set_populations(self._h, _dp(f))

    def populations(self) -> np.ndarray:
        out = np.zeros((19, *self.shape))
        self._lib.orc_get_populations(self._h, _dp(out))
        return out

    def step(self, n: int = 1, threads: int = 0) -> None:
        self._lib.orc_step(self._h, int(n), int(threads))

    def fields(self, threads: int = 0) -> dict:
        """drho, u, |S|, theta = tau_e - 1/2 of the current state."""
        drho = np.zeros(self.shape)
        u = np.zeros((3, *self.shape))
        sn = np.zeros(self.shape)
        th = np.zeros(self.shape)
        self._lib.orc_fields(self._h, _dp(drho), _dp(u), _dp(sn), _dp(th), int(threads))
        return {"drho": drho, "u": u, "snorm": sn, "theta": th}

    def force_field(self) -> np.ndarray:
        F = np.zeros((3, *self.shape))
        tmp = np.zeros(3)
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    self._lib.orc_force_at(self._h, x, y, z, _dp(tmp))
                    F[:, z, y, x] = tmp
        return F


from .params import derive_nu0, forcing_amplitude, bare_shear_rate  # noqa: E402,F401
from . import diagnostics  # noqa: E402,F401
