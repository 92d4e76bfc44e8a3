"""ctypes front end of the plain-C FP64 oracle march (test infrastructure only).

The arithmetic lives in ``lbm_oracle.c`` (scheme of Eqs. 1, 5-9 with the
paper's first-order splitting / upwind / explicit-Euler discretisation; the
readings are listed in that file's header).  This module only builds the
shared object, marshals numpy arrays and offers a ``Problem`` convenience
wrapper.  Pinned by tests that use closed forms, conservation, symmetry and an
independent matrix assembly of the same scheme (``fixed_point``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

COUETTE, CAVITY = 0, 1


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into liboracle.so next to it (gcc, OpenMP over cells)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("xi_x", ctypes.POINTER(ctypes.c_double)),
                ("xi_y", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
                ("geom", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("kn", ctypes.c_double), ("u_bottom", ctypes.c_double), ("u_top", ctypes.c_double),
                ("cfl", ctypes.c_double)]


class _Coeffs(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("omega", ctypes.c_double), ("u_ref", ctypes.c_double),
                ("d_x", ctypes.c_double), ("d_y", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, C = ctypes.POINTER(_Problem), ctypes.POINTER(_Coeffs)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.orc_coeffs_compute.argtypes = [P, C]
        lib.orc_coeffs_compute.restype = ctypes.c_int
        lib.orc_step.argtypes = [P, C, dp, dp]
        lib.orc_step.restype = None
        lib.orc_relax.argtypes = [P, C, dp, dp, ctypes.c_double]
        lib.orc_relax.restype = None
        lib.orc_relax_exp.argtypes = [P, C, dp, dp, ctypes.c_double]
        lib.orc_relax_exp.restype = None
        lib.orc_transport2.argtypes = [P, C, dp, dp]
        lib.orc_transport2.restype = None
        lib.orc_face_flux2_y.argtypes = [P, C, dp, dp]
        lib.orc_face_flux2_y.restype = None
        lib.orc_face_flux2_x.argtypes = [P, C, dp, dp]
        lib.orc_face_flux2_x.restype = None
        lib.orc_step_cells.argtypes = [P, C, dp, lp, ctypes.c_long, dp]
        lib.orc_step_cells.restype = None
        lib.orc_step2_cells.argtypes = [P, C, dp, lp, ctypes.c_long, dp]
        lib.orc_step2_cells.restype = None
        lib.orc_residual.argtypes = [dp, dp, ctypes.c_long, dp, dp]
        lib.orc_residual.restype = ctypes.c_double
        lib.orc_march.argtypes = [P, C, dp, ctypes.c_long, ctypes.c_long, ctypes.c_double, dp]
        lib.orc_march.restype = ctypes.c_long
        lib.orc_moments.argtypes = [P, C, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_moments.restype = None
        lib.orc_face_flux_y.argtypes = [P, C, dp, dp]
        lib.orc_face_flux_y.restype = None
        lib.orc_face_flux_x.argtypes = [P, C, dp, dp]
        lib.orc_face_flux_x.restype = None
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """One boundary-value problem of the paper: Couette channel or lid-driven cavity."""
    xi_x: np.ndarray
    xi_y: np.ndarray
    w: np.ndarray
    geom: int
    nx: int
    ny: int
    kn: float
    u_bottom: float
    u_top: float
    cfl: float = 0.9

    def __post_init__(self):
        self.xi_x = np.ascontiguousarray(self.xi_x, dtype=np.float64)
        self.xi_y = np.ascontiguousarray(self.xi_y, dtype=np.float64)
        self.w = np.ascontiguousarray(self.w, dtype=np.float64)
        self._p = _Problem(len(self.w), _dp(self.xi_x), _dp(self.xi_y), _dp(self.w), self.geom,
                           self.nx, self.ny, self.kn, self.u_bottom, self.u_top, self.cfl)
        self._c = _Coeffs()
        if _load().orc_coeffs_compute(ctypes.byref(self._p), ctypes.byref(self._c)) != 0:
            raise ValueError("invalid problem")

    @property
    def n(self) -> int:
        return len(self.w)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    @property
    def coeffs(self) -> dict:
        return {k: getattr(self._c, k) for k, _ in _Coeffs._fields_}

    def zeros(self) -> np.ndarray:
        return np.zeros((self.n, self.ncells), dtype=np.float64)

    def step(self, h: np.ndarray, nsteps: int = 1, omega: float | None = None) -> np.ndarray:
        """Return the state after `nsteps` steps (h is not modified); `omega` replaces the
        relaxation factor dt/Kn of the relaxation sub-step if given."""
        lib = _load()
        c = self._c
        if omega is not None:
            c = _Coeffs()
            ctypes.pointer(c)[0] = self._c
            c.omega = float(omega)
        cur = np.ascontiguousarray(h, dtype=np.float64).copy()
        nxt = np.empty_like(cur)
        for _ in range(nsteps):
            lib.orc_step(ctypes.byref(self._p), ctypes.byref(c), _dp(cur), _dp(nxt))
            cur, nxt = nxt, cur
        return cur

    def relax(self, h: np.ndarray, frac: float) -> np.ndarray:
        """Relaxation alone over frac * dt (explicit Euler, cell-local)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty_like(h)
        _load().orc_relax(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out), float(frac))
        return out

    def step_strang(self, h: np.ndarray, nsteps: int = 1) -> np.ndarray:
        """`nsteps` steps of the symmetric splitting relaxation(dt/2), transport(dt),
        relaxation(dt/2), composed literally from the relaxation and transport operators of
        this oracle (the transport+relaxation step run with omega halved supplies the
        transport and the second half step)."""
        cur = np.ascontiguousarray(h, dtype=np.float64).copy()
        for _ in range(nsteps):
            cur = self.step(self.relax(cur, 0.5), 1, omega=0.5 * self._c.omega)
        return cur

    def relax_exp(self, h: np.ndarray, frac: float) -> np.ndarray:
        """Relaxation alone over frac * dt, exact exponential decay to the equilibrium."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty_like(h)
        _load().orc_relax_exp(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out), float(frac))
        return out

    def transport2(self, h: np.ndarray) -> np.ndarray:
        """Second-order (Beam-Warming flux) transport alone over dt."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty_like(h)
        _load().orc_transport2(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out))
        return out

    def face_flux2_y(self, h: np.ndarray) -> np.ndarray:
        """x-momentum flux through horizontal faces with the second-order transport's face
        values, shape (ny+1, nx)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty((self.ny + 1) * self.nx)
        _load().orc_face_flux2_y(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out))
        return out.reshape(self.ny + 1, self.nx)

    def face_flux2_x(self, h: np.ndarray) -> np.ndarray:
        """Same through vertical faces (cavity), shape (ny, nx+1)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty(self.ny * (self.nx + 1))
        _load().orc_face_flux2_x(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out))
        return out.reshape(self.ny, self.nx + 1)

    def step_second_order(self, h: np.ndarray, nsteps: int = 1) -> np.ndarray:
        """`nsteps` steps of the second-order variant: exact relaxation over dt/2, second-order
        transport over dt, exact relaxation over dt/2 (symmetric splitting)."""
        cur = np.ascontiguousarray(h, dtype=np.float64).copy()
        for _ in range(nsteps):
            cur = self.relax_exp(self.transport2(self.relax_exp(cur, 0.5)), 0.5)
        return cur

    def step_cells(self, h: np.ndarray, cells) -> np.ndarray:
        """One step's result at the listed cells only: array (len(cells), n)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((len(cells), self.n), dtype=np.float64)
        _load().orc_step_cells(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h),
                               cells.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                               len(cells), _dp(out))
        return out

    def step2_cells(self, h: np.ndarray, cells) -> np.ndarray:
        """One step of the second-order variant in stored-state form (second-order transport,
        then the exact relaxation over dt) at the listed cells only: array (len(cells), n)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((len(cells), self.n), dtype=np.float64)
        _load().orc_step2_cells(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h),
                                cells.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                len(cells), _dp(out))
        return out

    def march(self, h: np.ndarray, max_steps: int, every: int = 100, tol: float = 0.0):
        """March to r < tol (checked every `every` steps); returns (h, steps, last r)."""
        cur = np.ascontiguousarray(h, dtype=np.float64).copy()
        r = ctypes.c_double()
        s = _load().orc_march(ctypes.byref(self._p), ctypes.byref(self._c), _dp(cur),
                              int(max_steps), int(every), float(tol), ctypes.byref(r))
        return cur, int(s), r.value

    def moments(self, h: np.ndarray) -> dict:
        h = np.ascontiguousarray(h, dtype=np.float64)
        outs = {k: np.empty(self.ncells) for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy")}
        _load().orc_moments(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h),
                            *[_dp(outs[k]) for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy")])
        return {k: v.reshape(self.ny, self.nx) for k, v in outs.items()}

    def face_flux_y(self, h: np.ndarray) -> np.ndarray:
        """x-momentum flux through horizontal faces, shape (ny+1, nx)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty((self.ny + 1) * self.nx)
        _load().orc_face_flux_y(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out))
        return out.reshape(self.ny + 1, self.nx)

    def face_flux_x(self, h: np.ndarray) -> np.ndarray:
        """y-momentum flux through vertical faces (cavity), shape (ny, nx+1)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty(self.ny * (self.nx + 1))
        _load().orc_face_flux_x(ctypes.byref(self._p), ctypes.byref(self._c), _dp(h), _dp(out))
        return out.reshape(self.ny, self.nx + 1)


def residual(hn: np.ndarray, h: np.ndarray) -> float:
    hn = np.ascontiguousarray(hn, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    return _load().orc_residual(_dp(hn), _dp(h), hn.size, None, None)


def make_problem(kind: str, n: int, geom: int, nx: int, ny: int, kn: float,
                 u_bottom: float, u_top: float, cfl: float = 0.9) -> Problem:
    """Problem on the oracle's own tensor-product velocity set ('half' N or 'full' M)."""
    from .quadrature import velocity_set_2d
    xi_x, xi_y, w = velocity_set_2d(kind, n)
    return Problem(np.array(xi_x), np.array(xi_y), np.array(w), geom, nx, ny,
                   math.inf if kn == math.inf else kn, u_bottom, u_top, cfl)
