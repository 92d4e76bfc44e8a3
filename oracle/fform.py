"""Literal f-form FP64 step of the scheme (TEST INFRASTRUCTURE ONLY: only tests use it).

The distribution f itself is stored, and each step follows the paper's equations as printed,
without the perturbation rewriting of ``lbm_oracle.c``:
  - first-order upwind transport of f with the scheme's Courant numbers (Eq. 1 and the
    discretisation paragraph), the upwind value across a wall face being the population
    the wall emits;
  - that population: f_a = w_a rho_w (1 + xi_t,a U) for velocities leaving the wall (Eq. 8,
    with the discrete weight w_a), where rho_w makes the normal mass flux through the face
    vanish (Eq. 9 as a discrete flux balance):
    rho_w = sum_{in} |xi_n| f_a / sum_{out} xi_n w_a (1 + xi_t,a U);
  - relaxation towards the equilibrium of Eq. (5), f^eq_a = w_a rho (1 + xi_a . u), with the
    velocity u = (sum xi_a f_a) / rho of Eqs. (6)-(7), i.e. with the division by rho.
Geometry, time step and splitting are the same readings as the h-form oracle (cell-centred
grid with walls on faces, Couette periodic in x, transport then relaxation, dt = CFL over
the largest |xi_d| / d_d summed over the directions that move, dt <= Kn), re-derived here.

Its states agree with the h-form oracle's h = (f - w) / u_ref up to rounding.  The f-form
computes with values near w_a, so it loses digits to cancellation: it serves as a
1e-10-level cross-check of the h-form, not as the primary oracle.
"""
from __future__ import annotations

import math

import numpy as np

COUETTE, CAVITY = 0, 1


class FFormProblem:
    def __init__(self, xi_x, xi_y, w, geom: int, nx: int, ny: int, kn: float, u_bottom: float, u_top: float,
                 cfl: float = 0.9):
        self.xi_x = np.asarray(xi_x, dtype=np.float64)
        self.xi_y = np.asarray(xi_y, dtype=np.float64)
        self.w = np.asarray(w, dtype=np.float64)
        self.geom, self.nx, self.ny = geom, nx, ny
        self.kn, self.u_bottom, self.u_top = kn, u_bottom, u_top
        if geom == COUETTE:
            self.dy = 1.0 / ny
            self.dx = self.dy
        else:
            self.dx, self.dy = 1.0 / nx, 1.0 / ny
        self.x_moves = not (geom == COUETTE and nx == 1)
        rate = np.abs(self.xi_y).max() / self.dy
        if self.x_moves:
            rate += np.abs(self.xi_x).max() / self.dx
        self.dt = cfl / rate
        if math.isfinite(kn):
            self.dt = min(self.dt, kn)
        self.omega = self.dt / kn if math.isfinite(kn) else 0.0

    def _wall_rho(self, f_cell, normal: str, u_wall: float):
        """rho_w of Eq. (9) for a wall face with the gas on the side of `normal` ('+y', '-y',
        '+x', '-x'), from the wall-adjacent cells' populations f_cell (n, cells)."""
        xn = {"+y": self.xi_y, "-y": -self.xi_y, "+x": self.xi_x, "-x": -self.xi_x}[normal]
        xt = self.xi_x if normal in ("+y", "-y") else self.xi_y
        incoming = (-xn * (xn < 0))[:, None] * f_cell
        outgoing = (xn * (xn > 0) * self.w * (1.0 + xt * u_wall)).sum()
        return incoming.sum(0) / outgoing

    def _emitted(self, rho_w, normal: str, u_wall: float):
        """Eq. (8): w_a rho_w (1 + xi_t U) for every velocity (used only where it leaves)."""
        xt = self.xi_x if normal in ("+y", "-y") else self.xi_y
        return (self.w * (1.0 + xt * u_wall))[:, None] * rho_w[None, :]

    def step(self, f: np.ndarray) -> np.ndarray:
        """One time step; f has shape (n, ny, nx)."""
        n, ny, nx = f.shape
        cav = self.geom == CAVITY
        # upwind neighbour along y: below for xi_y > 0 (the bottom wall's emission in row 0),
        # above for xi_y < 0 (the top wall's emission in row ny - 1)
        below = np.empty_like(f)
        above = np.empty_like(f)
        below[:, 1:, :] = f[:, :-1, :]
        above[:, :-1, :] = f[:, 1:, :]
        below[:, 0, :] = self._emitted(self._wall_rho(f[:, 0, :], "+y", self.u_bottom), "+y", self.u_bottom)
        above[:, ny - 1, :] = self._emitted(self._wall_rho(f[:, ny - 1, :], "-y", self.u_top), "-y", self.u_top)
        # along x: periodic for Couette, side walls at rest for the cavity
        left = np.empty_like(f)
        right = np.empty_like(f)
        left[:, :, 1:] = f[:, :, :-1]
        right[:, :, :-1] = f[:, :, 1:]
        if cav:
            left[:, :, 0] = self._emitted(self._wall_rho(f[:, :, 0], "+x", 0.0), "+x", 0.0)
            right[:, :, nx - 1] = self._emitted(self._wall_rho(f[:, :, nx - 1], "-x", 0.0), "-x", 0.0)
        else:
            left[:, :, 0] = f[:, :, nx - 1]
            right[:, :, nx - 1] = f[:, :, 0]
        nux = np.abs(self.xi_x) * self.dt / self.dx if self.x_moves else np.zeros_like(self.xi_x)
        nuy = np.abs(self.xi_y) * self.dt / self.dy
        up_x = np.where((self.xi_x > 0)[:, None, None], left, np.where((self.xi_x < 0)[:, None, None], right, f))
        up_y = np.where((self.xi_y > 0)[:, None, None], below, np.where((self.xi_y < 0)[:, None, None], above, f))
        fs = f - nux[:, None, None] * (f - up_x) - nuy[:, None, None] * (f - up_y)
        # Eqs. (5)-(7)
        rho = fs.sum(0)
        ux = np.tensordot(self.xi_x, fs, axes=1) / rho
        uy = np.tensordot(self.xi_y, fs, axes=1) / rho
        feq = self.w[:, None, None] * rho[None] * (1.0 + self.xi_x[:, None, None] * ux[None]
                                                   + self.xi_y[:, None, None] * uy[None])
        return fs - self.omega * (fs - feq)


def make_fform_problem(kind: str, n: int, geom: int, nx: int, ny: int, kn: float, u_bottom: float, u_top: float,
                       cfl: float = 0.9) -> FFormProblem:
    """Problem on the oracle's tensor-product velocity set ('half' N or 'full' M)."""
    from .quadrature import velocity_set_2d
    xi_x, xi_y, w = velocity_set_2d(kind, n)
    return FFormProblem(xi_x, xi_y, w, geom, nx, ny, kn, u_bottom, u_top, cfl)
