"""Hybrid half-range / full-range Couette march in plain numpy, FP64 (test infrastructure
only: tests, the package's smoke check and the bench's CPU leg may use it, the product
path never does).

The paper's conclusion proposes, without giving an algorithm, to couple a half-range model
(D2Q^h_{(2N)^2}, accurate in the Knudsen layers) near the walls with the full-range model it
reduces to far from the walls (N^2 velocities, a 2^d-fold saving) in the bulk.  This module
is this project's reading of that proposal for the Couette channel (the scheme of Eqs. 1,
5-9 elsewhere unchanged):

  * cells y < L and y >= ny - L carry the half-range set H of N nodes per half-axis, the
    cells between them the full-range Gauss-Hermite set F of N nodes per axis;
  * each cell is transported (first-order upwind in y, walls of Eqs. 8-9 on its own set)
    and relaxed (Eqs. 1, 5-7) in its own set; dt = cfl / (max |xi_y| / dy) over the sets
    present, and dt <= Kn;
  * across an interface face the upwind value of a velocity of the downstream cell comes
    from the upstream cell (the other set) through the tensor Hermite projection of order
    N - 1
        c_mn = sum_a h_a He_m(xi_x,a) He_n(xi_y,a) / (m! n!),
        h~_b = w_b sum_{m,n <= N-1} c_mn He_m(xi_x,b) He_n(xi_y,b)
    (He the probabilists' Hermite polynomials; exact on F data);
  * the flux through an interface face is the half-range one: both half-space fluxes are
    summed in H, the full-range side taken as its projection onto H.  The half-range cell
    sees exactly that exchange; the full-range cell's transported state gets the correction
    (lam + mu_x xi_x + mu_y xi_y) w_b with which its mass and momentum exchange through that
    face equals the half-range one (its own quadrature's half-space integrals are the
    inaccurate ones: sum over xi_y > 0 of xi_y w is 0.444 for N = 4 against 1/sqrt(2 pi)).
    Mass and momentum cross the interface exactly, and a state at rest stays at rest.
  * `HybridCavity` is the same coupling in the lid-driven cavity: half-range cells within
    L cells of any wall, unsplit upwind transport in x and y, the correction on every
    interface face (x or y).

Pins (tests): L >= ny/2 reduces to the half-range march and L = 0 to the full-range march
of the C oracle; the projection is exact on F data and on polynomials of degree <= N - 1
per axis; total mass is conserved exactly; a state at rest stays at rest; at the steady
state the face momentum flux is the same through every face, the interfaces included.
"""
from __future__ import annotations

import math

import numpy as np

from .quadrature import velocity_set_2d


def hermite_table(x: np.ndarray, order: int) -> np.ndarray:
    """He_0..He_order at the points x: array [order + 1][len(x)] (He_{k+1} = x He_k - k He_{k-1})."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((order + 1, len(x)))
    out[0] = 1.0
    if order >= 1:
        out[1] = x
    for k in range(1, order):
        out[k + 1] = x * out[k] - k * out[k - 1]
    return out


class VelocitySet:
    """Tensor-product set with its per-velocity nodes, weights and Hermite tables."""

    def __init__(self, kind: str, n: int, order: int):
        xi_x, xi_y, w = velocity_set_2d(kind, n)
        self.kind = kind
        self.xi_x = np.array(xi_x)
        self.xi_y = np.array(xi_y)
        self.w = np.array(w)
        self.n = len(w)
        self.hx = hermite_table(self.xi_x, order)
        self.hy = hermite_table(self.xi_y, order)
        # wall-flux normaliser of Eq. 9 (discrete flux balance): sum over xi_y > 0 of xi_y w
        self.d_y = float(np.sum(np.where(self.xi_y > 0, self.xi_y * self.w, 0.0)))


def hermite_coefficients(h: np.ndarray, s: VelocitySet, order: int) -> np.ndarray:
    """c_mn = sum_a h_a He_m(xi_x,a) He_n(xi_y,a) / (m! n!), m, n = 0..order."""
    c = np.zeros((order + 1, order + 1))
    for m in range(order + 1):
        for n in range(order + 1):
            c[m, n] = np.sum(h * s.hx[m] * s.hy[n]) / (math.factorial(m) * math.factorial(n))
    return c


def project(h: np.ndarray, src: VelocitySet, dst: VelocitySet, order: int) -> np.ndarray:
    """Tensor Hermite projection of a distribution of `src` onto the velocities of `dst`."""
    c = hermite_coefficients(h, src, order)
    out = np.zeros(dst.n)
    for m in range(order + 1):
        for n in range(order + 1):
            out += c[m, n] * dst.hx[m] * dst.hy[n]
    return dst.w * out


class HybridCouette:
    """Couette channel (one periodic column of ny cells, plates u_bottom at y = 0 and u_top at
    y = 1) with half-range cells within `layer` cells of either wall and full-range cells
    between them; N nodes per half-axis (half-range) and per axis (full-range)."""

    def __init__(self, n_half: int, ny: int, kn: float, u_bottom: float, u_top: float, layer: int,
                 cfl: float = 0.9):
        if ny < 2 or layer < 0 or not (kn > 0) or n_half < 1:
            raise ValueError("invalid hybrid problem")
        self.order = n_half - 1
        self.H = VelocitySet("half", n_half, self.order)
        self.F = VelocitySet("full", n_half, self.order)
        self.ny, self.kn, self.layer = ny, kn, layer
        self.u_bottom, self.u_top = u_bottom, u_top
        self.half = [j < layer or j >= ny - layer for j in range(ny)]
        present = [s for s, used in ((self.H, any(self.half)), (self.F, not all(self.half))) if used]
        self.dy = 1.0 / ny
        rate = max(float(np.max(np.abs(s.xi_y))) for s in present) / self.dy
        self.dt = cfl / rate
        if math.isfinite(kn) and self.dt > kn:
            self.dt = kn
        self.omega = self.dt / kn if math.isfinite(kn) else 0.0
        ur = max(abs(u_bottom), abs(u_top))
        self.u_ref = ur if ur > 0 else 1.0

    def vset(self, j: int) -> VelocitySet:
        return self.H if self.half[j] else self.F

    def zeros(self) -> list:
        return [np.zeros(self.vset(j).n) for j in range(self.ny)]

    def unknowns(self) -> int:
        return sum(self.vset(j).n for j in range(self.ny))

    def _wall_density(self, h: np.ndarray, s: VelocitySet, bottom: bool) -> float:
        # Eq. 9 as a discrete flux balance over the cell's own set; normal into the gas
        xn = s.xi_y if bottom else -s.xi_y
        return float(np.sum(np.where(xn < 0, -xn * h, 0.0))) / s.d_y

    def _ghost(self, s: VelocitySet, rho_w: float, bottom: bool) -> np.ndarray:
        # Eq. 8 in perturbation form for the velocities leaving the wall
        u = self.u_bottom if bottom else self.u_top
        return s.w * (rho_w * (1.0 + s.xi_x * u) + s.xi_x * u / self.u_ref)

    def upwind_from(self, h: list, j: int, k: int) -> np.ndarray:
        """Values of cell k as seen by cell j's set (k = j -+ 1): its own values for the same
        set, else their projection."""
        sj, sk = self.vset(j), self.vset(k)
        if sj is sk:
            return h[k]
        return project(h[k], sk, sj, self.order)

    @staticmethod
    def _face_moments(s: VelocitySet, v: np.ndarray, upward: bool):
        """(mass, x-momentum, y-momentum) flux sum |xi_y| (1, xi_x, xi_y) v over the velocities
        of s moving up (upward) or down."""
        m = (s.xi_y > 0) if upward else (s.xi_y < 0)
        t = np.where(m, np.abs(s.xi_y) * v, 0.0)
        return np.array([np.sum(t), np.sum(t * s.xi_x), np.sum(t * s.xi_y)])

    def half_fluxes_h(self, h: list, k: int):
        """Face k (between cells k - 1 and k, 1 <= k <= ny - 1) evaluated in the half-range
        set: the (mass, x-momentum, y-momentum) fluxes carried upward and downward, each
        side's distribution in H (projected when full-range)."""
        H = self.H
        lo = h[k - 1] if self.half[k - 1] else project(h[k - 1], self.F, H, self.order)
        hi = h[k] if self.half[k] else project(h[k], self.F, H, self.order)
        return self._face_moments(H, lo, True), self._face_moments(H, hi, False)

    def interface_correction(self, h: list, j: int) -> np.ndarray:
        """Correction added to the transported state of full-range cell j next to half-range
        cells: (lam + mu_x xi_x + mu_y xi_y) w with which its net mass and momentum exchange
        through each interface face equals the half-range evaluation of that face
        (sum w = sum xi_x^2 w = sum xi_y^2 w = 1, cross sums 0, for the full-range rule)."""
        s = self.vset(j)
        corr = np.zeros(s.n)
        if self.half[j]:
            return corr
        for k, other in ((j, j - 1), (j + 1, j + 1)):     # lower face k = j, upper face k = j + 1
            if other < 0 or other >= self.ny or not self.half[other]:
                continue
            up, dn = self.half_fluxes_h(h, k)
            recv = self.upwind_from(h, j, other)
            if k == j:    # j is above the face: receives the upward velocities, sends the downward
                want = up - dn
                have = self._face_moments(s, recv, True) - self._face_moments(s, h[j], False)
            else:         # j is below the face
                want = dn - up
                have = self._face_moments(s, recv, False) - self._face_moments(s, h[j], True)
            d = want - have
            corr += self.dt / self.dy * (d[0] + d[1] * s.xi_x + d[2] * s.xi_y) * s.w
        return corr

    def step(self, h: list, nsteps: int = 1) -> list:
        cur = [np.array(v, dtype=np.float64) for v in h]
        for _ in range(nsteps):
            nxt = []
            for j in range(self.ny):
                s = self.vset(j)
                hc = cur[j]
                # upwind y neighbours: below for xi_y > 0, above for xi_y < 0
                if j > 0:
                    below = self.upwind_from(cur, j, j - 1)
                else:
                    below = self._ghost(s, self._wall_density(hc, s, True), True)
                if j < self.ny - 1:
                    above = self.upwind_from(cur, j, j + 1)
                else:
                    above = self._ghost(s, self._wall_density(hc, s, False), False)
                hy = np.where(s.xi_y > 0, below, above)
                nuy = np.abs(s.xi_y) * self.dt / self.dy
                hs = hc - nuy * (hc - hy) + self.interface_correction(cur, j)
                rho = np.sum(hs)
                jx = np.sum(s.xi_x * hs)
                jy = np.sum(s.xi_y * hs)
                heq = s.w * (rho + s.xi_x * jx + s.xi_y * jy)
                nxt.append(hs - self.omega * (hs - heq))
            cur = nxt
        return cur

    @staticmethod
    def residual(hn: list, h: list) -> float:
        d = sum(float(np.sum((a - b) ** 2)) for a, b in zip(hn, h))
        n = sum(float(np.sum(a ** 2)) for a in hn)
        return math.sqrt(d / n) if n > 0 else (0.0 if d == 0 else math.inf)

    def march(self, h: list, max_steps: int, every: int = 100, tol: float = 0.0):
        """March to r < tol checked every `every` steps; returns (h, steps, last r)."""
        cur, steps, r = h, 0, math.inf
        while steps < max_steps:
            prev = self.step(cur, every - 1)
            cur = self.step(prev, 1)
            steps += every
            r = self.residual(cur, prev)
            if r < tol:
                break
        return cur, steps, r

    def mass(self, h: list) -> float:
        return float(sum(np.sum(v) for v in h))

    def ux(self, h: list) -> np.ndarray:
        """u_x per cell from the cell's own set: u_ref sum xi_x h / (1 + u_ref sum h)."""
        out = np.empty(self.ny)
        for j in range(self.ny):
            s = self.vset(j)
            out[j] = self.u_ref * np.sum(s.xi_x * h[j]) / (1.0 + self.u_ref * np.sum(h[j]))
        return out

    def face_flux(self, h: list) -> np.ndarray:
        """x-momentum flux u_ref sum xi_x xi_y h_upwind through the ny + 1 faces; the upward
        velocities counted in the lower cell's set, the downward ones in the upper cell's,
        except at an interface face, which is evaluated in the half-range set."""
        out = np.empty(self.ny + 1)
        for k in range(self.ny + 1):
            if 0 < k < self.ny and self.half[k - 1] != self.half[k]:
                up, dn = self.half_fluxes_h(h, k)
                out[k] = self.u_ref * (up[1] - dn[1])
                continue
            up = 0.0
            if k == 0:
                s = self.vset(0)
                g = self._ghost(s, self._wall_density(h[0], s, True), True)
                up = np.sum(np.where(s.xi_y > 0, s.xi_x * s.xi_y * g, 0.0))
            else:
                s = self.vset(k - 1)
                up = np.sum(np.where(s.xi_y > 0, s.xi_x * s.xi_y * h[k - 1], 0.0))
            if k == self.ny:
                s = self.vset(self.ny - 1)
                g = self._ghost(s, self._wall_density(h[self.ny - 1], s, False), False)
                down = np.sum(np.where(s.xi_y < 0, s.xi_x * s.xi_y * g, 0.0))
            else:
                s = self.vset(k)
                down = np.sum(np.where(s.xi_y < 0, s.xi_x * s.xi_y * h[k], 0.0))
            out[k] = self.u_ref * (up + down)
        return out


class HybridCavity:
    """Lid-driven cavity (nx x ny cells, walls on all four faces, the bottom moving at
    u_bottom and the top at u_top, the sides at rest) with half-range cells within `layer`
    cells of any wall and full-range cells inside.  Unsplit first-order upwind transport in x
    and y on each cell's own set; at an interface face (x or y) the upwind values are the
    projection of the neighbour, the face flux is the half-range evaluation, and the
    full-range cell's transported state gets (lam + mu_x xi_x + mu_y xi_y) w so that its
    mass and momentum exchange through the face equals it (sum w = sum xi_x^2 w =
    sum xi_y^2 w = 1, the cross sums 0, for the full-range rule)."""

    def __init__(self, n_half: int, nx: int, ny: int, kn: float, u_bottom: float, u_top: float, layer: int,
                 cfl: float = 0.9):
        if nx < 2 or ny < 2 or layer < 0 or not (kn > 0) or n_half < 1:
            raise ValueError("invalid hybrid problem")
        self.order = n_half - 1
        self.H = VelocitySet("half", n_half, self.order)
        self.F = VelocitySet("full", n_half, self.order)
        for s in (self.H, self.F):
            s.d_x = float(np.sum(np.where(s.xi_x > 0, s.xi_x * s.w, 0.0)))
        self.nx, self.ny, self.kn, self.layer = nx, ny, kn, layer
        self.u_bottom, self.u_top = u_bottom, u_top
        self.half = [min(x, nx - 1 - x, y, ny - 1 - y) < layer for y in range(ny) for x in range(nx)]
        present = [s for s, used in ((self.H, any(self.half)), (self.F, not all(self.half))) if used]
        self.dx, self.dy = 1.0 / nx, 1.0 / ny
        mx = max(float(np.max(np.abs(s.xi_x))) for s in present)
        my = max(float(np.max(np.abs(s.xi_y))) for s in present)
        self.dt = cfl / (mx / self.dx + my / self.dy)
        if math.isfinite(kn) and self.dt > kn:
            self.dt = kn
        self.omega = self.dt / kn if math.isfinite(kn) else 0.0
        ur = max(abs(u_bottom), abs(u_top))
        self.u_ref = ur if ur > 0 else 1.0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    def vset(self, c: int) -> VelocitySet:
        return self.H if self.half[c] else self.F

    def zeros(self) -> list:
        return [np.zeros(self.vset(c).n) for c in range(self.ncells)]

    def unknowns(self) -> int:
        return sum(self.vset(c).n for c in range(self.ncells))

    def mass(self, h: list) -> float:
        return float(sum(np.sum(v) for v in h))

    def _ghost(self, s: VelocitySet, h: np.ndarray, face: str) -> np.ndarray:
        """Eq. 8 ghost for the velocities leaving wall `face` (rho_w by Eq. 9 over the cell's
        own set, normal into the gas)."""
        if face in ("bottom", "top"):
            xn = s.xi_y if face == "bottom" else -s.xi_y
            d, xt, u = s.d_y, s.xi_x, (self.u_bottom if face == "bottom" else self.u_top)
        else:
            xn = s.xi_x if face == "left" else -s.xi_x
            d, xt, u = s.d_x, s.xi_y, 0.0
        rho_w = float(np.sum(np.where(xn < 0, -xn * h, 0.0))) / d
        return s.w * (rho_w * (1.0 + xt * u) + xt * u / self.u_ref)

    def seen(self, h: list, c: int, k: int) -> np.ndarray:
        """Cell k's values in cell c's set."""
        sc, sk = self.vset(c), self.vset(k)
        return h[k] if sc is sk else project(h[k], sk, sc, self.order)

    def _face_moments(self, s: VelocitySet, v: np.ndarray, axis: int, positive: bool):
        """(mass, x-momentum, y-momentum) flux sum |xi_d| (1, xi_x, xi_y) v over the velocities
        of s moving along +axis (positive) or -axis."""
        xd = s.xi_x if axis == 0 else s.xi_y
        m = (xd > 0) if positive else (xd < 0)
        t = np.where(m, np.abs(xd) * v, 0.0)
        return np.array([np.sum(t), np.sum(t * s.xi_x), np.sum(t * s.xi_y)])

    def correction(self, h: list, c: int, recv: dict) -> np.ndarray:
        """Correction of full-range cell c for its interface faces; recv[(axis, side)] are the
        values it received through that face (its own set)."""
        s = self.vset(c)
        corr = np.zeros(s.n)
        if self.half[c]:
            return corr
        x, y = c % self.nx, c // self.nx
        for axis, side, k in ((0, -1, c - 1 if x > 0 else -1), (0, 1, c + 1 if x < self.nx - 1 else -1),
                              (1, -1, c - self.nx if y > 0 else -1), (1, 1, c + self.nx if y < self.ny - 1 else -1)):
            if k < 0 or not self.half[k]:
                continue
            H = self.H
            mine_h = project(h[c], s, H, self.order)
            lo, hi = (h[k], mine_h) if side < 0 else (mine_h, h[k])
            up = self._face_moments(H, lo, axis, True)     # along +axis, from the lower-side cell
            dn = self._face_moments(H, hi, axis, False)    # along -axis, from the upper-side cell
            want = up - dn if side < 0 else dn - up
            got = self._face_moments(s, recv[(axis, side)], axis, side < 0)
            sent = self._face_moments(s, h[c], axis, side > 0)
            diff = want - (got - sent)
            fac = self.dt / (self.dx if axis == 0 else self.dy)
            corr += fac * (diff[0] + diff[1] * s.xi_x + diff[2] * s.xi_y) * s.w
        return corr

    def step(self, h: list, nsteps: int = 1) -> list:
        cur = [np.array(v, dtype=np.float64) for v in h]
        nx, ny = self.nx, self.ny
        for _ in range(nsteps):
            nxt = []
            for c in range(self.ncells):
                s = self.vset(c)
                hc = cur[c]
                x, y = c % nx, c // nx
                left = self.seen(cur, c, c - 1) if x > 0 else self._ghost(s, hc, "left")
                right = self.seen(cur, c, c + 1) if x < nx - 1 else self._ghost(s, hc, "right")
                below = self.seen(cur, c, c - nx) if y > 0 else self._ghost(s, hc, "bottom")
                above = self.seen(cur, c, c + nx) if y < ny - 1 else self._ghost(s, hc, "top")
                hx = np.where(s.xi_x > 0, left, np.where(s.xi_x < 0, right, hc))
                hy = np.where(s.xi_y > 0, below, np.where(s.xi_y < 0, above, hc))
                nux = np.abs(s.xi_x) * self.dt / self.dx
                nuy = np.abs(s.xi_y) * self.dt / self.dy
                recv = {(0, -1): left, (0, 1): right, (1, -1): below, (1, 1): above}
                hs = hc - nux * (hc - hx) - nuy * (hc - hy) + self.correction(cur, c, recv)
                rho, jx, jy = np.sum(hs), np.sum(s.xi_x * hs), np.sum(s.xi_y * hs)
                heq = s.w * (rho + s.xi_x * jx + s.xi_y * jy)
                nxt.append(hs - self.omega * (hs - heq))
            cur = nxt
        return cur

    def velocity(self, h: list):
        """(u_x, u_y) per cell [ny][nx] from each cell's own set."""
        ux, uy = np.empty(self.ncells), np.empty(self.ncells)
        for c in range(self.ncells):
            s = self.vset(c)
            rho = 1.0 + self.u_ref * np.sum(h[c])
            ux[c] = self.u_ref * np.sum(s.xi_x * h[c]) / rho
            uy[c] = self.u_ref * np.sum(s.xi_y * h[c]) / rho
        return ux.reshape(self.ny, self.nx), uy.reshape(self.ny, self.nx)
