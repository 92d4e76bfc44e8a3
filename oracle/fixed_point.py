"""Direct solve of the fully discrete steady state (oracle; test infrastructure only).

The march of ``lbm_oracle.c`` is an affine map h -> R (T h + t) per step
(first-order splitting: upwind transport T with wall ghosts, then explicit
Euler relaxation R; Eqs. 1, 5-9 and the discretisation paragraph of the
paper).  Its limit is the solution of (I - R T) h = R t.  Here the same scheme
is assembled as sparse matrices, independently of the C loops (different code,
different order of operations), and solved directly:

* T: per velocity a and cell c, (1 - nu_x - nu_y) on h_a(c), nu_x on the
  upwind x value, nu_y on the upwind y value; an upwind value across a wall is
  the ghost w_a [rho'_F (1 + xi_t U_F) + xi_t U_F / u_ref] whose rho'_F is linear
  in the incoming populations of the wall cell (Eq. 9 as a discrete flux
  balance) -- its constant part goes into t;
* R: per cell, (1 - omega) I + omega W with W_ab = w_a (1 + xi_a . xi_b);
* I - R T is singular along the uniform-density state h_a = w_a (any
  constant density perturbation is steady); the march conserves total mass,
  so the bordered system [[I - R T, z], [m^T, 0]] with z_a(c) = w_a and
  m = all-ones (total mass) fixes the solution with zero total mass, which is
  the one a cold start reaches.

Used to pin the march's limit without marching (e.g. the near-continuum
Couette case, where marching to 1e-12 takes many steps).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

COUETTE, CAVITY = 0, 1


def assemble(xi_x, xi_y, w, geom, nx, ny, kn, u_bottom, u_top, cfl=0.9):
    """Return (A, b, info) with the step map h -> A h + b, unknown index a * ncells + c."""
    xi_x = np.asarray(xi_x, float)
    xi_y = np.asarray(xi_y, float)
    w = np.asarray(w, float)
    n = len(w)
    nc = nx * ny
    N = n * nc
    # coefficients (same reading as the march: dt from the CFL number, dt <= Kn)
    if geom == COUETTE:
        dy = 1.0 / ny
        dx = dy
    else:
        dx, dy = 1.0 / nx, 1.0 / ny
    rate = np.max(np.abs(xi_y)) / dy
    if not (geom == COUETTE and nx == 1):
        rate += np.max(np.abs(xi_x)) / dx
    dt = cfl / rate
    if math.isfinite(kn):
        dt = min(dt, kn)
    omega = dt / kn if math.isfinite(kn) else 0.0
    u_ref = max(abs(u_bottom), abs(u_top)) or 1.0
    Dx = float(np.sum(np.where(xi_x > 0, xi_x * w, 0.0)))
    Dy = float(np.sum(np.where(xi_y > 0, xi_y * w, 0.0)))

    def idx(a, x, y):
        return a * nc + y * nx + x

    rows, cols, vals = [], [], []
    t = np.zeros(N)

    def add(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    # faces: (normal component function, D, tangential component, wall speed)
    faces = {
        "bottom": (xi_y, Dy, xi_x, u_bottom),
        "top": (-xi_y, Dy, xi_x, u_top),
        "left": (xi_x, Dx, xi_y, 0.0),
        "right": (-xi_x, Dx, xi_y, 0.0),
    }

    def add_ghost(row, a, face, x, y, nu):
        """row += nu * ghost_a(face of cell (x,y)): linear part into A, constant into t."""
        xn, D, xt, U = faces[face]
        lin = w[a] * (1.0 + xt[a] * U)
        for b in range(n):
            if xn[b] < 0:
                add(row, idx(b, x, y), nu * lin * (-xn[b]) / D)
        t[row] += nu * w[a] * xt[a] * U / u_ref

    for a in range(n):
        nux = abs(xi_x[a]) * dt / dx
        nuy = abs(xi_y[a]) * dt / dy
        for y in range(ny):
            for x in range(nx):
                r = idx(a, x, y)
                add(r, r, 1.0 - nux - nuy)
                if xi_x[a] != 0:
                    xs = x - 1 if xi_x[a] > 0 else x + 1
                    if 0 <= xs < nx:
                        add(r, idx(a, xs, y), nux)
                    elif geom == COUETTE:
                        add(r, idx(a, xs % nx, y), nux)
                    else:
                        add_ghost(r, a, "left" if xi_x[a] > 0 else "right", x, y, nux)
                if xi_y[a] != 0:
                    ys = y - 1 if xi_y[a] > 0 else y + 1
                    if 0 <= ys < ny:
                        add(r, idx(a, x, ys), nuy)
                    else:
                        add_ghost(r, a, "bottom" if xi_y[a] > 0 else "top", x, y, nuy)
    T = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))

    W = np.outer(w, np.ones(n)) * (1.0 + np.outer(xi_x, xi_x) + np.outer(xi_y, xi_y))
    Rcell = (1.0 - omega) * np.eye(n) + omega * W          # acts on the n velocities of a cell
    # R acts on index a*nc + c : R = kron(Rcell, I_nc)
    R = sp.kron(sp.csr_matrix(Rcell), sp.identity(nc, format="csr"), format="csr")
    A = (R @ T).tocsr()
    b = R @ t
    info = {"dt": dt, "omega": omega, "u_ref": u_ref, "n": n, "ncells": nc}
    return A, b, info


def solve_steady(xi_x, xi_y, w, geom, nx, ny, kn, u_bottom, u_top, cfl=0.9):
    """Steady state of the fully discrete scheme with zero total mass: h of shape (n, ncells)."""
    A, b, info = assemble(xi_x, xi_y, w, geom, nx, ny, kn, u_bottom, u_top, cfl)
    n, nc = info["n"], info["ncells"]
    N = n * nc
    z = np.repeat(np.asarray(w, float), nc)        # uniform-density null vector
    M = sp.bmat([[sp.identity(N, format="csr") - A, sp.csr_matrix(z.reshape(-1, 1))],
                 [sp.csr_matrix(np.ones((1, N))), None]], format="csc")
    rhs = np.concatenate([b, [0.0]])
    sol = spla.spsolve(M, rhs)
    return sol[:N].reshape(n, nc), info, float(sol[N])
