"""Steady planar Couette flow without space/time discretisation (oracle; test infrastructure only).

Semi-discrete solution: velocity space is discrete (any symmetric 1-D rule on
the y axis, the x axis only entering through sum_i w_i xi_i^2 = 1), y is
continuous.  Follows the construction the paper attributes to the moment
method of its Ref. [fgf09] and uses for Eqs. (10)-(11): the shear part of the
linearised solution is h_a = w_a xi_x,a g_j(y) with j the y-index of a, and
Eq. (1) at steady state reduces to

    xi_j g_j'(s) = sum_k w_k g_k(s) - g_j(s),     s = y / Kn,

whose solutions are the linear mode A (s - xi_j), the constant B and the
exponential eigenmodes of Xi^{-1} (1 w^T - I) (dispersion relation
sum_j w_j / (1 - lambda xi_j) = 1).  Walls (Eq. 8, with rho_w = 0 for this
odd-in-xi_x part): g_j(0) = U_bottom / u_ref for xi_j > 0 and
g_j(1/Kn) = U_top / u_ref for xi_j < 0.

Outputs in the units of Eq. (1):  u_x(y) = u_ref sum_j w_j g_j,
p_xy = u_ref sum_j w_j xi_j g_j = -u_ref A (the same at every y).

Also the paper's closed form for D2Q^h_16 (Eqs. 10-11) with the readings
needed to evaluate it (constant 0.9404 in both hyperbolic functions, velocities
scaled by sqrt(2 R T0) so that its Knudsen number is k = sqrt(2) Kn, y measured
from the channel centre, upper plate at +u_w).  Pinned against each other:
the closed form's 4-digit constants fix the semi-discrete solution for N = 2
to about 1e-4; the Kn -> inf limit is the free-molecular value
p_xy = -sqrt(2/pi) u_w (paper, text after Eqs. 10-11, in Eq. (1) units).
"""
from __future__ import annotations

import math

import numpy as np


def couette_semidiscrete(nodes, weights, kn: float, u_bottom: float, u_top: float,
                         u_ref: float | None = None):
    """Solve the semi-discrete steady Couette problem.

    nodes, weights: the 1-D y-axis rule (ascending, weights summing to 1).
    Returns a dict with callables u(y) (y in [0,1]) and g(y), and the constant p_xy.
    """
    xi = np.asarray(nodes, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    m = len(xi)
    if u_ref is None:
        u_ref = max(abs(u_bottom), abs(u_top)) or 1.0
    S = 1.0 / kn
    K = (np.outer(np.ones(m), w) - np.eye(m)) / xi[:, None]       # Xi^{-1} (1 w^T - I)
    lam, vec = np.linalg.eig(K)
    lam = lam.real
    vec = vec.real
    nonzero = np.abs(lam) > 1e-10
    kappa = lam[nonzero]
    V = vec[:, nonzero]
    assert len(kappa) == m - 2, "expected m-2 exponential modes"

    def basis(s):
        """Columns: linear mode, constant mode, exponential modes (scaled to be <= 1 on [0,S])."""
        cols = [s - xi, np.ones(m)]
        for q in range(len(kappa)):
            if kappa[q] < 0:
                e = math.exp(kappa[q] * s)
            else:
                e = math.exp(kappa[q] * (s - S))
            cols.append(V[:, q] * e)
        return np.stack(cols, axis=1)

    rows, rhs = [], []
    b0, bS = basis(0.0), basis(S)
    for j in range(m):
        if xi[j] > 0:
            rows.append(b0[j])
            rhs.append(u_bottom / u_ref)
        else:
            rows.append(bS[j])
            rhs.append(u_top / u_ref)
    coef = np.linalg.solve(np.array(rows), np.array(rhs))

    def g(y):
        return basis(y * S) @ coef

    def u(y):
        return u_ref * float(w @ g(y))

    pxy = u_ref * float(w @ (xi * g(0.5 * 1.0)))
    return {"u": u, "g": g, "pxy": pxy, "A": coef[0], "u_ref": u_ref,
            "decay_rates": np.sort(np.abs(kappa))}


def couette_d2qh16_closed_form(kn: float, y_center: float, u_w: float = 1.0):
    """Eqs. (10)-(11) of the paper for D2Q^h_16, upper plate at +u_w, lower at -u_w.

    kn is the Knudsen number of Eq. (1); the formula's own Knudsen number is
    k = sqrt(2) kn.  y_center = y/l measured from the channel centre in [-1/2, 1/2].
    Returns (u_x(y), p_xy) with p_xy in the units of Eq. (1).
    """
    k = math.sqrt(2.0) * kn
    a = 0.9404 / k
    den = (0.7071 * k + 0.3989) * math.cosh(a) + (1.128 * k + 0.5) * math.sinh(a)
    u = u_w * ((math.sinh(a) + 0.7978 * math.cosh(a)) * y_center
               + 0.5642 * k * math.sinh(1.881 / k * y_center)) / den
    lhs = -k * (math.sinh(a) + 0.7979 * math.cosh(a)) / den    # sqrt(2 R T0) p_xy / (u_w p0)
    pxy = lhs * u_w / math.sqrt(2.0)
    return u, pxy


def free_molecular_pxy(u_bottom: float, u_top: float) -> float:
    """Collisionless Couette shear in Eq. (1) units: (U_bottom - U_top) / sqrt(2 pi).

    With plates at -u_w and +u_w this is -sqrt(2/pi) u_w, the paper's
    p_fm = -2 p0 u_w / sqrt(pi R T0) written with velocities scaled by sqrt(R T0)
    instead of sqrt(2 R T0)."""
    return (u_bottom - u_top) / math.sqrt(2.0 * math.pi)
