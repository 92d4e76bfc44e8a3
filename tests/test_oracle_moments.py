"""Pins of the oracle's cell moments (rho, u, P_ij of Eqs. 6-7 and the stress output) against
what the mathematics fixes, independently of the oracle's own formula.

P_ij is the second moment of f = w + u_ref h (Eq. 1 units, RT = 1): for every velocity set used
here sum w xi_i xi_j = delta_ij, so the oracle forms it as delta_ij + u_ref sum xi_i xi_j h.  The
pins below use other routes to the same numbers:
  * a global equilibrium h = w (rho' + xi.j') has rho = 1 + u_ref rho', u = u_ref j' / rho and an
    isotropic stress P_ij = rho delta_ij (the isothermal pressure), by quadrature exactness to
    degree 3 (pinned in test_oracle_quadrature.py);
  * the second-order Hermite state h = w [rho' + xi.j' + 1/2 Pi_kl (xi_k xi_l - delta_kl)] has
    P_ij = rho delta_ij + u_ref Pi_ij on sets exact to degree 4;
  * the collisionless Couette state is uniform per velocity with closed-form moments:
    rho = 1, u_x = (U_b + U_t)/2, P_xx = P_yy = 1, P_xy = (U_b - U_t)/sqrt(2 pi);
  * the steady Couette cell stress converges at first order in dy to the constant shear of the
    semi-discrete solution;
  * a test compiles the oracle with planted mistakes (dropped delta_ij, rho in place of 1, u not
    divided by rho, transposed indices, u_ref dropped) and checks that each one fails a pin.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import quadrature as q
from oracle.couette_exact import couette_semidiscrete
from oracle.fixed_point import solve_steady
from oracle.march import CAVITY, COUETTE, Problem, make_problem

SETS = [("half", 2), ("half", 3), ("half", 4), ("half", 6), ("full", 3), ("full", 4)]
SETS_DEG4 = [s for s in SETS if not (s[0] == "half" and s[1] == 2)]   # exact to degree >= 4
NAMES = ("rho", "ux", "uy", "pxx", "pxy", "pyy")


def _oracle_moments(p, h):
    return p.moments(h)


def _equilibrium_state(p, seed):
    """h = w (rho' + xi . j') with rho', j' drawn per cell (returns h, rho', jx', jy')."""
    rng = np.random.default_rng(seed)
    rho_p = rng.uniform(-1.5, 1.5, p.ncells)
    jx, jy = rng.uniform(-1.0, 1.0, (2, p.ncells))
    h = p.w[:, None] * (rho_p[None, :] + p.xi_x[:, None] * jx[None, :] + p.xi_y[:, None] * jy[None, :])
    return h, rho_p, jx, jy


# --- the pins, written against a moments function so that the planted-mistake test can rerun them


def pin_equilibrium(moments, kind, n):
    p = make_problem(kind, n, CAVITY, 5, 4, 0.1, 0.0, 0.3)          # u_ref = 0.3: rho far from 1
    u_ref = p.coeffs["u_ref"]
    h, rho_p, jx, jy = _equilibrium_state(p, seed=5)
    m = moments(p, h)
    rho = 1.0 + u_ref * rho_p
    tol = 1e-13
    np.testing.assert_allclose(m["rho"].ravel(), rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["ux"].ravel(), u_ref * jx / rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["uy"].ravel(), u_ref * jy / rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pxx"].ravel(), rho, rtol=0, atol=tol)     # isothermal pressure
    np.testing.assert_allclose(m["pyy"].ravel(), rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pxy"].ravel(), 0.0, rtol=0, atol=tol)


def pin_hermite_second_order(moments, kind, n):
    p = make_problem(kind, n, CAVITY, 4, 3, 0.1, 0.0, 0.2)
    u_ref = p.coeffs["u_ref"]
    rng = np.random.default_rng(17)
    rho_p, jx, jy, pi_xx, pi_xy, pi_yy = rng.uniform(-1.0, 1.0, (6, p.ncells))
    X, Y, W = p.xi_x[:, None], p.xi_y[:, None], p.w[:, None]
    h = W * (rho_p + X * jx + Y * jy
             + 0.5 * (pi_xx * (X * X - 1.0) + 2.0 * pi_xy * X * Y + pi_yy * (Y * Y - 1.0)))
    m = moments(p, h)
    rho = 1.0 + u_ref * rho_p
    tol = 1e-12
    np.testing.assert_allclose(m["rho"].ravel(), rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["ux"].ravel(), u_ref * jx / rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["uy"].ravel(), u_ref * jy / rho, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pxx"].ravel(), rho + u_ref * pi_xx, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pxy"].ravel(), u_ref * pi_xy, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pyy"].ravel(), rho + u_ref * pi_yy, rtol=0, atol=tol)


def pin_free_molecular_couette(moments, n_half):
    ub, ut, ny = 0.01, 0.004, 12
    p = make_problem("half", n_half, COUETTE, 1, ny, math.inf, ub, ut)
    h, steps, r = p.march(p.zeros(), 200000, 50, 1e-15)
    assert r < 1e-15
    m = moments(p, h)
    tol = 1e-15
    np.testing.assert_allclose(m["rho"], 1.0, rtol=0, atol=tol)
    np.testing.assert_allclose(m["ux"], 0.5 * (ub + ut), rtol=0, atol=tol)
    np.testing.assert_allclose(m["uy"], 0.0, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pxx"], 1.0, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pyy"], 1.0, rtol=0, atol=tol)
    np.testing.assert_allclose(m["pxy"], (ub - ut) / math.sqrt(2.0 * math.pi), rtol=1e-12, atol=0)


def pin_couette_stress_first_order(moments, n_half):
    uw = 0.01
    x, w = q.halfrange_1d(n_half)
    sol = couette_semidiscrete([float(v) for v in x], [float(v) for v in w], 0.1, -uw, uw)
    xi_x, xi_y, ww = q.velocity_set_2d("half", n_half)
    errs = []
    for ny in (50, 100, 200):
        h, _, _ = solve_steady(xi_x, xi_y, ww, COUETTE, 1, ny, 0.1, -uw, uw)
        p = Problem(np.array(xi_x), np.array(xi_y), np.array(ww), COUETTE, 1, ny, 0.1, -uw, uw)
        errs.append(np.abs(moments(p, h)["pxy"][:, 0] - sol["pxy"]).max() / abs(sol["pxy"]))
    assert errs[-1] < 0.03, errs
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.1 for r in ratios), (errs, ratios)


def pin_single_velocity(moments, kind, n):
    """One velocity of one cell excited: P_ij - delta_ij = u_ref s xi_i xi_j there, the cell's
    other moments follow from Eqs. 6-7, every other cell is at rest."""
    p = make_problem(kind, n, CAVITY, 3, 2, 0.1, 0.0, 0.25)
    u_ref = p.coeffs["u_ref"]
    a = max((i for i in range(p.n) if p.xi_y[i] >= 0), key=lambda i: p.xi_x[i] - p.xi_y[i])  # xi_x > xi_y >= 0
    s, cell = 1.7, 4
    h = p.zeros()
    h[a, cell] = s
    m = {k: v.ravel() for k, v in moments(p, h).items()}
    rho = 1.0 + u_ref * s
    rest = np.arange(p.ncells) != cell
    tol = 1e-14
    for k, want in (("rho", rho), ("ux", u_ref * s * p.xi_x[a] / rho), ("uy", u_ref * s * p.xi_y[a] / rho),
                    ("pxx", 1.0 + u_ref * s * p.xi_x[a] ** 2), ("pxy", u_ref * s * p.xi_x[a] * p.xi_y[a]),
                    ("pyy", 1.0 + u_ref * s * p.xi_y[a] ** 2)):
        assert abs(m[k][cell] - want) <= tol * max(1.0, abs(want)), (k, m[k][cell], want)
    for k, rest_value in (("rho", 1.0), ("ux", 0.0), ("uy", 0.0), ("pxx", 1.0), ("pxy", 0.0), ("pyy", 1.0)):
        np.testing.assert_array_equal(m[k][rest], rest_value)


# --- the pins as tests of the oracle


@pytest.mark.parametrize("kind,n", SETS)
def test_equilibrium_state_has_isotropic_pressure_and_eq6_7_moments(kind, n):
    pin_equilibrium(_oracle_moments, kind, n)


@pytest.mark.parametrize("kind,n", SETS_DEG4)
def test_second_order_hermite_state_reproduces_its_stress(kind, n):
    pin_hermite_second_order(_oracle_moments, kind, n)


@pytest.mark.parametrize("n_half", [2, 4])
def test_free_molecular_couette_cell_moments_closed_form(n_half):
    pin_free_molecular_couette(_oracle_moments, n_half)


@pytest.mark.parametrize("n_half", [2, 4])
def test_steady_couette_cell_stress_converges_to_semidiscrete_shear(n_half):
    pin_couette_stress_first_order(_oracle_moments, n_half)


@pytest.mark.parametrize("kind,n", [("half", 4), ("full", 3)])
def test_single_velocity_state(kind, n):
    pin_single_velocity(_oracle_moments, kind, n)


def test_moments_are_the_f_form_sums_of_eqs_6_7():
    """On a random state the moments equal sum f, sum xi f / sum f and sum xi_i xi_j f with
    f = w + u_ref h formed here, on every set (this ties the delta_ij of the h-form to the
    quadrature's second moments)."""
    for kind, n in SETS:
        p = make_problem(kind, n, CAVITY, 4, 5, 0.1, 0.0, 0.05)
        u_ref = p.coeffs["u_ref"]
        h = 0.3 * np.random.default_rng(3).standard_normal((p.n, p.ncells))
        f = p.w[:, None] + u_ref * h
        X, Y = p.xi_x[:, None], p.xi_y[:, None]
        rho = f.sum(0)
        want = {"rho": rho, "ux": (X * f).sum(0) / rho, "uy": (Y * f).sum(0) / rho,
                "pxx": (X * X * f).sum(0), "pxy": (X * Y * f).sum(0), "pyy": (Y * Y * f).sum(0)}
        m = p.moments(h)
        for k in NAMES:
            np.testing.assert_allclose(m[k].ravel(), want[k], rtol=1e-13, atol=1e-14, err_msg=f"{kind}{n} {k}")


# --- planted mistakes: each one must fail at least one pin

MUTANTS = {
    "dropped delta_xx": ("if (pxx) pxx[cell] = 1.0 + c->u_ref * sxx;", "if (pxx) pxx[cell] = c->u_ref * sxx;"),
    "dropped delta_yy": ("if (pyy) pyy[cell] = 1.0 + c->u_ref * syy;", "if (pyy) pyy[cell] = c->u_ref * syy;"),
    "rho in place of 1 in P_xx": ("if (pxx) pxx[cell] = 1.0 + c->u_ref * sxx;", "if (pxx) pxx[cell] = r + c->u_ref * sxx;"),
    "rho in place of 1 in P_yy": ("if (pyy) pyy[cell] = 1.0 + c->u_ref * syy;", "if (pyy) pyy[cell] = r + c->u_ref * syy;"),
    "u_x not divided by rho": ("if (ux) ux[cell] = c->u_ref * sx / r;", "if (ux) ux[cell] = c->u_ref * sx;"),
    "u_y not divided by rho": ("if (uy) uy[cell] = c->u_ref * sy / r;", "if (uy) uy[cell] = c->u_ref * sy;"),
    "transposed index in P_xy": ("sxy += p->xi_x[a] * p->xi_y[a] * v;", "sxy += p->xi_x[a] * p->xi_x[a] * v;"),
    "P_yy from xi_x": ("syy += p->xi_y[a] * p->xi_y[a] * v;", "syy += p->xi_x[a] * p->xi_x[a] * v;"),
    "u_y from xi_x": ("sy += p->xi_y[a] * v;", "sy += p->xi_x[a] * v;"),
    "u_ref dropped from rho": ("double r = 1.0 + c->u_ref * s0;", "double r = 1.0 + s0;"),
    "u_ref dropped from P_xy": ("if (pxy) pxy[cell] = c->u_ref * sxy;", "if (pxy) pxy[cell] = sxy;"),
}


def _build_mutant(tmp_path, name, old, new):
    src_path = os.path.join(os.path.dirname(q.__file__), "lbm_oracle.c")
    with open(src_path) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"planted mistake {name!r}: the oracle text it replaces is not unique"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    c_file, so_file = tmp_path / f"{tag}.c", tmp_path / f"{tag}.so"
    c_file.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           str(c_file), "-o", str(so_file), "-lm"])
    lib = ctypes.CDLL(str(so_file))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_moments.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [dp] * 7
    lib.orc_moments.restype = None

    def moments(p, h):
        h = np.ascontiguousarray(h, dtype=np.float64)
        outs = {k: np.empty(p.ncells) for k in NAMES}
        lib.orc_moments(ctypes.addressof(p._p), ctypes.addressof(p._c), h.ctypes.data_as(dp),
                        *[outs[k].ctypes.data_as(dp) for k in NAMES])
        return {k: v.reshape(p.ny, p.nx) for k, v in outs.items()}
    return moments


def _pins():
    yield "equilibrium", lambda m: pin_equilibrium(m, "half", 4)
    yield "hermite", lambda m: pin_hermite_second_order(m, "half", 3)
    yield "single velocity", lambda m: pin_single_velocity(m, "half", 4)
    yield "free molecular", lambda m: pin_free_molecular_couette(m, 2)
    yield "couette stress", lambda m: pin_couette_stress_first_order(m, 2)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_in_moments_fails_a_pin(tmp_path, name):
    mutant = _build_mutant(tmp_path, name, *MUTANTS[name])
    caught = []
    for pin_name, pin in _pins():
        try:
            pin(mutant)
        except AssertionError:
            caught.append(pin_name)
    assert caught, f"planted mistake {name!r} passed every moments pin"
