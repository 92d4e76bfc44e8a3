"""Pins of the oracle march (plain-C FP64 scheme) against what the paper and mathematics fix."""
import math

import numpy as np
import pytest

from oracle import quadrature as q
from oracle.couette_exact import (couette_d2qh16_closed_form, couette_semidiscrete,
                                  free_molecular_pxy)
from oracle.fixed_point import assemble, solve_steady
from oracle.march import CAVITY, COUETTE, Problem, make_problem, residual
from paper_1308_0692_gb300.inputs import random_state


def _one_d(kind, n):
    nodes, weights = q.halfrange_1d(n) if kind == "half" else q.fullrange_1d(n)
    return [float(v) for v in nodes], [float(v) for v in weights]


@pytest.mark.parametrize("kind,n,geom,nx,ny,kn,ub,ut", [
    ("half", 2, CAVITY, 5, 4, 0.3, 0.0, 0.02),
    ("half", 4, CAVITY, 3, 3, 0.05, 0.01, -0.02),
    ("full", 3, CAVITY, 4, 5, 0.1, 0.0, 0.01),
    ("half", 2, COUETTE, 1, 9, 0.1, 0.01, -0.01),
    ("half", 2, COUETTE, 3, 4, 1.0, -0.01, 0.01),
    ("half", 3, COUETTE, 1, 6, math.inf, -0.01, 0.01),
])
def test_step_equals_independent_matrix_assembly(kind, n, geom, nx, ny, kn, ub, ut):
    """One step of the C loops equals A h + b of the separately assembled sparse scheme."""
    p = make_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h = random_state(p.n, p.ncells, seed=7)
    A, b, info = assemble(p.xi_x, p.xi_y, p.w, geom, nx, ny, kn, ub, ut)
    ref = (A @ h.ravel() + b).reshape(h.shape)
    got = p.step(h)
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    assert info["dt"] == p.coeffs["dt"]


def test_step_cells_matches_full_step():
    p = make_problem("half", 4, CAVITY, 7, 6, 0.1, 0.0, 0.01)
    h = random_state(p.n, p.ncells, seed=3)
    full = p.step(h)
    cells = [0, 6, 20, 41, 35, 17]
    part = p.step_cells(h, cells)
    np.testing.assert_array_equal(part, full[:, cells].T)


@pytest.mark.parametrize("geom,nx,ny,n", [(CAVITY, 7, 6, 4), (CAVITY, 9, 8, 6), (COUETTE, 1, 12, 4),
                                         (COUETTE, 5, 7, 2)])
def test_step2_cells_matches_transport2_then_exact_relaxation(geom, nx, ny, n):
    """The per-cell second-order step is the whole-grid second-order transport followed by
    the exact relaxation over dt, at every cell (walls, corners, the second cell from a
    wall, periodic columns), bit for bit."""
    p = make_problem("half", n, geom, nx, ny, 0.1, 0.0 if geom == CAVITY else 0.01, 0.01 if geom == CAVITY else -0.01)
    h = random_state(p.n, p.ncells, seed=5)
    full = p.relax_exp(p.transport2(h), 1.0)
    cells = list(range(p.ncells))[::-1]
    np.testing.assert_array_equal(p.step2_cells(h, cells), full[:, cells].T)


@pytest.mark.parametrize("geom,nx,ny", [(CAVITY, 13, 11), (COUETTE, 1, 30), (COUETTE, 4, 9)])
def test_total_mass_conserved(geom, nx, ny):
    """Transport with impermeable walls (Eq. 9) and relaxation (Eqs. 5-7) conserve total mass."""
    p = make_problem("half", 4, geom, nx, ny, 0.05, 0.01, -0.02)
    h = random_state(p.n, p.ncells, seed=11)
    m0 = h.sum()
    h2 = p.step(h, 300)
    assert abs(h2.sum() - m0) <= 1e-13 * np.abs(h).sum()


def test_collision_conserves_density_and_momentum_per_cell():
    """With collisions only (transport of a uniform field in a periodic column is the identity
    away from walls), rho and j of every cell are unchanged by the relaxation step."""
    # periodic channel 8 x 5 at rest, each velocity uniform over all cells: transport is the
    # identity in the three interior rows, so only the relaxation acts there
    p = make_problem("half", 4, COUETTE, 8, 5, 0.01, 0.0, 0.0)
    rng = np.random.default_rng(5)
    h = np.repeat(rng.standard_normal((p.n, 1)), 40, axis=1)
    out = p.step(h)
    interior = [c for c in range(40) if 8 <= c < 32]
    for c in interior:
        for mom in (np.ones(p.n), p.xi_x, p.xi_y):
            assert abs(mom @ out[:, c] - mom @ h[:, c]) <= 1e-14 * np.abs(h[:, c]).sum()
    # and the relaxation actually acted (h is not an equilibrium)
    assert np.abs(out - h)[:, interior].max() > 1e-3


@pytest.mark.parametrize("n_half", [2, 4])
def test_couette_antisymmetry(n_half):
    """Plates at +u and -u: u_x(y) = -u_x(1 - y) (config: plates +0.01 at y=0, -0.01 at y=1)."""
    p = make_problem("half", n_half, COUETTE, 1, 40, 0.1, 0.01, -0.01)
    h, steps, r = p.march(p.zeros(), 4000, 100, 1e-9)
    ux = p.moments(h)["ux"][:, 0]
    assert np.abs(ux + ux[::-1]).max() <= 1e-15
    assert ux[0] > 0 > ux[-1]


@pytest.mark.parametrize("n_half,ny", [(2, 7), (4, 40), (3, 15)])
def test_free_molecular_closed_form_shear(n_half, ny):
    """Kn = inf: the steady shear on every face is the collisionless value (U_b - U_t)/sqrt(2 pi),
    i.e. -sqrt(2/pi) u_w for plates at -u_w/+u_w (p_fm of the text after Eqs. 10-11)."""
    u = 0.01
    p = make_problem("half", n_half, COUETTE, 1, ny, math.inf, -u, u)
    h, steps, r = p.march(p.zeros(), 200000, 50, 1e-15)
    flux = p.face_flux_y(h)[:, 0]
    ref = free_molecular_pxy(-u, u)
    assert abs(ref + math.sqrt(2 / math.pi) * u) < 1e-17
    np.testing.assert_allclose(flux, ref, rtol=1e-12, atol=0)


def test_kn10_is_not_free_molecular():
    """Kn = 10 is close to but measurably away from the collisionless limit (about 5.6 %)."""
    x, w = _one_d("half", 4)
    sol = couette_semidiscrete(x, w, 10.0, -1.0, 1.0)
    fm = free_molecular_pxy(-1.0, 1.0)
    assert 0.04 < (sol["pxy"] - fm) / abs(fm) < 0.07


@pytest.mark.parametrize("kn", [0.01, 0.1, 1.0, 10.0])
def test_semidiscrete_couette_matches_paper_closed_form(kn):
    """Eqs. (10)-(11) (D2Q^h_16 closed form, 4-digit constants) agree with the semi-discrete
    eigen-solution for N = 2 to the precision of the printed constants."""
    x, w = _one_d("half", 2)
    sol = couette_semidiscrete(x, w, kn, -1.0, 1.0)
    for yc in (-0.5, -0.25, 0.0, 0.1, 0.5):
        u_cf, _ = couette_d2qh16_closed_form(kn, yc)
        assert abs(sol["u"](yc + 0.5) - u_cf) < 3e-4
    _, p_cf = couette_d2qh16_closed_form(kn, 0.5)
    assert abs(sol["pxy"] - p_cf) < 3e-4 * abs(p_cf)
    # decay rate of the Knudsen-layer mode: 1.881 in the closed form's units = sqrt(2)/(xi_1 xi_2)
    assert abs(sol["decay_rates"][0] * math.sqrt(2) - 1.881) < 1e-3
    assert abs(sol["decay_rates"][0] - 1.0 / (x[2] * x[3])) < 1e-12


def test_semidiscrete_couette_free_molecular_limit():
    x, w = _one_d("half", 4)
    sol = couette_semidiscrete(x, w, 1e5, -1.0, 1.0)
    assert abs(sol["pxy"] - free_molecular_pxy(-1.0, 1.0)) < 1e-4


def test_first_order_grid_convergence_to_semidiscrete_solution():
    """The discrete steady shear converges to the semi-discrete value at first order in dy."""
    x, w = _one_d("half", 2)
    exact = couette_semidiscrete(x, w, 0.1, -1.0, 1.0)["pxy"]
    xi_x, xi_y, ww = q.velocity_set_2d("half", 2)
    errs = []
    for ny in (50, 100, 200, 400):
        h, info, _ = solve_steady(xi_x, xi_y, ww, COUETTE, 1, ny, 0.1, -1.0, 1.0)
        p = Problem(np.array(xi_x), np.array(xi_y), np.array(ww), COUETTE, 1, ny, 0.1, -1.0, 1.0)
        flux = p.face_flux_y(h)[:, 0]
        assert np.ptp(flux) < 1e-10                      # same shear through every face
        errs.append(abs(flux.mean() - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), ratios


def test_march_converges_to_direct_steady_solution():
    """The march's limit is the fully discrete fixed point (Couette, 64 velocities, Kn = 0.1)."""
    p = make_problem("half", 4, COUETTE, 1, 100, 0.1, 0.01, -0.01)
    h, steps, r = p.march(p.zeros(), 100000, 100, 1e-13)
    hd, info, lam = solve_steady(p.xi_x, p.xi_y, p.w, COUETTE, 1, 100, 0.1, 0.01, -0.01)
    assert r < 1e-13 and abs(lam) < 1e-15
    assert np.abs(h - hd).max() <= 1e-10 * np.abs(hd).max()


def test_near_continuum_linear_profile_with_slip():
    """Kn = 0.01: the core of the steady profile is linear, with a velocity slip at the plates
    and a shear stress equal to the (numerical + physical) viscous stress of the core."""
    u = 0.01
    xi_x, xi_y, w = q.velocity_set_2d("half", 4)
    ny = 100
    h, info, _ = solve_steady(xi_x, xi_y, w, COUETTE, 1, ny, 0.01, u, -u)
    p = Problem(np.array(xi_x), np.array(xi_y), np.array(w), COUETTE, 1, ny, 0.01, u, -u)
    ux = p.moments(h)["ux"][:, 0] / u
    y = (np.arange(ny) + 0.5) / ny
    core = (y > 0.25) & (y < 0.75)
    slope = np.polyfit(y[core], ux[core], 1)[0]
    d2 = np.abs(np.diff(ux[core], 2)).max()
    assert d2 < 1e-6 * abs(slope) / ny                      # linear core
    # extrapolate the core line to the plates: the gas does not reach the plate speed (slip)
    fit = np.polyfit(y[core], ux[core], 1)
    u_at_wall = np.polyval(fit, 0.0)
    slip = 1.0 - u_at_wall
    assert 0.005 < slip < 0.2
    flux = p.face_flux_y(h)[:, 0] / u
    assert np.ptp(flux) < 1e-10 * abs(flux).max()           # one shear stress through every face
    assert flux.mean() * slope < 0                          # p_xy = -mu du/dy: opposite signs
    # effective viscosity of the core: physical Kn plus first-order upwind diffusion, same order
    mu_eff = -flux.mean() / slope
    assert 0.01 < mu_eff < 0.013
    # the semi-discrete (exact in y) value is approached but first-order error remains at dy = Kn
    x1, w1 = _one_d("half", 4)
    exact = couette_semidiscrete(x1, w1, 0.01, 1.0, -1.0)["pxy"]
    assert 0.05 < (flux.mean() - exact) / exact < 0.2


def test_x_axis_rule_does_not_change_couette():
    """Text after the Couette setup: full-range nodes on the x axis give the same Couette results."""
    xh, wh = _one_d("half", 2)
    xf, wf = _one_d("full", 4)
    set_half = q.mixed_set_2d(xh, wh, xh, wh)
    set_mixed = q.mixed_set_2d(xf, wf, xh, wh)
    res = []
    for xi_x, xi_y, w in (set_half, set_mixed):
        h, info, _ = solve_steady(xi_x, xi_y, w, COUETTE, 1, 50, 0.1, -0.01, 0.01)
        p = Problem(np.array(xi_x), np.array(xi_y), np.array(w), COUETTE, 1, 50, 0.1, -0.01, 0.01)
        res.append((p.moments(h)["ux"][:, 0], p.face_flux_y(h)[:, 0]))
    np.testing.assert_allclose(res[0][0], res[1][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(res[0][1], res[1][1], rtol=1e-12, atol=0)


def test_cavity_mirror_symmetry_in_the_linear_limit():
    """Lid-driven cavity at a tiny lid speed: u_x is even and u_y odd about x = 1/2."""
    u = 1e-8
    xi_x, xi_y, w = q.velocity_set_2d("half", 2)
    h, info, _ = solve_steady(xi_x, xi_y, w, CAVITY, 12, 12, 0.2, 0.0, u)
    p = Problem(np.array(xi_x), np.array(xi_y), np.array(w), CAVITY, 12, 12, 0.2, 0.0, u)
    m = p.moments(h)
    ux, uy = m["ux"] / u, m["uy"] / u
    assert np.abs(ux - ux[:, ::-1]).max() < 1e-6 * np.abs(ux).max()
    assert np.abs(uy + uy[:, ::-1]).max() < 1e-6 * np.abs(uy).max()
    assert ux[-1].mean() > 0                  # the gas under the lid follows it


def test_residual_definition():
    a = np.array([[3.0, 4.0]])
    b = np.zeros_like(a)
    assert residual(a, b) == 1.0
    assert residual(b, b) == 0.0
    assert abs(residual(a, a * 0.5) - 0.5) < 1e-16


# ---- symmetric (Strang) splitting: relaxation(dt/2), transport(dt), relaxation(dt/2) ----

@pytest.mark.parametrize("geom,nx,ny", [(COUETTE, 1, 12), (CAVITY, 6, 5)])
def test_strang_without_collisions_is_the_lie_step(geom, nx, ny):
    p = make_problem("half", 2, geom, nx, ny, math.inf, 0.0 if geom == CAVITY else 0.01, 0.01)
    h = random_state(p.n, p.ncells, seed=3)
    np.testing.assert_array_equal(p.step_strang(h, 4), p.step(h, 4))


@pytest.mark.parametrize("geom,nx,ny", [(COUETTE, 1, 12), (CAVITY, 6, 5)])
def test_strang_conserves_mass(geom, nx, ny):
    p = make_problem("half", 4, geom, nx, ny, 0.05, 0.0 if geom == CAVITY else 0.01, 0.01)
    h = random_state(p.n, p.ncells, seed=4)
    assert abs(p.step_strang(h, 5).sum() - h.sum()) <= 1e-12 * np.abs(h).sum()


@pytest.mark.parametrize("kn", [0.03, 0.4])
def test_strang_stored_state_is_a_lie_march_with_squared_half_factor(kn):
    """The identity the library's Strang mode rests on: with g = R(dt/2) h, one Strang step
    of h is g' = transport then a relaxation with factor (1 - omega/2)^2 (the two half
    relaxations share their equilibrium, which relaxation leaves unchanged)."""
    p = make_problem("half", 4, CAVITY, 7, 6, kn, 0.0, 0.01)
    w = p.coeffs["omega"]
    h0 = random_state(p.n, p.ncells, seed=5)
    literal = p.relax(p.step_strang(h0, 6), 0.5)
    g_form = p.step(p.relax(h0, 0.5), 6, omega=1.0 - (1.0 - 0.5 * w) ** 2)
    assert np.abs(literal - g_form).max() <= 1e-13 * np.abs(literal).max()


def test_relaxation_half_steps_compose_to_squared_factor_on_non_equilibrium():
    p = make_problem("half", 4, CAVITY, 5, 4, 0.1, 0.0, 0.01)
    h = random_state(p.n, p.ncells, seed=6)
    w = p.coeffs["omega"]
    twice = p.relax(p.relax(h, 0.5), 0.5)
    eq = p.relax(h, 1.0 / w)          # relaxing over dt/omega (= Kn) lands on the equilibrium
    np.testing.assert_allclose(twice - eq, (1 - 0.5 * w) ** 2 * (h - eq), rtol=0, atol=1e-14)


# ---- second-order variant: exact relaxation halves around a second-order transport ----

def _march_second_order(p, tol=1e-13, chunk=100, max_chunks=4000):
    g = p.zeros()
    for _ in range(max_chunks):
        g2 = p.step_second_order(g, chunk)
        r = np.linalg.norm(g2 - g) / max(np.linalg.norm(g2), 1e-300)
        g = g2
        if r < tol:
            return g
    raise AssertionError("no steady state")


def test_exact_relaxation_composes_and_conserves():
    p = make_problem("half", 4, CAVITY, 5, 4, 0.07, 0.0, 0.01)
    h = random_state(p.n, p.ncells, seed=8)
    np.testing.assert_allclose(p.relax_exp(p.relax_exp(h, 0.3), 0.45), p.relax_exp(h, 0.75), rtol=0, atol=1e-14)
    r = p.relax_exp(h, 0.5)
    m0, m1 = p.moments(h), p.moments(r)
    for k in ("rho", "ux", "uy"):
        np.testing.assert_allclose(m1[k], m0[k], rtol=0, atol=1e-15)


@pytest.mark.parametrize("geom,nx,ny", [(COUETTE, 1, 9), (COUETTE, 4, 6), (CAVITY, 7, 6)])
def test_second_order_transport_conserves_mass(geom, nx, ny):
    p = make_problem("half", 4, geom, nx, ny, 0.1, 0.0 if geom == CAVITY else 0.01, 0.01)
    h = random_state(p.n, p.ncells, seed=9)
    assert abs(p.transport2(h).sum() - h.sum()) <= 1e-12 * np.abs(h).sum()
    assert abs(p.step_second_order(h, 3).sum() - h.sum()) <= 1e-12 * np.abs(h).sum()


@pytest.mark.parametrize("n_half", [2, 4])
def test_second_order_free_molecular_shear_is_exact(n_half):
    """Without collisions every population is uniform at steady state; the second-order face
    values reproduce it, so p_xy = (U_b - U_t)/sqrt(2 pi) on every face (as for first order)."""
    ub, ut = 0.01, -0.01
    p = make_problem("half", n_half, COUETTE, 1, 16, math.inf, ub, ut)
    g = _march_second_order(p, tol=1e-14)
    f = p.face_flux2_y(g)[:, 0]
    np.testing.assert_allclose(f, free_molecular_pxy(ub, ut), rtol=1e-11, atol=0)


@pytest.mark.slow
def test_second_order_variant_converges_at_second_order():
    """Couette, D2Q^h_16, Kn = 0.1: the steady shear of the second-order variant converges to
    the semi-discrete (space- and time-continuous) value with error ratios near 4 per halving
    of dy (first-order upwind: near 2, test above), and the momentum flux is the same through
    every face (the discrete x-momentum balance of the scheme)."""
    x, w = _one_d("half", 2)
    exact = couette_semidiscrete(x, w, 0.1, -1.0, 1.0)["pxy"]
    errs = []
    for ny in (25, 50, 100):
        p = make_problem("half", 2, COUETTE, 1, ny, 0.1, -1.0, 1.0)
        g = _march_second_order(p)
        f = p.face_flux2_y(p.relax_exp(g, 0.5))[:, 0]      # the transported state
        assert np.ptp(f) < 1e-11 * abs(exact)
        errs.append(abs(f.mean() - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.2 < r < 4.6 for r in ratios), (errs, ratios)


def _transpose_state(p, h):
    """The state mirrored in the diagonal x = y: cells (x, y) -> (y, x), each velocity to the
    one with xi_x and xi_y swapped (found by exact node equality)."""
    perm = np.array([int(np.flatnonzero((p.xi_x == p.xi_y[a]) & (p.xi_y == p.xi_x[a]))[0]) for a in range(p.n)])
    out = np.empty_like(h)
    out[perm] = h.reshape(p.n, p.ny, p.nx).transpose(0, 2, 1).reshape(p.n, -1)
    return out


@pytest.mark.parametrize("kind,n", [("half", 2), ("half", 3), ("full", 3), ("full", 4)])
def test_square_cavity_at_rest_is_symmetric_under_transposition(kind, n):
    """With every wall at rest a square cavity is its own mirror image in the diagonal x = y:
    the step (first-order transport, walls, relaxation) and the second-order transport
    commute with the mirror, and the momentum flux sum xi_x xi_y h_upwind through the
    vertical faces equals that through the horizontal faces of the mirrored state (first and
    second order).  An x-transport or x-wall term that differed from its y counterpart (a
    sign, an upwind side, a wall density, an index) breaks the step's equality; a wrong
    upwind side or index in an x-face flux breaks the flux equality.  (A wall at rest emits
    w_a rho_w, whose xi_x xi_y moment vanishes, so the wall faces' fluxes are checked by
    their interior neighbours' values only.)"""
    p = make_problem(kind, n, CAVITY, 7, 7, 0.2, 0.0, 0.0)
    h = random_state(p.n, p.ncells, seed=20 + n)
    hT = _transpose_state(p, h)
    tol = 1e-14
    for f in (lambda v: p.step(v, 3), p.transport2, lambda v: p.step_second_order(v, 2)):
        a, b = _transpose_state(p, f(h)), f(hT)
        assert np.abs(a - b).max() <= tol * np.abs(a).max()
    for fx, fy in ((p.face_flux_x, p.face_flux_y), (p.face_flux2_x, p.face_flux2_y)):
        a, b = fx(h), fy(hT).T
        assert a.shape == b.shape and np.abs(a - b).max() <= tol * np.abs(a).max()


@pytest.mark.parametrize("n_half,geom,nx,ny,xi_max", [
    (4, COUETTE, 1, 100, 3.19989079049),      # largest node of the N = 4 half-range rule (Table 1)
    (4, CAVITY, 128, 128, 3.19989079049),
    (6, CAVITY, 2048, 2048, 4.29471226994),   # largest node of the N = 6 rule
    (4, COUETTE, 3, 40, 3.19989079049),       # a Couette channel several columns wide keeps the x term
])
def test_time_step_and_coefficients_closed_forms(n_half, geom, nx, ny, xi_max):
    """dt = CFL / sum_d (max |xi_d| / dx_d) with CFL 0.9 (the single Couette column has no x
    term), dx = 1/nx, dy = 1/ny (the Couette column's dx = dy), omega = dt / Kn, u_ref the
    larger wall speed; the half-range wall-flux normalisers sum_{xi_d > 0} xi_d w equal
    1/sqrt(2 pi) (the factor of Eq. 9) on both axes."""
    p = make_problem("half", n_half, geom, nx, ny, 0.1, 0.004, -0.01)
    c = p.coeffs
    column = geom == COUETTE and nx == 1
    rate = xi_max * ny + (0.0 if column else xi_max * (ny if geom == COUETTE else nx))
    assert c["dt"] == pytest.approx(0.9 / rate, rel=1e-10)
    assert c["omega"] == pytest.approx(c["dt"] / 0.1, rel=1e-15)
    assert c["u_ref"] == 0.01
    assert c["d_x"] == pytest.approx(1.0 / math.sqrt(2.0 * math.pi), rel=1e-14)
    assert c["d_y"] == pytest.approx(1.0 / math.sqrt(2.0 * math.pi), rel=1e-14)


def test_time_step_is_clamped_to_kn_and_walls_at_rest_give_unit_reference_speed():
    p = make_problem("half", 2, CAVITY, 8, 8, 1e-4, 0.0, 0.0)
    c = p.coeffs
    assert c["dt"] == 1e-4 and c["omega"] == 1.0 and c["u_ref"] == 1.0
    # the time steps of the benchmark workloads to 5 significant digits, computed by hand
    assert make_problem("half", 4, COUETTE, 1, 100, 0.1, 0.01, -0.01).coeffs["dt"] == pytest.approx(2.8126e-3, rel=2e-5)
    assert make_problem("half", 4, CAVITY, 128, 128, 0.1, 0.0, 0.01).coeffs["dt"] == pytest.approx(1.0987e-3, rel=5e-5)
    assert make_problem("half", 6, CAVITY, 2048, 2048, 0.05, 0.0, 0.01).coeffs["dt"] == pytest.approx(5.116e-5, rel=1e-4)
