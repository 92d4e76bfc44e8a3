"""Pins of the hybrid half-range / full-range oracle (oracle/hybrid.py), Couette channel and
lid-driven cavity: reductions to the C oracle's pure half-range and pure full-range
marches, exactness of the Hermite projection, conservation, the state at rest, the Couette
antisymmetry and the constancy of the face momentum flux at the steady state, the
cavity's mirror symmetry at a small lid speed."""
import math

import numpy as np
import pytest

from oracle import hybrid as hy
from oracle.march import COUETTE, make_problem

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_hermite_table_closed_forms():
    x = np.linspace(-3.0, 3.0, 13)
    t = hy.hermite_table(x, 4)
    np.testing.assert_allclose(t[2], x ** 2 - 1.0, atol=1e-14)
    np.testing.assert_allclose(t[3], x ** 3 - 3.0 * x, atol=1e-13)
    np.testing.assert_allclose(t[4], x ** 4 - 6.0 * x ** 2 + 3.0, atol=1e-12)


@pytest.mark.parametrize("n_half", [2, 3, 4])
def test_projection_exact_on_full_range_data(n_half):
    """F -> F is the identity (the K^2 tensor Hermite functions interpolate at the K-point
    nodes), and F -> H -> F too (H integrates the products exactly)."""
    q = n_half - 1
    H, F = hy.VelocitySet("half", n_half, q), hy.VelocitySet("full", n_half, q)
    rng = np.random.default_rng(n_half)
    for _ in range(3):
        h = rng.standard_normal(F.n)
        np.testing.assert_allclose(hy.project(h, F, F, q), h, atol=1e-12 * np.abs(h).max())
        back = hy.project(hy.project(h, F, H, q), H, F, q)
        np.testing.assert_allclose(back, h, atol=1e-12 * np.abs(h).max())


@pytest.mark.parametrize("n_half", [2, 4])
def test_projection_reproduces_polynomials(n_half):
    """w phi with phi a tensor polynomial of degree <= N - 1 per axis maps to w phi on the
    other set, both ways."""
    q = n_half - 1
    H, F = hy.VelocitySet("half", n_half, q), hy.VelocitySet("full", n_half, q)
    rng = np.random.default_rng(7)
    c = rng.standard_normal((q + 1, q + 1))

    def phi(s):
        return sum(c[m, n] * s.xi_x ** m * s.xi_y ** n for m in range(q + 1) for n in range(q + 1))

    np.testing.assert_allclose(hy.project(H.w * phi(H), H, F, q), F.w * phi(F), rtol=0, atol=1e-12)
    np.testing.assert_allclose(hy.project(F.w * phi(F), F, H, q), H.w * phi(H), rtol=0, atol=1e-12)


@pytest.mark.parametrize("kn", [0.1, 2.0])
def test_all_half_range_reduces_to_half_range_march(kn):
    ny = 14
    p = hy.HybridCouette(4, ny, kn, 0.01, -0.01, layer=ny // 2)
    got = np.array(p.step(p.zeros(), 25)).T
    ref = make_problem("half", 4, COUETTE, 1, ny, kn, 0.01, -0.01)
    want = ref.step(ref.zeros(), 25)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("kn", [0.1, 2.0])
def test_all_full_range_reduces_to_full_range_march(kn):
    ny = 14
    p = hy.HybridCouette(4, ny, kn, 0.01, -0.01, layer=0)
    got = np.array(p.step(p.zeros(), 25)).T
    ref = make_problem("full", 4, COUETTE, 1, ny, kn, 0.01, -0.01)
    want = ref.step(ref.zeros(), 25)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_mass_conserved_and_rest_state_kept():
    p = hy.HybridCouette(3, 18, 0.2, 0.01, -0.01, layer=4)
    rng = np.random.default_rng(3)
    h = [rng.standard_normal(p.vset(j).n) * 1e-2 for j in range(p.ny)]
    m0 = p.mass(h)
    assert abs(p.mass(p.step(h, 30)) - m0) < 1e-15
    rest = hy.HybridCouette(3, 18, 0.2, 0.0, 0.0, layer=4)
    h = [0.25 * rest.vset(j).w for j in range(rest.ny)]
    for a, b in zip(rest.step(h, 20), h):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-16)


def test_antisymmetry_and_constant_face_flux_at_steady_state():
    """Plates +u / -u with layers placed symmetrically: u(y) = -u(1 - y); at the steady state
    the momentum flux through every face (interfaces included) is the same."""
    p = hy.HybridCouette(4, 24, 0.3, 0.01, -0.01, layer=5)
    h, steps, r = p.march(p.zeros(), 100000, 100, 1e-12)
    assert r < 1e-12
    u = p.ux(h)
    np.testing.assert_allclose(u, -u[::-1], rtol=0, atol=1e-13 * np.abs(u).max())
    f = p.face_flux(h)
    assert (f.max() - f.min()) <= 1e-8 * np.abs(f).max()


def test_interfaces_move_the_result_between_the_two_models():
    """At Kn = 1 the hybrid's shear stress lies between the full-range and the half-range
    results and approaches the latter as the half-range layers grow."""
    ny, kn = 24, 1.0

    def pxy(layer):
        p = hy.HybridCouette(4, ny, kn, 0.01, -0.01, layer=layer)
        h, _, r = p.march(p.zeros(), 100000, 100, 1e-11)
        return p.face_flux(h).mean()

    half, full = pxy(ny // 2), pxy(0)
    e = [abs(pxy(L) - half) for L in (2, 6)]
    assert e[1] < e[0] < abs(full - half)
    assert math.copysign(1, pxy(6) - half) == math.copysign(1, full - half)


@pytest.mark.parametrize("layer,kind", [(4, "half"), (0, "full")])
def test_cavity_reduces_to_pure_marches(layer, kind):
    """All cells half-range (layer beyond the half width) or all full-range: the C oracle's
    cavity march on that set."""
    p = hy.HybridCavity(3, 7, 6, 0.2, 0.0, 0.01, layer)
    got = np.array(p.step(p.zeros(), 12)).T
    from oracle.march import CAVITY
    ref = make_problem(kind, 3, CAVITY, 7, 6, 0.2, 0.0, 0.01)
    want = ref.step(ref.zeros(), 12)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_cavity_mass_conserved_and_rest_state_kept():
    p = hy.HybridCavity(3, 9, 8, 0.2, 0.003, 0.01, 2)
    rng = np.random.default_rng(2)
    h = [rng.standard_normal(p.vset(c).n) * 1e-2 for c in range(p.ncells)]
    assert abs(p.mass(p.step(h, 15)) - p.mass(h)) < 1e-14
    r = hy.HybridCavity(3, 9, 8, 0.2, 0.0, 0.0, 2)
    h = [0.2 * r.vset(c).w for c in range(r.ncells)]
    for a, b in zip(r.step(h, 6), h):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-16)


def test_cavity_mirror_symmetry_at_small_lid_speed():
    """u_x(1 - x, y) = u_x(x, y) and u_y(1 - x, y) = -u_y(x, y), broken only at O(u_w) by the
    wall product rho_w u_w (Eq. 8): checked at u_w = 1e-8 with half-range layers placed
    symmetrically."""
    p = hy.HybridCavity(3, 10, 9, 0.3, 0.0, 1e-8, 3)
    ux, uy = p.velocity(p.step(p.zeros(), 30))
    scale = max(np.abs(ux).max(), np.abs(uy).max())
    np.testing.assert_allclose(ux, ux[:, ::-1], rtol=0, atol=1e-6 * scale)
    np.testing.assert_allclose(uy, -uy[:, ::-1], rtol=0, atol=1e-6 * scale)
    assert scale > 0


def _mirror_diagonal(p, h):
    """Cell (x, y) -> (y, x) of a square hybrid cavity, each cell's velocities permuted so
    that xi_x and xi_y swap (the layers are symmetric, so every cell keeps its set)."""
    out = [None] * p.ncells
    for y in range(p.ny):
        for x in range(p.nx):
            c, cm = y * p.nx + x, x * p.nx + y
            s = p.vset(c)
            assert p.vset(cm) is s
            perm = [int(np.flatnonzero((s.xi_x == s.xi_y[a]) & (s.xi_y == s.xi_x[a]))[0]) for a in range(s.n)]
            v = np.empty(s.n)
            v[perm] = h[c]
            out[cm] = v
    return out


@pytest.mark.parametrize("n_half,layer", [(2, 1), (3, 2), (4, 3)])
def test_cavity_at_rest_is_symmetric_under_transposition(n_half, layer):
    """With every wall at rest a square hybrid cavity is its own mirror image in the diagonal
    x = y: stepping a random state commutes with the mirror, so the x-interface projections,
    face fluxes and full-range corrections match their y counterparts term by term."""
    p = hy.HybridCavity(n_half, 8, 8, 0.2, 0.0, 0.0, layer)
    rng = np.random.default_rng(40 + n_half)
    h = [rng.standard_normal(p.vset(c).n) * 1e-2 for c in range(p.ncells)]
    a = _mirror_diagonal(p, p.step(h, 5))
    b = p.step(_mirror_diagonal(p, h), 5)
    scale = max(np.abs(v).max() for v in a)
    for va, vb in zip(a, b):
        np.testing.assert_allclose(va, vb, rtol=0, atol=1e-14 * scale)
