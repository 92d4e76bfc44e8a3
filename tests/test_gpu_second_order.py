"""GPU parity of the second-order variant (transport order 2, symmetric splitting with exact
half relaxations) and of its face fluxes, against the oracle's literal composition."""
import math

import numpy as np
import pytest

from oracle.march import CAVITY, COUETTE, make_problem as oracle_problem
from paper_1308_0692_gb300 import lbm
from paper_1308_0692_gb300.inputs import random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL_PER_STEP = 2e-6

CASES = [
    # kind, n, geom, nx, ny, kn, u_bottom, u_top
    ("half", 4, COUETTE, 1, 100, 0.1, 0.01, -0.01),
    ("half", 2, COUETTE, 4, 30, 0.05, -0.01, 0.01),      # periodic columns
    ("half", 4, CAVITY, 37, 29, 0.1, 0.0, 0.01),          # ragged segments, four walls
    ("half", 6, CAVITY, 45, 38, 0.05, 0.003, 0.01),       # D2Q^h_144, moving bottom
    ("full", 3, CAVITY, 23, 19, 0.2, 0.0, 0.01),          # D2Q9
    ("half", 4, CAVITY, 3, 3, 0.1, 0.0, 0.01),            # every cell next to a wall
]


def _kind(kind):
    return lbm.LBM_HALF_RANGE_GH if kind == "half" else lbm.LBM_FULL_RANGE_GH


def _sim(case, prec, g0, splitting):
    kind, n, geom, nx, ny, kn, ub, ut = case
    vs = lbm.lbm_make_velocity_set(_kind(kind), n)
    sim = lbm.lbm_init(vs, lbm.make_problem(geom, nx, ny, kn, ub, ut, prec=prec, residual_every=4), g0,
                       stream=torch.cuda.Stream())
    lbm.lbm_set_transport(sim, 2)
    lbm.lbm_set_splitting(sim, splitting)
    assert lbm.lbm_get_transport(sim) == 2
    return sim


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}{c[1]}-{'cav' if c[2] else 'cou'}-{c[3]}x{c[4]}" for c in CASES])
def test_second_order_step_parity_fp64(case):
    kind, n, geom, nx, ny, kn, ub, ut = case
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h0 = random_state(p.n, p.ncells, seed=71)
    steps = 8
    sim = _sim(case, lbm.LBM_FP64, p.relax_exp(h0, 0.5), lbm.LBM_SPLIT_STRANG_EXACT)
    lbm.lbm_step(sim, steps)
    h = p.step_second_order(h0, steps)
    g = p.relax_exp(h, 0.5)
    got = lbm.lbm_get_state(sim)
    assert np.abs(got - g).max() <= FP64_TOL * np.abs(g).max()
    fy, fx = lbm.lbm_face_flux(sim)
    ry = p.face_flux2_y(g)
    assert np.abs(fy - ry).max() <= 1e-11 * max(np.abs(ry).max(), 1e-300)
    if geom == CAVITY:
        rx = p.face_flux2_x(g)
        assert np.abs(fx - rx).max() <= 1e-11 * max(np.abs(rx).max(), 1e-300)
    m, mr = lbm.lbm_moments(sim, wall_shear=False), p.moments(h)
    for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy"):
        base = 1.0 if k in ("rho", "pxx", "pyy") else 0.0
        assert np.abs(m[k] - mr[k]).max() <= 1e-11 * max(np.abs(mr[k] - base).max(), 1e-300), k


@pytest.mark.parametrize("case", CASES[:4], ids=["cou100", "cou-periodic", "cav37x29", "cav45x38-144"])
def test_second_order_step_parity_fp32(case):
    kind, n, geom, nx, ny, kn, ub, ut = case
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    g0 = p.relax_exp(random_state(p.n, p.ncells, seed=72), 0.5).astype(np.float32).astype(np.float64)
    steps = 6
    sim = _sim(case, lbm.LBM_FP32_PERTURB, g0, lbm.LBM_SPLIT_STRANG_EXACT)
    lbm.lbm_step(sim, steps)
    # the stored-state form (pinned against the literal composition in the FP64 test):
    # transport then the exact-relaxation factor exp(-omega) on g
    w = p.coeffs["omega"]
    ref = g0
    for _ in range(steps):
        t = p.transport2(ref)
        eq = p.relax(t, 1.0 / w)
        ref = eq + math.exp(-w) * (t - eq)
    got = lbm.lbm_get_state(sim)
    assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * steps * np.abs(ref).max()


def test_second_order_transport_with_lie_splitting():
    case = CASES[2]
    kind, n, geom, nx, ny, kn, ub, ut = case
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h0 = random_state(p.n, p.ncells, seed=73)
    sim = _sim(case, lbm.LBM_FP64, h0, lbm.LBM_SPLIT_LIE)
    lbm.lbm_step(sim, 5)
    ref = h0
    for _ in range(5):
        ref = p.relax(p.transport2(ref), 1.0)
    got = lbm.lbm_get_state(sim)
    assert np.abs(got - ref).max() <= FP64_TOL * np.abs(ref).max()


def test_second_order_couette_converges_at_second_order():
    """Steady Couette shear of the library's second-order variant (FP64, D2Q^h_64, Kn = 0.1)
    against the semi-discrete solution: error ratios near 4 per halving of dy."""
    from oracle import quadrature as q
    from oracle.couette_exact import couette_semidiscrete
    nodes, weights = q.halfrange_1d(4)
    exact = couette_semidiscrete([float(v) for v in nodes], [float(v) for v in weights], 0.1, -0.01, 0.01)["pxy"]
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    errs = []
    for ny in (50, 100, 200):
        sim = lbm.lbm_init(vs, lbm.make_problem(COUETTE, 1, ny, 0.1, -0.01, 0.01, prec=lbm.LBM_FP64, residual_every=100),
                           stream=torch.cuda.Stream())
        lbm.lbm_set_transport(sim, 2)
        lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_STRANG_EXACT)
        info = lbm.lbm_solve(sim, 1e-13, 5_000_000, 0)
        assert info["residual"] < 1e-13
        fy, _ = lbm.lbm_face_flux(sim)
        assert np.ptp(fy[:, 0]) < 1e-10 * abs(exact)
        errs.append(abs(fy[:, 0].mean() - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.3 < r < 4.5 for r in ratios), (errs, ratios)


def test_order_study_against_semidiscrete_references():
    """The order study of the package, given the semi-discrete Couette shear as its reference
    (D2Q^h_64, Kn = 0.1): the paper's scheme converges at first order (error ratios near 2,
    observed order near 1), the second-order variant at second order (ratios near 4)."""
    from oracle import quadrature as q
    from oracle.couette_exact import couette_semidiscrete
    from paper_1308_0692_gb300 import experiments
    nodes, weights = q.halfrange_1d(4)
    exact = couette_semidiscrete([float(v) for v in nodes], [float(v) for v in weights], 0.1, -0.01, 0.01)["pxy"]
    out = experiments.order_study(kns=(0.1,), nys=(50, 100, 200), n_half=4, exact_pxy={0.1: exact})
    runs = {(r["order"], r["ny"]): r for r in out["runs"]}
    assert len(runs) == 6
    for order, lo, hi in ((1, 1.7, 2.3), (2, 3.3, 4.5)):
        for ny in (100, 200):
            assert lo < runs[(order, ny)]["ratio"] < hi, (order, ny, runs[(order, ny)])
        assert abs(runs[(order, 200)]["observed_order"] - order) < 0.3, runs[(order, 200)]


def test_second_order_rejections():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, 64, 64, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB))
    lbm.lbm_set_transport(sim, 2)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_set_variant(sim, 4, 0)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_solve(sim, 1e-8, 1000, 2)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    lbm.lbm_step(sim, 1)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_transport(sim, 1)
