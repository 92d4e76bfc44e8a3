"""GPU parity of the second-order variant (transport order 2, symmetric splitting with exact
half relaxations) and of its face fluxes, against the oracle's literal composition."""
import math

import numpy as np
import pytest

from oracle.march import CAVITY, COUETTE, make_problem as oracle_problem
from paper_1308_0692_gb300 import lbm
from paper_1308_0692_gb300.inputs import random_cells, random_state

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


def _stored_form_steps(p, g0, steps):
    """The oracle's stored-state form of the variant: second-order transport, then the
    exact relaxation over dt; every state along the way."""
    out = [g0]
    for _ in range(steps):
        out.append(p.relax_exp(p.transport2(out[-1]), 1.0))
    return out


MARCH2 = [
    # n per half-axis, nx, ny, kn, u_bottom, u_top, warps per segment
    (6, 192, 45, 0.05, 0.003, 0.01, 6),    # D2Q^h_144, moving bottom, ragged chunks
    (4, 256, 70, 0.1, 0.0, 0.01, 4),       # D2Q^h_64
    (6, 128, 12, 0.05, 0.0, 0.01, 6),      # the smallest grid the march takes
]


@pytest.mark.parametrize("path", [8, 9])
@pytest.mark.parametrize("case", MARCH2, ids=["cav192x45-144", "cav256x70-64", "cav128x12-144"])
def test_second_order_column_march_matches_oracle(case, path):
    """The second-order column march on the strip-tiled state (its interior rows 2 .. ny-3,
    the wall kernel beside it on the rest) against the oracle's stored-state steps, the
    residual of a residual step included; the segment kernel (load path 0) agrees with it
    to a few FP32 roundings."""
    n, nx, ny, kn, ub, ut, g = case
    p = oracle_problem("half", n, CAVITY, nx, ny, kn, ub, ut)
    g0 = p.relax_exp(random_state(p.n, p.ncells, seed=81), 0.5).astype(np.float32).astype(np.float64)
    steps = 6
    refs = _stored_form_steps(p, g0, steps)
    sim = _sim(("half", n, CAVITY, nx, ny, kn, ub, ut), lbm.LBM_FP32_PERTURB, g0, lbm.LBM_SPLIT_STRANG_EXACT)
    lbm.lbm_set_variant(sim, g, path)
    assert lbm.lbm_get_variant(sim) == (g, path)
    assert lbm.lbm_state_tiling(sim)[0] == 64
    lbm.lbm_step(sim, steps)
    got = lbm.lbm_get_state(sim)
    ref = refs[-1]
    assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * steps * np.abs(ref).max()
    # residual_every = 4: the residual of step 4
    r, st = lbm.lbm_residual(sim)
    d, m = refs[4] - refs[3], refs[4]
    r_ref = math.sqrt(float(np.sum(d * d)) / float(np.sum(m * m)))
    assert st == 4 and abs(r - r_ref) <= 1e-3 * r_ref
    seg = _sim(("half", n, CAVITY, nx, ny, kn, ub, ut), lbm.LBM_FP32_PERTURB, g0, lbm.LBM_SPLIT_STRANG_EXACT)
    lbm.lbm_step(seg, steps)
    assert np.abs(lbm.lbm_get_state(seg) - got).max() <= 4e-7 * steps * np.abs(ref).max()
    # outputs read through the tiles
    fy, fx = lbm.lbm_face_flux(sim)
    ry = p.face_flux2_y(got)
    assert np.abs(fy - ry).max() <= 1e-11 * max(np.abs(ry).max(), 1e-300)
    sim.close()
    seg.close()


@pytest.fixture(scope="module")
def so_bench_case():
    """The benchmark's workload (cavity 2048 x 2048, D2Q^h_144, Kn 0.05, lid 0.01, FP32) with
    the second-order variant: one FP32-representable state and the oracle's stored-state
    step at 400 sampled cells, among them the rows and columns next to the walls and to the
    march's strip and interior edges."""
    nx = ny = 2048
    p = oracle_problem("half", 6, CAVITY, nx, ny, 0.05, 0.0, 0.01)
    h0 = random_state(p.n, p.ncells, seed=83).astype(np.float32).astype(np.float64)
    edges = [(x, y) for y in (0, 1, 2, 3, ny // 2, ny - 4, ny - 3, ny - 2, ny - 1)
             for x in (0, 1, 2, 31, 32, 33, 95, 96, 1023, 1024, nx - 34, nx - 33, nx - 32, nx - 31, nx - 2, nx - 1)]
    cells = random_cells(p.ncells, 400, seed=84, include=[y * nx + x for x, y in edges])
    return p, h0, cells, p.step2_cells(h0, cells)


@pytest.mark.parametrize("variant", [(6, 8), (6, 9), (4, 0)], ids=["march-path8", "march-path9", "segments"])
def test_second_order_full_size_sampled_step(so_bench_case, variant):
    """One second-order step at the benchmark's size through each kernel variant, on
    sampled cells, with and without the residual."""
    p, h0, cells, ref = so_bench_case
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 6)
    idx = torch.as_tensor(np.asarray(cells, dtype=np.int64), device="cuda")
    cy, cx = idx // 2048, idx % 2048
    for residual_every in (1, 2):
        prob = lbm.make_problem(CAVITY, 2048, 2048, 0.05, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB,
                                residual_every=residual_every)
        buf = torch.empty(lbm.lbm_sim_bytes(vs, prob), dtype=torch.uint8, device="cuda")
        sim = lbm.lbm_init(vs, prob, h0, device_buf=buf, stream=torch.cuda.Stream())
        lbm.lbm_set_transport(sim, 2)
        lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_STRANG_EXACT)
        lbm.lbm_set_variant(sim, *variant)
        lbm.lbm_step(sim, 1)
        ptr, step = lbm.lbm_state_device(sim)
        assert step == 1
        tw, shift, tp, rp = lbm.lbm_state_tiling(sim)
        off = ptr - buf.data_ptr()
        if tw:
            nbytes = 4 * (2048 // tw + 1) * tp
            xs = cx + shift
            elems = torch.arange(p.n, device="cuda")[:, None] * tw + ((xs // tw) * tp + cy * rp + xs % tw)[None, :]
        else:
            pa, py = lbm.lbm_state_layout(sim)
            nbytes = 4 * p.n * p.ncells
            elems = torch.arange(p.n, device="cuda")[:, None] * pa + (cy * py + cx)[None, :]
        torch.cuda.synchronize()
        state = buf[off:off + nbytes].view(torch.float32)
        got = state[elems].double().cpu().numpy().T
        assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * np.abs(ref).max(), (variant, residual_every)
        if residual_every == 1:
            r, st = lbm.lbm_residual(sim)
            assert st == 1 and np.isfinite(r) and r > 0
        sim.close()
        del buf, state
    torch.cuda.empty_cache()


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
    # the segment kernel has one warps-per-segment choice (2 for D2Q^h_64 in FP32); the
    # column march exists for load paths 8 and 9 and needs nx a multiple of 64, >= 128
    for variant in ((4, 0), (4, 4), (4, 8), (3, 9)):
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_set_variant(sim, *variant)
        assert e.value.status == lbm.LBM_EUNSUPPORTED, variant
    lbm.lbm_set_variant(sim, 2, 0)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_solve(sim, 1e-8, 1000, 2)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    lbm.lbm_step(sim, 1)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_transport(sim, 1)
