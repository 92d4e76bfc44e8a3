"""Batched persistent sweep: every instance of a mixed batch against the FP64 oracle, the
convergence bookkeeping, and the bounded-wait error path of the grid barrier."""
import math

import numpy as np
import pytest

from oracle.march import CAVITY, COUETTE, make_problem as oracle_problem
from paper_1308_0692_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# per step the FP32 batch kernel differs from the FP64 oracle by single-precision rounding
FP32_TOL_PER_STEP = 2e-6

INSTANCES = [
    # geom, nx, ny, kn, u_bottom, u_top
    (COUETTE, 1, 64, 0.01, 0.01, -0.01),
    (COUETTE, 1, 131, 0.5, 0.007, -0.007),
    (COUETTE, 1, 97, 10.0, 0.02, -0.02),
    (CAVITY, 33, 33, 0.1, 0.0, 0.01),
    (CAVITY, 64, 64, 0.03, 0.0, 0.015),
    (CAVITY, 40, 40, 2.0, 0.0, 0.005),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_0692_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _probs(residual_every=10):
    return [lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP32_PERTURB, residual_every=residual_every)
            for g, nx, ny, kn, ub, ut in INSTANCES]


# cavities of awkward shapes for the column march: ragged strips, one- and two-row chunks,
# a strip narrower than a warp, a non-zero bottom-wall speed
ODD = [
    (CAVITY, 70, 9, 0.2, 0.0, 0.01),
    (CAVITY, 3, 2, 1.0, 0.0, 0.02),
    (CAVITY, 97, 131, 0.05, 0.004, 0.012),
    (COUETTE, 1, 7, 0.3, 0.01, -0.01),
]


@pytest.mark.parametrize("schedule", [(4, 0, 0), (2, 0, 2), (1, 1, 1)])
@pytest.mark.parametrize("march", [True, False])
def test_batch_matches_oracle_per_instance(schedule, march):
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    b = lbm.lbm_batch_init(vs, _probs(), stream=torch.cuda.Stream())
    lbm.lbm_batch_set_schedule(b, *schedule)
    lbm.lbm_batch_set_march(b, march)
    steps = 30
    lbm.lbm_batch_advance(b, 13, 0.0)      # two launches, uneven split
    lbm.lbm_batch_advance(b, steps - 13, 0.0)
    n_active, step = lbm.lbm_batch_poll(b)
    assert n_active == len(INSTANCES) and step == steps
    for i, (g, nx, ny, kn, ub, ut) in enumerate(INSTANCES):
        p = oracle_problem("half", 4, g, nx, ny, kn, ub, ut)
        ref = p.step(p.zeros(), steps)
        got = lbm.lbm_batch_get_state(b, i)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= FP32_TOL_PER_STEP * steps, (i, err)


@pytest.mark.parametrize("n_half,rows_per_warp", [(2, 1), (2, 2), (4, 1), (4, 2), (4, 4)])
def test_batch_column_march_odd_shapes(n_half, rows_per_warp):
    """The column march on ragged strips, short chunks and tiny cavities agrees with the FP64
    oracle step by step (and the Couette instance beside them with the segment kernel)."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    probs = [lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP32_PERTURB, residual_every=10)
             for g, nx, ny, kn, ub, ut in ODD]
    b = lbm.lbm_batch_init(vs, probs, stream=torch.cuda.Stream())
    m = 2 * n_half
    lbm.lbm_batch_set_march(b, True, 0, m // rows_per_warp)     # warps per item
    info = lbm.lbm_batch_get_march(b)
    assert info["on"] and info["items"] > 0 and info["warps_per_item"] == m // rows_per_warp
    steps = 25
    lbm.lbm_batch_advance(b, steps, 0.0)
    assert lbm.lbm_batch_poll(b) == (len(ODD), steps)
    for i, (g, nx, ny, kn, ub, ut) in enumerate(ODD):
        p = oracle_problem("half", n_half, g, nx, ny, kn, ub, ut)
        ref = p.step(p.zeros(), steps)
        got = lbm.lbm_batch_get_state(b, i)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= FP32_TOL_PER_STEP * steps, (i, err)


def test_batch_convergence_and_freezing():
    """Instances converge at different step counts; each is frozen at the residual check that
    first saw r < tol and its state stays put while the others march on."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    b = lbm.lbm_batch_init(vs, _probs(residual_every=50), stream=torch.cuda.Stream())
    tol = 1e-6
    for _ in range(400):
        lbm.lbm_batch_advance(b, 500, tol)
        n_active, step = lbm.lbm_batch_poll(b)
        if n_active == 0:
            break
    assert n_active == 0
    stats = [lbm.lbm_batch_status(b, i) for i in range(len(INSTANCES))]
    assert all(s["converged"] and s["residual"] < tol for s in stats)
    assert all(s["steps"] % 50 == 0 for s in stats)
    assert len({s["steps"] for s in stats}) > 1            # they did converge at different times
    # a frozen state does not move: one more launch leaves every state unchanged
    before = [lbm.lbm_batch_get_state(b, i) for i in range(len(INSTANCES))]
    lbm.lbm_batch_advance(b, 100, tol)
    lbm.lbm_batch_poll(b)
    for i in range(len(INSTANCES)):
        np.testing.assert_array_equal(lbm.lbm_batch_get_state(b, i), before[i])
    # the converged Couette state agrees with the single-simulation FP32 march of the same length
    g, nx, ny, kn, ub, ut = INSTANCES[2]
    sim = lbm.lbm_init(vs, lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP32_PERTURB, residual_every=50))
    lbm.lbm_step(sim, stats[2]["steps"])
    ref = lbm.lbm_get_state(sim)
    assert np.abs(before[2] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_batch_barrier_timeout_reports_error():
    """A grid-barrier wait limit of a few cycles makes the waits give up: the kernel returns
    and the next poll reports LBM_ETIMEOUT (no hang, the context stays usable)."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    b = lbm.lbm_batch_init(vs, _probs(), stream=torch.cuda.Stream())
    lbm.lbm_batch_set_timeout(b, 1)
    lbm.lbm_batch_advance(b, 50, 0.0)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_batch_poll(b)
    assert e.value.status == lbm.LBM_ETIMEOUT
    # the device is still fine
    x = torch.ones(10, device="cuda")
    assert float(x.sum()) == 10.0


def test_batch_rejects_mixed_or_unsupported():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    probs = _probs()
    probs[1].prec = lbm.LBM_FP64
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_batch_bytes(vs, probs)
    assert e.value.status == lbm.LBM_EINVAL
    vs6 = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 6)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_batch_bytes(vs6, _probs())
    assert e.value.status == lbm.LBM_EUNSUPPORTED


def _fp64_steady(vs, g, nx, ny, kn, ub, ut):
    sim = lbm.lbm_init(vs, lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP64, residual_every=100),
                       stream=torch.cuda.Stream())
    info = lbm.lbm_solve(sim, 1e-12, 2_000_000, 0)
    assert info["residual"] < 1e-12
    m = lbm.lbm_moments(sim)
    return m["ux"], m["uy"]


@pytest.mark.parametrize("n_half,two_rows", [(4, False), (2, False), (4, True)])
def test_batch_refine_meets_1e5_per_instance(n_half, two_rows):
    """Batched FP32 march to 1e-6, then the batched refinement (FP64 defect, FP32 correction
    march of all instances in one launch) to a defect target of 1e-10: every instance's
    steady velocity field is within 1e-5 of the FP64 steady state (max |du| / u_w); step
    counts and convergence flags are unchanged; and max_sweeps = 0 changes nothing."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    b = lbm.lbm_batch_init(vs, _probs(residual_every=100), stream=torch.cuda.Stream())
    if two_rows:
        lbm.lbm_batch_set_march(b, True, 0, n_half)
    for _ in range(400):
        lbm.lbm_batch_advance(b, 500, 1e-6)
        if lbm.lbm_batch_poll(b)[0] == 0:
            break
    stats = [lbm.lbm_batch_status(b, i) for i in range(len(INSTANCES))]
    assert all(s["converged"] != s["stalled"] for s in stats), stats      # every instance frozen
    assert all(s["residual"] < 1e-6 for s in stats if s["converged"]), stats
    before = [lbm.lbm_batch_get_state(b, i) for i in range(len(INSTANCES))]
    info0 = lbm.lbm_batch_refine(b, 1e-10, 0)
    assert all(r["sweeps"] == 0 and r["correction_steps"] == 0 for r in info0)
    for i in range(len(INSTANCES)):
        np.testing.assert_array_equal(lbm.lbm_batch_get_state(b, i), before[i])
    info = lbm.lbm_batch_refine(b, 1e-10, 3)
    assert [lbm.lbm_batch_status(b, i) for i in range(len(INSTANCES))] == stats
    for i, (g, nx, ny, kn, ub, ut) in enumerate(INSTANCES):
        assert info[i]["sweeps"] >= 1 and info[i]["correction_steps"] > 0, (i, info[i])
        assert info[i]["defect"] < info0[i]["defect"], (i, info[i], info0[i])
        uw = max(abs(ub), abs(ut))
        m = oracle_problem("half", n_half, g, nx, ny, kn, ub, ut).moments(lbm.lbm_batch_get_state(b, i))
        ux, uy = _fp64_steady(vs, g, nx, ny, kn, ub, ut)
        err = max(np.abs(m["ux"] - ux).max(), np.abs(m["uy"] - uy).max()) / uw
        assert err < 1e-5, (i, err, info[i])


def test_batch_refine_matches_single_simulation_refinement():
    """The batched refinement and lbm_solve's refinement of the same converged FP32 state
    (lbm_solve marches one more residual interval first) take about the same number of
    sweeps and end within FP32 rounding of each other."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    g, nx, ny, kn, ub, ut = INSTANCES[4]
    prob = lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP32_PERTURB, residual_every=100)
    b = lbm.lbm_batch_init(vs, [prob], stream=torch.cuda.Stream())
    for _ in range(400):
        lbm.lbm_batch_advance(b, 500, 1e-6)
        if lbm.lbm_batch_poll(b)[0] == 0:
            break
    h0 = lbm.lbm_batch_get_state(b, 0)
    sim = lbm.lbm_init(vs, prob, h0, stream=torch.cuda.Stream())
    sinfo = lbm.lbm_solve(sim, 1e-10, 1_000_000, 3)
    binfo = lbm.lbm_batch_refine(b, 1e-10, 3)[0]
    assert abs(binfo["sweeps"] - sinfo["sweeps"]) <= 1
    hb, hs = lbm.lbm_batch_get_state(b, 0), lbm.lbm_get_state(sim)
    assert np.abs(hb - hs).max() <= 1e-5 * np.abs(hs).max()


def test_batch_chunk_height_does_not_change_results():
    """Any rows-per-chunk choice of the column march (planned or fixed) gives the same states:
    the items tile each cavity exactly and every item's arithmetic is independent of its
    chunk; heights below 4 are rejected."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    states = []
    for rows in (0, 4, 7, 64):
        b = lbm.lbm_batch_init(vs, _probs(), stream=torch.cuda.Stream())
        lbm.lbm_batch_set_march(b, True, rows)
        info = lbm.lbm_batch_get_march(b)
        assert info["on"] and (rows == 0 or info["rows_per_chunk"] == rows)
        lbm.lbm_batch_advance(b, 15, 0.0)
        lbm.lbm_batch_poll(b)
        states.append([lbm.lbm_batch_get_state(b, i) for i in range(len(INSTANCES))])
        if rows == 64:
            with pytest.raises(lbm.LBMError) as e:
                lbm.lbm_batch_set_march(b, True, 3)
            assert e.value.status == lbm.LBM_EINVAL
            with pytest.raises(lbm.LBMError) as e:
                lbm.lbm_batch_set_march(b, True, 0, 3)        # warps per item: 8, 4 or 2 here
            assert e.value.status == lbm.LBM_EINVAL
        b.close()
    for other in states[1:]:
        for a, c in zip(states[0], other):
            np.testing.assert_array_equal(a, c)


def test_batch_freezes_instances_at_the_fp32_floor():
    """A tolerance below the FP32 rounding floor of the per-step change: every instance still
    freezes -- by the stagnation rule (no 1 % improvement over 20 checks) at its floor, or by
    the tolerance where its FP32 state stops changing altogether -- in finitely many steps."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    b = lbm.lbm_batch_init(vs, _probs(residual_every=50), stream=torch.cuda.Stream())
    tol = 1e-13
    done = 0
    while done < 400_000:
        lbm.lbm_batch_advance(b, 1000, tol)
        done += 1000
        if lbm.lbm_batch_poll(b)[0] == 0:
            break
    stats = [lbm.lbm_batch_status(b, i) for i in range(len(INSTANCES))]
    assert all(s["converged"] != s["stalled"] for s in stats), stats      # every instance frozen
    assert all(s["residual"] < 1e-6 for s in stats), [s["residual"] for s in stats]
    assert any(s["stalled"] for s in stats), stats
    # converged means below the tolerance; a stalled instance stopped at or above it
    assert all((s["residual"] < tol) == s["converged"] for s in stats), stats
    assert max(s["steps"] for s in stats) < done


def test_compensated_fp32_wall_sums_at_the_worst_case():
    """The batched column march forms the wall densities of Eq. 9 in compensated FP32 (TwoSum),
    the FP64 march in FP64.  At the hardest case for those sums -- a 256^2 cavity at Kn = 0.01,
    the longest walls and the slowest modes, next to a 512-cell Kn = 0.01 channel -- the batch
    marched to 5e-8 and refined to a defect of 1e-10 agrees with the FP64 march (to 1e-11) on
    the lid shear (every lid face and their mean, the drag), the density of the wall rows, the
    side-wall shear and the velocity field, all to 1e-5 relative."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    insts = [(CAVITY, 256, 256, 0.01, 0.0, 0.01), (COUETTE, 1, 512, 0.01, 0.01, -0.01)]
    probs = [lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP32_PERTURB, residual_every=100)
             for g, nx, ny, kn, ub, ut in insts]
    b = lbm.lbm_batch_init(vs, probs, stream=torch.cuda.Stream())
    lbm.lbm_batch_set_march(b, True)
    for _ in range(2000):
        lbm.lbm_batch_advance(b, 1000, 5e-8)
        if lbm.lbm_batch_poll(b)[0] == 0:
            break
    info = lbm.lbm_batch_refine(b, 1e-10, 3, 1e-10, 4_000_000)
    for i, (g, nx, ny, kn, ub, ut) in enumerate(insts):
        uw = max(abs(ub), abs(ut))
        p = oracle_problem("half", 4, g, nx, ny, kn, ub, ut)
        h32 = lbm.lbm_batch_get_state(b, i)
        sim = lbm.lbm_init(vs, lbm.make_problem(g, nx, ny, kn, ub, ut, prec=lbm.LBM_FP64, residual_every=100),
                           stream=torch.cuda.Stream())
        ref = lbm.lbm_solve(sim, 1e-11, 4_000_000, 0)
        assert ref["residual"] < 1e-11
        h64 = lbm.lbm_get_state(sim)
        sim.close()
        m32, m64 = p.moments(h32), p.moments(h64)
        du = max(np.abs(m32["ux"] - m64["ux"]).max(), np.abs(m32["uy"] - m64["uy"]).max()) / uw
        assert du < 1e-5, (i, du, info[i])
        # wall rows: density perturbation rho - 1 relative to its largest value there (or to u_w
        # where it vanishes: the antisymmetric channel has rho = 1 exactly)
        for row in (0, ny - 1):
            scale = max(np.abs(m64["rho"][row] - 1.0).max(), uw)
            assert np.abs(m32["rho"][row] - m64["rho"][row]).max() <= 1e-5 * scale, (i, row)
        fy32, fy64 = p.face_flux_y(h32), p.face_flux_y(h64)
        for j in (0, ny):                               # bottom wall and lid
            scale = np.abs(fy64[j]).max()
            assert np.abs(fy32[j] - fy64[j]).max() <= 1e-5 * scale, (i, j)
            assert abs(fy32[j].mean() - fy64[j].mean()) <= 1e-5 * abs(fy64[j].mean()), (i, j)
        if g == CAVITY:
            fx32, fx64 = p.face_flux_x(h32), p.face_flux_x(h64)
            for j in (0, nx):                           # side walls
                assert np.abs(fx32[:, j] - fx64[:, j]).max() <= 1e-5 * np.abs(fx64[:, j]).max(), (i, j)
    b.close()
