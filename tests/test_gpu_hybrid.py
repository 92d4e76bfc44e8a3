"""Hybrid half-range / full-range coupling on the GPU (lbm_hybrid_*), Couette column and
lid-driven cavity, against the FP64 numpy oracle (oracle/hybrid.py): state after a number
of steps from seeded random and cold states (FP64, 1e-12 relative), steady profiles,
conservation and the error paths."""
import numpy as np
import pytest

from oracle import hybrid as hy
from paper_1308_0692_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # n_half, ny, kn, u_bottom, u_top, layer
    (4, 30, 0.1, 0.01, -0.01, 6),
    (2, 17, 1.0, 0.02, 0.005, 3),      # odd ny, plates not antisymmetric
    (6, 20, 0.5, 0.01, -0.01, 4),      # 36 Hermite coefficients, 144 half-range velocities
    (3, 12, 0.2, 0.0, 0.015, 0),       # all full-range
    (3, 12, 0.2, 0.015, 0.0, 6),       # all half-range
    (4, 9, 0.05, 0.01, -0.01, 8),      # layer > ny / 2
    (4, 2, 0.3, 0.01, -0.01, 1),       # two cells
    (4, 25, 10.0, 0.01, -0.01, 1),     # one half-range cell per plate
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_0692_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _pack(h):
    return np.concatenate([np.asarray(v, dtype=np.float64) for v in h])


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("start", ["cold", "random"])
def test_hybrid_steps_match_oracle(case, start):
    n, ny, kn, ub, ut, layer = case
    p = hy.HybridCouette(n, ny, kn, ub, ut, layer)
    hb = lbm.lbm_hybrid_init(lbm.LBM_COUETTE, n, 1, ny, kn, ub, ut, layer, stream=torch.cuda.Stream())
    q = lbm.lbm_hybrid_query(hb)
    assert q["unknowns"] == p.unknowns()
    assert q["half_range_cells"] == sum(p.half)
    assert q["dt"] == pytest.approx(p.dt, rel=1e-15)
    if start == "random":
        rng = np.random.default_rng(ny * 100 + layer)
        h0 = [rng.standard_normal(p.vset(j).n) * 1e-2 for j in range(ny)]
        lbm.lbm_hybrid_set_state(hb, _pack(h0))
    else:
        h0 = p.zeros()
    steps = 37
    lbm.lbm_hybrid_step(hb, 20)
    lbm.lbm_hybrid_step(hb, steps - 20)
    got = lbm.lbm_hybrid_get_state(hb)
    want = _pack(p.step(h0, steps))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the residual of the last step, and the profile of the state reached
    prev = _pack(p.step(h0, steps - 1))
    r = lbm.lbm_hybrid_residual(hb)
    r_want = np.linalg.norm(want - prev) / np.linalg.norm(want)
    assert r == pytest.approx(r_want, rel=1e-9)
    ux = lbm.lbm_hybrid_velocity(hb)[0][:, 0]
    pxy = lbm.lbm_hybrid_face_flux(hb)
    hw = p.step(h0, steps)
    np.testing.assert_allclose(ux, p.ux(hw), rtol=0, atol=1e-13 * max(np.abs(p.ux(hw)).max(), 1e-300))
    fw = p.face_flux(hw)
    np.testing.assert_allclose(pxy, fw, rtol=0, atol=1e-12 * max(np.abs(fw).max(), 1e-300))
    hb.close()


def test_hybrid_steady_state_matches_oracle_and_conserves():
    n, ny, kn, ub, ut, layer = 4, 30, 0.3, 0.01, -0.01, 6
    p = hy.HybridCouette(n, ny, kn, ub, ut, layer)
    href, _, r = p.march(p.zeros(), 200000, 100, 1e-12)
    assert r < 1e-12
    hb = lbm.lbm_hybrid_init(lbm.LBM_COUETTE, n, 1, ny, kn, ub, ut, layer, stream=torch.cuda.Stream())
    info = lbm.lbm_hybrid_solve(hb, 1e-12, 200000, 100)
    assert info["residual"] < 1e-12
    ux = lbm.lbm_hybrid_velocity(hb)[0][:, 0]
    pxy = lbm.lbm_hybrid_face_flux(hb)
    assert np.abs(ux - p.ux(href)).max() / 0.01 < 1e-9
    fr = p.face_flux(href)
    assert np.abs(pxy - fr).max() / np.abs(fr).max() < 1e-9
    assert (pxy.max() - pxy.min()) <= 1e-8 * np.abs(pxy).max()      # constant through every face
    # mass conservation from a random state
    rng = np.random.default_rng(5)
    h0 = [rng.standard_normal(p.vset(j).n) * 1e-2 for j in range(ny)]
    lbm.lbm_hybrid_set_state(hb, _pack(h0))
    lbm.lbm_hybrid_step(hb, 200)
    assert abs(lbm.lbm_hybrid_get_state(hb).sum() - _pack(h0).sum()) < 1e-14
    hb.close()


CAVITY_CASES = [
    # n_half, nx, ny, kn, u_bottom, u_top, layer
    (3, 9, 8, 0.2, 0.003, 0.01, 2),
    (4, 12, 12, 0.1, 0.0, 0.01, 3),
    (2, 11, 7, 1.0, 0.0, 0.02, 1),
    (3, 7, 6, 0.2, 0.0, 0.01, 0),      # all full-range
    (3, 7, 6, 0.2, 0.0, 0.01, 4),      # all half-range
    (6, 6, 5, 0.5, 0.0, 0.01, 1),      # 144 half-range velocities next to 36 full-range
    (4, 96, 80, 0.1, 0.002, 0.01, 5),  # tiles of 32 cells, runs across row ends, tiles mixing interface cells
    (5, 70, 37, 0.3, 0.0, 0.01, 3),    # odd full-range set, ragged tiles
]


@pytest.mark.parametrize("case", CAVITY_CASES)
@pytest.mark.parametrize("start", ["cold", "random"])
def test_hybrid_cavity_steps_match_oracle(case, start):
    n, nx, ny, kn, ub, ut, layer = case
    p = hy.HybridCavity(n, nx, ny, kn, ub, ut, layer)
    hb = lbm.lbm_hybrid_init(lbm.LBM_CAVITY, n, nx, ny, kn, ub, ut, layer, stream=torch.cuda.Stream())
    q = lbm.lbm_hybrid_query(hb)
    assert q["unknowns"] == p.unknowns() and q["half_range_cells"] == sum(p.half)
    assert q["dt"] == pytest.approx(p.dt, rel=1e-15)
    if start == "random":
        rng = np.random.default_rng(nx * 31 + layer)
        h0 = [rng.standard_normal(p.vset(c).n) * 1e-2 for c in range(p.ncells)]
        lbm.lbm_hybrid_set_state(hb, _pack(h0))
    else:
        h0 = p.zeros()
    steps = 23
    lbm.lbm_hybrid_step(hb, steps)
    got = lbm.lbm_hybrid_get_state(hb)
    hw = p.step(h0, steps)
    want = _pack(hw)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    ux, uy = lbm.lbm_hybrid_velocity(hb)
    wx, wy = p.velocity(hw)
    scale = max(np.abs(wx).max(), np.abs(wy).max())
    np.testing.assert_allclose(ux, wx, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(uy, wy, rtol=0, atol=1e-12 * scale)
    if start == "random":
        assert abs(got.sum() - _pack(h0).sum()) < 1e-13
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_hybrid_face_flux(hb)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    hb.close()


def test_hybrid_rejects_invalid_arguments():
    C, V = lbm.LBM_COUETTE, lbm.LBM_CAVITY
    for args in [(C, 1, 1, 10, 0.1, 0.0, 0.01, 2), (C, 7, 1, 10, 0.1, 0.0, 0.01, 2), (C, 4, 1, 1, 0.1, 0.0, 0.01, 0),
                 (C, 4, 1, 10, 0.0, 0.0, 0.01, 2), (C, 4, 1, 10, 0.1, 0.0, 0.01, -1), (C, 4, 3, 10, 0.1, 0.0, 0.01, 2),
                 (V, 4, 1, 10, 0.1, 0.0, 0.01, 2), (5, 4, 8, 8, 0.1, 0.0, 0.01, 2)]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_hybrid_init(*args)
        assert e.value.status == lbm.LBM_EINVAL
    hb = lbm.lbm_hybrid_init(C, 4, 1, 10, 0.1, 0.0, 0.01, 2)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_hybrid_residual(hb)           # no step taken yet
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(ValueError):
        lbm.lbm_hybrid_set_state(hb, np.zeros(3))
    hb.close()


# ---- FP32 hybrid march with FP64 defect correction (lbm_hybrid_set_precision, lbm_hybrid_refine)

FP32_CASES = [
    # n_half, nx, ny, kn, u_bottom, u_top, layer
    (4, 48, 40, 0.1, 0.0, 0.01, 4),
    (2, 33, 30, 1.0, 0.0, 0.02, 3),
    (6, 20, 18, 0.5, 0.003, 0.01, 2),
    (3, 7, 6, 0.2, 0.0, 0.01, 0),      # all full-range
]


@pytest.mark.parametrize("case", FP32_CASES)
def test_hybrid_fp32_steps_match_oracle(case):
    """The FP32 march (every cell in FP32, the interface projections with FP32 tables)
    against the FP64 oracle from an FP32-representable state, to FP32 accuracy per step."""
    n, nx, ny, kn, ub, ut, layer = case
    p = hy.HybridCavity(n, nx, ny, kn, ub, ut, layer)
    rng = np.random.default_rng(nx * 7 + layer)
    h0 = [(rng.standard_normal(p.vset(c).n) * 1e-2).astype(np.float32).astype(np.float64) for c in range(p.ncells)]
    hb = lbm.lbm_hybrid_init(lbm.LBM_CAVITY, n, nx, ny, kn, ub, ut, layer, stream=torch.cuda.Stream())
    lbm.lbm_hybrid_set_state(hb, _pack(h0))
    lbm.lbm_hybrid_set_precision(hb, lbm.LBM_FP32_PERTURB)
    assert np.array_equal(lbm.lbm_hybrid_get_state(hb), _pack(h0))        # FP32-representable: exact
    steps = 6
    lbm.lbm_hybrid_step(hb, steps)
    got = lbm.lbm_hybrid_get_state(hb)
    want = _pack(p.step(h0, steps))
    assert np.abs(got - want).max() <= 2e-6 * steps * np.abs(want).max()
    assert np.isfinite(lbm.lbm_hybrid_residual(hb))
    ux, uy = lbm.lbm_hybrid_velocity(hb)
    assert np.isfinite(ux).all() and np.isfinite(uy).all()
    # back to FP64: the state carries over
    lbm.lbm_hybrid_set_precision(hb, lbm.LBM_FP64)
    assert np.array_equal(lbm.lbm_hybrid_get_state(hb), got)
    hb.close()


@pytest.mark.parametrize("case", [(4, 40, 40, 0.1, 0.0, 0.01, 4), (4, 32, 24, 1.0, 0.0, 0.01, 3)])
def test_hybrid_fp32_refined_reaches_the_fp64_steady_state(case):
    """FP32 march to its floor, then the FP64-defect refinement: the steady velocity field
    agrees with the FP64 hybrid march to 1e-12 within 1e-5 of the lid speed.  The defect of
    the refined state stops at the FP32 storage floor (the rounding of the stored state itself,
    about 1e-8 of the field), as in the plain march's refinement."""
    n, nx, ny, kn, ub, ut, layer = case
    ref = lbm.lbm_hybrid_init(lbm.LBM_CAVITY, n, nx, ny, kn, ub, ut, layer, stream=torch.cuda.Stream())
    info = lbm.lbm_hybrid_solve(ref, 1e-12, 400000, 100)
    assert info["residual"] < 1e-12
    wx, wy = lbm.lbm_hybrid_velocity(ref)
    ref.close()
    hb = lbm.lbm_hybrid_init(lbm.LBM_CAVITY, n, nx, ny, kn, ub, ut, layer, stream=torch.cuda.Stream())
    lbm.lbm_hybrid_set_precision(hb, lbm.LBM_FP32_PERTURB)
    m = lbm.lbm_hybrid_solve(hb, 5e-8, 400000, 100)
    assert m["steps"] < 400000
    r = lbm.lbm_hybrid_refine(hb, 1e-10, 3, 0.0, 400000, 100)
    assert r["defect"] < 3e-8 and r["correction_steps"] > 0
    ux, uy = lbm.lbm_hybrid_velocity(hb)
    err = max(np.abs(ux - wx).max(), np.abs(uy - wy).max()) / ut
    assert err < 1e-5, err
    with pytest.raises(lbm.LBMError):
        lbm.lbm_hybrid_refine(lbm.lbm_hybrid_init(lbm.LBM_CAVITY, n, 8, 8, kn, ub, ut, 1), 1e-10)   # FP64: refused
    hb.close()
