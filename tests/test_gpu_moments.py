"""Moments of FP32 states (double-float row sums, FP64 outer sums) against an FP64 evaluation
of the same stored values, for half-range and full-range sets and non-square grids."""
import numpy as np
import pytest

from paper_1308_0692_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_0692_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("kind,n,nx,ny", [(lbm.LBM_HALF_RANGE_GH, 6, 70, 33), (lbm.LBM_HALF_RANGE_GH, 4, 128, 96),
                                          (lbm.LBM_FULL_RANGE_GH, 3, 40, 41)])
def test_fp32_moments_match_fp64_evaluation(kind, n, nx, ny):
    vs = lbm.lbm_make_velocity_set(kind, n)
    xi_x, xi_y, w, _ = lbm.lbm_vset_query(vs)
    u_ref = 0.01
    prob = lbm.make_problem(lbm.LBM_CAVITY, nx, ny, 0.1, 0.0, u_ref, prec=lbm.LBM_FP32_PERTURB)
    sim = lbm.lbm_init(vs, prob, stream=torch.cuda.Stream())
    rng = np.random.default_rng(nx)
    lbm.lbm_set_state(sim, rng.standard_normal((len(w), nx * ny)))
    h = lbm.lbm_get_state(sim)                      # the stored FP32 values, as FP64
    m = lbm.lbm_moments(sim, wall_shear=False)
    xi_x, xi_y = np.asarray(xi_x)[:, None], np.asarray(xi_y)[:, None]
    s0 = h.sum(0)
    rho = 1.0 + u_ref * s0
    want = {"rho": rho, "ux": u_ref * (xi_x * h).sum(0) / rho, "uy": u_ref * (xi_y * h).sum(0) / rho,
            "pxx": 1.0 + u_ref * (xi_x ** 2 * h).sum(0), "pxy": u_ref * (xi_x * xi_y * h).sum(0),
            "pyy": 1.0 + u_ref * (xi_y ** 2 * h).sum(0)}
    for k, v in want.items():
        got = m[k].reshape(-1)
        np.testing.assert_allclose(got, v, rtol=0, atol=1e-13 * max(np.abs(v).max(), 1.0), err_msg=k)
    sim.close()


@pytest.mark.parametrize("n,nx,ny,variant,planar_variant", [(6, 192, 40, (6, 9), (6, 0)), (4, 128, 70, (4, 8), (4, 0)),
                                                             (2, 128, 33, (2, 9), (1, 0))])
def test_moments_read_the_tiled_state_in_place(n, nx, ny, variant, planar_variant):
    """On the strip-tiled state the moments are read through the tiles: the same values as
    from the planar layout, bit for bit, with or without the P_ij outputs requested."""
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n)
    prob = lbm.make_problem(lbm.LBM_CAVITY, nx, ny, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB)
    h = np.random.default_rng(nx + n).standard_normal(((2 * n) ** 2, nx * ny)) * 1e-2
    planar = lbm.lbm_init(vs, prob, h, stream=torch.cuda.Stream())
    lbm.lbm_set_variant(planar, *planar_variant)
    tiled = lbm.lbm_init(vs, prob, h, stream=torch.cuda.Stream())
    lbm.lbm_set_variant(tiled, *variant)
    assert lbm.lbm_state_tiling(tiled)[0] == 64 and lbm.lbm_state_tiling(planar)[0] == 0
    want = lbm.lbm_moments(planar)
    got = lbm.lbm_moments(tiled)
    for k in lbm.MOMENT_NAMES:
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(got["wall_shear"], want["wall_shear"])
    u_only = lbm.lbm_moments(tiled, wall_shear=False, which=("ux", "uy"))
    assert set(u_only) == {"ux", "uy"}
    assert np.array_equal(u_only["ux"], want["ux"]) and np.array_equal(u_only["uy"], want["uy"])
    # the state itself is untouched by the reads
    assert np.array_equal(lbm.lbm_get_state(tiled), lbm.lbm_get_state(planar))
    planar.close()
    tiled.close()
