"""FP32 host transfers of the state (lbm_get_state_f32 / lbm_set_state_f32) against the FP64
ones: for an FP32 simulation they move the stored values themselves, on the planar and on
the strip-tiled layout; for an FP64 simulation set widens exactly and get rounds to
nearest."""
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


# (half-range N, nx, ny, variant): planar default, the tiled column march (load path 9)
CASES = [(4, 128, 96, None), (4, 128, 96, (4, 9)), (6, 192, 40, (6, 9)), (2, 70, 33, None)]


@pytest.mark.parametrize("n,nx,ny,variant", CASES)
def test_fp32_transfers_move_the_stored_values(n, nx, ny, variant):
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n)
    prob = lbm.make_problem(lbm.LBM_CAVITY, nx, ny, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB)
    rng = np.random.default_rng(nx + ny)
    h64 = rng.standard_normal(((2 * n) ** 2, nx * ny)) * 1e-2
    a = lbm.lbm_init(vs, prob, stream=torch.cuda.Stream())
    b = lbm.lbm_init(vs, prob, stream=torch.cuda.Stream())
    if variant:
        lbm.lbm_set_variant(a, *variant)
        lbm.lbm_set_variant(b, *variant)
    lbm.lbm_set_state(a, h64)
    lbm.lbm_set_state_f32(b, h64.astype(np.float32))
    ha = lbm.lbm_get_state(a)
    assert np.array_equal(ha, h64.astype(np.float32).astype(np.float64))
    assert np.array_equal(lbm.lbm_get_state(b), ha)
    assert np.array_equal(lbm.lbm_get_state_f32(b), ha.astype(np.float32))
    # the same state marches the same way
    lbm.lbm_step(a, 3)
    lbm.lbm_step(b, 3)
    ga = lbm.lbm_get_state_f32(a)
    assert np.array_equal(lbm.lbm_get_state_f32(b), ga)
    assert np.array_equal(ga.astype(np.float64), lbm.lbm_get_state(a))
    a.close()
    b.close()


def test_fp32_transfers_of_an_fp64_simulation():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    prob = lbm.make_problem(lbm.LBM_CAVITY, 40, 24, 0.1, 0.0, 0.01, prec=lbm.LBM_FP64)
    sim = lbm.lbm_init(vs, prob, stream=torch.cuda.Stream())
    rng = np.random.default_rng(5)
    x32 = (rng.standard_normal((64, 40 * 24)) * 1e-2).astype(np.float32)
    lbm.lbm_set_state_f32(sim, x32)
    assert np.array_equal(lbm.lbm_get_state(sim), x32.astype(np.float64))       # widened exactly
    h64 = rng.standard_normal((64, 40 * 24)) * 1e-2
    lbm.lbm_set_state(sim, h64)
    assert np.array_equal(lbm.lbm_get_state_f32(sim), h64.astype(np.float32))   # rounded to nearest
    assert np.array_equal(lbm.lbm_get_state(sim), h64)                          # the state is untouched
    sim.close()
