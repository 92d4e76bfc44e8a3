"""CPU-side checks of the C-ABI library: it builds, loads, exports every declared entry
point, and its host logic (velocity sets, validation, memory sizing) is right.
No GPU compute is called here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import quadrature as q
from paper_1308_0692_gb300 import build as lbm_build
from paper_1308_0692_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module", autouse=True)
def built_library():
    lbm_build.build()
    return lbm.library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:lbm_status|void|const char \*)\s*\*?\s*(lbm_\w+)\s*\(",
                                 text, flags=re.M)))


def test_every_declared_entry_point_is_exported():
    names = _declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(lbm.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("kind,n", [(lbm.LBM_HALF_RANGE_GH, 2), (lbm.LBM_HALF_RANGE_GH, 3),
                                    (lbm.LBM_HALF_RANGE_GH, 4), (lbm.LBM_HALF_RANGE_GH, 6),
                                    (lbm.LBM_FULL_RANGE_GH, 3), (lbm.LBM_FULL_RANGE_GH, 4),
                                    (lbm.LBM_FULL_RANGE_GH, 8), (lbm.LBM_FULL_RANGE_GH, 12)])
def test_library_velocity_set_matches_oracle(kind, n):
    """The library's double-double quadrature (Hankel-Cholesky + Sturm bisection) rounds to
    the same doubles as the oracle's 80-digit Golub-Welsch construction."""
    vs = lbm.lbm_make_velocity_set(kind, n)
    xi_x, xi_y, w, m = lbm.lbm_vset_query(vs)
    ox, oy, ow = q.velocity_set_2d("half" if kind == lbm.LBM_HALF_RANGE_GH else "full", n)
    assert m * m == len(w) == len(ow)
    np.testing.assert_allclose(xi_x, ox, rtol=4.5e-16, atol=1e-300)
    np.testing.assert_allclose(xi_y, oy, rtol=4.5e-16, atol=1e-300)
    np.testing.assert_allclose(w, ow, rtol=4.5e-16, atol=0)


def test_library_table1_values():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    xi_x, xi_y, w, m = lbm.lbm_vset_query(vs)
    nodes = xi_x[:m]
    assert abs(nodes[-1] - 3.199890790) < 5e-10 and abs(nodes[4] - 0.1891884657) < 5e-11


@pytest.mark.parametrize("kind,n", [(lbm.LBM_HALF_RANGE_GH, 0), (lbm.LBM_HALF_RANGE_GH, 9),
                                    (lbm.LBM_FULL_RANGE_GH, 1), (7, 3)])
def test_velocity_set_rejects_bad_sizes(kind, n):
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_make_velocity_set(kind, n)
    assert e.value.status == lbm.LBM_EINVAL


def _vs(n=4):
    return lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n)


@pytest.mark.parametrize("field,value,status", [
    ("kn", 0.0, lbm.LBM_EINVAL), ("kn", -1.0, lbm.LBM_EINVAL), ("kn", float("nan"), lbm.LBM_EINVAL),
    ("cfl", 0.0, lbm.LBM_EINVAL), ("cfl", 1.5, lbm.LBM_EINVAL), ("ny", 1, lbm.LBM_EINVAL),
    ("nx", 0, lbm.LBM_EINVAL), ("geom", 5, lbm.LBM_EINVAL), ("prec", 9, lbm.LBM_EINVAL),
    ("residual_every", 0, lbm.LBM_EINVAL), ("u_top", float("inf"), lbm.LBM_EINVAL),
])
def test_problem_validation(field, value, status):
    prob = lbm.make_problem(lbm.LBM_CAVITY, 16, 16, 0.1, 0.0, 0.01)
    setattr(prob, field, value)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_sim_bytes(_vs(), prob)
    assert e.value.status == status
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(_vs(), prob)
    assert e.value.status == status


def test_unsupported_velocity_set_size():
    """N = 5 (10 nodes per axis) is a valid rule but has no compiled step kernel."""
    prob = lbm.make_problem(lbm.LBM_CAVITY, 16, 16, 0.1, 0.0, 0.01)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_sim_bytes(_vs(5), prob)
    assert e.value.status == lbm.LBM_EUNSUPPORTED


def test_infinite_kn_is_collisionless_not_an_error():
    prob = lbm.make_problem(lbm.LBM_COUETTE, 1, 10, math.inf, -0.01, 0.01)
    assert lbm.lbm_sim_bytes(_vs(), prob) > 0


def test_sim_bytes_scale_with_the_state():
    p64 = lbm.make_problem(lbm.LBM_CAVITY, 64, 64, 0.1, 0.0, 0.01, prec=lbm.LBM_FP64)
    p32 = lbm.make_problem(lbm.LBM_CAVITY, 64, 64, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB)
    state = 64 * 64 * 64
    b64 = lbm.lbm_sim_bytes(_vs(), p64)
    b32 = lbm.lbm_sim_bytes(_vs(), p32)
    assert b64 >= 2 * 8 * state          # double-buffered FP64 state
    assert b32 >= 4 * 4 * state          # FP32 state, its partner, defect and correction arrays
    assert b64 < 2 * 8 * state * 1.2 + 4e6


def test_norms_argument_checks():
    b = lbm.lbm_norms_scratch_bytes(10 ** 6)
    assert b >= 16
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_norms(1, None, 10 ** 6, lbm.LBM_FP64, 2, b - 8, 3)
    assert e.value.status == lbm.LBM_ENOMEM
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_norms(1, None, -1, lbm.LBM_FP64, 2, b, 3)
    assert e.value.status == lbm.LBM_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the CUDA library there is no fallback: the binding raises."""
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "liblbm.so"))
    with pytest.raises(RuntimeError, match="not built"):
        lbm.lbm_make_velocity_set(0, 4)


def test_grid_beyond_the_index_range_is_rejected():
    """Cell indices are 32-bit in the segment lists: grids of more than 2^31 cells are refused."""
    prob = lbm.make_problem(lbm.LBM_CAVITY, 65536, 32769, 0.1, 0.0, 0.01)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_sim_bytes(_vs(), prob)
    assert e.value.status == lbm.LBM_EINVAL
    ok = lbm.make_problem(lbm.LBM_CAVITY, 65536, 32768, 0.1, 0.0, 0.01)
    assert lbm.lbm_sim_bytes(_vs(), ok) > 8 * 64 * 65536 * 32768


def test_hybrid_init_argument_checks_need_no_device():
    """lbm_hybrid_init refuses invalid problems before it touches the device: N outside
    [2, 6], a Couette channel wider than one column, a grid beyond 16M cells, and a state
    beyond the 32-bit cell offsets (4000 x 4000 cells of D2Q^h_144: 2.3e9 unknowns)."""
    C, V = lbm.LBM_COUETTE, lbm.LBM_CAVITY
    for args in [(C, 1, 1, 10, 0.1, 0.0, 0.01, 2), (C, 7, 1, 10, 0.1, 0.0, 0.01, 2),
                 (C, 4, 3, 10, 0.1, 0.0, 0.01, 2), (V, 4, 5000, 4000, 0.1, 0.0, 0.01, 2),
                 (V, 6, 4000, 4000, 0.1, 0.0, 0.01, 2000)]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_hybrid_init(*args)
        assert e.value.status == lbm.LBM_EINVAL, args
