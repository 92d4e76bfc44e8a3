"""GPU parity of the fused step kernels against the FP64 CPU oracle, through the C-ABI.

Tolerances: FP64 path 1e-12 relative (max |delta h| / max |h|) at equal step counts;
FP32 path per step: 2e-6 of max |h| per step marched (single-precision rounding of
the O(10) operations and the velocity sums per value, which are far below any
indexing, sign or coefficient mistake, those being O(1)).
"""
import math

import numpy as np
import pytest

from oracle.march import CAVITY, COUETTE, make_problem as oracle_problem, residual as oracle_residual
from paper_1308_0692_gb300 import lbm
from paper_1308_0692_gb300.inputs import random_cells, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL_PER_STEP = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_0692_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _kind(kind):
    return lbm.LBM_HALF_RANGE_GH if kind == "half" else lbm.LBM_FULL_RANGE_GH


def gpu_run(kind, n, geom, nx, ny, kn, ub, ut, prec, h0, steps, stream=None, device_buf=False,
            residual_every=1):
    vs = lbm.lbm_make_velocity_set(_kind(kind), n)
    prob = lbm.make_problem(geom, nx, ny, kn, ub, ut, prec=prec, residual_every=residual_every)
    buf = None
    if device_buf:
        buf = torch.empty(lbm.lbm_sim_bytes(vs, prob), dtype=torch.uint8, device="cuda")
    sim = lbm.lbm_init(vs, prob, h0, device_buf=buf, stream=stream)
    lbm.lbm_step(sim, steps)
    return lbm.lbm_get_state(sim), sim


CASES = [
    # kind, n, geom, nx, ny, kn, u_bottom, u_top
    ("half", 4, COUETTE, 1, 100, 0.1, 0.01, -0.01),        # configuration of the Couette runs
    ("half", 4, COUETTE, 1, 100, 0.01, 0.01, -0.01),
    ("half", 4, COUETTE, 1, 100, 10.0, 0.01, -0.01),
    ("half", 4, COUETTE, 1, 37, math.inf, -0.01, 0.01),    # collisionless
    ("half", 2, COUETTE, 3, 41, 0.3, -0.02, 0.01),         # several periodic columns
    ("half", 4, CAVITY, 37, 29, 0.1, 0.0, 0.01),           # ragged: 1073 cells
    ("half", 4, CAVITY, 130, 67, 0.05, 0.003, 0.01),       # several tiles, moving bottom
    ("full", 3, CAVITY, 23, 19, 0.1, 0.0, 0.01),           # D2Q9
    ("full", 4, CAVITY, 23, 19, 0.2, 0.0, 0.01),           # D2Q16
    ("half", 2, CAVITY, 31, 33, 1.0, 0.0, 0.01),           # D2Q^h_16
    ("half", 3, CAVITY, 21, 17, 0.1, 0.0, 0.01),           # D2Q^h_36
    ("half", 6, CAVITY, 45, 38, 0.05, 0.0, 0.01),          # D2Q^h_144
    ("half", 4, CAVITY, 2, 2, 0.1, 0.0, 0.01),             # smallest cavity
    ("half", 4, COUETTE, 1, 2, 0.1, 0.01, -0.01),          # smallest channel
    ("half", 2, COUETTE, 70, 20, 0.2, 0.01, -0.01),        # several periodic columns, longer rows
    ("half", 6, CAVITY, 96, 33, 0.05, 0.0, 0.01),          # D2Q^h_144, 3 segments per row
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}{c[1]}-{'cav' if c[2] else 'cou'}-{c[3]}x{c[4]}-kn{c[5]}" for c in CASES])
def test_fp64_step_parity_random_state(case):
    kind, n, geom, nx, ny, kn, ub, ut = case
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h0 = random_state(p.n, p.ncells, seed=1000 + nx * ny)
    steps = 7
    got, sim = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP64, h0, steps)
    ref = p.step(h0, steps)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= FP64_TOL, err
    # residual of the last step against the oracle's definition
    r, st = lbm.lbm_residual(sim)
    assert st == steps
    r_ref = oracle_residual(ref, p.step(h0, steps - 1))
    assert abs(r - r_ref) <= 1e-10 * r_ref


@pytest.mark.parametrize("case", CASES[:2] + CASES[5:9] + CASES[11:12])
def test_fp32_step_parity_random_state(case):
    kind, n, geom, nx, ny, kn, ub, ut = case
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h0 = random_state(p.n, p.ncells, seed=2000 + nx * ny).astype(np.float32).astype(np.float64)
    steps = 5
    got, _ = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP32_PERTURB, h0, steps)
    ref = p.step(h0, steps)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= FP32_TOL_PER_STEP * steps, err


def test_fp64_cold_start_march_cavity_128():
    """Lid-driven cavity 128 x 128, 64 velocities, Kn 0.1, from f = w: 300 steps agree to 1e-12."""
    kind, n, geom, nx, ny, kn, ub, ut = "half", 4, CAVITY, 128, 128, 0.1, 0.0, 0.01
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    got, sim = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP64, None, 300)
    ref = p.step(p.zeros(), 300)
    assert np.abs(got - ref).max() <= FP64_TOL * np.abs(ref).max()
    m = lbm.lbm_moments(sim)
    mr = p.moments(ref)
    for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy"):
        scale = np.abs(mr[k] - (1.0 if k in ("rho", "pxx", "pyy") else 0.0)).max()
        assert np.abs(m[k] - mr[k]).max() <= 1e-12 * scale, k
    fy, fx = lbm.lbm_face_flux(sim)
    fyr, fxr = p.face_flux_y(ref), p.face_flux_x(ref)
    assert np.abs(fy - fyr).max() <= 1e-12 * np.abs(fyr).max()
    assert np.abs(fx - fxr).max() <= 1e-12 * np.abs(fxr).max()
    ws = m["wall_shear"]
    assert abs(ws[1] - fyr[-1].mean()) <= 1e-12 * abs(fyr[-1].mean())
    assert abs(ws[0] - fyr[0].mean()) <= 1e-12 * np.abs(fyr).max()
    assert abs(ws[2] - fxr[:, 0].mean()) <= 1e-12 * np.abs(fxr).max()


def test_couette_converged_to_steady_state_fp64():
    """Couette ny=100, 64 velocities, Kn = 0.1, marched to r < 1e-10 on the GPU, matches the
    oracle marched the same number of steps to 1e-12; face shear equals the oracle's."""
    kind, n, geom, nx, ny, kn, ub, ut = "half", 4, COUETTE, 1, 100, 0.1, 0.01, -0.01
    vs = lbm.lbm_make_velocity_set(_kind(kind), n)
    prob = lbm.make_problem(geom, nx, ny, kn, ub, ut, residual_every=100)
    sim = lbm.lbm_init(vs, prob)
    steps = 0
    while True:
        lbm.lbm_step(sim, 100)
        steps += 100
        r, _ = lbm.lbm_residual(sim)
        if r < 1e-10 or steps > 50000:
            break
    assert r < 1e-10
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    ref = p.step(p.zeros(), steps)
    got = lbm.lbm_get_state(sim)
    assert np.abs(got - ref).max() <= FP64_TOL * np.abs(ref).max()
    fy, _ = lbm.lbm_face_flux(sim)
    assert np.ptp(fy) < 1e-6 * np.abs(fy).max()        # one shear stress through every face


def test_caller_buffer_and_stream_give_identical_bits():
    kind, n, geom, nx, ny, kn, ub, ut = "half", 4, CAVITY, 50, 40, 0.1, 0.0, 0.01
    h0 = random_state(64, nx * ny, seed=5)
    a, _ = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP64, h0, 11)
    s = torch.cuda.Stream()
    b, _ = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP64, h0, 11, stream=s, device_buf=True)
    np.testing.assert_array_equal(a, b)       # deterministic: no atomics, fixed order


def test_sims_sharing_a_stream_from_two_threads():
    """Two simulations on one stream, stepped from two host threads at once, give the bits
    they give one after the other: each sim captures its step graphs on a private stream, so
    neither capture can swallow the other thread's launches on the shared stream."""
    import concurrent.futures as cf
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    probs = [lbm.make_problem(CAVITY, 96, 80, kn, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB, residual_every=5)
             for kn in (0.1, 0.03)]
    h0 = [random_state(64, 96 * 80, seed=s) for s in (5, 6)]

    def run(args):
        prob, h, stream = args
        sim = lbm.lbm_init(vs, prob, h, stream=stream)
        for _ in range(8):
            lbm.lbm_step(sim, 10)
        r = lbm.lbm_residual(sim)
        return lbm.lbm_get_state(sim), r

    alone = [run((p, h, lbm.PrivateStream())) for p, h in zip(probs, h0)]
    shared = torch.cuda.Stream()
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        both = list(ex.map(run, [(p, h, shared) for p, h in zip(probs, h0)]))
    for (ga, ra), (gb, rb) in zip(alone, both):
        assert np.array_equal(ga, gb) and ra == rb


@pytest.mark.parametrize("nx,ny", [(40, 30), (96, 70)])
@pytest.mark.parametrize("prec,tol", [(lbm.LBM_FP64, 1e-13), (lbm.LBM_FP32_PERTURB, 1e-6)])
def test_set_moments_matches_oracle_and_round_trips(prec, tol, nx, ny):
    """lbm_set_moments builds the oracle's Hermite state from six moment fields, and
    lbm_moments gives the fields back (the set D2Q^h_64 is exact to degree 4)."""
    from oracle.mlp import moments_to_h
    u_ref = 0.01
    p = oracle_problem("half", 4, CAVITY, nx, ny, 0.1, 0.0, u_ref)
    y, x = np.mgrid[0:ny, 0:nx] / np.array([[[ny]], [[nx]]])
    mom = {"rho": 1 + u_ref * 0.3 * np.sin(3 * x) * np.cos(2 * y), "ux": u_ref * 0.8 * np.cos(4 * y),
           "uy": -u_ref * 0.5 * np.sin(5 * x), "pxx": 1 + u_ref * 0.2 * x * y, "pxy": u_ref * 0.4 * (x - y),
           "pyy": 1 - u_ref * 0.25 * np.cos(x + y)}
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.1, 0.0, u_ref, prec=prec), stream=torch.cuda.Stream())
    lbm.lbm_set_moments(sim, mom)
    got = lbm.lbm_get_state(sim)
    ref = moments_to_h({k: v.reshape(-1) for k, v in mom.items()}, p.xi_x, p.xi_y, p.w, u_ref)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    back = lbm.lbm_moments(sim, wall_shear=False)
    for k in mom:
        assert np.abs(back[k] - mom[k]).max() <= 10 * tol * u_ref, k


@pytest.mark.parametrize("prec,tol,variant", [(lbm.LBM_FP64, FP64_TOL, None),
                                              (lbm.LBM_FP32_PERTURB, FP32_TOL_PER_STEP * 6, None),
                                              (lbm.LBM_FP32_PERTURB, FP32_TOL_PER_STEP * 6, (6, 4)),
                                              (lbm.LBM_FP32_PERTURB, FP32_TOL_PER_STEP * 6, (6, 7)),
                                              (lbm.LBM_FP32_PERTURB, FP32_TOL_PER_STEP * 6, (6, 8))])
def test_strang_splitting_matches_oracle(prec, tol, variant):
    """Symmetric splitting: the library's stored state g = R(dt/2) h after 6 steps equals the
    oracle's literal composition relaxation(dt/2), transport(dt), relaxation(dt/2), and the
    physical moments (lbm_moments) equal the oracle's moments of h."""
    n_half, nx, ny = (6, 192, 40) if variant else (4, 50, 37)
    p = oracle_problem("half", n_half, CAVITY, nx, ny, 0.08, 0.0, 0.01)
    h0 = random_state(p.n, p.ncells, seed=61)
    g0 = p.relax(h0, 0.5)
    if prec == lbm.LBM_FP32_PERTURB:
        g0 = g0.astype(np.float32).astype(np.float64)
        h0 = None
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.08, 0.0, 0.01, prec=prec, residual_every=3), g0,
                       stream=torch.cuda.Stream())
    lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_STRANG)
    assert lbm.lbm_get_splitting(sim) == lbm.LBM_SPLIT_STRANG
    if variant:
        lbm.lbm_set_variant(sim, *variant)
    lbm.lbm_step(sim, 6)
    # oracle: undo the first half relaxation to get h0 from g0 only in FP64; in FP32 start
    # from the rounded g0 through the g form (the identity is pinned on the CPU)
    w = p.coeffs["omega"]
    if h0 is not None:
        ref_g = p.relax(p.step_strang(h0, 6), 0.5)
        ref_h = p.step_strang(h0, 6)
    else:
        ref_g = p.step(g0, 6, omega=1.0 - (1.0 - 0.5 * w) ** 2)
        eq = p.relax(ref_g, 1.0 / w)
        ref_h = eq + (ref_g - eq) / (1.0 - 0.5 * w)
    got = lbm.lbm_get_state(sim)
    assert np.abs(got - ref_g).max() <= tol * np.abs(ref_g).max()
    m = lbm.lbm_moments(sim, wall_shear=False)
    mr = p.moments(ref_h)
    for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy"):
        scale = np.abs(mr[k] - (1.0 if k in ("rho", "pxx", "pyy") else 0.0)).max()
        assert np.abs(m[k] - mr[k]).max() <= max(tol, 1e-12) * 10 * scale, k
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_LIE)       # only before the first step


def test_zero_steps_and_set_get_roundtrip():
    kind, n, geom, nx, ny, kn, ub, ut = "half", 4, CAVITY, 9, 7, 0.1, 0.0, 0.01
    h0 = random_state(64, 63, seed=9)
    got, sim = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP64, h0, 0)
    np.testing.assert_array_equal(got, h0)
    h1 = random_state(64, 63, seed=10)
    lbm.lbm_set_state(sim, h1)
    np.testing.assert_array_equal(lbm.lbm_get_state(sim), h1)


def test_nonfinite_state_is_reported():
    kind, n, geom, nx, ny, kn, ub, ut = "half", 2, CAVITY, 8, 8, 0.1, 0.0, 0.01
    h0 = random_state(16, 64, seed=3)
    h0[5, 17] = np.nan           # planted on the host before upload
    _, sim = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, lbm.LBM_FP64, h0, 3)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_residual(sim)
    assert e.value.status == lbm.LBM_ENONFINITE


def test_small_device_buffer_rejected():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    prob = lbm.make_problem(CAVITY, 16, 16, 0.1, 0.0, 0.01)
    need = lbm.lbm_sim_bytes(vs, prob)
    buf = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(vs, prob, device_buf=buf)
    assert e.value.status == lbm.LBM_ENOMEM


@pytest.mark.parametrize("prec,dtype", [(lbm.LBM_FP64, torch.float64), (lbm.LBM_FP32_PERTURB, torch.float32)])
@pytest.mark.parametrize("count", [1, 1000, 3 * 10 ** 6 + 17])
def test_norms_against_host(prec, dtype, count):
    g = torch.Generator(device="cpu").manual_seed(count)
    a = torch.randn(count, generator=g, dtype=torch.float64).to(dtype)
    b = torch.randn(count, generator=g, dtype=torch.float64).to(dtype)
    ad, bd = a.cuda(), b.cuda()
    nbytes = lbm.lbm_norms_scratch_bytes(count)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    lbm.lbm_norms(ad.data_ptr(), bd.data_ptr(), count, prec, scratch.data_ptr(), nbytes, out.data_ptr(), s)
    torch.cuda.synchronize()
    a64, b64 = a.double().numpy(), b.double().numpy()
    ref = np.array([np.sum((a64 - b64) ** 2), np.sum(a64 ** 2)])
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12)


# ---- full-size configurations: sampled outputs the oracle computes one by one ----

FULL = [
    # (kind, n, geom, nx, ny, kn, ub, ut, prec) at the sizes the benchmark and the examples use
    ("half", 6, CAVITY, 2048, 2048, 0.05, 0.0, 0.01, lbm.LBM_FP32_PERTURB),
    ("half", 6, CAVITY, 2048, 2048, 0.05, 0.0, 0.01, lbm.LBM_FP64),
    ("half", 4, CAVITY, 256, 256, 0.1, 0.0, 0.01, lbm.LBM_FP32_PERTURB),
    ("half", 4, COUETTE, 1, 512, 0.02, 0.01, -0.01, lbm.LBM_FP32_PERTURB),
]


@pytest.mark.parametrize("case", FULL, ids=["cavity2048-144-fp32", "cavity2048-144-fp64",
                                            "cavity256-64-fp32", "couette512-64-fp32"])
def test_full_size_sampled_step(case):
    kind, n, geom, nx, ny, kn, ub, ut, prec = case
    p = oracle_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h0 = random_state(p.n, p.ncells, seed=77)
    if prec == lbm.LBM_FP32_PERTURB:
        h0 = h0.astype(np.float32).astype(np.float64)
    corners = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, nx // 2, (ny // 2) * nx, (ny // 2) * nx + nx - 1,
               (ny - 1) * nx + nx // 2, (ny // 2) * nx + nx // 2]
    cells = random_cells(p.ncells, 400, seed=78, include=corners)
    got, sim = gpu_run(kind, n, geom, nx, ny, kn, ub, ut, prec, h0, 1)
    del h0
    ref = p.step_cells(_host_state_for(p, seed=77, prec=prec), cells)
    g = got[:, cells].T
    tol = FP64_TOL if prec == lbm.LBM_FP64 else FP32_TOL_PER_STEP
    assert np.abs(g - ref).max() <= tol * np.abs(ref).max()


@pytest.fixture(scope="module")
def bench_case():
    """The benchmark's workload (cavity 2048 x 2048, D2Q^h_144, Kn 0.05, lid 0.01, FP32):
    one FP32-representable state and the oracle's step at 400 sampled cells."""
    p = oracle_problem("half", 6, CAVITY, 2048, 2048, 0.05, 0.0, 0.01)
    h0 = _host_state_for(p, seed=77, prec=lbm.LBM_FP32_PERTURB)
    nx, ny = 2048, 2048
    corners = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, 31 * nx + 31, 32 * nx + 32, nx + 32, 2 * nx - 33,
               (ny - 2) * nx + 32, (ny - 2) * nx + nx - 33, (ny // 2) * nx + 95, (ny // 2) * nx + 96]
    cells = random_cells(p.ncells, 400, seed=79, include=corners)
    return p, h0, cells, p.step_cells(h0, cells)


def _bench_variants():
    import bench
    return bench.VARIANTS


@pytest.mark.parametrize("variant", _bench_variants(), ids=lambda v: f"g{v[0]}-path{v[1]}")
def test_full_size_bench_variants(bench_case, variant):
    """Every kernel variant the benchmark may choose, at the benchmark's size, on sampled
    cells (walls, corners, strip and chunk edges of the column march), for the step with
    and without the residual."""
    p, h0, cells, ref = bench_case
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 6)
    idx = torch.as_tensor(np.asarray(cells, dtype=np.int64), device="cuda")
    rs = []
    for residual_every in (1, 2):
        prob = lbm.make_problem(CAVITY, 2048, 2048, 0.05, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB,
                                residual_every=residual_every)
        buf = torch.empty(lbm.lbm_sim_bytes(vs, prob), dtype=torch.uint8, device="cuda")
        sim = lbm.lbm_init(vs, prob, h0, device_buf=buf, stream=torch.cuda.Stream())
        lbm.lbm_set_variant(sim, *variant)
        lbm.lbm_step(sim, 1)
        ptr, step = lbm.lbm_state_device(sim)
        assert step == 1
        tw, shift, tp, rp = lbm.lbm_state_tiling(sim)
        off = ptr - buf.data_ptr()
        cy, cx = idx // 2048, idx % 2048
        if tw:
            # strip-tiled state (load path 8)
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
            rs.append(r)
        sim.close()
        del buf, state
    torch.cuda.empty_cache()


def _host_state_for(p, seed, prec):
    h = random_state(p.n, p.ncells, seed=seed)
    if prec == lbm.LBM_FP32_PERTURB:
        h = h.astype(np.float32).astype(np.float64)
    return h


@pytest.mark.parametrize("n_half,nx,ny,variants", [
    (4, 68, 40, [(1, 0), (2, 0), (4, 0), (2, 1), (4, 1), (2, 2), (4, 2), (2, 3), (4, 3)]),
    (6, 64, 36, [(2, 0), (3, 0), (4, 0), (6, 0), (3, 1), (4, 1), (6, 1), (3, 2), (4, 2), (6, 2), (3, 3), (6, 3)]),
    (6, 100, 36, [(2, 0), (3, 0), (4, 0), (6, 0), (3, 1), (4, 1), (6, 1), (6, 2), (6, 3)]),
])
def test_fp32_kernel_variants_agree(n_half, nx, ny, variants):
    """Every kernel variant (warps per segment; register, prefetched or TMA-staged loads) gives
    the oracle's result to FP32 accuracy, and variants with the same warps per segment agree
    to within a few FP32 roundings (same arithmetic, only the load path differs)."""
    p = oracle_problem("half", n_half, CAVITY, nx, ny, 0.1, 0.0, 0.01)
    h0 = random_state(p.n, p.ncells, seed=31).astype(np.float32).astype(np.float64)
    ref = p.step(h0, 4)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    by_g = {}
    for g, pf in variants:
        sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB,
                                                residual_every=2), h0, stream=torch.cuda.Stream())
        lbm.lbm_set_variant(sim, g, pf)
        lbm.lbm_step(sim, 4)
        got = lbm.lbm_get_state(sim)
        r, st = lbm.lbm_residual(sim)
        assert st == 4 and np.isfinite(r)
        assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * 4 * np.abs(ref).max(), (g, pf)
        if g in by_g:
            assert np.abs(got - by_g[g]).max() <= 1e-6 * np.abs(ref).max(), (g, pf)
        else:
            by_g[g] = got


@pytest.mark.parametrize("n_half,nx,ny,variants", [
    # 2 strips x 5 chunks: fewer items than blocks (most blocks find no work)
    (6, 192, 45, [(6, 0), (6, 4), (6, 5), (6, 6), (6, 7), (6, 8), (6, 9), (12, 4), (12, 5)]),
    # 5 strips x 65 chunks of 8 rows: more items than blocks, item-to-item pipelining
    (6, 384, 522, [(6, 0), (6, 4), (6, 5), (6, 6), (6, 7), (6, 8), (6, 9), (12, 5)]),
    (4, 256, 70, [(2, 0), (2, 5), (4, 0), (4, 5), (4, 8), (4, 9)]),
    # 15 strips x 41+ chunks: items beyond the fixed first three per block come from the counter
    (6, 1024, 1000, [(6, 0), (6, 4), (6, 6), (6, 7), (6, 8), (6, 9), (12, 5)]),
])
def test_fp32_column_march_matches_oracle(n_half, nx, ny, variants):
    """The column-march interior (load paths 4 to 9; 8 and 9 on the strip-tiled state, 9 with
    bulk asynchronous stores) gives the oracle's result to FP32 accuracy
    over several steps, with and without the residual, and agrees with the segment kernels
    to within a few FP32 roundings."""
    p = oracle_problem("half", n_half, CAVITY, nx, ny, 0.07, 0.002, 0.01)
    h0 = random_state(p.n, p.ncells, seed=41).astype(np.float32).astype(np.float64)
    steps = 3
    ref = p.step(h0, steps)
    ref_r = oracle_residual(ref, p.step(h0, steps - 1))
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    base = None
    for g, pf in variants:
        sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.07, 0.002, 0.01, prec=lbm.LBM_FP32_PERTURB,
                                                residual_every=steps), h0, stream=torch.cuda.Stream())
        lbm.lbm_set_variant(sim, g, pf)
        assert lbm.lbm_get_variant(sim) == (g, pf)
        lbm.lbm_step(sim, steps)
        got = lbm.lbm_get_state(sim)
        r, st = lbm.lbm_residual(sim)
        assert st == steps and abs(r - ref_r) <= 1e-4 * ref_r, (g, pf, r, ref_r)
        assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * steps * np.abs(ref).max(), (g, pf)
        if base is None:
            base = got
        else:
            assert np.abs(got - base).max() <= 1e-6 * np.abs(ref).max(), (g, pf)


@pytest.mark.parametrize("kind,n_half,nx,ny", [("half", 2, 128, 40), ("full", 4, 256, 70), ("half", 2, 192, 23)],
                         ids=["Dh16-128x40", "D16-256x70", "Dh16-192x23"])
def test_fp32_column_march_16_velocity_sets(kind, n_half, nx, ny):
    """The tiled column march (load paths 8 and 9) on the 16-velocity sets of the paper's
    half- versus full-range comparison (two warps, two velocity rows each) against the
    oracle over several steps with the residual, and against the register kernel."""
    p = oracle_problem(kind, n_half, CAVITY, nx, ny, 0.2, 0.0, 0.01)
    h0 = random_state(p.n, p.ncells, seed=43).astype(np.float32).astype(np.float64)
    steps = 4
    ref = p.step(h0, steps)
    ref_r = oracle_residual(ref, p.step(h0, steps - 1))
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH if kind == "half" else lbm.LBM_FULL_RANGE_GH, n_half)
    base = None
    for g, pf in [(1, 0), (2, 8), (2, 9)]:
        sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.2, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB,
                                                residual_every=steps), h0, stream=torch.cuda.Stream())
        lbm.lbm_set_variant(sim, g, pf)
        assert lbm.lbm_get_variant(sim) == (g, pf)
        lbm.lbm_step(sim, steps)
        got = lbm.lbm_get_state(sim)
        r, st = lbm.lbm_residual(sim)
        assert st == steps and abs(r - ref_r) <= 1e-4 * ref_r, (g, pf, r, ref_r)
        assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * steps * np.abs(ref).max(), (g, pf)
        if base is None:
            base = got
        else:
            assert np.abs(got - base).max() <= 1e-6 * np.abs(ref).max(), (g, pf)
        sim.close()


def test_column_march_rejected_where_strips_do_not_fit():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 6)
    for nx, ny in [(160, 64), (64, 64), (128, 9)]:
        sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB))
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_set_variant(sim, 6, 4)
        assert e.value.status == lbm.LBM_EUNSUPPORTED
    sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, 128, 64, 0.1, 0.0, 0.01, prec=lbm.LBM_FP64))
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_variant(sim, 6, 4)


def test_tma_variant_rejected_where_lines_are_unaligned():
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, 37, 29, 0.1, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB))
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_set_variant(sim, 2, 2)
    assert e.value.status == lbm.LBM_EUNSUPPORTED


def test_strip_tiled_state_layout_changes_and_refinement():
    """Load path 8 moves the state into the strip-tiled layout and any other path moves it
    back, bit for bit; host transfers stay planar; the tiling is reported and the planar
    pitches are refused while tiled; lbm_solve's refinement sweeps (run on the planar layout)
    give the same state as on the planar column march and leave the state tiled."""
    n_half, nx, ny = 6, 192, 45
    p = oracle_problem("half", n_half, CAVITY, nx, ny, 0.07, 0.002, 0.01)
    h0 = random_state(p.n, p.ncells, seed=43).astype(np.float32).astype(np.float64)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    prob = lbm.make_problem(CAVITY, nx, ny, 0.07, 0.002, 0.01, prec=lbm.LBM_FP32_PERTURB, residual_every=3)
    sim = lbm.lbm_init(vs, prob, h0, stream=torch.cuda.Stream())
    assert lbm.lbm_state_tiling(sim) == (0, 0, 0, 0)
    lbm.lbm_set_variant(sim, 6, 8)
    assert lbm.lbm_state_tiling(sim) == (64, 32, ny * p.n * 64, p.n * 64)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_state_layout(sim)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    np.testing.assert_array_equal(lbm.lbm_get_state(sim), h0)
    h1 = random_state(p.n, p.ncells, seed=44).astype(np.float32).astype(np.float64)
    lbm.lbm_set_state(sim, h1)
    np.testing.assert_array_equal(lbm.lbm_get_state(sim), h1)
    lbm.lbm_set_variant(sim, 6, 4)
    assert lbm.lbm_state_tiling(sim)[0] == 0
    np.testing.assert_array_equal(lbm.lbm_get_state(sim), h1)
    lbm.lbm_set_variant(sim, 6, 8)
    ref = p.step(h1, 3)
    lbm.lbm_step(sim, 3)
    got = lbm.lbm_get_state(sim)
    assert np.abs(got - ref).max() <= FP32_TOL_PER_STEP * 3 * np.abs(ref).max()
    m = lbm.lbm_moments(sim)
    mr = p.moments(got)
    for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy"):
        np.testing.assert_allclose(m[k], mr[k], rtol=0, atol=1e-12)
    fy, fx = lbm.lbm_face_flux(sim)
    np.testing.assert_allclose(fy, p.face_flux_y(got), rtol=0, atol=1e-12)
    np.testing.assert_allclose(fx, p.face_flux_x(got), rtol=0, atol=1e-12)
    sim.close()
    # the same solve on the planar and on the tiled column march
    out = []
    for pf in (4, 8):
        sim = lbm.lbm_init(vs, lbm.make_problem(CAVITY, nx, ny, 0.07, 0.0, 0.01, prec=lbm.LBM_FP32_PERTURB,
                                                residual_every=100), stream=torch.cuda.Stream())
        lbm.lbm_set_variant(sim, 6, pf)
        info = lbm.lbm_solve(sim, 1e-8, 400_000, 3, 1e-8)
        assert lbm.lbm_get_variant(sim) == (6, pf) and (lbm.lbm_state_tiling(sim)[0] == 64) == (pf == 8)
        out.append((info, lbm.lbm_get_state(sim)))
        sim.close()
    (i4, s4), (i8, s8) = out
    # same march steps, and the refinement ends at the same FP32 floor of the defect
    assert i8["steps"] == i4["steps"] and i8["sweeps"] == i4["sweeps"], (i4, i8)
    assert abs(i8["defect"] - i4["defect"]) <= 0.1 * i4["defect"] and i8["defect"] < 2e-8, (i4, i8)
    assert np.abs(s8 - s4).max() <= 1e-5 * np.abs(s4).max()
