"""Warm-start MLP kernels (BF16 tensor-core GEMMs, FP32 accumulation) against the FP64
oracle network with the same bfloat16 rounding points; training reduces the loss; the
warm-start state equals the oracle's second-order Hermite reconstruction."""
import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import quadrature as q
from paper_1308_0692_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_0692_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("rows", [1, 100, 1000, 4200])
def test_forward_and_gradients_match_oracle(rows):
    """Rows 1 to 4200: one partial 128-row tile up to 33 tiles with a ragged last one; the
    weight gradients (K = rows) take 1, 4 and 16 K-splits (some splits past the end of K)."""
    rng = np.random.default_rng(rows)
    params = omlp.init_params(seed=7)
    x = rng.uniform(-1, 1, (rows, 4)).astype(np.float32)
    t = rng.standard_normal((rows, 6)).astype(np.float32)
    m = lbm.lbm_mlp_create(4200, seed=1)
    lbm.lbm_mlp_set_params(m, lbm.mlp_flatten(params))
    qparams = lbm.mlp_unflatten(lbm.lbm_mlp_get_params(m))       # the fp32 master weights
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    yd = torch.empty((rows, 6), dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_forward(m, xd.data_ptr(), rows, yd.data_ptr())
    torch.cuda.synchronize()
    y_ref, _ = omlp.forward(qparams, x.astype(np.float64), bf16=True)
    assert _rel(yd.cpu().numpy(), y_ref) < 2e-3
    loss, g = lbm.lbm_mlp_loss_grad(m, xd.data_ptr(), td.data_ptr(), rows)
    loss_ref, grads_ref = omlp.loss_and_grads(qparams, x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert abs(loss - loss_ref) < 2e-3 * loss_ref
    gp = lbm.mlp_unflatten(g)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(gp, grads_ref)):
        assert _rel(gW, rW) < 1e-2, (l, _rel(gW, rW))
        assert _rel(gb, rb) < 1e-2, (l, _rel(gb, rb))
    # and against the unrounded FP64 network: bf16 costs about 1 % on the gradients
    loss64, grads64 = omlp.loss_and_grads(qparams, x.astype(np.float64), t.astype(np.float64), bf16=False)
    for (gW, gb), (rW, rb) in zip(gp, grads64):
        assert _rel(gW, rW) < 5e-2


def test_training_reduces_the_loss():
    rng = np.random.default_rng(0)
    rows = 2048
    x = rng.uniform(-1, 1, (rows, 4)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], x[:, 2] ** 2, np.cos(x[:, 0] + x[:, 1]), x[:, 3],
                  x[:, 0] * x[:, 2], 0.3 * np.ones(rows)], axis=1).astype(np.float32)
    m = lbm.lbm_mlp_create(rows, seed=3)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = lbm.lbm_mlp_train_step(m, xd.data_ptr(), td.data_ptr(), rows, 1e-3, want_loss=True)
    for _ in range(300):
        lbm.lbm_mlp_train_step(m, xd.data_ptr(), td.data_ptr(), rows, 1e-3)
    last, _ = lbm.lbm_mlp_loss_grad(m, xd.data_ptr(), td.data_ptr(), rows, want_grad=False)
    assert last < 0.05 * first


def test_warm_start_state_is_the_hermite_expansion():
    nx = ny = 24
    kn, uw = 0.3, 0.012
    m = lbm.lbm_mlp_create(nx * ny, seed=5)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    sim = lbm.lbm_init(vs, lbm.make_problem(lbm.LBM_CAVITY, nx, ny, kn, 0.0, uw))
    lbm.lbm_warm_start(sim, m, kn, uw)
    h = lbm.lbm_get_state(sim)
    # the same network on the same features, evaluated through the forward entry point
    xd = torch.empty((nx * ny, 4), dtype=torch.float32, device="cuda")
    yd = torch.empty((nx * ny, 6), dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_features(m, nx, ny, kn, uw, xd.data_ptr())
    lbm.lbm_mlp_forward(m, xd.data_ptr(), nx * ny, yd.data_ptr())
    torch.cuda.synchronize()
    feats = xd.cpu().numpy()
    cx = ((np.arange(nx) + 0.5) / nx) * 2 - 1
    np.testing.assert_allclose(feats[:nx, 0], cx, rtol=0, atol=1e-6)
    np.testing.assert_allclose(feats[0, 2], (2 * np.log10(kn) + 1) / 3, rtol=1e-6)
    pred = yd.cpu().numpy().astype(np.float64)
    mom = {"rho": 1 + uw * pred[:, 0], "ux": uw * pred[:, 1] / (1 + uw * pred[:, 0]),
           "uy": uw * pred[:, 2] / (1 + uw * pred[:, 0]), "pxx": 1 + uw * pred[:, 3], "pxy": uw * pred[:, 4],
           "pyy": 1 + uw * pred[:, 5]}
    xi_x, xi_y, w = (np.array(v) for v in q.velocity_set_2d("half", 4))
    ref = omlp.moments_to_h(mom, xi_x, xi_y, w, uw)
    assert np.abs(h - ref).max() <= 1e-6 * np.abs(ref).max()


def test_trained_network_shortens_the_march_at_equal_accuracy():
    """What the learned part gains: with the committed trained network, held-out cavities
    (128^2, D2Q^h_64, pairs from a seed the training never saw) reach the FP32 march target in
    fewer steps than from the cold start f = w, and the refined fields agree with the cold
    start's and with an FP64 solve within 1e-5 of u_w."""
    import os

    from paper_1308_0692_gb300 import warmstart
    path = os.path.join(os.path.dirname(warmstart.__file__), "data", "warmstart_mlp.npy")
    mlp = warmstart.load_mlp(path)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    pairs = warmstart.draw_pairs(4, seed=99173)
    cold_steps, warm_steps = [], []
    for kn, uw in pairs:
        runs = {}
        for name, net in (("cold", None), ("warm", mlp)):
            sim, info, _ = warmstart.solve_cavity(vs, kn, uw, prec=lbm.LBM_FP32_PERTURB, tol=1e-8, refine=3,
                                                  mlp=net, refine_tol=1e-8)
            runs[name] = (info, lbm.lbm_moments(sim, wall_shear=False))
            sim.close()
        s64, _, _ = warmstart.solve_cavity(vs, kn, uw, prec=lbm.LBM_FP64, tol=1e-10, refine=0)
        m64 = lbm.lbm_moments(s64, wall_shear=False)
        s64.close()
        for name, (info, m) in runs.items():
            err = max(np.abs(m["ux"] - m64["ux"]).max(), np.abs(m["uy"] - m64["uy"]).max()) / uw
            assert err < 1e-5, (kn, uw, name, err)
        cold_steps.append(runs["cold"][0]["steps"])
        warm_steps.append(runs["warm"][0]["steps"])
    assert sum(warm_steps) < 0.8 * sum(cold_steps), (cold_steps, warm_steps)
    mlp.close()
