"""Pins of the FP64 MLP reference and of the warm-start reconstruction (CPU only)."""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle import quadrature as q


def _small_params(seed=1, widths=(4, 7, 5, 6, 6)):
    return mlp.init_params(seed, widths)


def test_gelu_closed_forms():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    # GELU(0) = 0, GELU(z) - GELU(-z) = z, GELU'(0) = 1/2
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-15)
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-16
    # derivative against central differences
    eps = 1e-6
    fd = (mlp.gelu(z + eps) - mlp.gelu(z - eps)) / (2 * eps)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-10)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    params = _small_params()
    x = rng.standard_normal((9, 4))
    t = rng.standard_normal((9, 6))
    loss, grads = mlp.loss_and_grads(params, x, t)
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[l][0][i, j] += eps
            Wm[l][0][i, j] -= eps
            fd = (mlp.loss_and_grads(Wp, x, t)[0] - mlp.loss_and_grads(Wm, x, t)[0]) / (2 * eps)
            assert abs(grads[l][0][i, j] - fd) < 1e-7 * max(1.0, abs(fd)), (l, i, j)
        for i in (0, b.shape[0] - 1):
            Bp = [(w.copy(), bb.copy()) for w, bb in params]
            Bm = [(w.copy(), bb.copy()) for w, bb in params]
            Bp[l][1][i] += eps
            Bm[l][1][i] -= eps
            fd = (mlp.loss_and_grads(Bp, x, t)[0] - mlp.loss_and_grads(Bm, x, t)[0]) / (2 * eps)
            assert abs(grads[l][1][i] - fd) < 1e-7 * max(1.0, abs(fd)), (l, i)


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.0 + 2 ** -8 + 2 ** -9, -3.0, 1e-30])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # tie at 1 + 2^-8 rounds to even (1.0)
    assert r[2] == 1.0 + 2 ** -7       # above the tie rounds up
    assert r[3] == -3.0
    assert abs(r[4] - 1e-30) / 1e-30 < 2 ** -8


def test_hermite_reconstruction_reproduces_moments():
    """With the 64-velocity half-range set (exact to degree 7 per half-line) the second-order
    expansion returns the six moments it was built from."""
    xi_x, xi_y, w = (np.array(v) for v in q.velocity_set_2d("half", 4))
    rng = np.random.default_rng(0)
    n = 17
    u = 0.01
    mom = {"rho": 1 + u * rng.standard_normal(n), "ux": u * rng.standard_normal(n), "uy": u * rng.standard_normal(n),
           "pxx": 1 + u * rng.standard_normal(n), "pxy": u * rng.standard_normal(n), "pyy": 1 + u * rng.standard_normal(n)}
    h = mlp.moments_to_h(mom, xi_x, xi_y, w, u)
    rho = 1 + u * h.sum(0)
    np.testing.assert_allclose(rho, mom["rho"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(u * (xi_x @ h) / rho, mom["ux"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(u * (xi_y @ h) / rho, mom["uy"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(1 + u * ((xi_x * xi_x) @ h), mom["pxx"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u * ((xi_x * xi_y) @ h), mom["pxy"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(1 + u * ((xi_y * xi_y) @ h), mom["pyy"], rtol=0, atol=1e-14)
