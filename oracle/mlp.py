"""FP64 reference of the warm-start coordinate MLP (oracle; test infrastructure only).

Network: 4 -> 256 -> 256 -> 256 -> 6, exact-erf GELU after the three hidden layers,
z_l = a_{l-1} W_l^T + b_l, loss = mean over batch and outputs of (y - t)^2.  Backward by
the chain rule, written out layer by layer.  Optionally the inputs of every matrix
product are rounded to bfloat16 (round to nearest even) at the same points as the GPU
kernels do (layer inputs, weights, and the back-propagated gradients that enter a
product), so that a comparison with the GPU measures accumulation and elementwise
rounding only.  Pinned by central finite differences of the loss in FP64
(tests/test_oracle_mlp.py).

The warm-start reconstruction of the distribution from predicted moments (second-order
Hermite expansion, text of the learned-warm-start configuration) is also here:
  h_a = w_a [ rho' + xi_a . j' + 1/2 sum_ij (P'_ij - rho' delta_ij)(xi_i xi_j - delta_ij) ].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

WIDTHS = (4, 256, 256, 256, 6)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int, widths=WIDTHS):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, FP64 (W_l is [out][in])."""
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(widths) - 1):
        bound = 1.0 / math.sqrt(widths[i])
        W = rng.uniform(-bound, bound, size=(widths[i + 1], widths[i]))
        b = rng.uniform(-bound, bound, size=widths[i + 1])
        params.append((W, b))
    return params


def forward(params, x, bf16: bool = False):
    """Returns (y, cache) for inputs x [M][4]."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a = np.asarray(x, dtype=np.float64)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        a_in = rnd(a)
        Wq = rnd(W)
        z = a_in @ Wq.T + b
        cache.append((a_in, Wq, z))
        a = gelu(z) if l < L - 1 else z
    return a, cache


def loss_and_grads(params, x, t, bf16: bool = False):
    """Mean-squared-error loss and its gradients [(dW, db), ...] (FP64)."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    y, cache = forward(params, x, bf16)
    M, n_out = y.shape
    diff = y - t
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff / (M * n_out)            # dL/dz of the last layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        a_in, Wq, z = cache[l]
        gq = rnd(g)
        grads[l] = (gq.T @ a_in, g.sum(axis=0))
        if l > 0:
            da = gq @ Wq
            g = da * gelu_grad(cache[l - 1][2])
    return loss, grads


def moments_to_h(mom, xi_x, xi_y, w, u_ref):
    """Second-order Hermite reconstruction of h_a from the six moments per cell.

    mom: dict with rho, ux, uy, pxx, pxy, pyy (Eq. (1) units, arrays over cells).
    Returns h [n][ncells]."""
    rho_p = (mom["rho"] - 1.0) / u_ref
    jx = mom["rho"] * mom["ux"] / u_ref
    jy = mom["rho"] * mom["uy"] / u_ref
    pxx = (mom["pxx"] - 1.0) / u_ref
    pxy = mom["pxy"] / u_ref
    pyy = (mom["pyy"] - 1.0) / u_ref
    xx = np.asarray(xi_x)[:, None]
    yy = np.asarray(xi_y)[:, None]
    ww = np.asarray(w)[:, None]
    return ww * (rho_p + xx * jx + yy * jy
                 + 0.5 * ((pxx - rho_p) * (xx * xx - 1.0) + 2.0 * pxy * xx * yy + (pyy - rho_p) * (yy * yy - 1.0)))
