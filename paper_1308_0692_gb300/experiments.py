"""The paper's comparison of half-range and full-range velocity sets (Figs. 1-2 and the
Kn = 1 shear-stress statement), computed with the library's FP64 march.

Couette flow between plates at -u_w and +u_w: for each Knudsen number and velocity set the
steady state is marched on the GPU to a residual tolerance, and the shear stress (the
momentum flux through the cell faces, the same on every face at steady state) is reported
as p_xy / p_fm with p_fm = -sqrt(2/pi) u_w the free-molecular value (Eq. (1) units).  No
external kinetic (BGKW) solution is available here, so the reference for "kinetic theory"
is the library's own march with the 144-velocity half-range set (N = 6), which the paper
names as converged.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbm

SETS = {
    "D2Q^h_16": (lbm.LBM_HALF_RANGE_GH, 2),
    "D2Q_16": (lbm.LBM_FULL_RANGE_GH, 4),
    "D2Q^h_64": (lbm.LBM_HALF_RANGE_GH, 4),
    "D2Q^h_144": (lbm.LBM_HALF_RANGE_GH, 6),
}


def couette_shear(kind: int, n: int, kn: float, ny: int = 200, u_w: float = 0.01, tol: float = 1e-11,
                  stream=None):
    """Steady Couette p_xy / p_fm and the slip 1 - u_x/u_w of the gas in the cell next to the
    upper plate, FP64 march on the GPU."""
    vs = lbm.lbm_make_velocity_set(kind, n)
    prob = lbm.make_problem(lbm.LBM_COUETTE, 1, ny, kn, -u_w, u_w, prec=lbm.LBM_FP64, residual_every=100)
    sim = lbm.lbm_init(vs, prob, stream=stream)
    info = lbm.lbm_solve(sim, tol, 5_000_000, 0)
    fy, _ = lbm.lbm_face_flux(sim)
    m = lbm.lbm_moments(sim, wall_shear=False)
    p_fm = -math.sqrt(2.0 / math.pi) * u_w
    out = {"kn": kn, "pxy_over_pfm": float(fy[:, 0].mean() / p_fm), "slip": float(1.0 - m["ux"][-1, 0] / u_w),
           "steps": info["steps"], "residual": info["residual"]}
    sim.close()
    return out


def kn_sweep(kns=(0.01, 0.03, 0.1, 0.3, 1.0, 3.0, 10.0), ny=200, sets=("D2Q^h_16", "D2Q_16", "D2Q^h_144")):
    """p_xy / p_fm and wall slip for each set over a Kn sweep; the last set is the reference."""
    import torch
    stream = torch.cuda.Stream()
    res = {name: [couette_shear(*SETS[name], kn, ny=ny, stream=stream) for kn in kns] for name in sets}
    ref = res[sets[-1]]
    summary = {}
    for name in sets[:-1]:
        summary[name] = {
            "max_rel_err_pxy": max(abs(a["pxy_over_pfm"] - b["pxy_over_pfm"]) / abs(b["pxy_over_pfm"])
                                   for a, b in zip(res[name], ref)),
            "max_abs_err_slip": max(abs(a["slip"] - b["slip"]) for a, b in zip(res[name], ref)),
        }
    return {"kns": list(kns), "ny": ny, "results": res, "vs_reference": summary}
