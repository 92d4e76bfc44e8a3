"""Learned warm start of the lid-driven cavity march.

Pipeline (all numerical work in the library's CUDA kernels; PyTorch holds device
memory and gathers minibatches):

1. ``generate``: steady 128 x 128 cavity states for many (Kn, u_w) pairs, marched by the
   batched persistent FP32 solver to a residual tolerance; their six normalised moments
   ((rho-1)/u_w, u_x/u_w, u_y/u_w, (P_xx-1)/u_w, P_xy/u_w, (P_yy-1)/u_w) per cell are the
   training targets.
2. ``train``: Adam on minibatches of (cell features, targets) with the library's BF16
   tensor-core MLP kernels.
3. ``lbm_warm_start`` (C-ABI) builds the initial state of a new cavity from the
   network's prediction; the march from there (the same march as from a cold start)
   decides convergence, and the cold start remains the fallback.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbm
from .inputs import BATCH_SEED

FEATURES = 4
TARGETS = 6


def draw_pairs(count: int, seed: int):
    """(Kn, u_w) with Kn log-uniform in [0.01, 10] and u_w uniform in [0.005, 0.02]."""
    rng = np.random.default_rng(seed)
    kn = 10.0 ** rng.uniform(-2.0, 1.0, count)
    uw = rng.uniform(0.005, 0.02, count)
    return list(zip(kn.tolist(), uw.tolist()))


def generate(pairs, side=128, tol=1e-6, chunk=512, max_steps=400_000, steps_per_launch=1000, n_half=4,
             log=print):
    """Steady cavity states for all pairs; returns a float32 CUDA tensor [len(pairs), side*side, 6]
    of normalised moments and per-instance step counts."""
    import torch
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, n_half)
    ncells = side * side
    out = torch.empty((len(pairs), ncells, TARGETS), dtype=torch.float32, device="cuda")
    steps = np.zeros(len(pairs), dtype=np.int64)
    stream = torch.cuda.Stream()
    mom = torch.empty((6, ncells), dtype=torch.float64, device="cuda")
    n_stall = 0
    for c0 in range(0, len(pairs), chunk):
        sub = pairs[c0:c0 + chunk]
        probs = [lbm.make_problem(lbm.LBM_CAVITY, side, side, kn, 0.0, uw, prec=lbm.LBM_FP32_PERTURB,
                                  residual_every=100) for kn, uw in sub]
        b = lbm.lbm_batch_init(vs, probs, stream=stream)
        t0 = time.perf_counter()
        done = 0
        while done < max_steps:
            lbm.lbm_batch_advance(b, steps_per_launch, tol)
            done += steps_per_launch
            n_active, _ = lbm.lbm_batch_poll(b)
            if n_active == 0:
                break
        with torch.cuda.stream(stream):
            for i, (kn, uw) in enumerate(sub):
                lbm.lbm_batch_moments(b, i, mom.data_ptr())
                m = mom
                out[c0 + i, :, 0] = ((m[0] - 1.0) / uw).float()
                out[c0 + i, :, 1] = (m[1] / uw).float()
                out[c0 + i, :, 2] = (m[2] / uw).float()
                out[c0 + i, :, 3] = ((m[3] - 1.0) / uw).float()
                out[c0 + i, :, 4] = (m[4] / uw).float()
                out[c0 + i, :, 5] = ((m[5] - 1.0) / uw).float()
                st = lbm.lbm_batch_status(b, i)
                steps[c0 + i] = st["steps"]
                n_stall += st["stalled"]
        stream.synchronize()
        log(f"generate: instances {c0}..{c0 + len(sub) - 1} marched (tol {tol:g}; {n_stall} stalled above "
            f"it so far) in {time.perf_counter() - t0:.1f} s, max steps {steps[c0:c0 + len(sub)].max()}")
        b.close()
    return out, steps


def features(pairs, side=128):
    """Feature tensor [len(pairs), side*side, 4] (float32, CUDA) built by the library kernel."""
    import torch
    m = lbm.lbm_mlp_create(side * side, seed=0)
    out = torch.empty((len(pairs), side * side, FEATURES), dtype=torch.float32, device="cuda")
    for i, (kn, uw) in enumerate(pairs):
        lbm.lbm_mlp_features(m, side, side, kn, uw, out[i].data_ptr())
    torch.cuda.synchronize()
    m.close()
    return out


def train(feats, targets, steps=20000, batch_rows=8192, lr=1e-3, lr_final=1e-5, seed=0, max_batch=None,
          log=print):
    """Adam with a cosine-decayed learning rate on uniformly sampled (instance, cell) rows."""
    import torch
    n_inst, ncells, _ = feats.shape
    flat_x = feats.reshape(-1, FEATURES)
    flat_t = targets.reshape(-1, TARGETS)
    mlp = lbm.lbm_mlp_create(max(max_batch or 0, batch_rows, ncells), seed=seed)
    g = torch.Generator(device="cuda").manual_seed(seed)
    xb = torch.empty((batch_rows, FEATURES), dtype=torch.float32, device="cuda")
    tb = torch.empty((batch_rows, TARGETS), dtype=torch.float32, device="cuda")
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        idx = torch.randint(0, flat_x.shape[0], (batch_rows,), device="cuda", generator=g)
        torch.index_select(flat_x, 0, idx, out=xb)
        torch.index_select(flat_t, 0, idx, out=tb)
        torch.cuda.synchronize()
        a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / steps))
        want = it % 1000 == 0 or it == steps - 1
        loss = lbm.lbm_mlp_train_step(mlp, xb.data_ptr(), tb.data_ptr(), batch_rows, a, want_loss=want)
        if want:
            hist.append((it, loss))
            log(f"train: step {it} loss {loss:.3e} lr {a:.2e} ({time.perf_counter() - t0:.1f} s)")
    torch.cuda.synchronize()
    return mlp, hist, time.perf_counter() - t0


def solve_cavity(vs, kn, uw, side=128, prec=lbm.LBM_FP32_PERTURB, tol=1e-8, refine=3, mlp=None, stream=None,
                 refine_tol=0.0):
    """Solve one cavity to tol (cold start or warm start); returns (sim, info, seconds)."""
    import torch
    prob = lbm.make_problem(lbm.LBM_CAVITY, side, side, kn, 0.0, uw, prec=prec, residual_every=100)
    sim = lbm.lbm_init(vs, prob, stream=stream or lbm.PrivateStream())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mlp is not None:
        lbm.lbm_warm_start(sim, mlp, kn, uw)
    info = lbm.lbm_solve(sim, tol, 2_000_000, refine if prec == lbm.LBM_FP32_PERTURB else 0, refine_tol)
    torch.cuda.synchronize()
    return sim, info, time.perf_counter() - t0


def save_params(mlp, path):
    np.save(path, lbm.lbm_mlp_get_params(mlp))


def load_mlp(path, max_batch=128 * 128):
    m = lbm.lbm_mlp_create(max_batch, seed=0)
    lbm.lbm_mlp_set_params(m, np.load(path))
    return m


def batch_solve(vs, pairs, tol, side=128, mlp=None, steps_per_launch=500, max_steps=1_000_000):
    """March all pairs as one batch (cold or warm start) to max(tol, 5e-8) -- the FP32 march's
    share of a refined solve (see lbm_solve); returns (batch, steps per instance, seconds).
    The warm-start reconstruction is included in the time."""
    tol = max(tol, 5e-8)
    import torch
    probs = [lbm.make_problem(lbm.LBM_CAVITY, side, side, kn, 0.0, uw, prec=lbm.LBM_FP32_PERTURB,
                              residual_every=100) for kn, uw in pairs]
    b = lbm.lbm_batch_init(vs, probs, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mlp is not None:
        for i, (kn, uw) in enumerate(pairs):
            lbm.lbm_batch_warm_start(b, i, mlp, kn, uw)
    done = 0
    while done < max_steps:
        lbm.lbm_batch_advance(b, steps_per_launch, tol)
        done += steps_per_launch
        if lbm.lbm_batch_poll(b)[0] == 0:
            break
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    steps = np.array([lbm.lbm_batch_status(b, i)["steps"] for i in range(len(pairs))])
    return b, steps, el


def refine_instances(vs, b, pairs, tol, side=128, threads=32, refine_tol=0.0):
    """Mixed-precision refinement of each converged batch instance (FP64 defect, FP32
    correction march) in single-simulation objects, each on its own stream and driven by
    its own host thread so that the instances' small kernels run concurrently; returns
    (sims, march + correction steps, seconds)."""
    import concurrent.futures as cf

    import torch
    sims = []
    for i, (kn, uw) in enumerate(pairs):
        prob = lbm.make_problem(lbm.LBM_CAVITY, side, side, kn, 0.0, uw, prec=lbm.LBM_FP32_PERTURB,
                                residual_every=100)
        sims.append(lbm.lbm_init(vs, prob, lbm.lbm_batch_get_state(b, i), stream=lbm.PrivateStream()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()

    def one(sim):
        info = lbm.lbm_solve(sim, tol, 1_000_000, 3, refine_tol)
        return info["steps"] + info["correction_steps"]

    with cf.ThreadPoolExecutor(max_workers=min(threads, len(sims))) as ex:
        corr = list(ex.map(one, sims))
    torch.cuda.synchronize()
    return sims, np.array(corr), time.perf_counter() - t0


def refine_batch(b, tol, refine_tol=0.0, max_sweeps=3):
    """Mixed-precision refinement of every batch instance in place, all instances in one
    persistent launch per chunk of correction steps (lbm_batch_refine); returns (per-instance
    records, seconds)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = lbm.lbm_batch_refine(b, tol, max_sweeps, refine_tol)
    torch.cuda.synchronize()
    return info, time.perf_counter() - t0


def batch_fields(b, i):
    """(u_x, u_y) of batch instance i, host FP64 [ny][nx]."""
    import torch
    p = b.probs[i]
    mom = torch.empty(6 * p.nx * p.ny, dtype=torch.float64, device="cuda")
    lbm.lbm_batch_moments(b, i, mom.data_ptr())
    torch.cuda.synchronize()
    m = mom.view(6, p.ny, p.nx).cpu().numpy()
    return m[1], m[2]


def main(argv=None):
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser(description="train / evaluate the warm-start network")
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--train-count", type=int, default=4096)
    ap.add_argument("--test-count", type=int, default=256)
    ap.add_argument("--train-seed", type=int, default=BATCH_SEED + 1)
    ap.add_argument("--test-seed", type=int, default=BATCH_SEED + 2)
    ap.add_argument("--gen-tol", type=float, default=1e-6)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--params", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                                                     "warmstart_mlp.npy"))
    ap.add_argument("--accuracy-count", type=int, default=256)
    ap.add_argument("--out", default=None, help="write a JSON report here")
    args = ap.parse_args(argv)
    report = {}
    if args.cmd == "train":
        pairs = draw_pairs(args.train_count, args.train_seed)
        t0 = time.perf_counter()
        targets, steps = generate(pairs, tol=args.gen_tol)
        t_gen = time.perf_counter() - t0
        feats = features(pairs)
        mlp, hist, t_train = train(feats, targets, steps=args.train_steps)
        os.makedirs(os.path.dirname(args.params), exist_ok=True)
        save_params(mlp, args.params)
        report = {"train_count": len(pairs), "gen_tol": args.gen_tol, "gen_seconds": t_gen,
                  "gen_steps_mean": float(steps.mean()), "gen_steps_max": int(steps.max()),
                  "train_steps": args.train_steps, "train_seconds": t_train, "loss_history": hist}
    else:
        import torch
        vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
        pairs = draw_pairs(args.test_count, args.test_seed)
        mlp = load_mlp(args.params)
        bc, cold_steps, t_cold = batch_solve(vs, pairs, args.tol)
        bw, warm_steps, t_warm = batch_solve(vs, pairs, args.tol, mlp=mlp)
        sub = list(range(min(args.accuracy_count, len(pairs))))
        sims_w, corr_w, t_ref_w = refine_instances(vs, bw, [pairs[i] for i in sub], args.tol)
        errs = []
        for k, i in enumerate(sub):
            kn, uw = pairs[i]
            s64, info64, _ = solve_cavity(vs, kn, uw, prec=lbm.LBM_FP64, tol=1e-11, refine=0)
            m64 = lbm.lbm_moments(s64)
            mw = lbm.lbm_moments(sims_w[k])
            errs.append(max(np.abs(mw[q] - m64[q]).max() for q in ("ux", "uy")) / uw)
            s64.close()
        report = {"test_count": len(pairs), "tol": args.tol,
                  "cold": {"seconds": t_cold, "steps_mean": float(cold_steps.mean()),
                           "steps_median": float(np.median(cold_steps))},
                  "warm": {"seconds": t_warm, "steps_mean": float(warm_steps.mean()),
                           "steps_median": float(np.median(warm_steps))},
                  "steps_ratio_mean": float(np.mean(cold_steps / np.maximum(warm_steps, 1))),
                  "accuracy_subset": len(sub), "max_velocity_error_vs_fp64": float(max(errs)),
                  "refine_seconds_subset": t_ref_w}
    print(json.dumps(report), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(report, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
