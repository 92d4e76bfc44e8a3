"""Batched parameter sweep: 512 seed-drawn independent instances (256 Couette channels with
ny uniform in {64..512}, 256 lid-driven cavities with side in {64, 96, 128, 192, 256}; Kn
log-uniform in [0.01, 10], u_w uniform in [0.005, 0.02]; 64 half-range velocities) marched
together in the persistent batched FP32 kernel with an autotuned schedule, refined with the
FP64 defect correction, and each instance's error reported against an FP64 steady state
(the FP64 GPU march, whose steps are parity-checked against the CPU oracle; every Couette
channel, and the cavities up to a size limit).

Tolerance: a state whose residual (or FP64 defect) is r is off the discrete steady state by
about r / (1 - lambda), lambda the slowest mode's per-step factor; for the Kn ~ 0.01
channels of 500 cells that factor is ~3e3, so a 1e-8 target leaves errors of a few 1e-5.
The refinement therefore targets 1e-10 (the FP32 batch march stops at 5e-8, or where its
residual stops improving), and the
FP64 references are marched to 1e-11.

    python -m paper_1308_0692_gb300.sweep [--count 512] [--out report.json]

Several GPUs (one process per GPU, torchrun): the instances are dealt round-robin to the
ranks (shard), each rank runs its share as its own batch on its own GPU with no
communication, and rank 0 gathers the per-instance records (merge_reports): the sweep's
wall time is the slowest rank's.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import time

import numpy as np

from . import lbm
from .inputs import BATCH_SEED, batch_table


def _problem(inst, prec):
    geom = lbm.LBM_COUETTE if inst["geom"] == "couette" else lbm.LBM_CAVITY
    if geom == lbm.LBM_COUETTE:   # plates +u_w at y = 0 and -u_w at y = 1
        return lbm.make_problem(geom, 1, inst["ny"], inst["kn"], inst["u_w"], -inst["u_w"], prec=prec,
                                residual_every=100)
    return lbm.make_problem(geom, inst["nx"], inst["ny"], inst["kn"], 0.0, inst["u_w"], prec=prec,
                            residual_every=100)


def _log(*a):
    print(*a, flush=True)


def shard(count: int, rank: int, world: int) -> list[int]:
    """Instance indices of one rank: round-robin, so every rank gets the same mix of sizes."""
    return list(range(rank, count, world))


def merge_reports(reports: list[dict]) -> dict:
    """One report from the ranks' reports (instances disjoint): times are the slowest
    rank's, counts add up, per-instance records are merged in index order."""
    per = sorted((r for rep in reports for r in rep["per_instance"]), key=lambda r: r["index"])
    checked = [r["err"] for r in per if "err" in r]
    steps = np.array([r["steps"] for r in per])
    out = {k: reports[0][k] for k in ("seed", "refinement") if k in reports[0]}
    out.update({
        "count": len(per), "ranks": len(reports), "unknowns": int(sum(rep["unknowns"] for rep in reports)),
        "schedule": [rep["schedule"] for rep in reports],
        "tune_seconds": max(rep["tune_seconds"] for rep in reports),
        "batch_seconds": max(rep["batch_seconds"] for rep in reports),
        "refine_seconds": max(rep["refine_seconds"] for rep in reports),
        "reference_seconds": max(rep["reference_seconds"] for rep in reports),
        "steps_min": int(steps.min()), "steps_median": float(np.median(steps)), "steps_max": int(steps.max()),
        "instances_checked": len(checked),
        "max_velocity_error": max((e["u"] for e in checked), default=None),
        "max_wall_shear_error": max((e["wall_shear"] for e in checked), default=None),
        "per_instance": per,
    })
    return out


def run(count=512, seed=BATCH_SEED, tol=1e-10, ref_max_cells=128 * 128, threads=32, log=_log, indices=None,
        refine="batched"):
    """Sweep over the instances `indices` of the seed-drawn table of `count` (all by default).
    refine: "batched" (lbm_batch_refine: every instance's FP64 defect and FP32 correction march
    in the batch's persistent kernels) or "per_instance" (one simulation per instance, each on
    its own stream and host thread)."""
    import torch
    full = batch_table(count, seed)
    indices = list(range(count)) if indices is None else list(indices)
    table = [full[i] for i in indices]
    count_local = len(table)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    probs = [_problem(t, lbm.LBM_FP32_PERTURB) for t in table]
    unknowns = sum(p.nx * p.ny for p in probs) * 64
    b = lbm.lbm_batch_init(vs, probs, stream=torch.cuda.Stream())
    t0 = time.perf_counter()
    best = lbm.lbm_batch_tune(b, 10)
    t_tune = time.perf_counter() - t0
    log(f"sweep: {count_local} instances, {unknowns / 1e6:.1f} M unknowns, schedule {best} (tuned in {t_tune:.1f} s)")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tol32 = max(tol, 5e-8)
    steps_done = 0
    while True:
        lbm.lbm_batch_advance(b, 1000, tol32)
        steps_done += 1000
        n_active, _ = lbm.lbm_batch_poll(b)
        if n_active == 0 or steps_done >= 2_000_000:
            break
    t_batch = time.perf_counter() - t0
    status = [lbm.lbm_batch_status(b, i) for i in range(count_local)]
    steps = np.array([st["steps"] for st in status])
    n_conv = sum(st["converged"] for st in status)
    n_stall = sum(st["stalled"] for st in status)
    log(f"sweep: batch march done, {n_conv} of {count_local} instances converged below {tol32:g}, "
        f"{n_stall} stalled at their FP32 floor above it (both go to the refinement)")
    cells = np.array([p.nx * p.ny for p in probs])
    log(f"sweep: FP32 batch march to {tol32:g} in {t_batch:.1f} s ({steps_done} steps launched, "
        f"{(steps * cells * 64).sum() / t_batch / 1e9:.1f} G updates/s on active instances)")

    idx = [i for i, p in enumerate(probs) if p.nx * p.ny <= ref_max_cells]
    if refine == "batched":
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = lbm.lbm_batch_refine(b, tol, 3, tol, 2_000_000)
        torch.cuda.synchronize()
        t_refine = time.perf_counter() - t0
        ref_info = [(r["correction_steps"], r["defect"]) for r in info]
        # the refined states of the checked instances into simulations for the diagnostics
        sims = {i: lbm.lbm_init(vs, probs[i], lbm.lbm_batch_get_state(b, i), stream=lbm.PrivateStream())
                for i in idx}
        b.close()
    else:
        # refinement of every instance, one stream and host thread each
        sims = {i: lbm.lbm_init(vs, p, lbm.lbm_batch_get_state(b, i), stream=lbm.PrivateStream())
                for i, p in enumerate(probs)}
        b.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def refine_one(sim):
            info = lbm.lbm_solve(sim, tol, 2_000_000, 3, tol)
            return info["correction_steps"], info["defect"]

        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            ref_info = list(ex.map(refine_one, [sims[i] for i in range(count_local)]))
        torch.cuda.synchronize()
        t_refine = time.perf_counter() - t0
    log(f"sweep: {refine} refinement of all instances in {t_refine:.1f} s")

    # FP64 references (GPU march), concurrently

    def reference(i):
        p64 = _problem(table[i], lbm.LBM_FP64)
        s64 = lbm.lbm_init(vs, p64, stream=lbm.PrivateStream())
        lbm.lbm_solve(s64, tol * 1e-1, 5_000_000, 0)
        m = lbm.lbm_moments(s64)
        s64.close()
        return m

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        refs = dict(zip(idx, ex.map(reference, idx)))
    t_ref = time.perf_counter() - t0
    errs = {}
    for i in idx:
        m32 = lbm.lbm_moments(sims[i])
        m64 = refs[i]
        uw = table[i]["u_w"]
        errs[i] = {"u": float(max(np.abs(m32["ux"] - m64["ux"]).max(), np.abs(m32["uy"] - m64["uy"]).max()) / uw),
                   "wall_shear": float(np.abs(m32["wall_shear"] - m64["wall_shear"]).max()
                                       / max(np.abs(m64["wall_shear"]).max(), 1e-300))}
    for s in sims.values():
        s.close()
    report = {
        "count": count_local, "seed": seed, "unknowns": int(unknowns), "schedule": best, "tune_seconds": t_tune,
        "batch_seconds": t_batch, "refinement": refine, "refine_seconds": t_refine, "reference_seconds": t_ref,
        "steps_min": int(steps.min()), "steps_median": float(np.median(steps)), "steps_max": int(steps.max()),
        "instances_checked": len(errs),
        "max_velocity_error": max((e["u"] for e in errs.values()), default=None),      # None: nothing checked
        "max_wall_shear_error": max((e["wall_shear"] for e in errs.values()), default=None),
        "per_instance": [{"index": indices[i], **table[i], "steps": int(steps[i]),
                          "correction_steps": int(ref_info[i][0]), "defect": float(ref_info[i][1]),
                          **({"err": errs[i]} if i in errs else {})}
                         for i in range(count_local)],
    }
    return report


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--ref-max-cells", type=int, default=128 * 128)
    ap.add_argument("--refine", choices=["batched", "per_instance"], default="batched")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    import os
    world, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend="gloo")   # only the final gather of Python records
    rep = run(args.count, tol=args.tol, ref_max_cells=args.ref_max_cells, indices=shard(args.count, rank, world),
              log=_log if rank == 0 else (lambda *a: None), refine=args.refine)
    if dist is not None:
        reps = [None] * world
        dist.all_gather_object(reps, rep)
        rep = merge_reports(reps)
        dist.destroy_process_group()
    else:
        rep = merge_reports([rep])
    if rank == 0:
        short = {k: v for k, v in rep.items() if k != "per_instance"}
        print(json.dumps(short), flush=True)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(rep, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
