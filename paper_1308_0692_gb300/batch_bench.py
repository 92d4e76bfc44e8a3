"""Time the batched march kernels on a batch of lid-driven cavities (all instances live).

    python -m paper_1308_0692_gb300.batch_bench [--count 32] [--side 128] [--n-half 4]
        [--march on|off] [--warmup 100] [--steps 500] [--launches 1]

Seed-drawn (Kn, u_w) as in the warm-start study, FP32 perturbation storage, tolerance 0 so
that no instance freezes; prints one JSON line: milliseconds per step, node-velocity
updates per second and the equivalent HBM rate at the algorithmic 8 bytes per update.
`--march off` puts every instance on the segment kernel.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=32)
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--n-half", type=int, default=4)
    ap.add_argument("--march", choices=["on", "off"], default="on")
    ap.add_argument("--rows-per-chunk", type=int, default=0, help="0: planned by the library")
    ap.add_argument("--warps-per-item", type=int, default=0, help="M, M/2 or 0 (library default)")
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--launches", type=int, default=1)
    args = ap.parse_args(argv)
    import torch

    from . import lbm, warmstart
    pairs = warmstart.draw_pairs(args.count, seed=20130805)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, args.n_half)
    probs = [lbm.make_problem(lbm.LBM_CAVITY, args.side, args.side, kn, 0.0, uw, prec=lbm.LBM_FP32_PERTURB,
                              residual_every=100) for kn, uw in pairs]
    stream = torch.cuda.Stream()
    b = lbm.lbm_batch_init(vs, probs, stream=stream)
    lbm.lbm_batch_set_march(b, args.march == "on", args.rows_per_chunk if args.march == "on" else 0,
                            args.warps_per_item if args.march == "on" else 0)
    if args.warmup > 0:
        lbm.lbm_batch_advance(b, args.warmup, 0.0)
        lbm.lbm_batch_poll(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.launches):
        lbm.lbm_batch_advance(b, args.steps, 0.0)
    e1.record(stream)
    lbm.lbm_batch_poll(b)
    steps = args.steps * args.launches
    ms = e0.elapsed_time(e1) / steps
    upd = args.count * args.side * args.side * (2 * args.n_half) ** 2 / (ms * 1e-3)
    print(json.dumps({"workload": f"{args.count} cavities {args.side}^2, D2Q^h_{(2 * args.n_half) ** 2}, FP32",
                      "march": lbm.lbm_batch_get_march(b), "schedule": lbm.lbm_batch_get_schedule(b),
                      "steps": steps, "ms_per_step": ms, "updates_per_s": upd,
                      "equivalent_GBs_at_8B": upd * 8 / 1e9}), flush=True)
    b.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
