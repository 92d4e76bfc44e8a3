"""Benchmark of the fused finite-difference LB step on GB300.

Workload (default): lid-driven cavity 2048 x 2048 cells, half-range Gauss-Hermite set
with N = 6 nodes per half-axis (12 per axis, 144 velocities, 603,979,776 unknowns),
Kn = 0.05, lid speed 0.01, FP32 perturbation storage, FP64 residual every 10 steps.
One bench step = one time step of the whole hot path (upwind transport with wall
ghosts, moments, relaxation; the residual reduction on every 10th step).

Metric: node-velocity updates per second (cells x velocities x steps / s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]

With --gpus N > 1 (launched by torchrun) every rank marches its own replica of the
workload (the single-domain march has no data-parallel split without a halo exchange,
so ranks are independent replicas); value = all ranks' updates / max rank time.
--impl reference times the CPU oracle (plain FP64 C, all host cores) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import contextlib
import gc
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {
    "name": "cavity2048_Dh144_fp32",
    "geom": 1, "nx": 2048, "ny": 2048, "n_half": 6, "kn": 0.05, "u_bottom": 0.0, "u_top": 0.01,
    "cfl": 0.9, "residual_every": 10,
}
METRIC = "node-velocity updates/s"
UNIT = "updates/s"
E2E_STEPS = 100            # time steps per end-to-end API call (one residual interval)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ---------------------------------------------------------------- distributed plumbing
class Dist:
    """Rank bookkeeping; N > 1 runs independent replicas, the only collectives are the
    timing barrier and the max-over-ranks of the elapsed time."""

    def __init__(self, backend: str | None = None):
        self.world = _env_int("WORLD_SIZE", 1)
        self.rank = _env_int("RANK", 0)
        self.local_rank = _env_int("LOCAL_RANK", 0)
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend or ("nccl" if _cuda_ok() else "gloo"))
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, value: float) -> float:
        if not self.pg:
            return value
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, value: float) -> float:
        if not self.pg:
            return value
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def _cuda_ok() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def aggregate(units_per_rank: float, seconds_per_rank: float, dist: Dist):
    """Whole-job throughput: all ranks' units / the slowest rank's time."""
    t = dist.max(seconds_per_rank)
    u = dist.sum(units_per_rank)
    return u / t, t


# ---------------------------------------------------------------- timing helpers
@contextlib.contextmanager
def gc_paused():
    """A full pass of Python's cyclic garbage collector takes tens of ms with torch loaded and
    falls at a fixed point of the allocation count: collect before a timed region and pause
    the collector inside it, as timeit does."""
    gc.collect()
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = os.path.join(os.environ.get("LBM_CLOCK_LOG_DIR", tempfile.gettempdir()),
                                 f"lbm_bench_clocks_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_index}",
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def clocks_bad(clk: dict) -> bool:
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if any(r in bad for r in clk.get("reasons", [])):
        return True
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and smax and sm < 0.6 * smax and "sw_power_cap" not in clk.get("reasons", []):
        return True
    return False


# ---------------------------------------------------------------- own arm
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _traffic_record(kernel_key: str, order: int = 1):
    """ncu DRAM bytes per launch for the kernel, if captured for the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel_key)
    if not rec:
        return None
    h = hashlib.sha256()
    names = ("step_kernel.cuh", "step_tma.cuh", "step_march.cuh")
    if order == 2:
        names += ("step_so.cuh", "step_so_march.cu")
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_1308_0692_gb300", "csrc", name), "rb").read())
    digest = h.hexdigest()[:16]
    if rec.get("source_sha256_16") != digest:
        return None
    return rec.get("dram_bytes_per_launch")


VARIANTS = [(4, 0), (6, 0), (6, 2), (6, 3), (6, 4), (6, 5), (6, 6), (6, 7), (6, 8), (6, 9), (12, 4), (12, 5)]
LOAD_PATHS = ["registers", "prefetch", "tma", "tma+walls merged", "column march (4 row slots)",
              "column march (5 row slots)", "column march (2 row slots, 2 blocks per SM)",
              "column march (4 row slots, relaxation deferred by one row)",
              "column march on the strip-tiled state (4 row slots)",
              "column march on the strip-tiled state (4 row slots, bulk asynchronous stores)"]
# second-order transport (lbm_set_transport(sim, 2)): the segment kernel, and the second-order
# column march on the strip-tiled state
VARIANTS_SO = [(6, 0), (6, 8), (6, 9)]
LOAD_PATHS_SO = {0: "second-order segment kernel (registers)",
                 8: "second-order column march on the strip-tiled state (5 row slots)",
                 9: "second-order column march on the strip-tiled state (4 row slots, bulk asynchronous stores)"}


def choose_variant(sim, stream, args, variants=None, steps_per_trial=8):
    """Autotune the step kernel on the workload itself: warps per segment x load path
    (0 registers, 2 TMA-staged halo, 3 the same with the walls in one launch, 4 to 9 the
    TMA column march), a few timed steps each; or the forced --variant."""
    import torch

    from paper_1308_0692_gb300 import lbm
    if args is not None and args.variant:
        g, pf = (int(v) for v in args.variant.split(","))
        lbm.lbm_set_variant(sim, g, pf)
        return (g, pf), None
    times = {}
    for g, pf in (variants or VARIANTS):
        try:
            lbm.lbm_set_variant(sim, g, pf)
        except lbm.LBMError:
            continue
        lbm.lbm_step(sim, 2)
        trials = []
        for _ in range(3):                      # best of three runs of steps_per_trial steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lbm.lbm_step(sim, steps_per_trial)
            e1.record(stream)
            torch.cuda.synchronize()
            trials.append(e0.elapsed_time(e1) / steps_per_trial)
        times[f"{g},{pf}"] = min(trials)
    best = min(times, key=times.get)
    g, pf = (int(v) for v in best.split(","))
    lbm.lbm_set_variant(sim, g, pf)
    return (g, pf), times


def run_own(args, dist: Dist):
    import numpy as np
    import torch

    from paper_1308_0692_gb300 import lbm

    torch.cuda.set_device(dist.local_rank)
    dev_index = torch.cuda.current_device()
    w = WORKLOAD
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, w["n_half"])
    n_vel = (2 * w["n_half"]) ** 2
    prob = lbm.make_problem(w["geom"], w["nx"], w["ny"], w["kn"], w["u_bottom"], w["u_top"], w["cfl"],
                            lbm.LBM_FP32_PERTURB, w["residual_every"])
    stream = torch.cuda.Stream()
    buf = torch.empty(lbm.lbm_sim_bytes(vs, prob), dtype=torch.uint8, device="cuda")
    sim = lbm.lbm_init(vs, prob, None, device_buf=buf, stream=stream)
    order = args.transport
    if order == 2:
        lbm.lbm_set_transport(sim, 2)
        lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_STRANG_EXACT)
    ncells = w["nx"] * w["ny"]
    units_per_step = ncells * n_vel
    variant, tuning = choose_variant(sim, stream, args, VARIANTS_SO if order == 2 else VARIANTS)
    load_path = LOAD_PATHS_SO[variant[1]] if order == 2 else LOAD_PATHS[variant[1]]

    def timed_block(K):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with gc_paused():
            t0.record(stream)
            for i in range(K):
                starts[i].record(stream)
                lbm.lbm_step(sim, 1)
                ends[i].record(stream)
            t1.record(stream)
            torch.cuda.synchronize()
        dist.barrier()
        total = t0.elapsed_time(t1) / 1e3
        per = [s.elapsed_time(e) / 1e3 for s, e in zip(starts, ends)]
        return total, per

    lbm.lbm_step(sim, args.warmup)
    torch.cuda.synchronize()
    for attempt in range(2):
        sampler = ClockSampler(dev_index)
        sampler.start()
        time.sleep(0.3)
        _, step0 = lbm.lbm_state_device(sim)
        total, per = timed_block(args.steps)
        clk = sampler.stop()
        if not clocks_bad(clk):
            break
    value, tmax = aggregate(units_per_step * args.steps, total, dist)
    r, rstep = lbm.lbm_residual(sim)

    # dominant kernel: the plain fused step (steps whose index is not a residual step)
    plain = [d for i, d in enumerate(per) if (step0 + i + 1) % w["residual_every"] != 0]
    resid = [d for i, d in enumerate(per) if (step0 + i + 1) % w["residual_every"] == 0]
    algo_bytes = 8 * units_per_step          # read + write of every FP32 value
    avg = sum(plain) / len(plain)
    peak, peak_kind = _peaks()
    achieved = algo_bytes / avg / 1e9
    n_resid = len(resid)
    per_step = 1 if variant[1] == 3 else 2  # interior and wall kernels (one merged launch for path 3)
    launches = args.steps * per_step + n_resid   # + residual finalisations

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"lid-driven cavity {w['nx']}x{w['ny']}, D2Q^h_144 (N=6 half-range Gauss-Hermite), "
                               "Kn=0.05, lid u=0.01, FP32 perturbation storage, FP64 residual every 10 steps"
                               + ("; second-order transport (Beam-Warming face fluxes), symmetric splitting "
                                  "with exact relaxation" if order == 2 else ""),
                   "nx": w["nx"], "ny": w["ny"], "velocities": n_vel, "unknowns": units_per_step,
                   "residual_every": w["residual_every"], "cold_start": True,
                   "variant": {"warps_per_segment": variant[0], "load_path": load_path,
                               "autotune_ms_per_step": tuning},
                   "l2": f"inputs larger than L2 ({units_per_step * 4 / 1e9:.2f} GB per state copy), no flush",
                   "parallelism": f"replicas{dist.world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": f"fused step (interior + wall launches), {variant[0]} warps/segment, "
                               f"{load_path} loads",
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "avg_launch_ms": avg * 1e3,
                     "traffic": _traffic_record(f"step_f32_m12_g{variant[0]}_pf{variant[1]}"
                                                + ("_so" if order == 2 else ""), order)},
        "residual_step_ms": (sum(resid) / len(resid) * 1e3) if resid else None,
        "last_residual": [r, rstep],
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_e2e:
        out["e2e"] = run_e2e(sim, prob, n_vel, ncells, stream, dist, args)
        # the same calls with the FP64 host upload (lbm_set_state), twice the uploaded bytes
        e64 = run_e2e(sim, prob, n_vel, ncells, stream, dist, args, host_fp64=True)
        out["e2e"]["fp64_host_upload"] = {"value": e64["value"], "ms_per_call": round(e64["ms_per_call"], 2),
                                          "h2d_bytes_per_step": e64["h2d_bytes_per_step"]}
    if not args.no_extras and dist.world == 1 and order == 1:
        out["fp64"] = run_fp64_same_workload(vs, dist)
        sim.close()
        del buf
        torch.cuda.empty_cache()
        out["second_order"] = run_second_order_same_workload(vs, dist)
        out["time_to_residual"] = run_time_to_residual(dist)
        return out
    sim.close()
    del buf
    return out


def run_e2e(sim, prob, n_vel, ncells, stream, dist, args, host_fp64: bool = False):
    """Same metric through the public C-ABI with host buffers: upload a host state (pinned;
    FP32, the simulation's storage precision, through lbm_set_state_f32, or FP64 through
    lbm_set_state), march E2E_STEPS steps, read back the residual and u_x, u_y."""
    import ctypes

    import torch

    from paper_1308_0692_gb300 import lbm

    lib = lbm.library()
    nvals = n_vel * ncells
    hdt = torch.float64 if host_fp64 else torch.float32
    host_h = torch.zeros(nvals, dtype=hdt).pin_memory()
    ux = torch.empty(ncells, dtype=torch.float64).pin_memory()
    uy = torch.empty(ncells, dtype=torch.float64).pin_memory()
    dp = ctypes.POINTER(ctypes.c_double)
    upload = lib.lbm_set_state if host_fp64 else lib.lbm_set_state_f32
    hp = ctypes.cast(host_h.data_ptr(), dp if host_fp64 else ctypes.POINTER(ctypes.c_float))

    def one(rec=None):
        t0 = time.perf_counter()
        lbm._check(upload(sim.handle, hp))
        t1 = time.perf_counter()
        lbm.lbm_step(sim, E2E_STEPS)
        lbm.lbm_residual(sim)               # waits for the march
        t2 = time.perf_counter()
        lbm._check(lib.lbm_moments(sim.handle, None, ctypes.cast(ux.data_ptr(), dp),
                                   ctypes.cast(uy.data_ptr(), dp), None, None, None, None))
        t3 = time.perf_counter()
        if rec is not None:
            rec.append((t1 - t0, t2 - t1, t3 - t2))

    one()
    reps = 5
    rec = []
    dist.barrier()
    torch.cuda.synchronize()
    with gc_paused():
        t = time.perf_counter()
        for _ in range(reps):
            one(rec)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
    value, _ = aggregate(float(nvals) * E2E_STEPS * reps, el, dist)
    # each call's parts by the host clock (every part ends synchronised); the upload's share
    # moves with the host<->device copy rate of the machine
    hb = host_h.element_size()
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": nvals * hb,
            "d2h_bytes_per_step": 2 * ncells * 8 + 32,
            "ms_per_call": el / reps * 1e3,
            "calls_ms": [{"set_state": round(p[0] * 1e3, 2), "step_and_residual": round(p[1] * 1e3, 2),
                          "moments": round(p[2] * 1e3, 2)} for p in rec],
            "h2d_gbs_in_set_state": nvals * hb / min(p[0] for p in rec) / 1e9,
            "definition": f"one API call = {'lbm_set_state(host FP64' if host_fp64 else 'lbm_set_state_f32(host FP32'}"
                          f", pinned) + lbm_step({E2E_STEPS}) + lbm_residual + lbm_moments(ux, uy); value counts "
                          "the marched updates; Python's cyclic garbage collector paused during the timed calls "
                          "(as timeit does)"}


def run_fp64_same_workload(vs, dist, order: int = 1):
    """The plain FP64 march of the same workload (FP64 storage and arithmetic), few steps;
    order 2: its second-order variant (profiling)."""
    import torch

    from paper_1308_0692_gb300 import lbm
    w = WORKLOAD
    prob = lbm.make_problem(w["geom"], w["nx"], w["ny"], w["kn"], w["u_bottom"], w["u_top"], w["cfl"],
                            lbm.LBM_FP64, w["residual_every"])
    stream = torch.cuda.Stream()
    sim = lbm.lbm_init(vs, prob, None, stream=stream)
    if order == 2:
        lbm.lbm_set_transport(sim, 2)
        lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_STRANG_EXACT)
    lbm.lbm_step(sim, 3)
    K = 20
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    lbm.lbm_step(sim, K)
    t1.record(stream)
    torch.cuda.synchronize()
    sec = t0.elapsed_time(t1) / 1e3
    units = w["nx"] * w["ny"] * (2 * w["n_half"]) ** 2 * K
    sim.close()
    # the FP64 pipe's measured rate (a throughput kernel of this library) and the FP64 pipe
    # instructions the step executes per update (ncu, sm__inst_executed_pipe_fp64 x 32 lanes /
    # updates, FP64 step kernel at 1024^2 x 144)
    fma_rate = lbm.lbm_probe_fp64_rate(200_000, stream)
    ops = FP64_PIPE_OPS_PER_UPDATE
    return {"value": units / sec, "unit": UNIT, "steps": K, "ms_per_step": sec / K * 1e3,
            "achieved_hbm_gbs": 16 * units / sec / 1e9,
            "fp64_pipe": {"bound": "alu", "measured_fp64_ops_per_s": fma_rate, "ops_per_update": ops,
                          "achieved_fp64_ops_per_s": units / sec * ops, "frac": units / sec * ops / fma_rate},
            "note": "FP64 storage+arithmetic; bounded by the FP64 pipe of GB300, not HBM"}


def run_second_order_same_workload(vs, dist, steps: int = 20):
    """The second-order variant of the same workload (Beam-Warming face fluxes, symmetric
    splitting with exact relaxation): the FP32 step through each of its kernel variants (the
    fastest reported with its HBM roofline at 8 B per update) and the FP64 step."""
    import torch

    from paper_1308_0692_gb300 import lbm
    w = WORKLOAD
    units = w["nx"] * w["ny"] * (2 * w["n_half"]) ** 2
    peak, peak_kind = _peaks()
    res = {}
    for prec in (lbm.LBM_FP32_PERTURB, lbm.LBM_FP64):
        prob = lbm.make_problem(w["geom"], w["nx"], w["ny"], w["kn"], w["u_bottom"], w["u_top"], w["cfl"], prec,
                                w["residual_every"])
        stream = torch.cuda.Stream()
        sim = lbm.lbm_init(vs, prob, None, stream=stream)
        lbm.lbm_set_transport(sim, 2)
        lbm.lbm_set_splitting(sim, lbm.LBM_SPLIT_STRANG_EXACT)
        if prec == lbm.LBM_FP32_PERTURB:
            # trials of one residual interval each: every trial holds one residual step
            variant, tuning = choose_variant(sim, stream, None, VARIANTS_SO, w["residual_every"])
        else:
            variant, tuning = lbm.lbm_get_variant(sim), None
        lbm.lbm_step(sim, 3)
        torch.cuda.synchronize()
        K = steps if prec == lbm.LBM_FP32_PERTURB else 5
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        lbm.lbm_step(sim, K)
        t1.record(stream)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3 / K
        sim.close()
        if prec == lbm.LBM_FP32_PERTURB:
            achieved = 8 * units / sec / 1e9
            res["fp32"] = {"value": units / sec, "unit": UNIT, "steps": K, "ms_per_step": sec * 1e3,
                           "variant": {"warps_per_segment": variant[0], "load_path": LOAD_PATHS_SO[variant[1]],
                                       "autotune_ms_per_step": tuning},
                           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                        "frac": achieved / peak,
                                        "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                                        "basis": "8 B per update (one FP32 read and write of every value), "
                                                 "residual steps included"}}
        else:
            # FP64 pipe operations of the step: the per-update counts of its two kernels (ncu,
            # 1024^2 x 144) weighted by the cells each takes here (the wall kernel: the bottom
            # and top rows and the 32-cell segments at both ends of every other row)
            nx, ny = w["nx"], w["ny"]
            wall_cells = 2 * nx + (ny - 2) * 64
            ops = (FP64_SO_OPS_BULK * (nx * ny - wall_cells) + FP64_SO_OPS_WALL * wall_cells) / (nx * ny)
            rate = lbm.lbm_probe_fp64_rate(200_000, stream)
            res["fp64"] = {"value": units / sec, "unit": UNIT, "steps": K, "ms_per_step": sec * 1e3,
                           "variant": {"warps_per_segment": variant[0], "load_path": LOAD_PATHS_SO[variant[1]]},
                           "fp64_pipe": {"bound": "alu", "measured_fp64_ops_per_s": rate, "ops_per_update": ops,
                                         "achieved_fp64_ops_per_s": units / sec * ops,
                                         "frac": units / sec * ops / rate},
                           "note": "FP64 storage+arithmetic, second-order segment kernel; FP64-pipe bound"}
    return res


# FP64 pipe instructions (lane operations) per update of the second-order FP64 step's bulk
# and wall kernels (ncu sm__inst_executed_pipe_fp64 x 32 / updates, 1024^2 x 144, six warps
# per segment; profiles/)
FP64_SO_OPS_BULK = 12.38
FP64_SO_OPS_WALL = 24.0


# FP64 pipe instructions (lane operations) per node-velocity update of the FP64 step, from the
# ncu count of sm__inst_executed_pipe_fp64 on the 1024^2 x 144 FP64 step (profiles/)
FP64_PIPE_OPS_PER_UPDATE = 10.1


# refinement design behind the time-to-residual headline: "per_instance" (one simulation per
# instance on concurrent streams) or "batched" (lbm_batch_refine)
REFINE_HEADLINE = "batched"


HELD_OUT_SEED = 20130805     # the warm-start network's 256 held-out (Kn, u_w) pairs
HELD_OUT_COUNT = 256
ABLATION_COUNT = 32         # the one-factor-at-a-time rows run on the first 32 of them


def run_time_to_residual(dist):
    """Time to steady state of held-out lid-driven cavities (128 x 128, 64 half-range
    velocities, Kn log-uniform in [0.01, 10], u_w in [0.005, 0.02]; residual 1e-8 checked
    every 100 steps).

    All 256 held-out pairs of the warm-start network (the headline):
      fp64        plain FP64 march of every instance, 32 instances at a time on their own
                  streams and host threads (graph-captured residual intervals);
      batch_dc    one persistent batched FP32 sweep, then the batched FP64-defect refinement;
      warm_dc     the same from the learned warm start.
    The first 32 pairs, one factor at a time:
      fp64        plain FP64 march, instances one after another;
      fp64_concurrent  the same solves, all 32 at once on their own streams;
      fp32_dc     FP32 march + FP64-defect refinement, one after another;
      batch_dc, warm_dc as above (the refinement also run one simulation per instance).
    The refinement marches the correction until its per-step change is below tol (the
    criterion the FP64 march meets), i.e. equal accuracy by construction; the measured
    accuracy of every variant, max |u - u_fp64| / u_w over every instance, is reported."""
    import numpy as np
    import torch

    from paper_1308_0692_gb300 import lbm, warmstart
    pairs_all = warmstart.draw_pairs(HELD_OUT_COUNT, seed=HELD_OUT_SEED)
    vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, 4)
    tol = 1e-8
    params = os.path.join(ROOT, "paper_1308_0692_gb300", "data", "warmstart_mlp.npy")
    mlp = warmstart.load_mlp(params) if os.path.exists(params) else None

    def fields(sim):
        m = lbm.lbm_moments(sim, wall_shear=False)
        return m["ux"], m["uy"]

    def fp64_concurrent(pairs, threads):
        """Every instance's FP64 solve on its own stream, `threads` solves in flight."""
        sims = []
        for kn, uw in pairs:
            prob = lbm.make_problem(lbm.LBM_CAVITY, 128, 128, kn, 0.0, uw, prec=lbm.LBM_FP64, residual_every=100)
            sims.append(lbm.lbm_init(vs, prob, stream=lbm.PrivateStream()))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            infos = list(ex.map(lambda sm: lbm.lbm_solve(sm, tol, 2_000_000, 0), sims))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        refs = [fields(sm) for sm in sims]
        for sm in sims:
            sm.close()
        return el, [i["steps"] for i in infos], refs

    def batched(pairs, ref, net, per_instance):
        def err(got, i):
            return max(np.abs(got[0] - ref[i][0]).max(), np.abs(got[1] - ref[i][1]).max()) / pairs[i][1]
        b, steps, tb = warmstart.batch_solve(vs, pairs, tol, mlp=net)
        per = None
        if per_instance:
            # refinement one simulation per instance (own stream and host thread), from the
            # same batch states, timed beside the batched refinement
            sims, corr, tp = warmstart.refine_instances(vs, b, pairs, tol, refine_tol=tol)
            per = {"refine_seconds": tp, "refine_steps": corr.tolist(),
                   "max_err_vs_fp64": max(err(fields(sm), i) for i, sm in enumerate(sims))}
            for sm in sims:
                sm.close()
        n_stall = sum(lbm.lbm_batch_status(b, i)["stalled"] for i in range(len(pairs)))
        info, tr = warmstart.refine_batch(b, tol, refine_tol=tol)
        errs = [err(warmstart.batch_fields(b, i), i) for i in range(len(pairs))]
        b.close()
        out = {"seconds": tb + tr, "batch_seconds": tb, "refine_seconds": tr, "refinement": "batched",
               "steps": steps.tolist(), "refine_steps": [r["correction_steps"] for r in info],
               "sweeps": [r["sweeps"] for r in info], "stalled_in_march": int(n_stall),
               "max_err_vs_fp64": max(errs), "checked": len(errs)}
        if per is not None:
            out["per_instance_refinement"] = per
        return out

    # ---- all 256 held-out pairs
    t64, steps64, ref_all = fp64_concurrent(pairs_all, 32)
    upd_all = float(sum(steps64)) * 128 * 128 * 64
    full = {"workload": f"{len(pairs_all)} held-out lid-driven cavities 128x128 (seed {HELD_OUT_SEED}), D2Q^h_64, "
                        f"Kn log-uniform [0.01,10], u_w U(0.005,0.02), residual {tol:g}",
            "fp64": {"seconds": t64, "steps": steps64, "updates_per_s": upd_all / t64,
                     "schedule": "32 instances in flight, each on its own stream and host thread"}}
    full["batch_dc"] = batched(pairs_all, ref_all, None, False)
    full["warm_dc"] = batched(pairs_all, ref_all, mlp, False) if mlp is not None else None
    for k in ("batch_dc", "warm_dc"):
        if full[k]:
            full[k]["speedup_vs_fp64"] = t64 / full[k]["seconds"]

    # ---- the first 32 pairs, one factor at a time
    pairs = pairs_all[:ABLATION_COUNT]
    ref, t64s, steps64s = [], 0.0, []
    for kn, uw in pairs:
        sim, info, el = warmstart.solve_cavity(vs, kn, uw, prec=lbm.LBM_FP64, tol=tol, refine=0)
        t64s += el
        steps64s.append(info["steps"])
        ref.append(fields(sim))
        sim.close()
    upd = float(sum(steps64s)) * 128 * 128 * 64
    sub = {"workload": f"the first {len(pairs)} of the held-out pairs", "pairs": pairs,
           "fp64": {"seconds": t64s, "steps": steps64s, "updates_per_s": upd / t64s}}
    t64c, _, _ = fp64_concurrent(pairs, len(pairs))
    sub["fp64_concurrent"] = {"seconds": t64c, "updates_per_s": upd / t64c}
    t32, e32, st32 = 0.0, 0.0, []
    for i, (kn, uw) in enumerate(pairs):
        sim, info, el = warmstart.solve_cavity(vs, kn, uw, prec=lbm.LBM_FP32_PERTURB, tol=tol, refine=3,
                                               refine_tol=tol)
        t32 += el
        st32.append(info["steps"] + info["correction_steps"])
        ux, uy = fields(sim)
        e32 = max(e32, max(np.abs(ux - ref[i][0]).max(), np.abs(uy - ref[i][1]).max()) / uw)
        sim.close()
    sub["fp32_dc"] = {"seconds": t32, "steps": st32, "max_err_vs_fp64": e32, "speedup_vs_fp64": t64s / t32}
    sub["batch_dc"] = batched(pairs, ref, None, True)
    sub["warm_dc"] = batched(pairs, ref, mlp, True) if mlp is not None else None
    for k in ("batch_dc", "warm_dc"):
        if sub[k]:
            sub[k]["speedup_vs_fp64"] = t64s / sub[k]["seconds"]
            sub[k]["speedup_vs_fp64_concurrent"] = t64c / sub[k]["seconds"]
    if mlp is not None:
        mlp.close()
    return {"held_out_256": full, "ablation_32": sub}


def ttr_summary(ttr: dict, oracle_rate: float | None) -> dict:
    """A short digest of the time-to-residual runs (seconds, speed-ups, worst velocity error
    against the FP64 march, instance counts), printed as the line's last key."""
    def r3(x):
        return None if x is None else float(f"{x:.4g}")
    full, sub = ttr["held_out_256"], ttr["ablation_32"]
    out = {"tol": 1e-8, "n": len(full["fp64"]["steps"]), "fp64_s": r3(full["fp64"]["seconds"]),
           "batch_dc_s": r3(full["batch_dc"]["seconds"]),
           "batch_dc_max_du": r3(full["batch_dc"]["max_err_vs_fp64"])}
    if full.get("warm_dc"):
        w = full["warm_dc"]
        out.update({"warm_dc_s": r3(w["seconds"]), "warm_dc_max_du": r3(w["max_err_vs_fp64"]),
                    "warm_vs_fp64": r3(w["speedup_vs_fp64"]), "checked": w["checked"]})
    out["first32"] = {"fp64_seq_s": r3(sub["fp64"]["seconds"]), "fp64_conc_s": r3(sub["fp64_concurrent"]["seconds"]),
                      "fp32_dc_s": r3(sub["fp32_dc"]["seconds"]), "batch_dc_s": r3(sub["batch_dc"]["seconds"]),
                      "warm_dc_s": r3(sub["warm_dc"]["seconds"]) if sub.get("warm_dc") else None}
    if oracle_rate:
        upd = float(sum(full["fp64"]["steps"])) * 128 * 128 * 64
        out["oracle_extrap_s"] = r3(upd / oracle_rate)
    return out


def run_configs_time_to_residual():
    """The small configurations solved to their residual tolerance three ways: the CPU oracle
    (FP64, all host cores), the GPU FP64 march, and the GPU FP32 march with FP64 defect
    correction; steps, seconds and the GPU results' distance to the oracle's (max |du|/u_w).
    Couette ny = 100 (D2Q^h_64, plates +-0.01, Kn 0.1 / 0.01 / 10, r < 1e-10); cavity 128^2
    (lid 0.01, D2Q^h_64 at Kn 0.1 and 1, D2Q9 at Kn 0.1, r < 1e-8); cold starts, residual
    checked every 100 steps."""
    import numpy as np
    import torch

    from oracle import march as om
    from paper_1308_0692_gb300 import lbm
    om.build()
    cases = [("couette", "half", 4, om.COUETTE, 1, 100, kn, 0.01, -0.01, 1e-10) for kn in (0.1, 0.01, 10.0)]
    cases += [("cavity", "half", 4, om.CAVITY, 128, 128, kn, 0.0, 0.01, 1e-8) for kn in (0.1, 1.0)]
    cases += [("cavity", "full", 3, om.CAVITY, 128, 128, 0.1, 0.0, 0.01, 1e-8)]
    out = []
    for name, kind, n, geom, nx, ny, kn, ub, ut, tol in cases:
        uw = max(abs(ub), abs(ut))
        p = om.make_problem(kind, n, geom, nx, ny, kn, ub, ut)
        t0 = time.perf_counter()
        h, steps_cpu, _ = p.march(p.zeros(), 5_000_000, every=100, tol=tol)
        t_cpu = time.perf_counter() - t0
        m_cpu = p.moments(h)
        vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH if kind == "half" else lbm.LBM_FULL_RANGE_GH, n)
        rec = {"case": f"{name} {nx}x{ny} {'D2Q^h' if kind == 'half' else 'D2Q'}_{p.n} Kn={kn}", "tol": tol,
               "oracle": {"seconds": t_cpu, "steps": steps_cpu, "threads": os.cpu_count()}}
        for label, prec, refine in (("gpu_fp64", lbm.LBM_FP64, 0), ("gpu_fp32_dc", lbm.LBM_FP32_PERTURB, 3)):
            prob = lbm.make_problem(geom, nx, ny, kn, ub, ut, prec=prec, residual_every=100)
            sim = lbm.lbm_init(vs, prob, stream=lbm.PrivateStream())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = lbm.lbm_solve(sim, tol, 5_000_000, refine, tol)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            m = lbm.lbm_moments(sim, wall_shear=False)
            err = max(np.abs(m["ux"] - m_cpu["ux"]).max(), np.abs(m["uy"] - m_cpu["uy"]).max()) / uw
            rec[label] = {"seconds": el, "steps": info["steps"] + info["correction_steps"],
                          "max_du_over_uw_vs_oracle": float(err), "speedup_vs_oracle": t_cpu / el}
            sim.close()
        out.append(rec)
    return out


# ---------------------------------------------------------------- CPU oracle arm
def _oracle_setup(rows: int):
    import numpy as np

    from oracle.march import CAVITY, make_problem
    w = WORKLOAD
    p = make_problem("half", w["n_half"], CAVITY, w["nx"], w["ny"], w["kn"], w["u_bottom"], w["u_top"], w["cfl"])
    nx = w["nx"]
    # a band of rows in the middle of the grid; the state is zero elsewhere (never read)
    rows = max(1, min(rows, w["ny"] - 2))
    r0 = max(1, w["ny"] // 2 - rows // 2)
    h = np.zeros((p.n, p.ncells))
    rng = np.random.default_rng(4)
    lo, hi = (r0 - 1) * nx, (r0 + rows + 1) * nx
    h[:, lo:hi] = rng.standard_normal((p.n, hi - lo))
    cells = np.arange(r0 * nx, (r0 + rows) * nx, dtype=np.int64)
    return p, h, cells


class OracleBand:
    """The oracle's FP64 step on a band of `rows` middle rows of the workload grid, split into
    one contiguous chunk of cells per host thread, with one thread pool kept for the whole
    timing (the C step releases the GIL, so the threads run in parallel)."""

    def __init__(self, rows: int, threads: int):
        import numpy as np
        self.p, self.h, cells = _oracle_setup(rows=rows)
        self.rows = rows
        self.threads = threads
        self.ncells = int(len(cells))
        self.chunks = [c for c in np.array_split(cells, threads) if len(c)]
        self.ex = cf.ThreadPoolExecutor(max_workers=threads)

    def step(self):
        list(self.ex.map(lambda c: self.p.step_cells(self.h, c), self.chunks))

    def updates_per_step(self) -> int:
        return self.ncells * self.p.n

    def close(self):
        self.ex.shutdown()


def oracle_sample(seconds_target: float, threads: int, rows: int = 256):
    """Time the oracle's step on a band of `rows` rows of the workload grid with `threads`
    host threads for about `seconds_target` seconds.  Returns (updates/s, sample)."""
    band = OracleBand(rows, threads)
    try:
        band.step()
        t = time.perf_counter()
        passes = 0
        while True:
            band.step()
            passes += 1
            el = time.perf_counter() - t
            if el >= seconds_target:
                break
    finally:
        band.close()
    ups = band.updates_per_step() * passes / el
    return ups, {"rows": rows, "cells_per_pass": band.ncells, "passes": passes, "seconds": el}


def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return None
    from oracle import march
    march.build()
    threads = os.cpu_count() or 1
    ups_probe, _ = oracle_sample(1.0, threads, rows=64)
    # size each bench step so that warmup + steps end in about a minute
    budget = 60.0
    per_step_updates = max(144 * 2048, ups_probe * budget / max(1, args.steps + args.warmup))
    rows = max(1, min(int(per_step_updates / (2048 * 144)), WORKLOAD["ny"] - 2))
    band = OracleBand(rows, threads)
    try:
        for _ in range(args.warmup):
            band.step()
        t = time.perf_counter()
        for _ in range(args.steps):
            band.step()
        el = time.perf_counter() - t
    finally:
        band.close()
    units = band.updates_per_step() * args.steps
    value = units / el
    sample = (f"{rows} grid rows ({band.ncells} cells x {band.p.n} velocities) of the 2048x2048 cavity per step, "
              f"oracle step evaluated cell by cell, one contiguous chunk per host thread, {threads} threads")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "lid-driven cavity 2048x2048, D2Q^h_144 (N=6 half-range Gauss-Hermite), "
                                   "Kn=0.05, lid u=0.01 (CPU oracle, FP64)", "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- main
def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", default=None, help="force the step kernel variant 'warps,loadpath'")
    ap.add_argument("--nx", type=int, default=None,
                    help="side of the cavity (default 2048); smaller sides are for profiling only")
    ap.add_argument("--transport", type=int, choices=[1, 2], default=1,
                    help="2: time the second-order variant of the workload instead (profiling)")
    ap.add_argument("--fp64-only", action="store_true",
                    help="time only the plain FP64 march of the workload (profiling of the FP64 step)")
    args = ap.parse_args(argv)
    if args.nx:
        WORKLOAD["nx"] = WORKLOAD["ny"] = args.nx
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        dist = Dist(backend="gloo") if _env_int("WORLD_SIZE", 1) > 1 else Dist()
        out = run_reference(args, dist)
        if out is not None:
            print(json.dumps(out), flush=True)
        dist.close()
        return 0
    dist = Dist()
    if args.fp64_only:
        import torch

        from paper_1308_0692_gb300 import lbm
        torch.cuda.set_device(dist.local_rank)
        vs = lbm.lbm_make_velocity_set(lbm.LBM_HALF_RANGE_GH, WORKLOAD["n_half"])
        print(json.dumps({"fp64": run_fp64_same_workload(vs, dist, args.transport), "nx": WORKLOAD["nx"],
                          "transport": args.transport}), flush=True)
        dist.close()
        return 0
    out = run_own(args, dist)
    if dist.rank == 0:
        if dist.world == 1 and not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            ups, sample = oracle_sample(12.0, threads, rows=256)
            ups1, sample1 = oracle_sample(4.0, 1, rows=16)
            out["cpu_baseline"] = {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle",
                                   "sample": f"oracle FP64 step on {sample['cells_per_pass']} cells "
                                             f"({sample['rows']} middle rows) of the 2048x2048 x 144 workload, "
                                             f"one contiguous chunk per thread, {sample['passes']} passes "
                                             f"in {sample['seconds']:.1f} s",
                                   "single_thread_value": ups1}
            if not args.no_extras:
                out["configs_time_to_residual"] = run_configs_time_to_residual()
        ttr = out.get("time_to_residual")
        if ttr:
            # the oracle marching the same 256 cavities to the same residual, extrapolated: the
            # FP64 march's step counts (equal to the oracle's, which the configurations'
            # cases check) times the updates per step at the oracle's rate measured on the
            # 128^2 cavity configurations (same grid and velocity set)
            cases = [c for c in out.get("configs_time_to_residual", []) if c["case"].startswith("cavity 128x128 D2Q^h_64")]
            rate = (sum(c["oracle"]["steps"] for c in cases) * 128 * 128 * 64 / sum(c["oracle"]["seconds"] for c in cases)
                    if cases else None)
            if rate:
                full = ttr["held_out_256"]
                upd = float(sum(full["fp64"]["steps"])) * 128 * 128 * 64
                full["oracle_extrapolated"] = {
                    "seconds": upd / rate, "updates_per_s": rate, "cores": os.cpu_count(),
                    "basis": "extrapolated: FP64 march steps x 128^2 x 64 updates at the oracle's rate measured "
                             "on the 128^2 D2Q^h_64 cavity configurations",
                    "vs_warm_dc": (upd / rate) / full["warm_dc"]["seconds"] if full.get("warm_dc") else None}
            out["ttr_summary"] = ttr_summary(ttr, rate)
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
