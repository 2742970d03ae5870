#!/usr/bin/env python
"""Benchmark of the FAS/fast-sweeping moment solver on GB300.

One step = one NMG V-cycle of Algorithm 2 in FP64 (FS smoothing on every level, residual, restriction,
coarse right-hand side, coarse-grid update), the mass correction and the residual norm, on the
lid-driven cavity 256x256, M = 10 (286 moments), BGK, Kn = 0.01, lid velocity 0.5, second-order
van Albada reconstruction, 6 levels (coarsest 8x8), s1 = s2 = 2, s3 = 4.

metric: cell-moment updates per second = 4 sweeps x cells x N_M per FS step, summed over the
FS steps of every level in the timed cycles (residual evaluations are not counted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload lid256|lid32|lid64|lid128|heat512|batch64|learned512]

The JSON line also reports the same cycle with the mixed-precision smoother (FP32 correction
sweeps inside FP64 defect correction) and, at N=1, the wall time to relative residual 1e-8 of
the plain, mixed and learned-start forms.  --workload learned512 prints the learned start's
line on the held-out 512x512, M=10 cavity; --workload batch64 the batched form's.

With --impl reference the CPU oracle (plain serial C) is timed on the host on a bounded sample
of the same workload.  Multi-GPU runs (torchrun) solve one independent replica per GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (nx, M, Kn, walls, model, Pr, order, slope, levels, description)
    "lid256": dict(nx=256, M=10, Kn=0.01, lid=0.5, heat=None, model=0, Pr=2 / 3, order=2, slope=2, levels=6,
                   desc="lid-driven cavity 256x256, M=10 (286 moments), BGK, Kn=0.01, lid 0.5, "
                        "2nd-order van Albada, 6-level FAS V-cycle (s1,s2,s3)=(2,2,4)"),
    "lid32": dict(nx=32, M=5, Kn=0.1, lid=0.1, heat=None, model=0, Pr=2 / 3, order=1, slope=0, levels=3,
                  desc="lid-driven cavity 32x32, M=5 (56 moments), BGK, Kn=0.1, lid 0.1, first order, "
                       "3-level FAS V-cycle (2,2,4)"),
    "lid64": dict(nx=64, M=10, Kn=0.01, lid=0.5, heat=None, model=0, Pr=2 / 3, order=2, slope=2, levels=4,
                  desc="lid-driven cavity 64x64, M=10 (286 moments), BGK, Kn=0.01, lid 0.5, "
                       "2nd-order van Albada, 4-level FAS V-cycle (2,2,4) (small profiling case)"),
    "lid128": dict(nx=128, M=10, Kn=0.01, lid=0.5, heat=None, model=0, Pr=2 / 3, order=2, slope=2, levels=5,
                   desc="lid-driven cavity 128x128, M=10 (286 moments), BGK, Kn=0.01, lid 0.5, "
                        "2nd-order van Albada, 5-level FAS V-cycle (2,2,4) (profiling case of the one-CTA sweep)"),
    "heat512": dict(nx=512, M=8, Kn=0.05, lid=0.0, heat=2.0, model=1, Pr=2 / 3, order=2, slope=2, levels=7,
                    desc="bottom-heated cavity 512x512, M=8 (165 moments), Shakhov Pr=2/3, Kn=0.05, "
                         "theta_bottom=2, 2nd-order van Albada, 7-level FAS V-cycle (2,2,4)"),
}


def batch64_instances(seed=0, count=64):
    """The batched cavity workload: per instance, in this order, Kn = 10^U(-2,0), lid velocity
    U(0.05,0.5), grid N in {64,128,256}, M in {5,8}; BGK, second order, coarsest grid 8x8; the
    local step is capped at 1/nu (Kn down to 0.01 with M = 5 makes the explicit collision step
    unstable on the coarse grids otherwise)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        Kn = float(10 ** rng.uniform(-2, 0))
        U = float(rng.uniform(0.05, 0.5))
        N = int(rng.choice([64, 128, 256]))
        M = int(rng.choice([5, 8]))
        levels = int(round(math.log2(N // 8))) + 1
        out.append(dict(nx=N, M=M, Kn=Kn, lid=U, heat=None, model=0, Pr=2 / 3, order=2, slope=2, levels=levels))
    return out


def batch_cycle_flops(inst):
    """Algorithmic FP64 flops of the FS updates of one batched V-cycle: 4 FS steps on every
    level, coarse levels with a right-hand side r."""
    fl = 0
    for w in inst:
        for l in range(w["levels"]):
            cells = (w["nx"] >> (w["levels"] - 1 - l)) ** 2
            fl += 4 * 4 * cells * flops_per_update(w["M"], 2, l < w["levels"] - 1)
    return fl


def batch64_measure(args, dev, world=1):
    """Batched V-cycles of the 64 cavities, timed: (record, kernel launches in the timed cycles)."""
    import torch

    from paper_2206_13164_gb300 import nrmg

    inst = batch64_instances()
    stream = torch.cuda.Stream(dev)
    groups = {}
    with torch.cuda.stream(stream):
        for w in inst:
            S = nrmg.Solver(w["nx"], w["nx"], w["M"], w["Kn"], walls_of(w), levels=w["levels"], model=0,
                            order=2, slope=2, dtnu=1.0, device=dev, stream=stream)
            groups.setdefault(w["M"], []).append((w, S))
        t0 = time.perf_counter()
        # one batch of all 64 problems (both M): one persistent launch per stage
        batches = {"all": nrmg.Batch([S for g in groups.values() for _, S in g])}
        t_build = time.perf_counter() - t0
        tune = {M: B.autotune(candidates=(2, 3, 4, 5, 6)) for M, B in batches.items()}
        for _ in range(args.warmup):
            for B in batches.values():
                B.fas_cycle()
        l0 = sum(B.launches for B in batches.values())
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for B in batches.values():
                B.fas_cycle()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    launches = sum(B.launches for B in batches.values()) - l0
    upd = sum(cycle_updates(w) for w in inst) * args.steps
    ms = max_over_ranks(ms, dev)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    ach = batch_cycle_flops(inst) * args.steps / (ms * 1e-3) / 1e12
    rec = {"value": replica_throughput(upd, world, ms * 1e-3), "unit": "cell-moment updates/s",
           "ms_per_step": ms / args.steps, "steps": args.steps,
           "instances": {str(M): len(g) for M, g in groups.items()},
           "batches": len(batches), "batch_build_s": t_build,
           "graph_replay": {str(M): B.graph for M, B in batches.items()},
           "autotune_ctas_per_sm": {str(M): B.tuned for M, B in batches.items()},
           "autotune_s": {str(M): t for M, t in tune.items()},
           "roofline": {"bound": "alu", "kernel": "fs_batch_kernel; achieved = algorithmic FS flops of the "
                                                 "batched cycle over the whole cycle's time (transfers included)",
                        "achieved": ach, "peak": fp64_peak(nsm), "unit": "TFLOP/s", "frac": ach / fp64_peak(nsm),
                        "peak_source": "derived FP64 pipe peak"}}
    del batches, groups
    torch.cuda.empty_cache()
    return rec, launches


def run_batch64(args):
    import torch

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    rec, launches = batch64_measure(args, dev, world)
    ms = rec["ms_per_step"] * args.steps
    if rank == 0:
        out = {"metric": "cell-moment updates/s", "value": rec["value"],
               "unit": "cell-moment updates/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "64 lid-driven cavities (seed 0): Kn 10^U(-2,0), lid U(0.05,0.5), N in "
                                      "{64,128,256}, M in {5,8}, BGK, 2nd order; one batch of all 64, one "
                                      "persistent FS launch per stage", "step": "one batched V-cycle of all 64 instances",
                          "instances": rec["instances"], "batch_build_s": rec["batch_build_s"],
                          "graph_replay": rec["graph_replay"], "autotune_ctas_per_sm": rec["autotune_ctas_per_sm"],
                          "autotune_s": rec["autotune_s"]},
               "roofline": rec["roofline"], "gpu_launches": launches}
        print(json.dumps(out), flush=True)


def nmom(M):
    return (M + 1) * (M + 2) * (M + 3) // 6


# DRAM bytes (read + write) per FS launch, averaged over the 11 FS launches of one V-cycle of
# the 256x256 M=10 workload, from one ncu capture of the current sweep kernels (one-CTA and
# two-CTA cluster sweeps); no figure for the other workloads
FS_TRAFFIC_BYTES_PER_LAUNCH = {"lid256": 393.3e6}

LEARNED_KEYS = ("status", "cycles", "final_cycles", "wasted_cycles", "rel_res", "rel_res_after_climb",
                "coarse_cycles", "t_coarse", "t_climb", "t_final", "t_total", "climb")


def net_flops(P, cin=19, hidden=64, cout=10):
    """Algorithmic flops of one forward pass over P pixels (real channel counts, 3x3 taps)."""
    return 2 * P * 9 * (cin * hidden + 2 * hidden * hidden + hidden * cout)


def net_forward_timing(net, H, W, reps=10, warmup=3):
    """CUDA-event time of the network's forward pass on one H x W image (inputs resident)."""
    import torch

    x = torch.randn((1, H, W, net.cin), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        net.forward(x)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        net.forward(x)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return ms, net_flops(H * W) / (ms * 1e-3) / 1e12


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (burst, cuBLAS)"
    except Exception:
        return 1900.0, "fallback 1.9 PFLOP/s bf16"


def mirror_symmetry_error(fields):
    """Largest deviation from the mirror symmetry about x = 1/2 of the bottom-heated cavity,
    relative to each field's largest magnitude: u1, s12, s13 and q1 change sign under the
    reflection, every other field is even."""
    import torch

    odd = torch.tensor([1 if k in (1, 6, 7, 11) else 0 for k in range(14)], device=fields.device)
    sign = 1.0 - 2.0 * odd.to(fields.dtype)
    mirrored = torch.flip(fields, dims=[1]) * sign
    dev = (fields - mirrored).abs().amax(dim=(0, 1))
    scale = fields.abs().amax(dim=(0, 1)).clamp_min(1e-300)
    keep = scale > 1e-12
    return float((dev[keep] / scale[keep]).max())


def learned_time_to_tol(w, tol=1e-8, grid=0, grid_mixed=None, dtnu=0.0, ref_fields=None):
    """Time to tol of the learned start on the workload (with and without the network, and with
    the mixed-precision smoother), or the reason it cannot run.  dtnu: the local-step cap of
    every solver context, the same as the plain solve's so that the cycles compare like for
    like; ref_fields: the plain FP64 solution, against which each form's fields are compared."""
    from paper_2206_13164_gb300 import learned

    if w["heat"] or not w["lid"]:
        return {"unavailable": "the learned start covers the lid-driven cavity family only"}
    if not os.path.exists(learned.WEIGHTS):
        return {"unavailable": "trained weights missing: " + learned.WEIGHTS}
    net = learned.Net.load(max_pixels=w["nx"] ** 2)
    out = {"start_grid": w["nx"] // 8, "weights": os.path.relpath(learned.WEIGHTS, ROOT), "solver_dtnu": dtnu}
    for key, nn, prec in (("no_net", None, 0), ("net", net, 0), ("net_mixed", net, 1)):
        ls = learned.LearnedSolve(w["nx"], w["M"], w["Kn"], w["lid"], start=w["nx"] // 8, net=nn, precision=prec,
                                  dtnu=dtnu)
        ls.set_grid(grid if prec == 0 or grid_mixed is None else grid_mixed)
        r = ls.run(tol=tol)
        out[key] = {k: r[k] for k in LEARNED_KEYS}
        if ref_fields is not None:
            out[key]["field_rel_err"] = learned.field_rel_errors(ls.target.fields(), ref_fields)
        del ls
    return out


def run_learned512(args):
    """The learned initial guess on the held-out 512x512, M = 10 cavity: seconds to relative
    residual 1e-8 (of the plain start's residual) against the plain FP64 solve."""
    import torch

    rank, local_rank, world = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    print(json.dumps(learned512_record(args, local_rank)), flush=True)


def learned512_record(args, local_rank=0):
    """The learned start's JSON record on the held-out 512x512 cavity."""
    import torch

    from paper_2206_13164_gb300 import learned

    N, M, Kn, U = 512, 10, 0.03, 0.35
    net = learned.Net.load(max_pixels=N * N)
    fwd_ms, fwd_tf = net_forward_timing(net, N, N, reps=max(args.steps, 3), warmup=max(args.warmup, 3))
    props = torch.cuda.get_device_properties(local_rank)
    try:
        gpu_id = "GPU-" + str(props.uuid)
    except Exception:
        gpu_id = str(local_rank)
    # sweep grid picked on a throwaway context of the same cavity (untimed)
    tuner = learned.lid_solver(N, M, Kn, U)
    tuner.fas_cycle()
    tune = tuner.autotune(candidates=(1, 2, 3), reps=1)
    grid = tuner.tuned
    del tuner
    with ClockSampler(gpu_id) as clk:
        ev = learned.evaluate(N, M, Kn, U, net, start=64, grid=grid, mixed=True)
    # the learned coarse-level correction on its held-out cavity (128x128, M = 8: the network
    # was trained on 64x64, M = 8 trajectories), plain cycle against the cycle with the
    # correction under the update-residual and the post-smoothing acceptance rules
    try:
        cnet = learned.Net.load(learned.CORR_WEIGHTS, max_pixels=128 * 128)
        corr = learned.evaluate_correction(128, 8, Kn, U, cnet, rules=(learned.ACCEPT_UPDATE,
                                                                      learned.ACCEPT_SMOOTHED))
        corr["weights"] = os.path.relpath(learned.CORR_WEIGHTS, ROOT)
        del cnet
    except Exception as e:  # the record of the learned start stands without it
        corr = {"error": f"{type(e).__name__}: {e}"}
    peak, src = bf16_peak()
    t_net, t_plain = ev["net"]["t_total"], ev["plain"]["t_total"]
    out = {"metric": "seconds to relative residual 1e-8 (learned start)", "value": t_net, "unit": "s",
           "n_gpus": 1, "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * t_net, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 solver; bf16 network with f32 accumulation",
           "data": "synthetic",
           "config": {"workload": f"held-out lid-driven cavity {N}x{N}, M={M}, BGK, Kn={Kn}, lid {U}, 2nd-order "
                                  "van Albada, 7 levels, local step capped at 1/nu; network trained on solver "
                                  "solutions at 64x64 and 128x128, M=8",
                      "weights": os.path.relpath(learned.WEIGHTS, ROOT), "meta": getattr(net, "meta", None),
                      "autotune_ctas_per_sm": grid, "autotune_s_per_cycle": tune},
           "plain": {k: ev["plain"][k] for k in ("status", "cycles", "rel_res", "t_total")},
           "no_net": {k: ev["no_net"][k] for k in LEARNED_KEYS + ("max_field_diff", "field_rel_err")},
           "net": {k: ev["net"][k] for k in LEARNED_KEYS + ("max_field_diff", "field_rel_err")},
           "plain_mixed": {k: ev["plain_mixed"][k] for k in ("status", "cycles", "rel_res", "t_total",
                                                             "max_field_diff", "field_rel_err")},
           "net_mixed": {k: ev["net_mixed"][k] for k in LEARNED_KEYS + ("max_field_diff", "field_rel_err")},
           "speedup_vs_plain": t_plain / t_net,
           "speedup_vs_plain_with_mixed_smoother": t_plain / ev["net_mixed"]["t_total"],
           "coarse_correction": corr,
           "roofline": {"bound": "tensor", "kernel": "network forward (4 conv3x3 launches, mma.sync BF16)",
                        "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s", "frac": fwd_tf / peak,
                        "traffic": None, "peak_source": src, "forward_ms": fwd_ms,
                        "flops_per_forward": net_flops(N * N)},
           "clocks": clk.summary()}
    return out


def walls_of(w):
    walls = [((0.0, 0.0, 0.0), 1.0, 1.0) for _ in range(4)]
    if w["lid"]:
        walls[2] = ((w["lid"], 0.0, 0.0), 1.0, 1.0)
    if w["heat"]:
        walls[0] = ((0.0, 0.0, 0.0), w["heat"], 1.0)
    return walls


def cycle_updates(w):
    """cell-moment updates of one V-cycle: 4 FS steps (s1+s2 or s3) on every level."""
    n = nmom(w["M"])
    tot = 0
    for l in range(w["levels"]):
        cells = (w["nx"] >> (w["levels"] - 1 - l)) ** 2
        steps = 4  # s1 + s2 = 2 + 2 on levels >= 1, s3 = 4 on level 0
        tot += steps * 4 * cells * n
    return tot


def flops_per_corr_update(M, order=2):
    """FP32 flops of one correction-sweep cell update (the linearized operator, no
    re-projection): at second order the 8 face states re-expanded into the cell basis
    (8 transforms) + 80 flops per moment (slopes, fluxes, collision); at first order the 4
    neighbours (4 transforms) + 60 flops per moment."""
    T = 6 * math.comb(M + 3, 4)
    return (8 * T + 80 * nmom(M)) if order == 2 else (4 * T + 60 * nmom(M))


def flops_per_update(M, order, has_r):
    """Algorithmic FP64 flops of one cell update: T per basis transform (2 flops x 3 directions x
    C(M+3,4) multiply-adds), 9 transforms + 80 flops per moment at second order (5 + 60 at first
    order), one more transform when the level has a right-hand side r."""
    T = 6 * math.comb(M + 3, 4)
    n = nmom(M)
    f = (9 * T + 80 * n) if order == 2 else (5 * T + 60 * n)
    return f + (T if has_r else 0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value, device=None):
    """Largest value over the ranks of the default process group (the value itself when there
    is none): the job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` independent replicas: all ranks' units / the slowest time."""
    return units_per_rank * world / seconds


def cpu_oracle_sample(w, level_shift: int, sweeps: int = 1, threads: int = 0):
    """Time the CPU oracle (as it stands: serial, or its OpenMP mode with `threads` > 1) on
    directional sweeps D1 of one level of the workload.  Returns (cell-moment updates/s,
    seconds, description)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle

    oracle.build()
    c = oracle.OrConfig()
    c.nx = c.ny = w["nx"]
    c.lx = c.ly = 1.0
    c.levels = w["levels"]
    c.M, c.Kn, c.model, c.Pr, c.omega, c.beta = w["M"], w["Kn"], w["model"], w["Pr"], 0.81, 1.0
    c.order, c.slope, c.cfl = w["order"], w["slope"], 0.9
    c.s1, c.s2, c.s3, c.gamma = 2, 2, 4, 1
    for k, (u, th, chi) in enumerate(walls_of(w)):
        for d in range(3):
            c.wall_u[k][d] = u[d]
        c.wall_theta[k], c.wall_chi[k] = th, chi
    S = oracle.Solver(c)
    if threads > 1:
        S.set_threads(threads)
    lev = w["levels"] - 1 - level_shift
    ny, nx = S.shape(lev)
    t0 = time.perf_counter()
    for _ in range(sweeps):
        S.sweep(lev, 1)
    dt = time.perf_counter() - t0
    upd = sweeps * nx * ny * nmom(w["M"])
    mode = f"oracle OpenMP mode, {threads} threads" if threads > 1 else "serial oracle"
    return upd / dt, dt, f"{sweeps} directional sweep(s) D1 over the {nx}x{ny} level of the workload " \
                         f"({nx * ny} cell updates), {mode}"


def run_reference(args, w):
    rank, _, world = dist_env()
    if rank != 0:
        return
    # each step: one D1 sweep of the level cpu_baseline times (the finest up to 256x256)
    shift = cpu_sample_level_shift(w)
    for _ in range(args.warmup):
        cpu_oracle_sample(w, shift)
    times, rates, desc = [], [], ""
    for _ in range(args.steps):
        r, dt, desc = cpu_oracle_sample(w, shift)
        times.append(dt)
        rates.append(r)
    tot_upd = sum(r * t for r, t in zip(rates, times))
    value = tot_upd / sum(times)
    out = {
        "impl": "reference", "metric": "cell-moment updates/s", "value": value, "unit": "cell-moment updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "sample": desc},
        "cpu_baseline": {"value": value, "unit": "cell-moment updates/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "cell-moment updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def workload_summary(w, args, dev, steps=3):
    """A workload's plain V-cycle (updates/s, the FS kernel's roofline), its mixed-precision
    cycle and both forms' seconds to 1e-8 with their field errors."""
    import torch

    from paper_2206_13164_gb300 import nrmg

    props = torch.cuda.get_device_properties(dev)

    def make(prec=0, dtnu=0.0):
        return nrmg.Solver(w["nx"], w["nx"], w["M"], w["Kn"], walls_of(w), levels=w["levels"], model=w["model"],
                           Pr=w["Pr"], order=w["order"], slope=w["slope"], precision=prec, dtnu=dtnu, device=dev)

    S = make()
    for _ in range(args.warmup):
        S.fas_cycle()
    tune = S.autotune(candidates=(1, 2, 3, 4), reps=1, clusters=CLUSTER_CANDIDATES)
    cluster_cells = S.cluster_cells
    S.set_profiling(True)
    S.fs_profile()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(S.stream)
    for _ in range(steps):
        S.fas_cycle()
    e1.record(S.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    fs_ms, fs_n, u0, u1 = S.fs_profile()
    S.set_profiling(False)
    grid = S.tuned
    del S
    torch.cuda.empty_cache()
    fl = u0 * flops_per_update(w["M"], w["order"], False) + u1 * flops_per_update(w["M"], w["order"], True)
    ach = fl / (fs_ms * 1e-3) / 1e12
    peak = fp64_peak(props.multi_processor_count)
    rec = {"workload": w["desc"], "value": cycle_updates(w) * steps / (ms * 1e-3), "unit": "cell-moment updates/s",
           "ms_per_step": ms / steps, "steps": steps, "autotune_ctas_per_sm": grid, "autotune_s_per_cycle": tune,
           "two_cta_cluster_sweeps_max_cells": cluster_cells,
           "roofline": {"bound": "alu", "kernel": "FP64 FS sweeps of all levels (fs_kernel and fs_cluster_kernel)",
                        "achieved": ach,
                        "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "fs_ms_per_step": fs_ms / steps,
                        "peak_source": "derived FP64 pipe peak"}}
    mixed, mgrid = mixed_cycle_timing(w, make, args, dev, props, 1, lambda: None, steps=steps)
    rec["mixed"] = mixed
    rec["time_to_tol"] = time_to_tol(w, make, dev, grid, mgrid, learned_forms=False)
    return rec


def extra_workloads(args, dev):
    """The other configurations, each in its own sub-object: the bottom-heated 512x512 Shakhov
    cavity (plain and mixed, mirror symmetry), the batch of 64 cavities, and the learned start
    on the held-out 512x512 cavity.  A failure is reported in place of that record."""
    import torch

    out = {}
    for name in ("heat512", "batch64", "learned512"):
        t0 = time.perf_counter()
        try:
            if name == "heat512":
                out[name] = workload_summary(WORKLOADS["heat512"], args, dev)
            elif name == "batch64":
                bargs = argparse.Namespace(steps=min(args.steps, 3), warmup=min(args.warmup, 2))
                rec, launches = batch64_measure(bargs, dev)
                rec["gpu_launches"] = launches
                rec["workload"] = ("64 lid-driven cavities (seed 0): Kn 10^U(-2,0), lid U(0.05,0.5), N in "
                                   "{64,128,256}, M in {5,8}, BGK, 2nd order, local step capped at 1/nu; one "
                                   "persistent FS launch per stage for all 64")
                out[name] = rec
            else:
                out[name] = learned512_record(args)
        except Exception as e:  # report, keep the main line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


# level sizes (cells) up to which the FP64 sweeps may run on two-CTA clusters, tried by the
# autotuner after the grid
CLUSTER_CANDIDATES = (0, 4096, 16384)


def fp64_peak(nsm):
    """Derived FP64 pipe peak in TFLOP/s: SMs x 2 DFMA/clk x 2 flops x 2070 MHz."""
    return nsm * 2 * 2 * 2.07e9 / 1e12


# executed FP64 flops per cell update of the FS kernel (2 x DFMA + DADD + DMUL thread
# instructions per update, ncu, finest-level launch of the 64x64 M=10 second-order cavity):
# the algorithmic count (flops_per_update) is 1.22x this
FS_EXECUTED_FLOPS = {10: 50340}


def mixed_cycle_timing(w, make, args, dev, props, world, barrier, steps=None):
    """The V-cycle with the mixed-precision smoother: ms per cycle, updates/s and the FP32
    correction sweep's roofline.  Returns (record, tuned grid)."""
    import torch

    steps = steps or args.steps
    S2 = make(1)
    for _ in range(args.warmup):
        S2.fas_cycle()
    tune_mixed = S2.autotune(reps=1)
    S2.set_profiling(True)
    S2.fs_profile()
    barrier()
    torch.cuda.synchronize(dev)
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record(S2.stream)
    for _ in range(steps):
        S2.fas_cycle()
    m1.record(S2.stream)
    torch.cuda.synchronize(dev)
    mms = m0.elapsed_time(m1)
    mlev = S2.fs_profile_levels()
    cms, cn, cu0, cu1 = S2.fs_profile()
    S2.set_profiling(False)
    corr_fl = (cu0 + cu1) * flops_per_corr_update(w["M"], w["order"])
    fp32_peak = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    rec = {"value": cycle_updates(w) * steps * world / (mms * 1e-3), "unit": "cell-moment updates/s",
           "ms_per_step": mms / steps, "steps": steps, "dtype": "f32 correction sweeps + f64 defect/transfers",
           "roofline": {"bound": "alu", "kernel": "fs_corr_kernel (FP32 correction sweeps, FS timings "
                                                 "of all levels; the coarsest level stays FP64)",
                        "achieved": corr_fl / (cms * 1e-3) / 1e12 if cms > 0 else None,
                        "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": (corr_fl / (cms * 1e-3) / 1e12 / fp32_peak) if cms > 0 else None,
                        "peak_source": "derived: SMs x 128 FFMA/clk x 2 flops x 2070 MHz",
                        "flops_per_cell_update": flops_per_corr_update(w["M"], w["order"]),
                        "sweep_ms_per_step": cms / steps,
                        "sweep_ms_per_step_by_level": [round(m / steps, 3) for m, _ in mlev]},
           "autotune_ctas_per_sm": S2.tuned, "autotune_s_per_cycle": tune_mixed}
    grid = S2.tuned
    del S2
    torch.cuda.empty_cache()
    return rec, grid


def time_to_tol(w, make, dev, grid, grid_mixed, learned_forms=True, tol=1e-8):
    """Seconds and cycles to relative residual tol from the global Maxwellian: plain FP64,
    mixed precision and (lid cavities) the learned start, every form with the same local
    step; each form's fields against the plain FP64 solution (per-field max relative error),
    and the mirror asymmetry of the bottom-heated cavity."""
    import torch

    from paper_2206_13164_gb300 import learned

    ttt = {"tol": tol, "solver_dtnu": 0.0}
    ref = None
    for prec, key in ((0, "plain_fp64"), (1, "mixed")):
        S3 = make(prec)
        S3.set_grid(grid if prec == 0 or grid_mixed is None else grid_mixed)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st, cyc, rr = S3.solve(tol, 400)
        torch.cuda.synchronize(dev)
        ttt[key] = {"seconds": time.perf_counter() - t0, "cycles": cyc, "rel_residual": rr, "status": int(st)}
        f = S3.fields()
        if prec == 0:
            ref = f
        else:
            ttt[key]["field_rel_err_vs_plain_fp64"] = learned.field_rel_errors(f, ref)
            ttt[key]["fell_back_to_fp64"] = bool(S3.mixed_fallback())
        if w["heat"]:
            ttt[key]["mirror_symmetry_rel_err"] = mirror_symmetry_error(f)
        del S3, f
        torch.cuda.empty_cache()
    ttt["mixed_over_plain_time"] = ttt["mixed"]["seconds"] / ttt["plain_fp64"]["seconds"]
    if learned_forms:
        ttt["learned"] = learned_time_to_tol(w, grid=grid, grid_mixed=grid_mixed, dtnu=0.0, ref_fields=ref)
        if "net" in ttt["learned"]:
            ttt["learned_over_plain_time"] = ttt["learned"]["net"]["t_total"] / ttt["plain_fp64"]["seconds"]
            ttt["learned_mixed_over_plain_time"] = (ttt["learned"]["net_mixed"]["t_total"]
                                                    / ttt["plain_fp64"]["seconds"])
    return ttt


def cpu_sample_level_shift(w):
    """The level the CPU oracle is timed on: the finest up to 256x256, else the next one."""
    return 0 if w["nx"] <= 256 else 1


def cpu_baseline(w):
    """The oracle as it stands on the host: serial (1 core), and its OpenMP mode on all cores,
    each on one D1 sweep of the same level of the workload."""
    shift = cpu_sample_level_shift(w)
    r, dt, desc = cpu_oracle_sample(w, shift)
    out = {"value": r, "unit": "cell-moment updates/s", "cores": 1, "kind": "oracle",
           "sample": desc + f" ({dt:.1f} s)"}
    ncores = os.cpu_count() or 1
    if ncores > 1:
        ro, dto, desco = cpu_oracle_sample(w, shift, threads=ncores)
        out["openmp"] = {"value": ro, "unit": "cell-moment updates/s", "cores": ncores, "kind": "oracle",
                         "sample": desco + f" ({dto:.1f} s)", "speedup_over_serial": ro / r}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lid256", choices=sorted(WORKLOADS) + ["batch64", "learned512"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-tol", action="store_true", help="skip the two solves to 1e-8")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision cycle timing")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-start solves to 1e-8")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (heated 512x512, batch of 64, held-out learned 512x512)")
    args = ap.parse_args()
    if args.workload == "learned512":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the learned start has no CPU counterpart"}))
            return
        run_learned512(args)
        return
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU sample"}))
            return
        run_batch64(args)
        return
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist

    from paper_2206_13164_gb300 import nrmg

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def make(prec=0, dtnu=0.0):
        return nrmg.Solver(w["nx"], w["nx"], w["M"], w["Kn"], walls_of(w), levels=w["levels"], model=w["model"],
                           Pr=w["Pr"], order=w["order"], slope=w["slope"], precision=prec, dtnu=dtnu, device=dev)

    S = make()
    stream = S.stream
    fp64_peak_meas = nrmg.peak_fma(0, 2048, stream)
    for _ in range(args.warmup):
        S.fas_cycle()
    # sweep grid: persistent CTAs per SM picked by timing one cycle each (untimed warm-up)
    tune_plain = S.autotune(candidates=(1, 2, 3, 4), reps=1, clusters=CLUSTER_CANDIDATES)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(props.uuid)
    except Exception:
        gpu_id = str(local_rank)
    S.set_profiling(True)
    S.fs_profile()  # reset
    S.residual_profile()
    l0 = S.launches
    with ClockSampler(gpu_id) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rel = None
        for _ in range(args.steps):
            rel = S.fas_cycle()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = e0.elapsed_time(e1)
    launches = S.launches - l0
    per_level = S.fs_profile_levels()
    fs_ms, fs_n, u0, u1 = S.fs_profile()
    res_ms, res_n, rc0, rc1 = S.residual_profile()
    S.set_profiling(False)
    ms = max_over_ranks(ms, dev)
    upd = cycle_updates(w) * args.steps
    value = replica_throughput(upd, world, ms * 1e-3)

    # end to end through the public C ABI with HOST buffers: every step copies the state from
    # pinned host memory into the solver (nrmg_set_state_host), runs one cycle and reads the
    # state back (nrmg_get_state_host); the copies are inside the timed region
    P, F = S.get_state()
    hP = torch.empty(P.shape, dtype=P.dtype, pin_memory=True)
    hF = torch.empty(F.shape, dtype=F.dtype, pin_memory=True)
    hP.copy_(P)
    hF.copy_(F)
    oP = torch.empty(P.shape, dtype=P.dtype, pin_memory=True)
    oF = torch.empty(F.shape, dtype=F.dtype, pin_memory=True)
    del P, F
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S.set_state_host(hP, hF)
        S.fas_cycle()
        S.get_state_host(oP, oF)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_value = replica_throughput(cycle_updates(w) * e2e_steps, world, e2e_s)
    bytes_state = (hP.numel() + hF.numel()) * 8

    # mixed precision: FP32 correction sweeps inside FP64 defect correction, same cycle
    mixed, mixed_grid = None, 0
    if not args.no_mixed:
        mixed, mixed_grid = mixed_cycle_timing(w, make, args, dev, props, world, barrier)

    # time to relative residual 1e-8 from the global Maxwellian, plain FP64 vs mixed vs learned
    ttt = None
    if world == 1 and not args.no_time_to_tol:
        ttt = time_to_tol(w, make, dev, S.tuned, mixed_grid if mixed else None,
                          learned_forms=not args.no_learned)

    # roofline of the dominant kernel (the persistent FS sweep kernel, all levels)
    fl = u0 * flops_per_update(w["M"], w["order"], False) + u1 * flops_per_update(w["M"], w["order"], True)
    achieved = fl / (fs_ms * 1e-3) / 1e12 if fs_ms > 0 else None
    nsm = props.multi_processor_count
    peak_nominal = fp64_peak(nsm)
    res_fl = rc0 * flops_per_update(w["M"], w["order"], False) + rc1 * flops_per_update(w["M"], w["order"], True)
    res_ach = res_fl / (res_ms * 1e-3) / 1e12 if res_ms > 0 else None
    clocks = clk.summary()
    plain_grid = S.tuned
    plain_cluster = {"max_cells": S.cluster_cells, "capacity": S.cluster_capacity,
                     "s_per_cycle": {str(k): v for k, v in S.cluster_times.items()}}
    del S
    torch.cuda.empty_cache()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(w)
        out = {
            "metric": "cell-moment updates/s", "value": value, "unit": "cell-moment updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "step": "one FAS V-cycle + mass correction + residual norm",
                       "cell_moment_updates_per_step": cycle_updates(w),
                       "l2": "inputs larger than L2 (finest-level coefficient array alone is "
                             f"{w['nx'] ** 2 * ((nmom(w['M']) + 3) // 4 * 4) * 8 / 1e6:.0f} MB)",
                       "parallelism": f"replicas x{world}", "rel_residual_after": rel,
                       "autotune_ctas_per_sm": plain_grid, "autotune_s_per_cycle": tune_plain,
                       "two_cta_cluster_sweeps": plain_cluster},
            "roofline": {"bound": "alu", "kernel": "FP64 FS sweeps of all levels (fs_kernel, one CTA per update, "
                                                  "and fs_cluster_kernel, two-CTA clusters on the small levels)",
                         "achieved": achieved, "peak": peak_nominal, "unit": "TFLOP/s",
                         "frac": (achieved / peak_nominal) if achieved else None,
                         "traffic": FS_TRAFFIC_BYTES_PER_LAUNCH.get(args.workload),
                         "traffic_note": "bytes per FS launch, average over one V-cycle's launches "
                                         "(ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "peak_source": "derived: SMs x 2 DFMA/clk x 2 flops x 2070 MHz (FP64 pipe)",
                         "fp64_fma_measured_tflops": fp64_peak_meas / 1e12,
                         "fs_ms_per_step": fs_ms / args.steps, "fs_launches": fs_n,
                         "fs_ms_per_step_by_level": [round(m / args.steps, 3) for m, _ in per_level],
                         "fs_us_per_cell_update_by_level": [round(1e3 * m / u, 3) if u else None
                                                            for m, u in per_level],
                         "flops_per_cell_update": flops_per_update(w["M"], w["order"], False),
                         "executed_flops_per_cell_update_ncu": FS_EXECUTED_FLOPS.get(w["M"])},
            "residual_roofline": {"bound": "alu", "kernel": "residual_kernel (norms, defects, coarse right-hand "
                                                            "sides of the timed cycles)",
                                  "achieved": res_ach, "peak": peak_nominal, "unit": "TFLOP/s",
                                  "frac": (res_ach / peak_nominal) if res_ach else None,
                                  "ms_per_step": res_ms / args.steps, "launches": res_n,
                                  "cells": rc0 + rc1, "flops_per_cell": flops_per_update(w["M"], w["order"], False),
                                  "peak_source": "derived FP64 pipe peak, as above"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "cell-moment updates/s", "h2d_bytes_per_step": bytes_state,
                    "d2h_bytes_per_step": bytes_state, "steps": e2e_steps,
                    "path": "nrmg_set_state_host (pinned host -> device) + nrmg_fas_cycle + nrmg_get_state_host "
                            "(device -> pinned host), one C ABI call each"},
            "gpu_launches": launches,
            "clocks": clocks,
            "mixed": mixed,
            "time_to_tol": ttt,
        }
        if world == 1 and not args.no_extras and args.workload == "lid256":
            out["extra_workloads"] = extra_workloads(args, dev)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
