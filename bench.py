#!/usr/bin/env python3
"""Benchmark of the GB300 Parareal path for the Cahn-Hilliard equation.

Workload (default): 1D nonlinear Parareal NPA-I (Newton fine solver, tolerance 1e-12), FP64
states and residuals, M = 1024 interior nodes, eps = 0.02, T = 1, N = 64 slices, 200 fine steps
per slice, one plain coarse step per slice, batch of 256 seeded initial conditions
u0 = 0.1 U(-1,1) (seeds 0..255), all slices of all problems in one persistent launch per
iteration, each iteration replayed as a CUDA graph.

A step is one pass of the whole path over the batch: the coarse initial sweep, one fine sweep
over every slice of every problem, and the sequential coarse sweep with the Parareal correction
and the convergence norms (ch_parareal_run with max_iters = 1). `value` is fine grid-point
steps per second (one fine time step applied to one interior node), whole job.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Parareal time-to-1e-8 (learned vs plain G) & grid-pt-steps/s; % HBM roofline"

WORKLOADS = {
    "c2": dict(name="1D nonlinear Parareal NPA-I M=1024 eps=0.02 T=1 N=64 J=200 newton_tol=1e-12 batch=256",
               n=1024, eps=0.02, T=1.0, N=64, J=200, batch=256, variant="NPA-I", newton_tol=1e-12,
               amp=0.1, precision=1, ttol=True),
    # profiling case of the same kernels: c2's batch, grid and slices, 10 fine steps per slice
    "c2-profile": dict(name="1D NPA-I M=1024 eps=0.02 N=64 J=10 (dt as c2) batch=256, profiling case",
                       n=1024, eps=0.02, T=0.05, N=64, J=10, batch=256, variant="NPA-I", newton_tol=1e-12,
                       amp=0.1, precision=1, ttol=False),
    "c3": dict(name="2D nonlinear Parareal NPA-I 256x256 grid (n=255) eps=0.01 T=0.5 N=32 J=100 u0=0.05*N(0,1) seed 1",
               dim=2, n=255, eps=0.01, T=0.5, N=32, J=100, batch=1, variant="NPA-I", newton_tol=1e-12,
               amp=0.05, kind="normal", seed0=1, precision=1, ttol=True),
    # profiling case of the 2D kernels: c3's grid, slices and step size, 10 fine steps per slice
    "c3-profile": dict(name="2D NPA-I 256x256 (n=255) eps=0.01 N=32 J=10 (dt as c3), profiling case",
                       dim=2, n=255, eps=0.01, T=0.05, N=32, J=10, batch=1, variant="NPA-I", newton_tol=1e-12,
                       amp=0.05, kind="normal", seed0=1, precision=1, ttol=False),
    "c4": dict(name="2D nonlinear Parareal NPA-I 512x512 grid (n=511) eps=0.01 T=2 N=64 J=100 u0=0.05*N(0,1) seed 2000",
               dim=2, n=511, eps=0.01, T=2.0, N=64, J=100, batch=1, variant="NPA-I", newton_tol=1e-12,
               amp=0.05, kind="normal", seed0=2000, precision=1, ttol=False),
    # profiling case of the 2D kernels at the 512 x 512 grid: c4's grid, slices and step size,
    # 2 fine steps per slice
    "c4-profile": dict(name="2D NPA-I 512x512 (n=511) eps=0.01 N=64 J=2 (dt as c4), profiling case",
                       dim=2, n=511, eps=0.01, T=0.04, N=64, J=2, batch=1, variant="NPA-I", newton_tol=1e-12,
                       amp=0.05, kind="normal", seed0=2000, precision=1, ttol=False),
    "c1": dict(name="1D linear Parareal PA-I M=128 eps=0.05 T=0.1 N=16 dt=1e-5 batch=1",
               n=128, eps=0.05, T=0.1, N=16, J=625, batch=1, variant="PA-I", newton_tol=1e-12,
               amp=0.1, precision=0, ttol=True),
    # c1 with the fine LIN1 steps as FP32 solves refined against their FP64 residual (to the FP64
    # rounding level; the coarse steps stay FP64 solves)
    "c1-mixed": dict(name="1D linear Parareal PA-I M=128 eps=0.05 T=0.1 N=16 dt=1e-5 batch=1, fine solves FP32 "
                          "refined in FP64",
                     n=128, eps=0.05, T=0.1, N=16, J=625, batch=1, variant="PA-I", newton_tol=1e-12,
                     amp=0.1, precision=1, ttol=True),
    # the Neumann-Neumann fine solver of Section 4.6 on the paper's grid for it (h = 1/128, 8 equal
    # subdomains, theta = 1/4, interface tolerance 1e-10), PA-I with eps = 0.0725, J = 200
    "c1-nn": dict(name="1D PA-I with the Neumann-Neumann fine solver, n=127 (h=1/128) eps=0.0725 T=0.1 N=16 J=200 "
                       "8 subdomains theta=1/4 tol=1e-10 batch=1",
                  n=127, eps=0.0725, T=0.1, N=16, J=200, batch=1, variant="PA-I", newton_tol=1e-12,
                  amp=0.1, precision=0, ttol=True, nn=(8, 0.25, 1e-10, 200)),
}
FINE_OF = {"PA-I": "lin1", "PA-II": "lin2", "PA-III": "lin2", "NPA-I": "nl", "NPA-II": "nl"}
COARSE_OF = {"PA-I": "lin1", "PA-II": "lin2", "PA-III": "lin1", "NPA-I": "lin1", "NPA-II": "nl"}

# FP64 arithmetic per grid point (FMA = 2 flops) that the nonlinear scheme needs in full
# precision: the right-hand side (I - dt D_h) u^n once per step, and per Newton iteration the
# residual H(Y) = Y - Yhat + D_h(eps^2 dt D_h Y - dt Y^3) and the update Y -= dY.
FP64_FLOPS_RHS = 5
FP64_FLOPS_NEWTON = 15
# A step of a linear scheme (Eq. 2.4 / 2.5) in FP64: the right-hand side and the assembly of the
# pentadiagonal rows (about 20 flops per point) and its banded LU solve (about 25).
FP64_FLOPS_LINEAR_STEP = 45
# The Neumann-Neumann fine solver: per iteration and node a Dirichlet and a Neumann block
# elimination with 2x2 blocks (about 30 flops each), per step the final Dirichlet solve and the
# right-hand side (about 35).
FP64_FLOPS_NN_ITER = 60
FP64_FLOPS_NN_STEP = 35
# GB300 FP64: 152 SMs x 2 FP64 FMA lanes x 2 flops x 2.07 GHz (maximum SM clock).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# DRAM bytes (read + write) of one 1D fine-sweep launch at c2's batch and slices (256 x 64 units,
# all slices iterating), from a one-launch ncu capture of dram__bytes_read.sum +
# dram__bytes_write.sum on the current kernel; independent of the fine steps per slice (the slice
# state stays in registers). None when the kernel has changed since the capture.
FINE_SWEEP_1D_TRAFFIC = {(1024, 256, 64): 218.5e6}


# 2D fine sweep, algorithmic DRAM/L2 bytes per grid point and unit, each array read or written
# once per phase (the executions fuse some phases; the count is the algorithm's, not a kernel's).
# CG iteration (5 phases): u to physical space (read u, write t: 8), times
# dt (wc - wbar) (read t, wc, write t2: 12), back to sine space (8), w = M u + That with (w, u)
# and (r, u) (read t, u, r, write w: 16), update of p, s, x, r, u (read u, w, p, s, x, r, write
# p, s, x, r, u: 44). Newton iteration: z = c1 lap Y - dt g (read Y, write z FP64: 16), H and
# weights (read Y, Yhat, z, write H, wc: 32), H to sine space and CG start (8 + 16: write x, r, u), correction to
# physical space (8), FP64 update (read d, Y, write Y: 20). Step: right-hand side (16) and
# predictor (read Y, Yprev, write both: 32).
BYTES_CG_2D = 8 + 12 + 8 + 16 + 44
BYTES_NEWTON_2D = 16 + 32 + 8 + 16 + 8 + 20
BYTES_STEP_2D = 16 + 32
# DRAM traffic of the 2D fine sweep on the 512 x 512 grid, from a one-pass ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum over the kernels of a batched propagation of 64
# slices (current kernels): the first two CG iterations of all 64 units move 565 + 1099 MB of DRAM
# traffic against 735 + 1471 MB of algorithmic bytes (the L2 keeps part of each phase's output for
# the next). The fine sweep's traffic per launch is reported as that ratio times its algorithmic
# bytes.
TRAFFIC_2D_OVER_ALGORITHMIC = {511: 0.754}


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (the slowest rank sets a weak-scaling time)."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def u0_batch(w, rank):
    import ch_inputs
    import numpy as np
    base = rank * w["batch"] + w.get("seed0", 0)
    dim = w.get("dim", 1)
    return np.stack([ch_inputs.initial_condition(dim, w["n"], base + b, kind=w.get("kind", "uniform"), amp=w["amp"])
                     for b in range(w["batch"])])


# ------------------------------------------------------------------------ clocks sampling


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------ CPU oracle leg


ORACLE_2D_STEPS = 2  # 2D sample: this many fine steps of one slice per process (sparse LU per step)
ORACLE_NN_STEPS = 20  # Neumann-Neumann sample: this many fine steps of one slice per process


def _oracle_step(args):
    """1D: one step of the workload (coarse sweep + one fine sweep + correction) for one problem.
    2D: ORACLE_2D_STEPS fine steps of one slice (a full 2D step takes hours with sparse LU)."""
    w, u0 = args
    t = time.perf_counter()
    if w.get("nn"):
        from oracle import nn1d
        nn1d.nn_propagate(w["n"], w["eps"], w["T"] / w["N"] / w["J"], ORACLE_NN_STEPS, u0, *w["nn"])
    elif w.get("dim", 1) == 2:
        from oracle import oracle2d as o2
        p = o2.Params(n=w["n"], eps=w["eps"], T=w["T"], N=w["N"], J=w["J"], newton_tol=w["newton_tol"],
                      solver="pcg")
        o2.propagate(p, FINE_OF[w["variant"]], w["T"] / w["N"] / w["J"], ORACLE_2D_STEPS, u0)
    else:
        from oracle import oracle1d as o
        p = o.Params(n=w["n"], eps=w["eps"], T=w["T"], N=w["N"], J=w["J"], fine=FINE_OF[w["variant"]],
                     coarse=COARSE_OF[w["variant"]], newton_tol=w["newton_tol"], max_iters=1)
        o.parareal(p, u0)
    return time.perf_counter() - t


def _serial_fine(args):
    """The sequential fine solve F^N(u0) of one problem (the classical serial method, Section 2),
    on one core; 2D: ORACLE_2D_STEPS fine steps."""
    w, u0 = args
    t = time.perf_counter()
    if w.get("dim", 1) == 2:
        from oracle import oracle2d as o2
        p = o2.Params(n=w["n"], eps=w["eps"], T=w["T"], N=w["N"], J=w["J"], newton_tol=w["newton_tol"],
                      solver="pcg")
        o2.propagate(p, FINE_OF[w["variant"]], w["T"] / w["N"] / w["J"], ORACLE_2D_STEPS, u0)
    elif w.get("nn"):
        from oracle import nn1d
        nn1d.nn_propagate(w["n"], w["eps"], w["T"] / w["N"] / w["J"], ORACLE_NN_STEPS, u0, *w["nn"])
    else:
        from oracle import oracle1d as o
        p = o.Params(n=w["n"], eps=w["eps"], T=w["T"], N=w["N"], J=w["J"], fine=FINE_OF[w["variant"]],
                     coarse=COARSE_OF[w["variant"]], newton_tol=w["newton_tol"])
        o.fine_solution(p, u0)
    return time.perf_counter() - t


def _sample_points(w):
    """Fine grid-point steps of one oracle sample (one problem's step of the workload in 1D; a few
    fine steps of one slice in 2D and for the Neumann-Neumann solver)."""
    if w.get("nn"):
        return ORACLE_NN_STEPS * w["n"]
    if w.get("dim", 1) == 2:
        return ORACLE_2D_STEPS * w["n"] ** 2
    return w["N"] * w["J"] * w["n"]


def cpu_model():
    """The host CPU's model name (x86: 'model name'; Arm: implementer / part of /proc/cpuinfo)."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        info = []
    for key in ("model name", "Model name"):
        for ln in info:
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    impl = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU implementer")]
    part = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU part")]
    if impl and part:
        return f"{platform.machine()} implementer {impl[0]} part {part[0]}"
    return platform.machine() or "unknown"


def cpu_oracle(w, problems, u0s, steps=1):
    """Times the oracle on `problems` problems, one single-threaded process per problem (spawned):
    the all-core sample when `problems` is the core count."""
    import oracle
    oracle.build()
    u0s = [u0s[b % len(u0s)] for b in range(problems)]  # a batch smaller than the sample repeats
    times = []
    with oracle.spawn_pool(problems) as pool:
        for _ in range(steps):
            t = time.perf_counter()
            pool.map(_oracle_step, [(w, u0s[b]) for b in range(problems)])
            times.append(time.perf_counter() - t)
    return problems * _sample_points(w), times


def cpu_serial_fine(w, u0):
    """The 1-core sequential fine solve of one problem, timed in a spawned process; returns
    (grid-point steps, seconds)."""
    import oracle
    oracle.build()
    with oracle.spawn_pool(1) as pool:
        secs = pool.map(_serial_fine, [(w, u0)])[0]
    if w.get("dim", 1) == 2 or w.get("nn"):
        pts = _sample_points(w)
    else:
        pts = w["N"] * w["J"] * w["n"]
    return pts, secs


def cpu_sample_size():
    """All host cores, one oracle process per core."""
    return max(1, os.cpu_count() or 1)


def cpu_baseline(w, u0, steps=1):
    """The CPU oracle as it stands on this host: the all-core sample (one problem per core) and
    the 1-core sequential fine solve (the serial method Parareal is measured against)."""
    problems = cpu_sample_size()
    pts, times = cpu_oracle(w, problems, u0, steps=steps)
    spts, ssecs = cpu_serial_fine(w, u0[0])
    what = (f"{problems} processes x {ORACLE_NN_STEPS} Neumann-Neumann fine steps of one slice (dense subdomain "
            "solves)" if w.get("nn") else
            f"{problems} processes x {ORACLE_2D_STEPS} fine steps of one slice (sparse solves by library CG)"
            if w.get("dim", 1) == 2 else
            f"{problems} problems of the batch (repeated when the batch is smaller), one process per core, each "
            "one step of the workload (coarse sweep + fine sweep of every slice + correction)")
    return {"value": steps * pts / sum(times), "unit": "grid-pt-steps/s", "cores": problems, "kind": "oracle",
            "sample": what, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "serial_fine_1core": {"value": spts / ssecs, "unit": "grid-pt-steps/s", "seconds": round(ssecs, 3),
                                  "sample": ("sequential fine solve F^N(u0) of problem 0 on one core"
                                             if w.get("dim", 1) == 1 and not w.get("nn") else
                                             "the fine steps of the all-core sample, one process")}}


# ----------------------------------------------------------------------------- our arm


def bench_ours(args, w, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2304_14074_gb300 as ch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    u0 = u0_batch(w, rank)
    B, n, N, J = w["batch"], w["n"], w["N"], w["J"]
    dim = w.get("dim", 1)
    pts = n ** dim
    cfg = ch.Config(dim=dim, n=n, eps=w["eps"], T=w["T"], n_slices=N, fine_steps=J, variant=w["variant"],
                    newton_tol=w["newton_tol"], max_iters=1, precision=w["precision"])
    u0_dev = torch.as_tensor(u0, dtype=torch.float64, device=dev).contiguous()
    pr = ch.Parareal(cfg, batch=B, stream=stream)
    if w.get("nn"):
        pr.set_fine_nn(*w["nn"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def one_step():
        pr.set_initial_device(u0_dev)
        pr.run()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    execution = pr.execution()
    fine_pts_per_step = B * N * J * pts
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fine_ms, newton_total, launches, cg_per_step = 0.0, 0, 0, 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
            st = [pr.stats(b) for b in (0,)]
            fine_ms += st[0]["fine_sweep_ms"]
            launches += st[0]["kernel_launches"]
            if i == 0:
                if dim == 1:
                    newton_total = sum(pr.stats(b)["newton_total"] for b in range(B))
                else:
                    newton_total = st[0]["newton_total"]
                    cg_per_step = st[0]["inner_iterations"]
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, dev)
    value = world * args.steps * fine_pts_per_step / (total_ms / 1e3)

    # roofline of the dominant kernel (the fine sweep), timed live between the iteration graphs
    fine_ms_per_launch = fine_ms / args.steps
    newton_per_step = newton_total  # Newton iterations (summed over problems) in one step
    if dim == 1:
        if FINE_OF[w["variant"]] == "nl":
            alg_flops = fine_pts_per_step * FP64_FLOPS_RHS + newton_per_step * n * FP64_FLOPS_NEWTON
        elif w.get("nn"):
            # newton_total counts NN iterations here
            alg_flops = fine_pts_per_step * FP64_FLOPS_NN_STEP + newton_per_step * n * FP64_FLOPS_NN_ITER
        else:
            alg_flops = fine_pts_per_step * FP64_FLOPS_LINEAR_STEP
        achieved = alg_flops / (fine_ms_per_launch / 1e3) / 1e9
        dgemm = fp64_dgemm_tflops() * 1e3 if rank == 0 else None
        # the denominator: the FP64 rate measured in this run (MEASURED_PEAKS.json has no FP64
        # entry), the nominal rate beside it
        peak = dgemm if dgemm else FP64_PEAK_GFLOPS
        roofline = {"bound": "alu", "kernel": ("k_nn_fine_sweep" if w.get("nn") else "k_fine_sweep") + " (FP64 pipe)",
                    "achieved": round(achieved, 2),
                    "peak": round(peak, 1), "unit": "GFLOP/s",
                    "frac": round(achieved / peak, 4),
                    "peak_source": ("measured in this run: cuBLAS DGEMM 6144^3 (no FP64 entry in MEASURED_PEAKS.json)"
                                    if dgemm else "nominal FP64: 152 SMs x 4 flop/clk x 2.07 GHz"),
                    "fp64_nominal_gflops": round(FP64_PEAK_GFLOPS, 1),
                    "frac_of_nominal": round(achieved / FP64_PEAK_GFLOPS, 4),
                    "traffic": FINE_SWEEP_1D_TRAFFIC.get((n, B, N)),
                    "fine_sweep_ms_per_launch": round(fine_ms_per_launch, 3),
                    "fine_sweep_share_of_step": round(fine_ms / total_ms, 4) if world == 1 else None,
                    "newton_iters_per_step_point": round(newton_per_step / (B * N * J), 3),
                    "algorithmic_fp64_flops_per_launch": alg_flops}
    else:
        roofline = roofline_2d(w, B, fine_ms_per_launch, newton_per_step, cg_per_step,
                               fine_ms / total_ms if world == 1 else None)

    # end to end through the public API: pinned host inputs in, every slice of the result out
    u0_pin = torch.from_numpy(u0).pin_memory()
    out_pin = torch.empty((B, N + 1, pts), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(max(1, args.steps // 2)):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr.set_initial_batch(u0_pin)
        pr.run()
        pr.get_slices_batch(out_pin)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e_mean = max_over_ranks(e2e_mean, dist, dev)
    e2e = {"value": world * fine_pts_per_step / (e2e_mean / 1e3), "unit": "grid-pt-steps/s",
           "h2d_bytes_per_step": int(u0.nbytes), "d2h_bytes_per_step": int(out_pin.numel() * 8),
           "ms_per_step": round(e2e_mean, 3)}
    pr.close()

    ttol = None
    if w.get("ttol") and not args.no_ttol and rank == 0:
        ttol = time_to_tolerance(ch, w, u0, stream, metrics_jsonl=args.metrics_jsonl)
        if w["variant"].startswith("PA"):
            ttol["theory_bound"] = theory_vs_measured(ch, w, u0, stream, ttol.pop("err_ratio"))
        else:
            ttol.pop("err_ratio")
    if not args.no_learned and rank == 0:
        ttol = dict(ttol or {})
        ttol["learned_vs_plain_G"] = learned_vs_plain(ch, stream)
    r2d = None
    if dim == 1 and not args.no_2d and rank == 0:
        r2d = c4_step_roofline(ch, stream)
    return dict(value=value, total_ms=total_ms, step_ms=step_ms, roofline=roofline, e2e=e2e,
                clocks=clk.summary(), launches=launches, ttol=ttol, roofline_2d=r2d, execution=execution)


def roofline_2d(w, B, fine_ms_per_launch, newton_total, cg_total, share):
    """HBM roofline of the 2D fine sweep: algorithmic bytes (BYTES_* per grid point, from the
    Newton and CG iterations summed over the units) over the live fine-sweep time."""
    n, N, J = w["n"], w["N"], w["J"]
    pts = n * n
    units = B * N
    alg_bytes = pts * (newton_total * BYTES_NEWTON_2D + cg_total * BYTES_CG_2D + units * J * BYTES_STEP_2D)
    achieved = alg_bytes / (fine_ms_per_launch / 1e3) / 1e9
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    field = 4 * pts * units  # one FP32 solver vector over all units
    work = 9 * field         # the CG's FP32 vectors (x, r, p, u, s, w, weights, two transform buffers)
    where = ("its working set fits the 129 MB L2: HBM bandwidth is a bound, not the limit" if work < 100e6 else
             "its working set is beyond the 129 MB L2: the sweeps stream from HBM")
    return {"bound": "hbm", "kernel": "2D fine sweep (sine-transform passes + pointwise sweeps)",
            "workload": w["name"], "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "peak_source": ("MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks
                            else "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"),
            "traffic": (round(TRAFFIC_2D_OVER_ALGORITHMIC[n] * alg_bytes) if n in TRAFFIC_2D_OVER_ALGORITHMIC
                        else None),
            "traffic_source": ("ncu DRAM bytes of full CG iterations (all units active) over their algorithmic "
                               f"bytes, {TRAFFIC_2D_OVER_ALGORITHMIC[n]}, times this launch's algorithmic bytes"
                               if n in TRAFFIC_2D_OVER_ALGORITHMIC else None),
            "fine_sweep_ms_per_launch": round(fine_ms_per_launch, 3),
            "fine_sweep_share_of_step": round(share, 4) if share is not None else None,
            "newton_iterations_per_unit_step": round(newton_total / (units * J), 3),
            "cg_iterations_per_unit_step": round(cg_total / (units * J), 3),
            "algorithmic_bytes_per_launch": alg_bytes,
            "note": f"one FP32 solver vector over all {units} units is {field / 1e6:.1f} MB and the CG "
                    f"touches about nine ({work / 1e6:.0f} MB): {where}"}


def c4_step_roofline(ch, stream, warmup=1, steps=1):
    """One step of the 512 x 512 configuration (coarse initial sweep + fine sweep of all 64 slices
    + coarse sweep with correction), timed live with CUDA events; the roofline of its fine sweep."""
    import torch
    w = WORKLOADS["c4"]
    u0 = u0_batch(w, 0)
    cfg = ch.Config(dim=2, n=w["n"], eps=w["eps"], T=w["T"], n_slices=w["N"], fine_steps=w["J"],
                    variant=w["variant"], newton_tol=w["newton_tol"], max_iters=1, precision=w["precision"])
    pr = ch.Parareal(cfg, batch=1, stream=stream)
    u0_dev = torch.as_tensor(u0, dtype=torch.float64, device="cuda").contiguous()
    for _ in range(warmup):
        pr.set_initial_device(u0_dev)
        pr.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fine_ms, newton, cg = 0.0, 0, 0
    a.record(stream)
    for _ in range(steps):
        pr.set_initial_device(u0_dev)
        pr.run()
        st = pr.stats(0)
        fine_ms += st["fine_sweep_ms"]
        newton += st["newton_total"]
        cg += st["inner_iterations"]
    b.record(stream)
    torch.cuda.synchronize()
    step_ms = a.elapsed_time(b) / steps
    execution = pr.execution()
    pr.close()
    r = roofline_2d(w, 1, fine_ms / steps, newton / steps, cg / steps, fine_ms / steps / step_ms)
    r["execution"] = execution
    r["step_ms"] = round(step_ms, 2)
    r["grid_pt_steps_per_s"] = w["N"] * w["J"] * w["n"] ** 2 / (step_ms / 1e3)
    return r


def sweep2d(w, args):
    """The fine propagation of all N slices of a 2D workload as one batched ch_propagate call
    (the kernels of a Parareal fine sweep, without the coarse sweeps), `args.fine` fine steps from
    the slice states of a short fine trajectory, timed with CUDA events; HBM roofline against the
    algorithmic bytes."""
    import numpy as np
    import torch

    import ch_inputs
    import paper_2304_14074_gb300 as ch
    torch.cuda.set_device(0)
    n, N, J = w["n"], w["N"], w["J"]
    dt = w["T"] / N / J
    u0 = np.stack([ch_inputs.initial_condition(2, n, w.get("seed0", 0) + s, kind="normal", amp=w["amp"])
                   for s in range(N)])
    cfg = ch.Config(dim=2, n=n, eps=w["eps"], T=w["T"], n_slices=N, fine_steps=J, newton_tol=w["newton_tol"],
                    lin_tol=args.lin_tol)
    X0 = torch.as_tensor(u0, device="cuda")
    # start from states past the initial transient (a few fine steps), as the slices of a sweep
    X0 = ch.propagate(cfg, "nl", dt, 8, X0)
    newton = torch.zeros(N, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        ch.propagate(cfg, "nl", dt, args.fine, X0)
    torch.cuda.synchronize()
    ms = []
    tot_newton = 0
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ch.propagate(cfg, "nl", dt, args.fine, X0, newton=newton)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        tot_newton += int(newton.sum().item())
    t = sum(ms) / len(ms)
    return {"experiment": "sweep2d", "workload": w["name"], "units": N, "fine_steps": args.fine,
            "lin_tol": args.lin_tol or 1e-3,
            "ms_per_propagation": round(t, 3), "grid_pt_steps_per_s": N * args.fine * n * n / (t / 1e3),
            "newton_per_unit_step": tot_newton / (args.steps * N * args.fine)}


C5_TRUNCATED = dict(problems=64, N=64, J=2, dt=0.5 / 64 / 100, seed=0)


def ensemble_c5(args):
    """The uneven-grid ensemble (c5: grids 64^2..512^2 drawn uniformly from {64, 128, 256, 512},
    eps ~ U[0.01, 0.05], N = 64 slices, plain coarse step), truncated to C5_TRUNCATED's problem
    count and fine steps per slice at c5's fine step (T = N J dt). One Parareal iteration (coarse
    initial sweep, fine sweep of every slice of every problem, coarse sweep with the correction),
    all grid-size groups run concurrently; timed over `args.steps` runs after `args.warmup`."""
    import torch

    import ch_inputs
    import paper_2304_14074_gb300 as ch
    torch.cuda.set_device(0)
    c = C5_TRUNCATED
    sizes, eps = ch_inputs.ensemble_draws(c["seed"], c["problems"])
    ns = [int(s) - 1 for s in sizes]
    T = c["N"] * c["J"] * c["dt"]
    cfg = ch.Config(dim=2, n=ns[0], eps=float(eps[0]), T=T, n_slices=c["N"], fine_steps=c["J"], variant="NPA-I",
                    newton_tol=1e-12, max_iters=1)
    ens = ch.Ensemble(cfg, ns, [float(e) for e in eps])
    for i, n in enumerate(ns):
        ens.set_initial(i, ch_inputs.initial_condition(2, n, 3000 + i, kind="normal", amp=0.05))
    for _ in range(args.warmup):
        ens.run()
    ts = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ens.run()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    pts = sum(c["N"] * c["J"] * n * n for n in ns)
    groups = {int(n): ns.count(n) for n in sorted(set(ns))}
    st = [ens.stats(i) for i in range(len(ns))]
    ens.close()
    t = sum(ts) / len(ts)
    return {"experiment": "c5-truncated",
            "workload": (f"ensemble of {len(ns)} 2D problems (c5 truncated from 1024), grids {groups} (n: count), "
                         f"eps in [{eps.min():.3f}, {eps.max():.3f}], N={c['N']}, J={c['J']} at c5's dt={c['dt']:.4g} "
                         f"(T={T:.3g}), NPA-I, plain coarse step, one Parareal iteration per run"),
            "seconds_per_iteration": round(t, 4), "grid_pt_steps_per_s": pts / t,
            "iterations": int(st[0]["iterations"])}


def fp64_dgemm_tflops(size=6144, reps=3):
    """FP64 rate measured on this GPU: a cuBLAS DGEMM (torch.matmul on float64), timed with CUDA
    events after a warm-up. A library measurement beside the nominal FP64 peak, as the BF16 peak is
    a cuBLAS GEMM."""
    import torch
    a = torch.randn(size, size, dtype=torch.float64, device="cuda")
    b = torch.randn(size, size, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        c = a @ b
    e1.record()
    torch.cuda.synchronize()
    del a, b, c
    return 2.0 * size ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def time_to_tolerance(ch, w, u0, stream, err_tol=1e-8, metrics_jsonl=None):
    """Plain-G Parareal until every problem is within err_tol (max_n L2_h) of the sequential fine
    solution; reports the device time of the Parareal run and of the serial fine solve. With
    metrics_jsonl, every problem's per-iteration history is appended to that file."""
    import torch
    B, N = w["batch"], w["N"]
    cfg = ch.Config(dim=w.get("dim", 1), n=w["n"], eps=w["eps"], T=w["T"], n_slices=N, fine_steps=w["J"],
                    variant=w["variant"], newton_tol=w["newton_tol"], max_iters=N, precision=w["precision"],
                    err_tol=err_tol)
    pr = ch.Parareal(cfg, batch=B, stream=stream)
    if w.get("nn"):
        pr.set_fine_nn(*w["nn"])
    pr.set_initial_batch(u0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pr.compute_reference()
    b.record(stream)
    torch.cuda.synchronize()
    serial_ms = a.elapsed_time(b)
    status = pr.run()
    stats = [pr.stats(i) for i in range(B)]
    if metrics_jsonl:
        for i, st in enumerate(stats):
            ch.append_jsonl(metrics_jsonl, ch.stats_records(st, workload=w["name"], run="time_to_1e-8", problem=i,
                                                            status=int(status)))
    iters = max(s["iterations"] for s in stats)
    t_ms = stats[0]["t_iter_ms"][iters]
    worst = max(s["err_l2"][s["iterations"]] for s in stats)
    e = stats[0]["err_l2"]
    pr.close()
    return {"coarse": "plain (one LIN1 step per slice)", "err_tol": err_tol, "seconds": round(t_ms / 1e3, 4),
            "iterations": int(iters), "converged_all": status == 0, "worst_final_err_l2": worst,
            "serial_fine_seconds_same_gpu": round(serial_ms / 1e3, 4),
            "err_ratio": [float(e[k] / e[0]) for k in range(1, min(len(e), 9))]}


def theory_vs_measured(ch, w, u0, stream, ratio_actual):
    """Section 3 bound (ch_parareal_theory_bound) beside measured error reductions E^k / E^0 of
    problem 0: the linear variant's run above, and the same configuration on the frozen model
    diag(u^2) = I for which the theorems are proved (Theorems 3.7, 3.9, 3.11)."""
    N = w["N"]
    kw = dict(dim=w.get("dim", 1), n=w["n"], eps=w["eps"], T=w["T"], n_slices=N, fine_steps=w["J"],
              variant=w["variant"], newton_tol=w["newton_tol"], max_iters=N, precision=w["precision"])
    alpha, beta, f = ch.theory_bound(ch.Config(**kw), N)
    pr = ch.Parareal(ch.Config(**kw, frozen=True), batch=1, stream=stream)
    if w.get("nn"):
        pr.set_fine_nn(*w["nn"])
    pr.set_initial(0, u0[0])
    pr.compute_reference()
    pr.run()
    e = pr.stats(0)["err_l2"]
    pr.close()
    kmax = min(len(ratio_actual), len(e) - 1)
    return {"alpha": alpha, "beta": beta, "k": list(range(1, kmax + 1)),
            "bound_factor": [float("%.4g" % f[k]) for k in range(1, kmax + 1)],
            "measured_frozen": [float("%.4g" % (e[k] / e[0])) for k in range(1, kmax + 1)],
            "measured_scheme": [float("%.4g" % r) for r in ratio_actual[:kmax]]}


# Learned against plain coarse propagator, time to 1e-8. LEARNED_CASE is small enough to train
# G_theta and run both Parareal forms inside the default benchmark; LEARNED_C4 is the 512 x 512
# configuration (eps = 0.01, T = 2, N = 64, J = 100) with 64 training trajectories (seeds
# 1000..1063) snapshotted every dT / 5: 64 x 315 = 20160 pairs (U(t), U(t + dT)), plus perturbed
# pairs, evaluated from the held-out seed 2000 (run by `--experiment learned-c4`).
LEARNED_CASE = dict(n=63, eps=0.05, T=0.3, N=16, J=8, stride=4, train_seeds=64, eval_seed=5000,
                    steps=((1e-3, 8000), (3e-4, 6000), (1e-4, 4000)), batch=32, perturbed=None, chunk=4096,
                    relative_loss=True)
LEARNED_C4 = dict(n=511, eps=0.01, T=2.0, N=64, J=100, stride=5, train_seeds=64, eval_seed=2000,
                  steps=((1e-3, 12000), (3e-4, 8000), (1e-4, 4000)), batch=32, perturbed=512, chunk=512,
                  relative_loss=True)


# G_theta forward arithmetic per pixel: four 32 -> 32 layers (2 x 32 x 288 flops each) and the
# 1 -> 32 and 32 -> 1 layers (2 x 32 x 9 and 2 x 288).
GTHETA_FLOPS_PER_PIXEL = 4 * 2 * 32 * 288 + 2 * 32 * 9 + 2 * 288


def gtheta_forward_roofline(ch, net, batch=8, n=511):
    """Tensor-core roofline of the G_theta forward pass on `batch` fields of the 512^2 grid, timed
    with CUDA events (the four 32 -> 32 layers are BF16 tcgen05.mma on the tensor cores)."""
    import torch
    x = (0.5 * torch.randn(batch, n, n, dtype=torch.float64, device="cuda")).contiguous()
    for _ in range(3):
        y = net.forward(x)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    a.record()
    for _ in range(reps):
        y = net.forward(x, out=y)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    flops = GTHETA_FLOPS_PER_PIXEL * batch * n * n
    peak = measured_peaks().get("bf16_tflops", 1900.0)
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "workload": f"G_theta forward, {batch} fields of {n}^2", "ms": round(ms, 4),
            "achieved": round(achieved, 1), "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "peak_source": ("MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)" if "bf16_tflops" in measured_peaks()
                            else "fallback 1.9 PFLOP/s bf16 (no MEASURED_PEAKS.json)"),
            "algorithmic_flops_per_pixel": GTHETA_FLOPS_PER_PIXEL}


def _propagate_chunked(ch, cfg, scheme, dt, nsteps, X, chunk):
    """ch.propagate over the rows of X in chunks of `chunk` fields (bounds the solver's work space)."""
    import torch
    out = torch.empty_like(X)
    for i in range(0, X.shape[0], chunk):
        ch.propagate(cfg, scheme, dt, nsteps, X[i:i + chunk].contiguous(), out[i:i + chunk])
    return out


def learned_vs_plain(ch, stream, err_tol=1e-8, case=None):
    """Trains G_theta (correction form G(U) + R(U)) on fine-solver snapshot pairs (and, when the case
    asks for them, on pairs from perturbed snapshots), all produced by the library on the GPU, then
    runs Parareal to err_tol with the plain and with the learned coarse step from a held-out
    initial condition."""
    import numpy as np
    import torch

    import ch_inputs
    c = case or LEARNED_CASE
    n, eps, T, N, J, stride = c["n"], c["eps"], c["T"], c["N"], c["J"], c["stride"]
    dT = T / N
    t0 = time.perf_counter()
    seeds = range(1000, 1000 + c["train_seeds"])
    one = ch.Config(dim=2, n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-12)
    # training trajectories: the sequential fine solution of every seed, snapshotted every dT/stride
    states = torch.empty((len(seeds), N * stride + 1, n * n), dtype=torch.float64, device="cuda")
    states[:, 0] = torch.as_tensor(np.stack([ch_inputs.initial_condition(2, n, s, kind="normal", amp=0.05)
                                             for s in seeds]), device="cuda")
    for j in range(N * stride):
        states[:, j + 1] = ch.propagate(one, "nl", dT / J, J // stride, states[:, j].contiguous())
    base = _propagate_chunked(ch, one, "lin1", dT, 1, states.reshape(-1, n * n), c["chunk"]).reshape(states.shape)
    # perturbed pairs (U + eta, F(U + eta)) around the slice-boundary states teach the step's
    # response to perturbations, which is what the Parareal correction differences
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    X = states[:, ::stride].reshape(-1, n * n)
    if c.get("perturbed"):
        idx = torch.randperm(X.shape[0], generator=g, device="cuda")[:c["perturbed"]]
        X = X[idx]
    pairs = []
    kinds = ((0.05, False), (0.2, True), (0.05, True)) if not c.get("perturbed") else ((0.2, True), (0.05, False))
    for amp, smooth in kinds:
        eta = torch.randn(X.shape, device="cuda", dtype=torch.float64, generator=g)
        if smooth:
            for _ in range(3):
                eta = _propagate_chunked(ch, one, "lin1", dT, 1, eta.contiguous(), c["chunk"])
            eta = eta / eta.abs().amax(dim=1, keepdim=True)
        Xp = (X + amp * eta).contiguous()
        pairs.append(torch.stack([Xp, _propagate_chunked(ch, one, "nl", dT / J, J, Xp, c["chunk"])], 1))
    pert = torch.cat(pairs).contiguous()
    pbase = _propagate_chunked(ch, one, "lin1", dT, 1, pert.reshape(-1, n * n), c["chunk"]).reshape(pert.shape)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = ch.GTheta(seed=1)
    net.set_loss(c.get("relative_loss", False))
    t1 = time.perf_counter()
    losses = []
    for lr, steps in c["steps"]:
        for rep in range(4):
            losses.append(net.train(states, stride=stride, steps=steps // 8, batch=c["batch"], lr=lr,
                                    seed=rep + int(lr * 1e6), base=base))
            losses.append(net.train(pert, stride=1, steps=steps // 8, batch=c["batch"], lr=lr,
                                    seed=50 + rep + int(lr * 1e6), base=pbase))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    params = net.get_params()
    losses = np.concatenate(losses)
    npairs = len(seeds) * (N * stride - stride + 1)
    del base, pbase, pert, pairs
    # one-step error of each coarse propagator on held-out states (slice boundaries of the
    # evaluation trajectory), relative to the change F(U) - U over the slice
    cfg = ch.Config(dim=2, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="NPA-I", newton_tol=1e-12,
                    err_tol=err_tol)
    u0 = ch_inputs.initial_condition(2, n, c["eval_seed"], kind="normal", amp=0.05)[None]
    out = {}
    for name, p in (("plain", None), ("learned", params)):
        h = ch.Parareal(cfg, batch=1, stream=stream)
        h.set_initial_batch(u0)
        h.compute_reference()
        if p is not None:
            h.set_coarse_model(p, "correction")
        if name == "plain":
            ref = torch.empty((1, N + 1, n * n), dtype=torch.float64, device="cuda")
            h.get_reference_device(ref)
        try:
            st, failed = h.run(), None
        except ch.ChError as e:  # reported, not fatal: the other form still runs
            st, failed = e.status, e.name + " (" + h.lib.ch_parareal_last_error(h._h).decode() + ")"
        s0 = h.stats(0)
        k = s0["iterations"]
        out[name] = {"iterations": int(k), "seconds": round(s0["t_iter_ms"][k] / 1e3, 4), "converged": st == 0,
                     "final_err_l2": float(s0["err_l2"][k]), "err_l2_history":
                     [float("%.3g" % v) for v in s0["err_l2"][:k + 1]],
                     "coarse_fallback_iter": int(s0["coarse_fallback_iter"]), "error": failed}
        h.close()
    U = ref[0, :N].contiguous()
    Fu = ref[0, 1:]
    Gu = _propagate_chunked(ch, one, "lin1", dT, 1, U, c["chunk"])
    Lu = torch.empty_like(U)
    net.forward(U.view(N, n, n), out=Lu.view(N, n, n), base=Gu.view(N, n, n))
    chg = (Fu - U).norm(dim=1)
    out["one_step_error_rel_to_change"] = {
        "plain": float(((Gu - Fu).norm(dim=1) / chg).median()),
        "learned": float(((Lu - Fu).norm(dim=1) / chg).median()),
        "over": f"the {N} slices of the held-out trajectory (median over slices)"}
    out["speedup_learned_over_plain"] = round(out["plain"]["seconds"] / max(out["learned"]["seconds"], 1e-9), 3)
    out["gtheta_forward_roofline"] = gtheta_forward_roofline(ch, net)
    net.close()
    out["config"] = (f"2D NPA-I n={n} eps={eps} T={T} N={N} J={J}, u0 = 0.05 N(0,1) seed {c['eval_seed']}; "
                     f"G_theta correction form trained on {len(seeds)} trajectories (seeds 1000..) "
                     f"x {N * stride - stride + 1} = {npairs} snapshot pairs + {X.shape[0] * len(kinds)} perturbed "
                     f"pairs, {len(losses)} Adam steps"
                     + (", relative loss (each crop's squared error over its target's energy)"
                        if c.get("relative_loss") else ", mean squared error"))
    out["data_seconds"] = round(t_data, 2)
    out["training_seconds"] = round(t_train, 2)
    out["final_training_loss"] = float(losses[-200:].mean())
    return out


# ------------------------------------------------------------------------------ main


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2")
    ap.add_argument("--no-ttol", action="store_true", help="skip the time-to-1e-8 run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain coarse propagator run")
    ap.add_argument("--no-2d", action="store_true", help="skip the 512 x 512 2D step (roofline_2d)")
    ap.add_argument("--metrics-jsonl", default=None,
                    help="append the time-to-1e-8 run's per-iteration history of every problem to this file")
    ap.add_argument("--experiment", choices=["learned-c4", "sweep2d", "c5", "gtheta-fwd"], default=None,
                    help="learned-c4: learned vs plain coarse propagator to 1e-8 on the 512 x 512 configuration "
                         "(training included); sweep2d: the 2D fine propagation of one Parareal fine sweep of a 2D "
                         "workload (all its slices batched), `--steps` times `--fine` steps, timed alone. One JSON "
                         "line each.")
    ap.add_argument("--fine", type=int, default=2, help="sweep2d: fine steps per timed propagation")
    ap.add_argument("--lin-tol", type=float, default=0.0, help="sweep2d: inner CG tolerance (0: the default)")
    args = ap.parse_args()
    if args.experiment == "gtheta-fwd":
        import torch

        import paper_2304_14074_gb300 as ch
        torch.cuda.set_device(0)
        net = ch.GTheta(seed=1)
        r = gtheta_forward_roofline(ch, net)
        r["conv"] = os.environ.get("CH_GTHETA_CONV", "tcgen05")
        net.close()
        print(json.dumps(r))
        return
    if args.experiment == "c5":
        print(json.dumps(ensemble_c5(args)))
        return
    if args.experiment == "sweep2d":
        print(json.dumps(sweep2d(WORKLOADS[args.workload if args.workload != "c2" else "c4"], args)))
        return
    if args.experiment == "learned-c4":
        import torch

        import paper_2304_14074_gb300 as ch
        torch.cuda.set_device(0)
        t = time.perf_counter()
        r = learned_vs_plain(ch, torch.cuda.current_stream(), case=LEARNED_C4)
        r["experiment"] = "learned-c4"
        r["wall_seconds"] = round(time.perf_counter() - t, 1)
        print(json.dumps(r))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    ubytes = w["batch"] * (w["N"] + 1) * w["n"] ** w.get("dim", 1) * 8
    l2 = (f"inputs larger than L2 (U, F, Gold {ubytes / 1e6:.0f} MB each) and" if ubytes > 129e6
          else f"U, F, Gold {ubytes / 1e6:.3g} MB each (smaller than L2);") + " a 256 MB L2 flush between steps"
    config = {"workload": w["name"], "global_batch": w["batch"] * world, "slices": w["N"], "fine_steps": w["J"],
              "grid": w["n"], "parallelism": f"replicas{world}" if world > 1 else "single", "l2": l2,
              "step": "coarse initial sweep + one fine sweep over all slices + coarse sweep/correction/norms"}

    if args.impl == "reference":
        if rank != 0:
            return
        u0 = u0_batch(w, 0)
        problems = cpu_sample_size()
        for _ in range(args.warmup):
            pass  # the oracle has no warm-up state; each step below is a fresh sample
        pts, times = cpu_oracle(w, problems, u0, steps=args.steps)
        total = sum(times)
        value = args.steps * pts / total
        what = (f"{problems} processes x {ORACLE_NN_STEPS} Neumann-Neumann fine steps of one slice per step"
                if w.get("nn") else
                f"{problems} processes x {ORACLE_2D_STEPS} fine steps of one slice per step (sparse solves by "
                "library CG)" if w.get("dim", 1) == 2 else
                f"{problems} problems of the batch per step (repeated when the batch is smaller), one process per "
                "core, each one step of the workload (coarse sweep + fine sweep of every slice + correction)")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grid-pt-steps/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": value, "unit": "grid-pt-steps/s", "cores": problems, "kind": "oracle",
                                 "sample": what, "nproc": os.cpu_count(), "cpu_model": cpu_model()},
                "e2e": {"value": value, "unit": "grid-pt-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    # CPU oracle baseline first (spawned processes, before any GPU work in this process)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(w, u0_batch(w, 0))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    r = bench_ours(args, w, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    config["execution"] = r["execution"]
    line = {"metric": METRIC, "value": r["value"], "unit": "grid-pt-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": r["launches"],
            "clocks": r["clocks"], "time_to_1e-8": r["ttol"], "roofline_2d": r["roofline_2d"],
            "precision": ("FP64 states, residuals, correction and norms; " +
                          ("inner solves of the fine steps FP32 (refined by the FP64 residual)" if w["precision"] == 1
                           else "all solves FP64"))}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
