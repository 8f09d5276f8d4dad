#!/usr/bin/env python
"""Benchmark of the sparse-grid WENO5 hot path on one GB300 (or N, one process each).

Workload: an uneven batch of 256 independent 3-D Burgers problems u_t + sum_k (u^2/2)_{x_k} = 0
on [0, 4]^3, u0 = 0.5 + a sin(pi (x+y+z)/2), a ~ U[0.5, 1], root cells N_r in {8, 12, 16},
finest level N_L in {3, 4, 5} (seeded draws), all advanced to t = 0.3 with CFL 0.4, FP32 state,
one persistent launch per RK stage over all members' grids, CUDA-graph replay.

One benchmark step = one pass of the whole path over the batch: on-device restriction of the
initial condition (Step 1), time marching to t = 0.3 (Step 2), WENO5 prolongation and signed
combination in FP64 for every member (Step 3), FP64 min/max of every combined solution.

Metric: grid-point updates per second (one point advanced one full RK3 step), whole job.
Prints one JSON line.  --impl reference times the FP64 CPU oracle on the host cores instead.

--workload relax2d / relax4d measures the Vlasov-Boltzmann relaxation model of Example 5
instead (one GPU): (a) N_r = 40, N_L = 3 in 2-D to t = 6, (b) N_r = 10, N_L = 3 in 4-D to t = 3,
CFL 0.4, FP32 batched; one step = restriction, time marching, combination and the two entropy
functionals of the combined solution.  Its state fits in L2, so L2 is flushed between steps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2007_10196_gb300 import inputs  # noqa: E402  (seeded workload draws only)

METRIC = "WENO5 grid-point updates/s and HBM GB/s fraction, FP32 batched vs FP64 plain at equal L1"
UNIT = "grid-point updates/s"
WORKLOAD = "burgers3d_batch256_t0.3_cfl0.4_f32_batched"

# Algorithmic work of the FP32 stage kernel per grid point per RK stage for 3-D Burgers (FLOPs,
# an FMA counts 2): per axis the LF split of the point (6), one interface flux with two
# one-sided WENO5 reconstructions (2 x 54) and their combination (7), the flux difference (3);
# plus the RK update (4 on average over the three stages).
FLOPS_PER_POINT_STAGE_3D = 3 * (6 + 2 * 54 + 7 + 3) + 4
# Algorithmic HBM bytes per point per full RK step, FP32 compensated state (u^n = U + C, stage
# increments D1, D2): stage 1 reads U, writes D1 (8); stage 2 reads U, D1, writes D2 (12);
# stage 3 reads U, D2, C, writes U and C (20).
BYTES_PER_POINT_STEP = 40
# FP64 Shu-Osher form: stage 1 reads u^n, writes u1 (16); stages 2 and 3 read their input and
# u^n and write the result (24 + 24).
BYTES_PER_POINT_STEP_F64 = 64
FP32_LANES_PER_SM = 128
# Burgers shock time of u0 = 0.5 + a sin(pi (x+y+z)/2): characteristics in s = x+y+z move at
# 3u, so they first cross at t = 1 / (3 a pi/2); members with a below this stay smooth to t_end.
A_SMOOTH_AT_T_END = 2.0 / (3.0 * math.pi * 0.3)
STAGE_SOURCES = ("sg_stage.cuh", "sg_sweep2.cuh", "sg_weno.cuh", "sg_device.h")  # the d = 3 sweep kernels and what they include
# Vlasov-Boltzmann (Example 5), FP32 line-buffer stage kernel, per point per RK stage: per axis
# the split of the point (2: the line speed times the value, twice), two one-sided WENO5
# reconstructions (2 x 54), their combination (7) and the flux difference (3); then the
# relaxation (mu rho - u) / tau added (4) and the RK update (4 on average).
FLOPS_PER_POINT_STAGE_RELAX = {2: 2 * (2 + 2 * 54 + 7 + 3) + 8, 4: 4 * (2 + 2 * 54 + 7 + 3) + 8}
RELAX = {"relax2d": (2, 40, 3, 6.0, "vlasov_boltzmann_example5a_nr40_nl3_t6_cfl0.4_f32_batched"),
         "relax4d": (4, 10, 3, 3.0, "vlasov_boltzmann_example5b_4d_nr10_nl3_t3_cfl0.4_f32_batched")}


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


N_MEMBERS = 256
# --stage-kernel: sg_params.stage_kernel by name (0 = SG_STAGE_AUTO, 2 = SG_STAGE_SWEEP, ...)
STAGE_KERNELS = {"auto": 0, "sweep": 2, "sweep2": 3}


def _members(rank):
    return inputs.burgers3d_batch(256, seed=2007 + rank)[:N_MEMBERS]


def _batch_points(members):
    """Grid counts and points per member (sparse-grid combination of Section 2.2)."""
    out = []
    for m in members:
        tot, grids = 0, 0
        for q in range(3):
            s = m.nl - q
            for l0 in range(s + 1):
                for l1 in range(s - l0 + 1):
                    l2 = s - l0 - l1
                    tot += (m.nr << l0) * (m.nr << l1) * (m.nr << l2)
                    grids += 1
        out.append((grids, tot))
    return out


# Algorithmic work of the prolongation + combination step (Step 3, Eqs. 8-15), FP32 arithmetic
# (FMA = 2 FLOP): one interpolation at a fine node from a prepared window -- the cubic N(s) and
# quadratic D(s) by Horner (10), their quotient (1), w2 + (s/2) q (3) -- is 14 FLOP; preparing
# a window (the differences, the three smoothness indicators of Eq. 10, the weights' factors and
# the coefficients of N and D) is 60 FLOP per coarse node and line; adding c_g v into the sum is
# 2 FLOP per grid and finest node.  Bytes: Û is written once, 8 B per finest node.
FLOP_INTERP, FLOP_PREPARE, FLOP_ACCUM = 14, 60, 2
BYTES_PER_FINEST_POINT = 8


def combine_work(members):
    """(finest points, FLOPs) of Step 3 over the members: per grid, every prolonged axis k < d-1
    interpolates each fine node of each line and prepares each coarse node once per line; the
    last axis does so at every finest node (grids whose last axis is coarse) and adds c_g v."""
    pts, flops = 0, 0
    for m in members:
        Nf = m.nr << m.nl
        pts += Nf ** 3
        for q in range(3):
            s = m.nl - q
            for l0 in range(s + 1):
                for l1 in range(s - l0 + 1):
                    n = [m.nr << l0, m.nr << l1, m.nr << (s - l0 - l1)]
                    cur = list(n)
                    for k in range(2):
                        if n[k] < Nf:
                            lines = (cur[0] * cur[1] * cur[2]) // cur[k]
                            flops += lines * (Nf * FLOP_INTERP + n[k] * FLOP_PREPARE)
                            cur[k] = Nf
                    if n[2] < Nf:
                        flops += Nf * Nf * (Nf * FLOP_INTERP + n[2] * FLOP_PREPARE)
                    flops += Nf ** 3 * FLOP_ACCUM
    return pts, flops


# ------------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ------------------------------------------------------------------------------------------
def _oracle_member(args):
    nr, nl, a, nsteps = args
    import oracle
    p = oracle.problem(3, nr, nl, pde=oracle.BURGERS, eps=1e-3, lo=0.0, hi=4.0)
    lev, co = oracle.grid_set(3, nl)
    grids = [oracle.restrict_sine(p, l, 0.5, a, math.pi / 2) for l in lev]
    t0 = time.perf_counter()
    out, steps, t = oracle.solve(p, lev, grids, inputs.BATCH_T_END, max_steps=nsteps, rule=oracle.DT_CFL,
                                 cfl=inputs.BATCH_CFL)
    dt = time.perf_counter() - t0
    return sum(g.size for g in out) * steps, dt


def oracle_sample(members, pool, cores, nsteps=1):
    """Runs the oracle on every member for `nsteps` time steps in a process pool; returns
    (point-updates, wall seconds)."""
    import oracle
    oracle.build()
    jobs = [(m.nr, m.nl, m.a, nsteps) for m in members]
    jobs.sort(key=lambda j: -(j[0] << j[1]))  # largest first for balance
    t0 = time.perf_counter()
    res = pool.map(_oracle_member, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    return sum(r[0] for r in res), wall


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.f:
            return None
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _cpu_model():
    """The host CPU's model name (lscpu) and the cores this process may run on."""
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        ncpu = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        ncpu = os.cpu_count() or 1
    return "%s (%d cores available)" % (name or "unknown", ncpu)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def stage_source_hash():
    """sha256 over the sources that define the stage kernels."""
    h = hashlib.sha256()
    for name in STAGE_SOURCES:
        with open(os.path.join(ROOT, "paper_2007_10196_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _stage_traffic(kernel, points_per_launch):
    """DRAM bytes per stage launch from the committed ncu summary (bytes per point-stage of the
    profiled launches), scaled by the points one launch processes -- if that summary is of the
    same kernel built from the same sources; else None."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        if rec["kernel"] != kernel or rec["sources_sha256"] != stage_source_hash():
            return None
        return rec["dram_bytes_per_point_stage"] * points_per_launch
    except (OSError, ValueError, KeyError):
        return None


def kernel_name(P, h):
    kern, tp, _ = P.sg_stage_config(h)
    if kern == P.SG_STAGE_SWEEP:
        return "sg_stage_sweep3_kernel<float, false>"
    if kern == P.SG_STAGE_SWEEP2:  # pairs of work items per block at the batch's sizes
        return "sg_stage_sweep3x2_kernel<false, 2>"
    return "sg_stage_box_kernel<float,3,%d>" % (tp // 256)


def compare_fp64_plain(P, stream, members, nmax=4, nshock=2):
    """The plain FP64 path (one launch per grid per RK stage) against the batched FP32 path on
    the same members: stepping rates to t_end, and accuracy.  Members still smooth at t_end: the
    L1 error of the combined solution against the exact (characteristic) solution for both.
    Members past their shock (no exact solution): the FP32 combined solution against the FP64
    one (identical to the oracle's, bit for bit), max and mean difference."""
    import torch
    sel = [m for m in members if m.a < A_SMOOTH_AT_T_END][:nmax]
    # the smallest shocked members (a full FP64 read of each combined solution)
    shk = sorted([m for m in members if m.a >= A_SMOOTH_AT_T_END], key=lambda m: m.nr << m.nl)[:nshock]
    if not sel:
        return None
    run = sel + shk
    ics = [(0.5, m.a, math.pi / 2, 0.0) for m in run]
    pts = [n for _, n in _batch_points(run)]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for prec, exe in ((P.SG_F64, P.SG_PLAIN), (P.SG_F32, P.SG_BATCHED)):
        hs = [P.create(3, m.nr, m.nl, P.SG_PDE_BURGERS, precision=prec, exec=exe, dt_rule=P.SG_DT_CFL,
                       cfl=inputs.BATCH_CFL, cuda_stream=stream.cuda_stream) for m in run]
        b = P.sg_batch_create(hs) if exe == P.SG_BATCHED else None
        try:
            ms = 0.0
            for rep in range(2):  # the first pass autotunes and warms up
                for h, ic in zip(hs, ics):
                    P.sg_init(h, P.SG_IC_SINE, ic)
                ev0.record(stream)
                if b is not None:
                    P.sg_step(b, inputs.BATCH_T_END)
                else:
                    for h in hs:
                        P.sg_step(h, inputs.BATCH_T_END)
                ev1.record(stream)
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
            upd = sum(P.sg_time(h)[1] * n for h, n in zip(hs, pts))
            l1, uh = [], []
            for h, m in zip(hs, run):
                P.sg_prolong_combine(h)
                if len(l1) < len(sel):
                    l1.append(P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT))
                else:
                    uh.append(P.sg_read(h, -1, count=(m.nr << m.nl) ** 3))
            res[prec] = (upd / (ms / 1e3), l1, ms, uh)
        finally:
            if b is not None:
                P.sg_destroy(b)
            for h in hs:
                P.sg_destroy(h)
    r64, l64, ms64, u64 = res[P.SG_F64]
    r32, l32, ms32, u32 = res[P.SG_F32]
    shocked = [{"member": (m.nr, m.nl, round(m.a, 4)), "max_abs_diff": float(np.max(np.abs(a - b))),
                "mean_abs_diff": float(np.mean(np.abs(a - b))), "range_fp64": [float(b.min()), float(b.max())]}
               for m, a, b in zip(shk, u32, u64)]
    return {"fp64_plain_value": r64, "fp32_batched_value": r32, "unit": UNIT, "speedup": r32 / r64,
            "fp64_plain_hbm_gbs": r64 * BYTES_PER_POINT_STEP_F64 / 1e9,
            "fp64_plain_ms": ms64, "fp32_batched_ms": ms32,
            "members": [(m.nr, m.nl, round(m.a, 4)) for m in sel],
            "l1_exact_fp64": l64, "l1_exact_fp32": l32,
            "l1_ratio_fp32_over_fp64_max": max(a / b for a, b in zip(l32, l64)),
            "shocked_fp32_vs_fp64": shocked,
            "note": "rates over smooth and shocked members together, both stepped to t_end and combined; "
                    "L1 against the exact solution on the smooth members"}


def fp64_plain_configs(P, stream, c3_steps=64):
    """The plain FP64 path and the batched FP32 path on the 2-D advection configuration
    (adv2d_nr10_nl4: full run to t = 1, L1 against the exact translate) and on the 3-D one
    (adv3d_nr8_nl6, finest 512^3: a fixed number of steps, rates only): point-updates/s and the
    FP64 path's algorithmic HBM bytes per second (64 B per point-step)."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    peaks, _ = _peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    for name, nsteps in (("adv2d_nr10_nl4", None), ("adv3d_nr8_nl6", c3_steps)):
        w = inputs.WORKLOADS[name]
        row = {}
        for prec, exe in ((P.SG_F64, P.SG_PLAIN), (P.SG_F32, P.SG_BATCHED)):
            h = P.create(w.dim, w.nr, w.nl, w.pde, precision=prec, exec=exe, dt_rule=w.dt_rule,
                         dt_coef=w.dt_coef, lo=w.lo, hi=w.hi, cuda_stream=stream.cuda_stream)
            try:
                G = P.sg_num_grids(h)
                pts = sum(int(np.prod(P.sg_grid_info(h, g, w.dim)[1])) for g in range(G))
                ms = 0.0
                for rep in range(2):  # the first pass autotunes and warms up
                    P.sg_init(h, P.SG_IC_SINE, w.ic)
                    ev0.record(stream)
                    P.sg_step(h, w.t_end, nsteps if nsteps else (1 << 62))
                    ev1.record(stream)
                    ev1.synchronize()
                    ms = ev0.elapsed_time(ev1)
                steps = P.sg_time(h)[1]
                rate = steps * pts / (ms / 1e3)
                r = {"value": rate, "ms": ms, "steps": steps, "points": pts}
                if prec == P.SG_F64:
                    gbs = rate * BYTES_PER_POINT_STEP_F64 / 1e9
                    r.update({"hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak})
                if nsteps is None:
                    P.sg_prolong_combine(h)
                    r["l1_exact"] = P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT)
                row["fp64_plain" if prec == P.SG_F64 else "fp32_batched"] = r
            finally:
                P.sg_destroy(h)
        row["speedup"] = row["fp32_batched"]["value"] / row["fp64_plain"]["value"]
        out[name] = row
    return out


def oracle_single_thread(members, every=8):
    """The oracle on one host thread, in this process: every `every`-th member's first time step
    (a bounded, representative sample of the batch); (point-updates/s, sample description)."""
    import oracle
    oracle.build()
    upd, wall = 0, 0.0
    sample = members[::every]
    for m in sample:
        u, w = _oracle_member((m.nr, m.nl, m.a, 1))
        upd += u
        wall += w
    return upd / wall, "%d members (every %dth), first time step each, one thread" % (len(sample), every), wall


def aggregate(local_ms, local_updates, dist=None, device="cpu"):
    """Whole-job figures over ranks: (max elapsed ms over ranks, sum of point-updates).  The
    members of every rank are independent problems, so nothing but these two scalars is
    exchanged (weak scaling)."""
    if dist is None:
        return float(local_ms), float(local_updates)
    import torch
    t = torch.tensor([float(local_ms), float(local_updates)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2007_10196_gb300 as P

    pool = None
    cores = 0
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = min(os.cpu_count() or 1, 64)
        pool = mp.get_context("spawn").Pool(cores)

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.Stream()
    members = _members(rank)
    info = _batch_points(members)
    P.build()
    hs = []
    with torch.cuda.stream(stream):
        for m in members:
            h = P.create(3, m.nr, m.nl, P.SG_PDE_BURGERS, precision=P.SG_F32, exec=P.SG_BATCHED,
                         dt_rule=P.SG_DT_CFL, cfl=inputs.BATCH_CFL, cuda_stream=stream.cuda_stream,
                         stage_kernel=STAGE_KERNELS[args.stage_kernel])
            hs.append(h)
        batch = P.sg_batch_create(hs)
    ics = [(0.5, m.a, math.pi / 2, 0.0) for m in members]
    all_h = hs + [batch]

    def one_pass(host_in=None, host_out=None):
        if host_in is None:
            for h, ic in zip(hs, ics):
                P.sg_init(h, P.SG_IC_SINE, ic)
        else:
            for h, buf in zip(hs, host_in):
                P.sg_init_grids(h, buf)
        ev_step0.record(stream)
        P.sg_step(batch, inputs.BATCH_T_END)
        ev_step1.record(stream)
        P.sg_prolong_combine(batch)  # every member, sharing the batch's intermediates
        ev_comb1.record(stream)
        ext = [(P.sg_reduce(h, -1, P.SG_REDUCE_MIN), P.sg_reduce(h, -1, P.SG_REDUCE_MAX)) for h in hs]
        if host_out is not None:
            for h, buf in zip(hs, host_out):
                P.sg_read(h, P.SG_WHICH_ALL_GRIDS, out=buf)
        return ext

    def updates():
        return sum(P.sg_time(h)[1] * n for h, (_, n) in zip(hs, info))

    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_step0, ev_step1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_comb1 = torch.cuda.Event(enable_timing=True)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_pass()
        upd_per_pass = updates()
        P.sg_set_profiling(batch, True)
        launches0 = sum(P.sg_launch_count(h) for h in all_h)
        step_ms = []
        comb_ms = []
        times = []
        barrier()
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        smi_id = vis.split(",")[local_rank].strip() if vis else str(local_rank)
        with ClockSampler(smi_id) as clk:
            for _ in range(args.steps):
                ev_a.record(stream)
                ext = one_pass()
                ev_b.record(stream)
                ev_b.synchronize()
                times.append(ev_a.elapsed_time(ev_b))
                step_ms.append(ev_step0.elapsed_time(ev_step1))
                comb_ms.append(ev_step1.elapsed_time(ev_comb1))
        barrier()
        launches = sum(P.sg_launch_count(h) for h in all_h) - launches0
        stage_ms, stage_launches = P.sg_profile(batch)
        P.sg_set_profiling(batch, False)
        assert updates() == upd_per_pass
        # shock-capturing bound of the combined solutions (report, not tuned): u0 in [0.5-a, 0.5+a]
        over = max(max(0.0, (0.5 - m.a) - lo, hi - (0.5 + m.a)) for m, (lo, hi) in zip(members, ext))

        # end to end through the C ABI from pinned host buffers, results read back to host
        e2e = None
        if not args.no_e2e:
            host_in, host_out = [], []
            for h, (_, n) in zip(hs, info):
                P.sg_init(h, P.SG_IC_SINE, ics[len(host_in)])
                pin = torch.empty(n, dtype=torch.float32, pin_memory=True).numpy()
                P.sg_read(h, P.SG_WHICH_ALL_GRIDS, out=pin)
                host_in.append(pin)
                host_out.append(torch.empty(n, dtype=torch.float32, pin_memory=True).numpy())
            one_pass(host_in, host_out)  # warm
            barrier()
            et = []
            for _ in range(max(1, args.steps // 2)):
                ev_a.record(stream)
                one_pass(host_in, host_out)
                ev_b.record(stream)
                ev_b.synchronize()
                et.append(ev_a.elapsed_time(ev_b))
            barrier()
            nbytes = sum(n for _, n in info) * 4
            e2e_ms = statistics.mean(et)
            e2e = {"value": upd_per_pass / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes + 16 * len(hs), "ms_per_step": e2e_ms,
                   "api": "sg_init_grids (pinned host) + sg_step + sg_prolong_combine + sg_reduce + sg_read"}

    mean_ms = statistics.mean(times)
    total_ms, total_upd = aggregate(sum(times), upd_per_pass * args.steps, dist, "cuda")

    kname = kernel_name(P, batch)
    for h in [batch] + hs:
        P.sg_destroy(h)
    compare = plain_cfg = None
    if rank == 0 and not args.no_compare:  # untimed: after the timed region and the e2e pass
        with torch.cuda.stream(stream):
            compare = compare_fp64_plain(P, stream, members)
            plain_cfg = fp64_plain_configs(P, stream)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, src = _peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    point_stages = 3 * upd_per_pass * args.steps
    achieved = point_stages * FLOPS_PER_POINT_STAGE_3D / (stage_ms / 1e3) / 1e12
    hbm_gbs = upd_per_pass * args.steps * BYTES_PER_POINT_STEP / (stage_ms / 1e3) / 1e9
    traffic = _stage_traffic(kname, point_stages / max(stage_launches, 1))
    # Step 3 (prolongation + signed combination of every member), timed by the events around it
    fpts, fflops = combine_work(members)
    comb_s = statistics.mean(comb_ms) / 1e3
    comb_gbs = fpts * BYTES_PER_FINEST_POINT / comb_s / 1e9
    comb_tf = fflops / comb_s / 1e12
    roof_comb = {"finest_points": fpts, "bytes_per_finest_point": BYTES_PER_FINEST_POINT, "flops": fflops,
                 "ms": comb_s * 1e3, "achieved_gbs": comb_gbs, "hbm_frac": comb_gbs / float(peaks.get("hbm_gbs", 6800.0)),
                 "achieved_tflops": comb_tf, "alu_frac": comb_tf / alu_peak,
                 "share_of_pass": statistics.mean(comb_ms) / mean_ms,
                 "kernels": "sg_prolong_multi_kernel<float,8>, sg_combine_last_axis_f32x2_kernel"}
    clocks = clk.summary()
    cpu = None
    if pool is not None:
        upd_c, wall_c = oracle_sample(members, pool, cores, nsteps=1)
        pool.close()
        v1, s1, w1 = oracle_single_thread(members)
        cpu = {"value": upd_c / wall_c, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "all %d members, first time step each (FP64 C oracle, one process per core)" % len(members),
               "seconds": wall_c, "cpu_model": _cpu_model(),
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": s1, "seconds": w1}}
    line = {
        "metric": METRIC, "value": total_upd / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "members": len(members), "seed": 2007, "domain": "[0,4]^3",
                   "grids": sum(g for g, _ in info), "points": sum(n for _, n in info),
                   "pt_updates_per_step": upd_per_pass, "t_end": inputs.BATCH_T_END, "cfl": inputs.BATCH_CFL,
                   "exec": "one persistent launch per RK stage over all members, graph replay",
                   "l2": "inputs larger than L2 (3 FP32 state arrays of %.2f GB)" % (sum(n for _, n in info) * 4 / 1e9),
                   "parallelism": "replicas" if world == 1 else "dp%d" % world},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "kernel": kname,
                     "peak_source": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (%s SM clock)" % (nsm, FP32_LANES_PER_SM, sm_max, src)},
        "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": float(peaks.get("hbm_gbs", 6800.0)),
                "frac": hbm_gbs / float(peaks.get("hbm_gbs", 6800.0)), "peak_source": src,
                "bytes_per_point_step": BYTES_PER_POINT_STEP},
        "roofline_combine": roof_comb,
        "breakdown_ms": {"step_to_t_end": statistics.mean(step_ms), "stage_kernels": stage_ms / args.steps,
                         "stage_launches": stage_launches // args.steps,
                         "prolong_combine": statistics.mean(comb_ms)},
        "stepping_rate": upd_per_pass / (statistics.mean(step_ms) / 1e3),
        "bound_overshoot": over,
        "fp64_plain_vs_fp32_batched": compare,
        "fp64_plain_configs": plain_cfg,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _oracle_relax_grid(args):
    dim, nr, nl, lev, nsteps = args
    import oracle
    p = oracle.problem(dim, nr, nl, pde=oracle.VLASOV_BOLTZMANN, eps=1e-3, lo=-5.0, hi=5.0)
    u = oracle.restrict_relax(p, lev)
    t0 = time.perf_counter()
    out, steps, _ = oracle.solve(p, [lev], [u], 100.0, max_steps=nsteps, rule=oracle.DT_CFL, cfl=0.4)
    return out[0].size * steps, time.perf_counter() - t0


def relax_oracle_sample(dim, nr, nl, pool):
    """The oracle on every grid of the sparse set for one time step (the CFL step is the same for
    every grid: each spans the whole domain), grids in parallel; (point-updates, wall seconds)."""
    import oracle
    oracle.build()
    lev, _ = oracle.grid_set(dim, nl)
    jobs = sorted([(dim, nr, nl, [int(x) for x in l], 1) for l in lev], key=lambda j: -sum(j[3]))
    t0 = time.perf_counter()
    res = pool.map(_oracle_relax_grid, jobs, chunksize=1)
    return sum(r[0] for r in res), time.perf_counter() - t0


def run_kinetic(args):
    """Example 5 (Vlasov-Boltzmann relaxation) on one GPU; prints one JSON line."""
    import torch
    import paper_2007_10196_gb300 as P

    dim, nr, nl, t_end, workload = RELAX[args.workload]
    cores = min(os.cpu_count() or 1, 64)
    pool = None if args.no_cpu else mp.get_context("spawn").Pool(cores)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    P.build()
    with torch.cuda.stream(stream):
        h = P.create(dim, nr, nl, P.SG_PDE_VLASOV_BOLTZMANN, precision=P.SG_F32, exec=P.SG_BATCHED,
                     dt_rule=P.SG_DT_CFL, cfl=0.4, lo=-5.0, hi=5.0, cuda_stream=stream.cuda_stream)
    G = P.sg_num_grids(h)
    pts = sum(int(np.prod(P.sg_grid_info(h, g, dim)[1])) for g in range(G))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def one_pass(host_in=None, host_out=None):
        if host_in is None:
            P.sg_init(h, P.SG_IC_RELAX, ())
        else:
            P.sg_init_grids(h, host_in)
        P.sg_step(h, t_end)
        P.sg_prolong_combine(h)
        ent = (P.sg_reduce(h, -1, P.SG_REDUCE_ENTROPY_H2), P.sg_reduce(h, -1, P.SG_REDUCE_ENTROPY_LOG))
        if host_out is not None:
            P.sg_read(h, P.SG_WHICH_ALL_GRIDS, out=host_out)
        return ent

    def timed(fn, n):
        out, ts = None, []
        for _ in range(n):
            flush.zero_()
            ev_a.record(stream)
            out = fn()
            ev_b.record(stream)
            ev_b.synchronize()
            ts.append(ev_a.elapsed_time(ev_b))
        return out, ts

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_pass()
        steps = P.sg_time(h)[1]
        upd = steps * pts
        P.sg_set_profiling(h, True)
        launches0 = P.sg_launch_count(h)
        torch.cuda.synchronize()
        with ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0].strip()) as clk:
            ent, times = timed(one_pass, args.steps)
        torch.cuda.synchronize()
        launches = P.sg_launch_count(h) - launches0
        stage_ms, stage_launches = P.sg_profile(h)
        P.sg_set_profiling(h, False)
        kern, tp, _ = P.sg_stage_config(h)
        e2e = None
        if not args.no_e2e:
            P.sg_init(h, P.SG_IC_RELAX, ())
            host_in = torch.empty(pts, dtype=torch.float32, pin_memory=True).numpy()
            P.sg_read(h, P.SG_WHICH_ALL_GRIDS, out=host_in)
            host_out = torch.empty(pts, dtype=torch.float32, pin_memory=True).numpy()
            _, et = timed(lambda: one_pass(host_in, host_out), max(1, args.steps))
            e2e_ms = statistics.mean(et)
            e2e = {"value": upd / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": pts * 4,
                   "d2h_bytes_per_step": pts * 4 + 16, "ms_per_step": e2e_ms,
                   "api": "sg_init_grids (pinned host) + sg_step + sg_prolong_combine + sg_reduce + sg_read"}
    P.sg_destroy(h)
    peaks, src = _peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    point_stages = 3 * upd * args.steps
    achieved = point_stages * FLOPS_PER_POINT_STAGE_RELAX[dim] / (stage_ms / 1e3) / 1e12
    mean_ms = statistics.mean(times)
    cpu = None
    if pool is not None:
        u_c, w_c = relax_oracle_sample(dim, nr, nl, pool)
        pool.close()
        cpu = {"value": u_c / w_c, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "all %d grids, first time step each (FP64 C oracle, one process per core)" % G,
               "seconds": w_c, "cpu_model": _cpu_model()}
    line = {
        "metric": METRIC, "value": upd * args.steps / (sum(times) / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "dim": dim, "root_cells": nr, "level": nl, "grids": G, "points": pts,
                   "t_end": t_end, "time_steps": steps, "pt_updates_per_step": upd,
                   "l2": "state fits in L2: a 256 MB buffer is written between timed steps"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": None,
                     "kernel": "sg_stage_line_kernel<float,%d,%d>" % (dim, tp // 256),
                     "peak_source": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (%s SM clock)" % (nsm, FP32_LANES_PER_SM, sm_max, src)},
        "breakdown_ms": {"stage_kernels": stage_ms / args.steps, "stage_launches": stage_launches // args.steps},
        "entropy_h2_hlog": ent, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    """The FP64 C oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return
    members = _members(0)
    cores = min(os.cpu_count() or 1, 64)
    pool = mp.get_context("spawn").Pool(cores)
    for _ in range(args.warmup):
        oracle_sample(members[:cores], pool, cores, nsteps=1)
    upd, wall = 0, 0.0
    for _ in range(args.steps):
        u, w = oracle_sample(members, pool, cores, nsteps=1)
        upd += u
        wall += w
    pool.close()
    v = upd / wall
    sample = "all %d members, first time step each (FP64 C oracle, one process per core)" % len(members)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "members": len(members), "seed": 2007},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-plain comparison")
    ap.add_argument("--members", type=int, default=256,
                    help="first M members of the batch only (small cases for profiling)")
    ap.add_argument("--stage-kernel", choices=sorted(STAGE_KERNELS), default="auto",
                    help="the stage kernel of the batch (default: the autotuner's choice)")
    ap.add_argument("--workload", choices=["burgers3d_batch"] + sorted(RELAX), default="burgers3d_batch",
                    help="the benchmark batch (default), or Example 5 (Vlasov-Boltzmann) in 2-D or 4-D")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least three untimed passes
    global N_MEMBERS
    N_MEMBERS = max(1, min(256, args.members))
    rank, world, local_rank = _env_rank()
    if args.workload != "burgers3d_batch":
        if args.impl == "reference" or world > 1:
            raise SystemExit("--workload %s: our arm on one GPU only" % args.workload)
        run_kinetic(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
