#!/usr/bin/env python
"""Benchmark: converged J solves/s of the 3DRT hot path on GB300.

One step = one converged solve of one synthetic slab from J = B: source
update, formal solution (J and, on the first pass, Lambda*), operator
splitting (Jacobi sweeps) and the convergence test, repeated until
max|dJ/J| < tol (Hauschildt & Baron 2011, Sect. 2-2.3).  The opacity is
re-set at the start of every step, so every step rebuilds Lambda*.

Default workload: 65^3 slab, 32 x 32 directions, plain FP64, tol 1e-8.
Inputs are resident on the GPU when the timed region starts; `e2e` repeats
the measurement through the host-pointer API with the host->device copies
of chi, eps and B and the device->host copy of J inside the timed region.

--impl reference times the FP64 CPU oracle (the reference arm) on bounded
samples of the same workload.  Under torchrun (N > 1) every rank solves its
own replica (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 arithmetic of one march step of the closed-form branch, counting an
# FMA as 2 flops: two bilinear interpolations (2 x 7), the trapezoid optical
# depth (2), exp(-x) (16: Tang's table-driven method, 8 FMA), 1 - e (1), the
# division (8: Newton from a reciprocal seed, 4 FMA), w_cur and w_up (2),
# the intensity update (5) and the transmission update (1).
FLOPS_PER_STEP_FP64 = 49
# Replay of the recorded FP64 march, per step: the bilinear interpolation
# of S (one multiply and three FMA, 7 flops) and I += c S (one FMA, 2): five
# FP64 instructions; 8 coefficient bytes streamed from memory.
FLOPS_PER_STEP_FP64_REPLAY = 9
# Peak FP64 of GB300 from the profiling recipe's figure (1.25 TFLOP/s,
# i.e. 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz).
PEAK_FP64_TFLOPS = 1.25
# FP32 arithmetic of one step of the FP32-sweep march (FMA = 2), common to
# both branches of the segment weights: chi interpolation 7, source
# differences S(p) - S_0 20, optical depth 2 and its running sum 1, the
# transmission's argument 1 (plus 1 MUFU ex2), the increment folded with
# the carried low part (2 FMA) 4 and the compensated sum 3: 38.  Closed
# form (x >= 2): e^-x argument, 1 - e, (1 - e)/x, 1 - q, q - e and the two
# transmission products, 7 (plus MUFU ex2, rcp): 45 per step.  Series
# (x < 2): z = x^2, two degree-4 Horner chains (16), x E, z Q, their
# difference and sum and two transmission products, 23 (no MUFU): 61 per
# step.  The branch mix is counted by the library's branch-counting march
# (rt_fs32_branch_counts).
FLOPS_COMMON_FP32 = 38
FLOPS_CLOSED_FP32 = 45
FLOPS_SERIES_FP32 = 61
FLOPS_PER_STEP_FP32 = FLOPS_CLOSED_FP32     # lower bound: every step on the closed form
# Replay of the recorded FP32 march, per voxel-step: 20 flops for the
# interpolated source difference, 5 for the Kahan update; DRAM bytes per
# replayed voxel-step from ncu on the 33^3 slab (4 coefficient bytes, the
# blocks of four steps padded, and the source records)
FLOPS_PER_STEP_FP32_REPLAY = 25
REPLAY32_DRAM_BYTES_PER_STEP = 5.48
# Thread instructions per step of k_fs32d (ncu, 65^3 slab, 32 x 32 directions)
INSTR_PER_STEP_FP32 = 74.2
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz.
PEAK_FP32_TFLOPS = 80.5
# DRAM bytes (read + write) per k_fs64 launch on slab65, from one ncu
# capture of the current kernel: chi, S, B and the direction tables stay
# L2-resident, so the march reads 7.8 MB per launch from DRAM and writes none.
TRAFFIC_FS64_SLAB65 = 7805184
# DRAM bytes per k_fs64rep launch on slab65: 8.35 bytes per replayed step
# (ncu on the 33^3 slab, whose recording fits a capture) x 3.576e9 steps
TRAFFIC_FS64REP_SLAB65 = 29843233564
# The double-float march executes 398 thread instructions per step (ncu,
# slab65); its bound is instruction issue: 152 SMs x 4 schedulers x 32 lanes
# x 2.07 GHz = 40.3e12 thread instructions/s.
INSTR_PER_STEP_DF64 = 398
PEAK_ISSUE_TINST = 40.3

# HBM bandwidth of the GB300s: the driver's measured copy
# (MEASURED_PEAKS.json, hbm_gbs), read at run time when the file is there.
def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6796.5


MEASURED_HBM_GBS = _measured_hbm()

# Outer iterations and Jacobi sweeps of one converged ORACLE solve (Ng every
# 4 iterations, tol 1e-8), from full oracle solves run once on the GPU machine's
# 16 Arm cores: the counts the sampled CPU timings are scaled by.
# 16 Arm cores (Neoverse-V2) of the GPU machine: slab65 converged in 633.4 s
# (18 iterations, 485 sweeps), slab17 in 0.82 s (17 iterations, 416 sweeps).
ORACLE_COUNTS = {
    "slab65": {"iters": 18, "sweeps": 485, "full_solve_s": 633.4, "cores": 16},
    "slab17": {"iters": 17, "sweeps": 416, "full_solve_s": 0.82, "cores": 16},
}
# DRAM bytes (read + write) of one k_jacobi launch on the 129^3 grid, from
# one ncu capture of the current kernel: 478.5 MB read + 16.4 MB written,
# the algorithmic 232 B per voxel.
TRAFFIC_JACOBI_129 = 494896128
# DRAM bytes (read + write) of one k_fs32d launch on slab65, from one ncu
# capture of the current kernel: 27.77 MB read (the padded pair planes,
# the tables) + 0.01 MB written; then everything is served from L2.
TRAFFIC_FS32_SLAB65 = 27855872

# The FP32-sweep iterate stops changing below a relative delta of ~1e-8
# (rounding), so its outer tolerance is at least 5e-8, and Ng extrapolation
# is skipped once delta < 1e-6 (it would amplify that rounding).
TOL_FP32 = 5e-8
NG_MIN_FP32 = 1e-6

WORKLOADS = {
    "slab65": dict(desc="65^3 slab (x,y periodic), chi = 10^(-4+8k/64) exp(0.3 N(0,1)), "
                        "eps = 10^(-4U) per voxel, B = (1+k/64)^4, 32x32 directions, tol 1e-8",
                   make="slab_65"),
    "slab17": dict(desc="17^3 slab, chi = 10^(-4+8k/16)(1+0.2(U-1/2)), eps = 1e-2, B = 1, "
                        "16x16 directions, tol 1e-8",
                   make="slab_small"),
    "slab33": dict(desc="33^3 slab, the 65^3 slab's laws on half the grid, 16x16 directions "
                        "(a small case for profiles)", make="slab_65",
                   kw=dict(n=33, n_theta=16, n_phi=16)),
    "batch": dict(desc="wavelength batch (see --lambdas)", make=None),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_problem(name, lambdas=512):
    from paper_1107_5719_gb300 import workloads as W
    if name == "batch":
        # one wavelength of the batch stands for the per-wavelength cost
        return W.batch_65(n_lambda=lambdas)[0]
    spec = WORKLOADS[name]
    return getattr(W, spec["make"])(**spec.get("kw", {}))


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7],
                                 pcap=f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def smi_id(dev):
    """nvidia-smi selector of a torch device (its UUID; index as fallback)."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(getattr(dev, "index", 0) or 0)


def flush_l2(buf):
    buf.add_(1.0)


def timed_solves(R, p, precision, dev, stream, flush, warmup, steps, max_iter, clk_id=None,
                 groups=0, ng=0, ng_min=0.0, tol=None, fs_method=0, src_order=0):
    """Converged solves of problem `p` through the device API: every step
    re-sets the opacity (Lambda* rebuilt) and J = B, then iterates to
    convergence.  Returns per-step ms, iteration counts, profiling counters,
    the last J (host) and the clock summary."""
    import torch
    chi = torch.from_numpy(p.chi).to(dev)
    eps = torch.from_numpy(p.eps).to(dev)
    Bt = torch.from_numpy(p.B).to(dev)
    Jout = torch.empty_like(Bt)
    ctx = R.rt_create(dev.index, precision)
    try:
        R.rt_set_stream(ctx, stream)
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
        R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
        R.rt_set_epsilon_dev(ctx, eps)
        if groups:
            R.rt_set_direction_groups(ctx, groups)
        if ng:
            R.rt_set_ng(ctx, ng, ng_min)
        if fs_method:
            R.rt_set_fs_method(ctx, fs_method)
        if src_order:
            R.rt_set_source_order(ctx, src_order)
        tol_used = p.tol if tol is None else tol

        def step():
            R.rt_set_opacity_dev(ctx, chi)      # new opacity: Lambda* is rebuilt
            R.rt_set_planck_dev(ctx, Bt)        # J = B
            it, delta, conv = R.rt_solve_dev(ctx, Jout, tol=tol_used, max_iter=max_iter)
            if not conv:
                raise RuntimeError(f"solve did not converge in {it} iterations ({delta:.3e})")
            return it

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        R.rt_reset_stats(ctx)
        R.rt_set_profiling(ctx, True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        times, iters = [], []
        replicas_barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(clk_id) if clk_id is not None else None
        if clk:
            clk.__enter__()
        try:
            for _ in range(steps):
                with torch.cuda.stream(stream):
                    flush_l2(flush)
                stream.synchronize()
                ev0.record(stream)
                iters.append(step())
                ev1.record(stream)
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1))
        finally:
            if clk:
                clk.__exit__(None, None, None)
        torch.cuda.synchronize()
        replicas_barrier()
        st = R.rt_get_stats(ctx)
        return dict(times=times, iters=iters, stats=st, J=Jout.cpu().numpy(),
                    clocks=clk.summary() if clk else None)
    finally:
        R.rt_destroy(ctx)


def march_rate(R, p, precision, dev, stream, launches=5, record=0):
    """Device time and executed steps per launch of the formal solution
    alone: the march itself (record 0), or the replay of the recorded march
    (record -1: the untimed first formal solution records); source
    S = eps B + (1 - eps) B, timed with the library's CUDA events."""
    import torch
    S = torch.from_numpy(p.eps * p.B + (1 - p.eps) * p.B).to(dev)
    J = torch.empty_like(S)
    ctx = R.rt_create(dev.index, precision)
    try:
        R.rt_set_stream(ctx, stream)
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
        R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
        R.rt_set_opacity(ctx, p.chi)
        R.rt_set_epsilon(ctx, p.eps)
        R.rt_set_planck(ctx, p.B)
        R.rt_set_fs_record(ctx, record)
        R.rt_formal_solution_dev(ctx, S, J, None)
        stream.synchronize()
        branches = {}
        if precision == R.RT_FP32_SWEEP and record == 0:
            # outside the timed launches: the branch-counting copy of the march
            n, ser = R.rt_fs32_branch_counts(ctx, S.cpu().numpy())
            branches = {"branch_count_steps": n, "series_steps": ser}
        R.rt_reset_stats(ctx)
        R.rt_set_profiling(ctx, True)
        for _ in range(launches):
            R.rt_formal_solution_dev(ctx, S, J, None)
        st = R.rt_get_stats(ctx)
    finally:
        R.rt_destroy(ctx)
    ms = st["fs_ms"] / max(st["fs_launches"], 1)
    steps = st["steps"] / max(st["fs_launches"], 1)
    return {"ms_per_launch": round(ms, 4), "steps_per_launch": round(steps),
            "fs_steps_per_s": round(steps / (ms / 1e3), 1), **branches}


def record_rate(R, p, dev, stream, reps=2):
    """The recorded FP64 march on problem p: device time of a recording
    formal solution (the march that records, then the replay that gives J)
    and of replays alone, with their steps; new opacities before each
    recording.  Source S = eps B + (1 - eps) B."""
    import torch
    S = torch.from_numpy(p.eps * p.B + (1 - p.eps) * p.B).to(dev)
    chi = torch.from_numpy(p.chi).to(dev)
    J = torch.empty_like(S)
    ctx = R.rt_create(dev.index, R.RT_FP64)
    try:
        R.rt_set_stream(ctx, stream)
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
        R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
        R.rt_set_opacity_dev(ctx, chi)
        R.rt_set_epsilon(ctx, p.eps)
        R.rt_set_planck(ctx, p.B)
        R.rt_formal_solution_dev(ctx, S, J, None)
        stream.synchronize()
        nbytes, valid = R.rt_fs_record_info(ctx)
        out = {"recorded": bool(valid), "bytes": nbytes}
        if not valid:
            return out
        R.rt_set_profiling(ctx, True)
        R.rt_reset_stats(ctx)
        for _ in range(reps):
            R.rt_formal_solution_dev(ctx, S, J, None)
        rep = R.rt_get_stats(ctx)
        R.rt_reset_stats(ctx)
        for _ in range(reps):
            R.rt_set_opacity_dev(ctx, chi)        # the next formal solution records
            R.rt_formal_solution_dev(ctx, S, J, None)
        both = R.rt_get_stats(ctx)
    finally:
        R.rt_destroy(ctx)
    rep_ms = rep["fs_ms"] / reps
    rep_steps = rep["steps"] / reps
    out.update(replay_ms=rep_ms, replay_steps=rep_steps,
               record_ms=both["fs_ms"] / reps - rep_ms,
               record_steps=both["steps"] / reps - rep_steps)
    return out


def replicas_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def e2e_solves(R, p, precision, dev, steps, max_iter, ng=0):
    """Solves/s through the host-pointer API from pinned host buffers, with
    the host->device copies of chi, eps, B and the device->host copy of J in
    the timed region."""
    import ctypes as C
    import torch
    chi_h = torch.from_numpy(p.chi).pin_memory()
    eps_h = torch.from_numpy(p.eps).pin_memory()
    B_h = torch.from_numpy(p.B).pin_memory()
    J_h = torch.empty_like(B_h).pin_memory()
    ctx = R.rt_create(dev.index, precision)
    lib = R.load()
    try:
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
        R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
        if ng:
            R.rt_set_ng(ctx, ng)

        def one():
            for f, t in ((lib.rt_set_opacity, chi_h), (lib.rt_set_epsilon, eps_h),
                         (lib.rt_set_planck, B_h)):
                if f(ctx, t.data_ptr()) != 0:
                    raise RuntimeError(R.rt_last_error(ctx))
            it = C.c_int()
            last = C.c_double()
            if lib.rt_solve(ctx, p.tol, max_iter, 1e-12, 1000, J_h.data_ptr(), C.byref(it),
                            C.byref(last), None, None) != 0:
                raise RuntimeError(R.rt_last_error(ctx))

        one()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        torch.cuda.synchronize()
        return steps / (time.perf_counter() - t0)
    finally:
        R.rt_destroy(ctx)


def init_ranks():
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1107_5719_gb300 import build as B
    B.build()
    from paper_1107_5719_gb300 import rt3d as R
    R.load()
    return ws, rank, local, dev, R


def run_only(args, dev, R):
    """One companion measurement alone (for profiling and diagnostics): its
    JSON object, not a bench line."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    flush = torch.zeros(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    name = args.only
    if name == "os_sweep":
        out = os_sweep_roofline(R, dev, args.os_sweeps)
    elif name == "precision":
        out = precision_check(R, dev, args.precision_n)
    elif name == "batched":
        out = batched_vs_fp64(R, dev, stream, flush, args.batch_lambdas, args.fp64_subset,
                              args.batch_tol, args.ng, args.max_iter)
    elif name == "config5":
        out = config5_iteration(R, dev, stream, args.ng)
    elif name == "march32":
        pw = make_problem(args.workload)
        m32 = march_rate(R, pw, R.RT_FP32_SWEEP, dev, stream)
        r32 = march_rate(R, pw, R.RT_FP32_SWEEP, dev, stream, record=-1)
        probe = R.rt_probe_peaks(dev.index)
        out = {"march": m32, "roofline": fp32_roofline(m32, probe),
               "replay": r32, "replay_roofline": fp32_replay_roofline(r32)}
    else:
        raise SystemExit(f"unknown companion {name}")
    print(json.dumps({"only": name, name: out}), flush=True)


def fp32_replay_roofline(r32):
    """The replay of the recorded FP32 march: per voxel-step the
    interpolated source difference (4 differences, 4 + 4 products and sums:
    20 flops) and the Kahan update (5), 4 coefficient bytes streamed; it
    waits on its loads (ncu: long-scoreboard stalls), so both the HBM
    fraction of its coefficient stream and its FP32 rate are given."""
    ms, n = r32["ms_per_launch"], r32["steps_per_launch"]
    gbs = REPLAY32_DRAM_BYTES_PER_STEP * n / (ms / 1e3) / 1e9
    tfl = FLOPS_PER_STEP_FP32_REPLAY * n / (ms / 1e3) / 1e12
    return {"kernel": "k_fs32rep (replay of the recorded FP32 march)", "bound": "hbm",
            "achieved": round(gbs, 1), "peak": round(MEASURED_HBM_GBS, 1), "unit": "GB/s",
            "frac": round(gbs / MEASURED_HBM_GBS, 4),
            "dram_bytes_per_step": REPLAY32_DRAM_BYTES_PER_STEP,
            "flops_per_step": FLOPS_PER_STEP_FP32_REPLAY,
            "achieved_tflops": round(tfl, 3), "frac_of_fp32_peak": round(tfl / PEAK_FP32_TFLOPS, 4),
            "note": "latency-bound (ncu on the 33^3 slab: long-scoreboard stalls 10 per issue, "
                    "issue 37%); DRAM bytes per step from that capture"}


def fp32_roofline(m32, probe):
    """Roofline of the FP32 march from march_rate's figures: algorithmic
    flops weighted by the counted branch mix, the closed-form-only lower
    bound beside it, and the instruction-issue rate that bounds it."""
    ms, n = m32["ms_per_launch"], m32["steps_per_launch"]
    ser = m32.get("series_steps")
    if ser is None:
        flops = FLOPS_PER_STEP_FP32 * n
    else:
        # the counting march ran the same source: its step count is this one's
        frac_ser = ser / max(m32["branch_count_steps"], 1)
        flops = n * (FLOPS_SERIES_FP32 * frac_ser + FLOPS_CLOSED_FP32 * (1 - frac_ser))
    ach32 = flops / (ms / 1e3) / 1e12
    low = FLOPS_PER_STEP_FP32 * n / (ms / 1e3) / 1e12
    issue = INSTR_PER_STEP_FP32 * n / (ms / 1e3) / 1e12
    return {"kernel": "k_fs32d (FP32-sweep march)", "bound": "alu",
            "achieved": round(ach32, 3), "peak": PEAK_FP32_TFLOPS,
            "unit": "TFLOP/s", "frac": round(ach32 / PEAK_FP32_TFLOPS, 4),
            "flops_per_step": round(flops / max(n, 1), 2),
            "flops_per_step_branches": {"series": FLOPS_SERIES_FP32,
                                        "closed": FLOPS_CLOSED_FP32},
            "series_fraction": round(frac_ser, 4) if ser is not None else None,
            "achieved_closed_form_only": round(low, 3),
            "frac_closed_form_only": round(low / PEAK_FP32_TFLOPS, 4),
            "issue": {"instr_per_step": INSTR_PER_STEP_FP32,
                      "achieved_tinst_s": round(issue, 2),
                      "peak_tinst_s": PEAK_ISSUE_TINST,
                      "frac": round(issue / PEAK_ISSUE_TINST, 4)},
            "peak_source": "unit counts and clock: 152 SMs x 128 lanes x 2 "
                           "flops x 2.07 GHz",
            "peak_measured": round(probe["fp32_tflops"], 3)
            if probe["fp32_tflops"] else None,
            "frac_of_measured": round(ach32 / probe["fp32_tflops"], 4)
            if probe["fp32_tflops"] else None,
            "traffic": TRAFFIC_FS32_SLAB65,
            "note": "ncu: bound by instruction issue (76.5% of issue slots; "
                    "74.2 thread instructions per step, 41.5 of them FP32 "
                    "arithmetic), L1 66%"}


def run_ours(args):
    import torch
    from paper_1107_5719_gb300 import replicas as RP
    ws, rank, local, dev, R = init_ranks()
    if args.only:
        return run_only(args, dev, R)
    if args.workload.startswith("batch"):
        return run_batch(args, ws, rank, dev, R)
    p = make_problem(args.workload)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.zeros(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MiB > L2

    r64 = timed_solves(R, p, R.RT_FP64, dev, stream, flush, args.warmup, args.steps,
                       args.max_iter, clk_id=smi_id(dev), ng=args.ng)
    st = r64["stats"]
    my_ms = float(sum(r64["times"]))
    solves_per_s, total_ms = RP.weak_throughput(args.steps, my_ms)
    ms_per_step = total_ms / args.steps
    fs_per_solve = st["fs_launches"] / args.steps
    pairs = p.nvox * p.ndir
    vd_per_s = RP.sum_over_ranks(st["fs_launches"] * pairs) / (total_ms / 1e3)
    steps_per_s = RP.sum_over_ranks(st["steps"]) / (total_ms / 1e3)

    # measured arithmetic peaks (FMA chains), reported beside the unit-count peaks
    try:
        probe = R.rt_probe_peaks(dev.index)
    except R.RtError:
        probe = {"fp64_tflops": None, "fp32_tflops": None}

    # dominant kernel: the replay of the recorded FP64 march (every formal
    # solution of a solve evaluates J from the recording; the first one
    # also records it), timed alone; the recording march beside it
    rec = record_rate(R, p, dev, stream)
    iters = st["iterations"] / args.steps
    if rec["recorded"]:
        rep_ms, rep_steps = rec["replay_ms"], rec["replay_steps"]
        achieved = FLOPS_PER_STEP_FP64_REPLAY * rep_steps / (rep_ms / 1e3) / 1e12
        roofline = {"kernel": "k_fs64rep (replay of the recorded FP64 march)", "bound": "alu",
                    "achieved": round(achieved, 4), "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(achieved / PEAK_FP64_TFLOPS, 4),
                    "traffic": TRAFFIC_FS64REP_SLAB65 if args.workload == "slab65" else None,
                    "flops_per_step": FLOPS_PER_STEP_FP64_REPLAY,
                    "fp64_instructions_per_step": 5,
                    "coefficient_bytes_per_step": 8,
                    "hbm_gbs_coefficients": round(8 * rep_steps / (rep_ms / 1e3) / 1e9, 1),
                    "steps_per_launch": round(rep_steps),
                    "ms_per_launch": round(rep_ms, 4),
                    "share_of_step": round(rep_ms * iters / (my_ms / args.steps), 4),
                    "record": {"kernel": "k_fs64<true> (the march, recording)",
                               "ms": round(rec["record_ms"], 3),
                               "steps": round(rec["record_steps"]),
                               "achieved_tflops": round(FLOPS_PER_STEP_FP64 * rec["record_steps"]
                                                        / (rec["record_ms"] / 1e3) / 1e12, 4),
                               "flops_per_step": FLOPS_PER_STEP_FP64,
                               "bytes_held": rec["bytes"]}}
    else:
        fs_ms = st["fs_ms"] / max(st["fs_launches"], 1)
        steps_per_launch = st["steps"] / max(st["fs_launches"], 1)
        achieved = FLOPS_PER_STEP_FP64 * steps_per_launch / (fs_ms / 1e3) / 1e12
        roofline = {"kernel": "k_fs64 (formal-solution march, FP64)", "bound": "alu",
                    "achieved": round(achieved, 4), "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(achieved / PEAK_FP64_TFLOPS, 4), "traffic": None,
                    "flops_per_step": FLOPS_PER_STEP_FP64,
                    "steps_per_launch": round(steps_per_launch),
                    "ms_per_launch": round(fs_ms, 4),
                    "share_of_step": round(st["fs_ms"] / my_ms, 4)}
    roofline.update({
        "peak_source": "unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz",
        "peak_measured": round(probe["fp64_tflops"], 4) if probe["fp64_tflops"] else None,
        "frac_of_measured": round(achieved / probe["fp64_tflops"], 4)
        if probe["fp64_tflops"] else None,
        "peak_measured_source": "rt_probe_peaks: register-resident DFMA chains on every "
                                "SM, CUDA events"})

    # the FP32-sweep form of the same workload on the same GPU: converged
    # solves of the form as created (finishing stage from delta < 1e-6),
    # at the headline's tolerance; the march's own rate from FP32-only
    # formal solutions (the finishing stage marches a source change)
    fp32 = None
    if args.fp32_steps > 0:
        r32 = timed_solves(R, p, R.RT_FP32_SWEEP, dev, stream, flush, 1, args.fp32_steps,
                           args.max_iter, ng=args.ng, ng_min=NG_MIN_FP32, tol=p.tol)
        st32 = r32["stats"]
        ms32 = float(sum(r32["times"]))
        m32 = march_rate(R, p, R.RT_FP32_SWEEP, dev, stream)
        rep32 = march_rate(R, p, R.RT_FP32_SWEEP, dev, stream, record=-1)
        fp32 = {"value": round(RP.weak_throughput(args.fp32_steps, ms32)[0], 6), "unit": "solves/s",
                "form": "FP32 sweep + finishing stage from delta < 1e-6 (the default)",
                "ms_per_step": round(ms32 / args.fp32_steps, 3),
                "iters_per_solve": st32["iterations"] / args.fp32_steps,
                "march_launches_per_solve": st32["fs_launches"] / args.fp32_steps,
                "tol": p.tol,
                "max_rel_dev_from_fp64_J": float(np.max(np.abs(r32["J"] - r64["J"]) / r64["J"])),
                "speedup_vs_fp64": round(my_ms / args.steps / (ms32 / args.fp32_steps), 3),
                "march": m32}
        fp32["roofline"] = fp32_roofline(m32, probe)
        fp32["replay"] = rep32
        fp32["replay_roofline"] = fp32_replay_roofline(rep32)

    # the double-float form (FP64-accurate march on the FP32 pipes)
    df64 = None
    if args.df64_steps > 0:
        rdf = timed_solves(R, p, R.RT_DF64, dev, stream, flush, 1, args.df64_steps,
                           args.max_iter, ng=args.ng)
        stdf = rdf["stats"]
        msdf = float(sum(rdf["times"]))
        # the march (every formal solution of an unrecorded context) and the
        # replay of its recording, each timed alone
        mdf = march_rate(R, p, R.RT_DF64, dev, stream)
        repdf = march_rate(R, p, R.RT_DF64, dev, stream, record=-1)
        eq = FLOPS_PER_STEP_FP64 * mdf["steps_per_launch"] / (mdf["ms_per_launch"] / 1e3) / 1e12
        df64 = {"value": round(RP.weak_throughput(args.df64_steps, msdf)[0], 6), "unit": "solves/s",
                "form": "double-float, the march recorded once per opacity and replayed",
                "ms_per_step": round(msdf / args.df64_steps, 3),
                "iters_per_solve": stdf["fs_launches"] / args.df64_steps,
                "march": mdf, "replay": repdf,
                "march_fp64_equivalent_tflops": round(eq, 3),
                "march_fp64_equivalent_frac_of_fp64_peak": round(eq / PEAK_FP64_TFLOPS, 3),
                "max_rel_dev_from_fp64_J": float(np.max(np.abs(rdf["J"] - r64["J"]) / r64["J"])),
                "speedup_vs_fp64": round(my_ms / args.steps / (msdf / args.df64_steps), 3)}
        issue = INSTR_PER_STEP_DF64 * mdf["steps_per_launch"] / (mdf["ms_per_launch"] / 1e3) / 1e12
        df64["roofline"] = {"kernel": "k_fsdf (double-float march)", "bound": "issue",
                            "achieved": round(issue, 3), "peak": PEAK_ISSUE_TINST,
                            "unit": "T thread-instructions/s",
                            "frac": round(issue / PEAK_ISSUE_TINST, 4),
                            "instructions_per_step": INSTR_PER_STEP_DF64}

    # the short-characteristics formal solution (O(1) per pair, FP64): a
    # different discretisation of the same problem, reported beside it
    short = None
    if args.sc_steps > 0:
        rsc = timed_solves(R, p, R.RT_FP64, dev, stream, flush, 1, args.sc_steps,
                           args.max_iter, ng=args.ng, fs_method=R.RT_FS_SHORT)
        stsc = rsc["stats"]
        mssc = float(sum(rsc["times"]))
        short = {"value": round(RP.weak_throughput(args.sc_steps, mssc)[0], 6), "unit": "solves/s",
                 "ms_per_step": round(mssc / args.sc_steps, 3),
                 "iters_per_solve": stsc["fs_launches"] / args.sc_steps,
                 "ms_per_fs_launch": round(stsc["fs_ms"] / max(stsc["fs_launches"], 1), 4),
                 "pairs_per_s_fs": round(stsc["fs_launches"] * pairs / (stsc["fs_ms"] / 1e3), 1)
                 if stsc["fs_ms"] else None,
                 "max_rel_diff_from_long_J": float(np.max(np.abs(rsc["J"] - r64["J"]) / r64["J"])),
                 "median_rel_diff_from_long_J": float(np.median(np.abs(rsc["J"] - r64["J"]) / r64["J"])),
                 "note": "different discretisation (I interpolated on each plane)"}
        rscd = timed_solves(R, p, R.RT_DF64, dev, stream, flush, 1, args.sc_steps,
                            args.max_iter, ng=args.ng, fs_method=R.RT_FS_SHORT)
        stscd = rscd["stats"]
        msscd = float(sum(rscd["times"]))
        short["double_float"] = {
            "value": round(RP.weak_throughput(args.sc_steps, msscd)[0], 6), "unit": "solves/s",
            "ms_per_step": round(msscd / args.sc_steps, 3),
            "ms_per_fs_launch": round(stscd["fs_ms"] / max(stscd["fs_launches"], 1), 4),
            "max_rel_dev_from_fp64_short_J": float(np.max(np.abs(rscd["J"] - rsc["J"]) / rsc["J"]))}

    # the parabolic-source variant of the FP64 march (second-order source)
    para = None
    if args.para_steps > 0:
        rpa = timed_solves(R, p, R.RT_FP64, dev, stream, flush, 1, args.para_steps,
                           args.max_iter, ng=args.ng, src_order=R.RT_SRC_PARABOLIC)
        stpa = rpa["stats"]
        mspa = float(sum(rpa["times"]))
        para = {"value": round(RP.weak_throughput(args.para_steps, mspa)[0], 6), "unit": "solves/s",
                "form": "FP64, the march recorded once per opacity and replayed",
                "ms_per_step": round(mspa / args.para_steps, 3),
                "iters_per_solve": stpa["fs_launches"] / args.para_steps,
                "ms_per_fs_launch": round(stpa["fs_ms"] / max(stpa["fs_launches"], 1), 4),
                "fs_steps_per_s": round(stpa["steps"] / (stpa["fs_ms"] / 1e3), 1)
                if stpa["fs_ms"] else None,
                "max_rel_diff_from_linear_J": float(np.max(np.abs(rpa["J"] - r64["J"]) / r64["J"])),
                "median_rel_diff_from_linear_J": float(np.median(np.abs(rpa["J"] - r64["J"]) / r64["J"])),
                "note": "different discretisation (second-order source)"}

    budget = Budget(args.budget_s)
    precision = precision_check(R, dev, args.precision_n) if args.precision_n > 0 else None
    os_sweep = os_sweep_roofline(R, dev, args.os_sweeps) if args.os_sweeps > 0 else None
    batched = None
    if args.batch_lambdas > 0 and budget.left() > 0:
        batched = batched_vs_fp64(R, dev, stream, flush, args.batch_lambdas, args.fp64_subset,
                                  args.batch_tol, args.ng, args.max_iter)
    config5 = None
    if args.config5 and budget.left() > 0:
        config5 = config5_iteration(R, dev, stream, args.ng)
    elif args.config5:
        config5 = {"skipped": f"time budget of {args.budget_s:.0f} s used up"}

    e2e = None
    if args.e2e_steps > 0:
        v = e2e_solves(R, p, R.RT_FP64, dev, args.e2e_steps, args.max_iter, args.ng)
        e2e = {"value": round(RP.sum_over_ranks(v), 6), "unit": "solves/s",
               "h2d_bytes_per_step": 3 * p.nvox * 8, "d2h_bytes_per_step": p.nvox * 8,
               "steps": args.e2e_steps, "api": "rt_set_opacity/epsilon/planck + rt_solve (host)"}

    line = {
        "metric": "converged J solves/s", "value": round(solves_per_s, 6), "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + ": " + WORKLOADS[args.workload]["desc"],
                   "nx": p.nx, "ny": p.ny, "nz": p.nz, "ndir": p.ndir, "tol": p.tol,
                   "precision": "FP64", "parallelism": f"replicas x{ws}",
                   "l2": "flushed between steps (512 MiB write)",
                   "lstar": "rebuilt every step",
                   "ng_acceleration": f"every {args.ng} iterations" if args.ng else "off"},
        "voxel_dir_updates_per_s": round(vd_per_s, 1),
        "march_steps_per_s": round(steps_per_s, 1),
        "iters_per_solve": round(fs_per_solve, 3),
        "roofline": roofline,
        "fp32_sweep": fp32,
        "df64": df64,
        "short_characteristics": short,
        "parabolic_source": para,
        "precision_eps1e-6": precision,
        "fp32_batched": batched,
        "os_sweep": os_sweep,
        "config5_iteration": config5,
        "measured_peaks": probe,
        "gpu_launches": int(st["launches"]),
        "clocks": r64["clocks"],
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        counts = ORACLE_COUNTS.get(args.workload, ORACLE_COUNTS["slab65"])
        line["cpu_baseline"] = cpu_baseline(p, counts["iters"], counts["sweeps"], args.cpu_seconds)
        line["cpu_baseline"]["extrapolated"] = True
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


class Budget:
    """Wall-clock budget of the companion measurements (seconds since the
    bench started); the last ones are skipped, and say so, when it is used
    up."""

    T0 = time.time()

    def __init__(self, seconds):
        self.seconds = seconds

    def left(self):
        return self.seconds - (time.time() - Budget.T0)


def _ctx_for(R, dev, p, precision):
    ctx = R.rt_create(dev.index, precision)
    R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
    R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
    R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
    R.rt_set_opacity(ctx, p.chi)
    R.rt_set_epsilon(ctx, p.eps)
    R.rt_set_planck(ctx, p.B)
    return ctx


def precision_check(R, dev, n=33):
    """Precision form at eps = 1e-6 (strong scattering): n x n x 129 slab
    with the 64 x 64 directions of the 129^3 configuration.  The FP32-sweep
    context as created (finishing stage from delta < 1e-6, Ng every 4)
    is solved to tol 1e-8; the reference continues the same iteration in
    double-float (FP64-accurate march) to delta < 1e-9, i.e. to the FP64
    fixed point within ~70 x 1e-9 at this eps."""
    from paper_1107_5719_gb300 import workloads as W
    pc = W.slab_precision(n=n, nzz=129, n_theta=64, n_phi=64)
    shape = (pc.nz, pc.ny, pc.nx)
    ctx = _ctx_for(R, dev, pc, R.RT_FP32_SWEEP)
    try:
        R.rt_set_ng(ctx, 4, NG_MIN_FP32)
        t0 = time.time()
        r = R.rt_solve(ctx, shape, tol=1e-8, max_iter=5000)
        t32 = time.time() - t0
        d = np.asarray(r["deltas"])
        n32 = int(np.argmax(d < 1e-6)) + 1 if np.any(d < 1e-6) else int(r["iters"])
        R.rt_set_precision(ctx, R.RT_DF64)
        R.rt_set_ng(ctx, 4, 0.0)
        t0 = time.time()
        rr = R.rt_solve(ctx, shape, tol=1e-9, max_iter=3000)
        tref = time.time() - t0
    finally:
        R.rt_destroy(ctx)
    err = np.abs(r["J"] - rr["J"]) / rr["J"]
    return {"workload": f"{n}x{n}x129 slab, strong-scattering chi law (tau 1e-4..1e4), eps = 1e-6, "
                        "B = 1, 64x64 directions",
            "fp32_default": {"form": "FP32 sweep, finishing stage from delta < 1e-6, Ng every 4",
                             "tol": 1e-8, "converged": bool(r["converged"]), "iters": int(r["iters"]),
                             "fp32_iters": n32, "finishing_iters": int(r["iters"]) - n32,
                             "s": round(t32, 2), "max_rel_err": float(err.max()),
                             "median_rel_err": float(np.median(err))},
            "reference": {"form": "same iteration continued in double-float to delta < 1e-9",
                          "iters": int(rr["iters"]), "converged": bool(rr["converged"]),
                          "s": round(tref, 2)},
            "target": 1e-6}


def os_sweep_roofline(R, dev, sweeps=200):
    """Operator-splitting Jacobi sweep (k_jacobi) alone: 232 algorithmic
    bytes per voxel and sweep (26 coefficients, r and J read, J written;
    J's stencil neighbours come from cache), timed over `sweeps` sweeps with
    CUDA events (host-driven sweeps, no graph), on the 65^3 slab (its 64 MB
    per sweep stays in the 129 MB L2) and on 129^3 (498 MB per sweep, from
    HBM).  Directions do not enter the sweep: 2x2 directions build Lambda*."""
    import torch
    from paper_1107_5719_gb300 import workloads as W
    out = {}
    for name, n in (("slab65", 65), ("slab129", 129)):
        p = W.slab_65(n=n, n_theta=2, n_phi=2)
        ctx = _ctx_for(R, dev, p, R.RT_FP64)
        try:
            R.rt_set_graphs(ctx, 0)
            Bt = torch.from_numpy(p.B).to(dev)
            Jfs, Jn = torch.empty_like(Bt), torch.empty_like(Bt)
            R.rt_formal_solution_dev(ctx, Bt, Jfs, None)
            R.rt_os_step_dev(ctx, Jfs, Bt, Jn, 0.0, 20)
            torch.cuda.synchronize()
            R.rt_reset_stats(ctx)
            R.rt_set_profiling(ctx, True)
            R.rt_os_step_dev(ctx, Jfs, Bt, Jn, 0.0, sweeps)
            st = R.rt_get_stats(ctx)
        finally:
            R.rt_destroy(ctx)
        ms = st["jacobi_ms"] / max(st["jacobi_launches"], 1)
        gbs = 232.0 * p.nvox / (ms / 1e3) / 1e9
        out[name] = {"voxels": p.nvox, "bytes_per_sweep": 232 * p.nvox, "ms_per_sweep": round(ms, 5),
                     "achieved_GBps": round(gbs, 1),
                     "frac_of_hbm": round(gbs / MEASURED_HBM_GBS, 4)}
    tfl = 2 * 26 * out["slab129"]["voxels"] / (out["slab129"]["ms_per_sweep"] / 1e3) / 1e12
    out["roofline"] = {"kernel": "k_jacobi (operator-splitting sweep, FP64), 129^3",
                       "bound": "alu", "achieved": round(tfl, 4), "peak": PEAK_FP64_TFLOPS,
                       "unit": "TFLOP/s", "frac": round(tfl / PEAK_FP64_TFLOPS, 4),
                       "flops_per_voxel": 52, "traffic": TRAFFIC_JACOBI_129,
                       "hbm_GBps": out["slab129"]["achieved_GBps"],
                       "hbm_frac": out["slab129"]["frac_of_hbm"],
                       "peak_source": "unit counts and clock (FP64); HBM: measured copy "
                                      "bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                       "note": "ncu: FP64 pipe 90% busy (26 stencil FMAs and the "
                               "convergence test, ~36 FP64 instructions per voxel), DRAM "
                               "traffic = the algorithmic 232 B per voxel, so the FP64 pipe, "
                               "not HBM, bounds the sweep on this GPU; slab65's sweep is "
                               "L2-resident"}
    return out


def batched_vs_fp64(R, dev, stream, flush, nl, nsub, tol, ng, max_iter):
    """FP32-batched form against FP64 plain on the same GPU.  The batch: all
    nl wavelengths of the 512-point configuration (65^3, 32x32 directions,
    chi x 10^(-2+4U), eps 10^(-5+5U) per wavelength), FP32 sweep with the
    default finishing stage, tol 1e-8, one fused march launch per outer
    iteration and the OS step of all active wavelengths as one CUDA graph.
    FP64 plain: nsub wavelengths spread evenly over the batch (every
    nl/nsub-th), one rt_solve each at the same tolerance; the ratio is the
    batch's wavelength-solves/s over FP64 plain's on that subset, and each
    subset wavelength's batch J is compared with its FP64 J."""
    import torch
    from paper_1107_5719_gb300 import workloads as W
    probs = W.batch_65(n_lambda=nl)
    t0 = time.time()
    bt = R.rt_batch_create(probs, device=dev.index, precision=R.RT_FP32_SWEEP)
    t_create = time.time() - t0
    sub = list(range(0, nl, max(1, nl // nsub)))[:nsub]
    try:
        R.rt_batch_set_ng(bt, ng, NG_MIN_FP32)
        R.rt_batch_set_stream(bt, stream)
        R.rt_batch_solve(bt, len(probs), tol=tol, max_iter=1)              # warm-up
        R.rt_batch_reset(bt, rebuild_lstar=True)
        R.rt_batch_reset_stats(bt)
        R.rt_batch_set_profiling(bt, True)
        with torch.cuda.stream(stream):
            flush_l2(flush)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(smi_id(dev)) as clk:
            e0.record(stream)
            rb = R.rt_batch_solve(bt, len(probs), tol=tol, max_iter=max_iter)
            e1.record(stream)
            e1.synchronize()
        msb = e0.elapsed_time(e1)
        stb = R.rt_batch_get_stats(bt)
        Jb = {i: R.rt_batch_get_J(bt, i, (probs[i].nz, probs[i].ny, probs[i].nx)) for i in sub}
    finally:
        R.rt_batch_destroy(bt)
    vb = len(probs) / (msb / 1e3)
    # FP64 plain on the subset
    per, ms64 = [], 0.0
    for i in sub:
        p = probs[i]
        ctx = _ctx_for(R, dev, p, R.RT_FP64)
        try:
            if ng:
                R.rt_set_ng(ctx, ng)
            R.rt_set_stream(ctx, stream)
            e0.record(stream)
            r = R.rt_solve(ctx, (p.nz, p.ny, p.nx), tol=tol, max_iter=max_iter)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        finally:
            R.rt_destroy(ctx)
        ms64 += ms
        per.append({"lambda": i, "chi_scale_eps": p.name.split(": ")[1],
                    "fp64_iters": int(r["iters"]), "fp64_s": round(ms / 1e3, 2),
                    "batch_iters": int(rb["iters"][i]),
                    "max_rel_err_vs_fp64": float(np.max(np.abs(Jb[i] - r["J"]) / r["J"]))})
    v64 = len(sub) / (ms64 / 1e3)
    march_steps = stb["steps"]
    ach = FLOPS_PER_STEP_FP32 * march_steps / (stb["fs_ms"] / 1e3) / 1e12 if stb["fs_ms"] else None
    return {"value": round(vb, 6), "unit": "wavelength-solves/s",
            "workload": f"{nl} wavelengths x 65^3, chi x 10^(-2+4U), eps 10^(-5+5U), 32x32 directions",
            "form": "FP32 sweep, finishing stage from delta < 1e-6 (one double-float formal "
                    "solution, then FP32 marches of the source change), FP64 J/Lambda*/OS",
            "tol": tol, "converged": bool(rb["converged"]), "s": round(msb / 1e3, 2),
            "create_s": round(t_create, 1),
            "iters_mean": float(np.mean(rb["iters"])), "iters_max": int(np.max(rb["iters"])),
            "outer_iterations": int(stb["iterations"]),
            "host_syncs_per_iteration": round(stb["host_syncs"] / max(stb["iterations"], 1), 3),
            "fused_march_s": round(stb["fs_ms"] / 1e3, 2),
            "os_graph_s": round(stb["jacobi_ms"] / 1e3, 2),
            "march_steps_per_s": round(march_steps / (stb["fs_ms"] / 1e3), 1) if stb["fs_ms"] else None,
            "march_roofline": {"bound": "alu", "achieved": round(ach, 3) if ach else None,
                               "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                               "frac": round(ach / PEAK_FP32_TFLOPS, 4) if ach else None,
                               "note": "all march launches of the solve (fused FP32 and the "
                                       "finishing stage), 45 FP32 flops per executed step: "
                                       "the closed-form count, a lower bound (series steps "
                                       "do 61)"},
            "clocks": clk.summary(),
            "fp64_plain_subset": {"lambdas": sub, "value": round(v64, 6), "unit": "wavelength-solves/s",
                                  "s": round(ms64 / 1e3, 2), "per_lambda": per},
            "vs_fp64_plain_same_wavelengths": round(vb / v64, 3),
            "max_rel_err_vs_fp64": max(q["max_rel_err_vs_fp64"] for q in per),
            "target": 1e-6}


def config5_iteration(R, dev, stream, ng):
    """The uneven batch at its configured 64x64 directions (8 x 257^2x129,
    24 x 129^3, 32 x 65^3; strong-scattering chi law x 10^(-2+4U), eps
    10^(-5+5U)): ONE outer iteration of the FP32-batched solve from J = B
    (the fused march over all 64 problems, Lambda* of every problem, the OS
    graph, the convergence tests), timed with CUDA events.  A converged
    solve is extrapolated from it with the iteration counts measured on the
    same batch at 16x8 directions and says so."""
    import torch
    from paper_1107_5719_gb300 import workloads as W
    t0 = time.time()
    probs = W.batch_uneven()
    bt = R.rt_batch_create(probs, device=dev.index, precision=R.RT_FP32_SWEEP)
    t_create = time.time() - t0
    try:
        R.rt_batch_set_ng(bt, ng, NG_MIN_FP32)
        # one iteration of all 64 problems: their recordings could not be held
        # together (a 65^3 problem's at 64x64 directions alone takes 156 GB),
        # so every problem marches
        R.rt_batch_set_fs_record(bt, 0)
        R.rt_batch_set_stream(bt, stream)
        R.rt_batch_reset_stats(bt)
        R.rt_batch_set_profiling(bt, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        R.rt_batch_solve(bt, len(probs), tol=1e-8, max_iter=1)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        st = R.rt_batch_get_stats(bt)
    finally:
        R.rt_batch_destroy(bt)
    ach = FLOPS_PER_STEP_FP32 * st["steps"] / (st["fs_ms"] / 1e3) / 1e12
    # iterations per class measured at 16x8 directions (FP32 sweep, double-float
    # finish from delta < 1e-6, tol 1e-8): mean 293 / 134 / 35
    iters = {257: 293, 129: 134, 65: 35}
    w = [p.nvox * p.nz for p in probs]
    it_w = sum(wi * iters[p.nx] for wi, p in zip(w, probs)) / sum(w)
    march_ms = st["fs_ms"]
    return {"workload": "8 x 257x257x129 + 24 x 129^3 + 32 x 65^3, 64x64 directions, "
                        "chi x 10^(-2+4U), eps 10^(-5+5U)",
            "voxels": int(sum(p.nvox for p in probs)), "create_s": round(t_create, 1),
            "first_iteration_ms": round(ms, 1), "fused_march_ms": round(march_ms, 1),
            "os_graph_ms": round(st["jacobi_ms"], 1),
            "lambda_star_and_rest_ms": round(ms - march_ms - st["jacobi_ms"], 1),
            "march_steps": int(st["steps"]),
            "march_steps_per_s": round(st["steps"] / (march_ms / 1e3), 1),
            "march_roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": PEAK_FP32_TFLOPS,
                               "unit": "TFLOP/s", "frac": round(ach / PEAK_FP32_TFLOPS, 4),
                               "note": "45 FP32 flops per executed step: the closed-form "
                                       "count, a lower bound (series steps do 61)"},
            "converged_s_extrapolated": round(march_ms / 1e3 * it_w, 0),
            "extrapolation": "fused march time x the march-work-weighted mean of the iteration "
                             "counts measured at 16x8 directions (293 / 134 / 35 for the three "
                             "sizes); EXTRAPOLATED, not run"}



def run_batch(args, ws, rank, dev, R):
    """Wavelength batch (FP32 sweep, fused launch): converged
    wavelength-solves/s; each rank solves its share of the wavelengths."""
    import torch
    from paper_1107_5719_gb300 import replicas as RP
    from paper_1107_5719_gb300 import workloads as W
    nl = args.lambdas
    mine = RP.shard([1] * nl, ws, rank)
    probs_all = W.batch_65(n_lambda=nl)
    probs = [probs_all[i] for i in mine]
    b = R.rt_batch_create(probs, device=dev.index, precision=R.RT_FP32_SWEEP)
    if args.ng:
        R.rt_batch_set_ng(b, args.ng, NG_MIN_FP32)
    stream = torch.cuda.Stream(device=dev)
    R.rt_batch_set_stream(b, stream)
    flush = torch.zeros(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    try:
        def step():
            R.rt_batch_reset(b, rebuild_lstar=True)
            r = R.rt_batch_solve(b, len(probs), tol=TOL_FP32, max_iter=args.max_iter)
            if not r["converged"]:
                raise RuntimeError("batch did not converge")
            return r
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        R.rt_batch_reset_stats(b)
        R.rt_batch_set_profiling(b, True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        times = []
        replicas_barrier()
        with ClockSampler(smi_id(dev)) as clk:
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush_l2(flush)
                stream.synchronize()
                ev0.record(stream)
                r = step()
                ev1.record(stream)
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1))
        replicas_barrier()
        st = R.rt_batch_get_stats(b)
    finally:
        R.rt_batch_destroy(b)
    my_ms = float(sum(times))
    value, total_ms = RP.weak_throughput(args.steps * len(probs), my_ms)
    fs_ms = st["fs_ms"] / max(st["fs_launches"], 1)
    line = {"metric": "converged J solves/s (wavelength points)", "value": round(value, 6),
            "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 march / f64 J, Lambda*, OS",
            "data": "synthetic",
            "config": {"workload": f"batch: {nl} wavelengths x 65^3 slab, chi x 10^(-2+4U), "
                                   f"eps 10^(-5+5U), 32x32 directions, tol {TOL_FP32:g}",
                       "precision": "FP32 sweep", "parallelism": f"wavelength shards x{ws}",
                       "l2": "flushed between steps (512 MiB write)",
                       "lstar": "rebuilt every step"},
            "march_steps_per_s": round(RP.sum_over_ranks(st["steps"]) / (total_ms / 1e3), 1),
            "fused_fs_ms_per_launch": round(fs_ms, 3),
            "fused_fs_steps_per_s": round(st["steps"] / (st["fs_ms"] / 1e3), 1) if st["fs_ms"] else None,
            "iters_max": int(np.max(r["iters"])), "iters_mean": float(np.mean(r["iters"])),
            "gpu_launches": int(st["launches"]), "clocks": clk.summary(), "e2e": None}
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_baseline(p, iters, sweeps, seconds, seed=0):
    """The oracle as it stands on this host's cores, on a bounded sample:
    J at sampled voxels (all directions) gives the formal-solution cost per
    voxel; one Jacobi sweep on the full grid gives the sweep cost; both are
    scaled by the measured iteration and sweep counts of one solve."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    S = p.eps * p.B + (1 - p.eps) * p.B
    n = 16
    t_vox = None
    total = 0
    t_all = 0.0
    while True:
        vox = rng.integers(0, p.nvox, n)
        t0 = time.perf_counter()
        oracle.mean_intensity_at(p, S, vox, nthreads=cores)
        dt = time.perf_counter() - t0
        total += n
        t_all += dt
        t_vox = t_all / total
        if t_all > 0.5 * seconds or total >= p.nvox:
            break
        n = int(min(max(n * 2, 0.25 * seconds / max(t_vox, 1e-9)), p.nvox))
    L = np.zeros((27, p.nz, p.ny, p.nx))
    L[13] = 0.5
    t0 = time.perf_counter()
    oracle.os_step(p, L, p.B, p.B, tol_inner=0.0, max_sweeps=1)
    t_sweep = time.perf_counter() - t0
    t_solve = iters * (t_vox * p.nvox) + sweeps * t_sweep
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"J at {total} random voxels x {p.ndir} directions ({t_all:.1f} s on "
                      f"{cores} threads) and one full-grid Jacobi sweep ({t_sweep:.2f} s), "
                      f"scaled to {iters:.0f} formal solutions and {sweeps:.0f} sweeps per solve"}


def oracle_full_solve(p, ng):
    """One full converged oracle solve (Ng every `ng` iterations) on this
    host's cores: seconds, iterations, Jacobi sweeps."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.solve(p, tol=p.tol, max_iter=1000, ng_period=ng, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"s": round(dt, 2), "solves_per_s": 1.0 / dt, "iters": int(r["iters"]),
            "sweeps": int(np.sum(r["sweeps"])), "converged": bool(r["converged"]), "cores": cores}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on this host's cores.

    Every step is one bounded sample of the bench workload (J at sampled
    voxels with all directions, plus one full-grid Jacobi sweep), timed;
    the line's value extrapolates the sampled costs to one converged solve
    with the oracle's own iteration and sweep counts (ORACLE_COUNTS, from
    full oracle solves on the GPU machine's cores) and says so
    ("extrapolated": true); ms_per_step is the sample's own wall time.  A
    full converged oracle solve of the 17^3 slab is run and timed too."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    p = make_problem(args.workload, args.lambdas)
    counts = ORACLE_COUNTS.get(args.workload, ORACLE_COUNTS["slab65"])
    vals, walls = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(p, counts["iters"], counts["sweeps"], args.cpu_seconds / 2, seed=i)
        if i >= args.warmup:
            vals.append(cb["value"])
            walls.append(time.perf_counter() - t0)
    v = float(np.mean(vals))
    full17 = oracle_full_solve(make_problem("slab17"), args.ng)
    line = {"impl": "reference", "metric": "converged J solves/s", "value": v, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * float(np.mean(walls)), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "extrapolated": True,
            "config": {"workload": args.workload + ": " + WORKLOADS[args.workload]["desc"],
                       "nx": p.nx, "ny": p.ny, "nz": p.nz, "ndir": p.ndir, "tol": p.tol},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"] + " (each step one such "
                             "sample; value extrapolated from the samples)"},
            "oracle_counts": counts,
            "full_solve_slab17": full17,
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="slab65")
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--df64-steps", type=int, default=2)
    ap.add_argument("--sc-steps", type=int, default=2)
    ap.add_argument("--para-steps", type=int, default=1)
    ap.add_argument("--batch-lambdas", type=int, default=512,
                    help="wavelengths of the FP32-batched companion (0 = skip)")
    ap.add_argument("--fp64-subset", type=int, default=8,
                    help="wavelengths of the batch solved in FP64 plain for the same-wavelength "
                         "ratio and the per-wavelength error")
    ap.add_argument("--batch-tol", type=float, default=1e-8,
                    help="outer tolerance of the batched companion and its FP64 subset")
    ap.add_argument("--precision-n", type=int, default=33,
                    help="horizontal size of the eps = 1e-6 precision check (n x n x 129, "
                         "64x64 directions; 0 = skip)")
    ap.add_argument("--no-precision-check", dest="precision_n", action="store_const", const=0,
                    help="skip the eps = 1e-6 precision check")
    ap.add_argument("--os-sweeps", type=int, default=200,
                    help="sweeps timed for the operator-splitting roofline (0 = skip)")
    ap.add_argument("--config5", type=int, default=1,
                    help="time one outer iteration of the uneven batch at 64x64 directions (0 = skip)")
    ap.add_argument("--only", choices=["os_sweep", "precision", "batched", "config5", "march32"],
                    help="run one companion measurement alone and print its JSON object "
                         "(profiling and diagnostics; not a bench line)")
    ap.add_argument("--budget-s", type=float, default=1500.0,
                    help="wall-clock seconds after which the remaining companions are skipped")
    ap.add_argument("--ng", type=int, default=4,
                    help="Ng acceleration period of the outer iteration (0 = off)")
    ap.add_argument("--lambdas", type=int, default=512, help="wavelengths of the batch workload")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
