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
# Peak FP64 of GB300 from the profiling recipe's figure (1.25 TFLOP/s,
# i.e. 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz).
PEAK_FP64_TFLOPS = 1.25

WORKLOADS = {
    "slab65": dict(desc="65^3 slab (x,y periodic), chi = 10^(-4+8k/64) exp(0.3 N(0,1)), "
                        "eps = 10^(-4U) per voxel, B = (1+k/64)^4, 32x32 directions, tol 1e-8",
                   make="slab_65"),
    "slab17": dict(desc="17^3 slab, chi = 10^(-4+8k/16)(1+0.2(U-1/2)), eps = 1e-2, B = 1, "
                        "16x16 directions, tol 1e-8",
                   make="slab_small"),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_problem(name):
    from paper_1107_5719_gb300 import workloads as W
    return getattr(W, WORKLOADS[name]["make"])()


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


def run_ours(args):
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

    p = make_problem(args.workload)
    chi = torch.from_numpy(p.chi).to(dev)
    eps = torch.from_numpy(p.eps).to(dev)
    Bt = torch.from_numpy(p.B).to(dev)
    Jout = torch.empty_like(Bt)
    stream = torch.cuda.Stream(device=dev)
    ctx = R.rt_create(local, R.RT_FP64)
    R.rt_set_stream(ctx, stream)
    R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
    R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
    R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
    R.rt_set_epsilon_dev(ctx, eps)
    flush = torch.zeros(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MiB > L2

    def step():
        R.rt_set_opacity_dev(ctx, chi)      # new opacity: Lambda* is rebuilt
        R.rt_set_planck_dev(ctx, Bt)        # J = B
        it, delta, conv = R.rt_solve_dev(ctx, Jout, tol=p.tol, max_iter=args.max_iter)
        if not conv:
            raise RuntimeError(f"solve did not converge in {it} iterations (delta {delta:.3e})")
        return it

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    R.rt_reset_stats(ctx)
    R.rt_set_profiling(ctx, True)
    times = []
    iters = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(smi_id(dev)) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            stream.synchronize()
            ev0.record(stream)
            iters.append(step())
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    st = R.rt_get_stats(ctx)
    R.rt_set_profiling(ctx, False)
    total_ms = float(sum(times))
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    solves_per_s = ws * args.steps / (total_ms / 1e3)
    fs_per_solve = st["fs_launches"] / args.steps
    pairs = p.nvox * p.ndir
    vd_per_s = ws * st["fs_launches"] * pairs / (total_ms / 1e3)
    steps_per_s = ws * st["steps"] / (total_ms / 1e3)

    # dominant kernel: the FP64 formal-solution march
    fs_ms = st["fs_ms"] / max(st["fs_launches"], 1)
    steps_per_launch = st["steps"] / max(st["fs_launches"], 1)
    flops_launch = FLOPS_PER_STEP_FP64 * steps_per_launch
    achieved = flops_launch / (fs_ms / 1e3) / 1e12
    roofline = {"kernel": "k_fs64 (formal-solution march, FP64)", "bound": "alu",
                "achieved": round(achieved, 4), "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": round(achieved / PEAK_FP64_TFLOPS, 4), "traffic": None,
                "peak_source": "recipe FP64 figure (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                "flops_per_step": FLOPS_PER_STEP_FP64, "steps_per_launch": steps_per_launch,
                "ms_per_launch": round(fs_ms, 4),
                "share_of_step": round(st["fs_ms"] / total_ms, 4)}

    # end to end through the host-pointer API (pinned host buffers)
    e2e = None
    if args.e2e_steps > 0:
        chi_h = torch.from_numpy(p.chi).pin_memory()
        eps_h = torch.from_numpy(p.eps).pin_memory()
        B_h = torch.from_numpy(p.B).pin_memory()
        J_h = torch.empty_like(B_h).pin_memory()
        ctx2 = R.rt_create(local, R.RT_FP64)
        R.rt_set_grid(ctx2, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_boundary(ctx2, p.top_bc, p.bottom_bc)
        R.rt_set_quadrature(ctx2, p.mu, p.phi, p.w)
        lib = R.load()
        import ctypes as C

        def e2e_step():
            lib.rt_set_opacity(ctx2, chi_h.data_ptr())
            lib.rt_set_epsilon(ctx2, eps_h.data_ptr())
            lib.rt_set_planck(ctx2, B_h.data_ptr())
            it = C.c_int()
            last = C.c_double()
            rc = lib.rt_solve(ctx2, p.tol, args.max_iter, 1e-12, 1000, J_h.data_ptr(),
                              C.byref(it), C.byref(last), None, None)
            if rc != 0:
                raise RuntimeError(R.rt_last_error(ctx2))

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        R.rt_destroy(ctx2)
        e2e = {"value": round(ws * args.e2e_steps / dt, 6), "unit": "solves/s",
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
                   "lstar": "rebuilt every step"},
        "voxel_dir_updates_per_s": round(vd_per_s, 1),
        "march_steps_per_s": round(steps_per_s, 1),
        "iters_per_solve": round(fs_per_solve, 3),
        "roofline": roofline,
        "gpu_launches": int(st["launches"]),
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(p, fs_per_solve, st["jacobi_launches"] / args.steps,
                                            args.cpu_seconds)
    R.rt_destroy(ctx)
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


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on bounded samples of the workload."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    p = make_problem(args.workload)
    iters = args.ref_iters
    sweeps = args.ref_sweeps
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(p, iters, sweeps, args.cpu_seconds / 2, seed=i)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": "converged J solves/s", "value": v, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload + ": " + WORKLOADS[args.workload]["desc"],
                       "nx": p.nx, "ny": p.ny, "nz": p.nz, "ndir": p.ndir, "tol": p.tol},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="slab65")
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-iters", type=float, default=60.0,
                    help="outer iterations per solve assumed by the reference arm")
    ap.add_argument("--ref-sweeps", type=float, default=2000.0,
                    help="Jacobi sweeps per solve assumed by the reference arm")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
