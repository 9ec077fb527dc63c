"""Benchmark of the batched Rusanov patch update on GB300.

Workload (default): 3D compressible Euler (s = 5, gamma = 1.4), FP64,
262,144 patches of 5x5x5 interior cells + one halo cell, arranged as a
64^3 periodic patch mesh (a 320^3-cell domain), every cell an i.i.d. random
state (rho ~ U[0.5,1.5], u,v,w ~ U[-0.5,0.5], p ~ U[0.5,1.5]).

One step = the whole hot path through the C ABI, fv_time_step: halo cells
gathered from the neighbours, Rusanov update with dt from the CFL condition
(CFL 0.4) on the device, and the maximum wave speed of the new state reduced
for the next step, in one kernel; buffers ping-pong.  The wave speed of the
initial state is seeded once (fv_halo_fill + fv_max_eigenvalue_reduce).  The
same step as three separate kernels (halo fill, reduce, update) and the FP32
path are measured as variants.

Metric: patch cell-updates per second (interior cells advanced per second).
The buffers (2 x 3.6 GB) are far larger than L2 (129 MB), so no flush is
needed between steps.

Arms:
  default            the CUDA library (value: device-resident timing; e2e: the
                     update through fv_patch_update_host on the pinned host
                     batch, advanced in place: chunked host->device copies of
                     each patch's span from its first to its last face-halo
                     cell, the update, device->host copies of each interior
                     plane, overlapped; wall clock)
  --impl reference   the FP64 CPU oracle on the host cores (a bounded sample
                     of the same workload per step)

Multi-GPU (torchrun): every rank advances its own replica of the workload
(independent patch meshes, no data-path collective; weak scaling); timing
is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "patch cell-updates/s"
UNIT = "cell-updates/s"

WORKLOADS = {
    # name: (d, p, n_patches, grid, precision)
    "euler3d_fp64_262144x5": (3, 5, 262144, (64, 64, 64), "f64"),
    "euler3d_fp32_262144x5": (3, 5, 262144, (64, 64, 64), "f32"),
    # small cases of the same kernels (profiling captures, quick checks)
    "euler3d_fp64_32768x5": (3, 5, 32768, (32, 32, 32), "f64"),
    "euler3d_fp32_32768x5": (3, 5, 32768, (32, 32, 32), "f32"),
    # the precision workload's size (4095^2 cells in 5 x 5 patches), random
    # states: the one-warp FP32 kernel for 2D (profiling captures)
    "euler2d_fp32_670761x5": (2, 5, 670761, (819, 819), "f32"),
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# FP64 pipe: 2 FP64 lanes per SM per clock (one DFMA/DADD/DMUL per lane per
# clock) on GB300, 152 SMs.  The peak uses the maximum SM clock.
FP64_LANES_PER_SM = 2
NUM_SMS = 152
# Special-function unit: 16 tanh.approx.f32 results per SM per clock (4 per
# SM sub-partition), the rate of the correction kernel's 128 GELUs per face.
SFU_TANH_PEAK = 16 * NUM_SMS * 2.07e9
# Instruction issue: one warp instruction per scheduler per clock, four
# schedulers per SM (the correction kernel's latency-bound chains run into it).
ISSUE_PEAK = 4 * NUM_SMS * 2.07e9


def fp64_ops_per_patch(d: int, p: int, mode: str = "carry") -> int:
    """FP64 pipe operations of one patch in the step kernel (the algorithm's
    count, the reciprocal and square root counted as the FP64 operations of
    their Newton refinements: 3 and 5).
      primitives of a cell: 3 (1/rho) + d (u) + d (j.u) + 2 (p) + 1 (E+p)
                            + 2 (c^2) + 5 (sqrt) = 13 + 2d;
      face flux G:          2 (a) + 2 (u_L + a, u_R - a) + 1 (p_L + p_R)
                            + 2 (rho) + 2d (momenta) + 4 (energy) = 2d + 11;
      cell update:          s (2d) (sum of G_+ - G_- over d directions, fma);
      next-step wave speed: primitives + d adds.
    mode "update": primitives of the interior and face-halo cells, faces,
    update; "step": that plus the next-step wave speed; "carry": the time
    step with the primitive carry (no conversion of the input state)."""
    s = d + 2
    interior = p ** d
    halo = 2 * d * p ** (d - 1)
    faces = d * (p + 1) * p ** (d - 1)
    prim = 13 + 2 * d
    ops = faces * (2 * d + 11) + interior * s * 2 * d
    if mode in ("update", "step"):
        ops += (interior + halo) * prim
    if mode in ("step", "carry"):
        ops += interior * (prim + d)
    return ops


def alg_bytes_per_patch(d: int, p: int, itemsize: int, carry: bool = False) -> int:
    """Algorithmic HBM bytes of one patch update: read the interior and the
    face-halo cells, write the interior; with the primitive carry also read
    the interior (d+3 values) and face-halo (4 values) primitives and write
    the interior ones."""
    s = d + 2
    interior = p ** d
    halo = 2 * d * p ** (d - 1)
    b = ((interior + halo) * s + interior * s) * itemsize
    if carry:
        b += (2 * interior * (d + 3) + halo * 4) * itemsize
    return b


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(name: str, seed: int = 0):
    from paper_2302_09005_gb300 import inputs
    d, p, n, grid, prec = WORKLOADS[name]
    dtype = np.float64 if prec == "f64" else np.float32
    q, off, sz = inputs.random_batch(n, p, d, seed=seed, dtype=dtype)
    nbr = inputs.grid_neighbours(grid)
    return q, off, sz, nbr


def _events(n):
    import torch
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n)]


def _interior_view(t, n, stride, p, d, s):
    """(n, p, .., p, s) view of the interior cells of a flat patch buffer."""
    ne = p + 2
    v = t[: n * stride].view(n, stride)[:, : ne ** d * s].reshape((n,) + (ne,) * d + (s,))
    return v[(slice(None),) + (slice(1, 1 + p),) * d]


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2302_09005_gb300 import _build, fv

    _build.build()
    torch.cuda.set_device(local)
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    d, p, n, grid, prec = WORKLOADS[args.workload]
    s = d + 2
    fvprec = fv.FV_FP64 if prec == "f64" else fv.FV_FP32
    itemsize = 8 if prec == "f64" else 4
    q, off, sz, nbr = make_workload(args.workload, seed=rank)
    stride = int(off[1] - off[0])
    h_q = torch.from_numpy(q).pin_memory()
    h_off = torch.from_numpy(off).pin_memory()
    h_sz = torch.from_numpy(sz).pin_memory()
    h_nbr = torch.from_numpy(nbr).pin_memory()
    h_out = torch.empty_like(h_q).pin_memory()
    del q
    stream = torch.cuda.Stream()
    qa = h_q.to("cuda")
    qb = qa.clone()
    toff, tsz, tnbr = h_off.cuda(), h_sz.cuda(), h_nbr.cuda()
    b = fv.Batch(d, precision=fvprec, max_patch_size=p, stream=stream)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    if prec == "f32":  # one patch size: the FP32 kernel built for it
        fv.fv_batch_plan(b.h, tsz, n)
    torch.cuda.synchronize()

    def seed(x):  # lambda of the initial state: halo fill + reduce, once
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)

    # FP64: primitive carry, each step reads the primitives the previous one
    # wrote; FP32 (issue- and memory-bound) runs faster without it
    use_carry = prec == "f64"
    prims = ([torch.empty(n * b.prim_stride(), dtype=torch.float64, device="cuda")
              for _ in range(2)] if use_carry else [])
    carry = {"in": None, "k": 0}

    def step(x, y):
        if not use_carry:
            b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
            return
        pout = prims[carry["k"] & 1]
        b.time_step_prim(x, y, carry["in"], pout, toff, tsz, tnbr, dx, cfl)
        carry["in"] = pout
        carry["k"] += 1

    with torch.cuda.stream(stream):
        seed(qa)
        for _ in range(args.warmup):
            step(qa, qb)
            qa, qb = qb, qa
    stream.synchronize()
    if b.status() != fv.FV_OK:
        raise RuntimeError("warm-up: " + fv.fv_last_error(b.h))

    # ---- device-resident timed region: K fused time steps -----------------
    ev = _events(args.steps)
    t0, t1 = _events(1)[0]
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            step(qa, qb)
            ev[k][1].record(stream)
            qa, qb = qb, qa
        t1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    if b.status() != fv.FV_OK:
        raise RuntimeError("timed region: " + fv.fv_last_error(b.h))
    if ws > 1:
        tt = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        dist.barrier()
    cells_per_step = n * p ** d
    value = ws * cells_per_step * args.steps / (ms / 1e3)
    kern_ms = sum(step_ms) / len(step_ms)

    variants = {}
    if not args.no_variants:
        # the same step without the primitive carry (fv_time_step)
        k2 = max(1, min(args.steps, 5))
        ev2 = _events(k2)
        with torch.cuda.stream(stream):
            for k in range(k2):
                ev2[k][0].record(stream)
                b.time_step(qa, qb, toff, tsz, tnbr, dx, cfl)
                ev2[k][1].record(stream)
                qa, qb = qb, qa
        stream.synchronize()
        nc_ms = sum(e[0].elapsed_time(e[1]) for e in ev2) / k2
        variants["time_step_no_carry"] = {
            "value": cells_per_step / (nc_ms / 1e3), "unit": UNIT, "ms_per_step": nc_ms,
            "steps": k2, "what": "fv_time_step: the same fused step converting its input "
                                "state to primitives itself"}
        # the same step as three separate kernels (halo fill, reduce, update)
        k2 = max(1, min(args.steps, 5))
        ev2 = _events(k2)
        with torch.cuda.stream(stream):
            for k in range(k2):
                ev2[k][0].record(stream)
                b.halo_fill(qa, toff, tsz, tnbr)
                b.max_eigenvalue(qa, toff, tsz, cfl, dx)
                b.update(qa, qb, toff, tsz, dx, -1.0)
                ev2[k][1].record(stream)
                qa, qb = qb, qa
        stream.synchronize()
        sep_ms = sum(e[0].elapsed_time(e[1]) for e in ev2) / k2
        variants["separate_kernels"] = {
            "value": cells_per_step / (sep_ms / 1e3), "unit": UNIT, "ms_per_step": sep_ms,
            "steps": k2, "what": "fv_halo_fill + fv_max_eigenvalue_reduce + "
                                "fv_patch_update_batch per step"}

    # ---- end-to-end through the C ABI with host buffers ----------------------
    # The paper's offload pattern: the host batch (patches with their halos)
    # goes through fv_patch_update_host, which overlaps chunked host->device
    # copies, the update and device->host copies.  The batch is advanced in
    # place, step after step, as an engine updates its patch storage: the
    # copies then take spans of the 5^3 boxes (in: from the first face-halo
    # cell to the last; back: each interior plane from its first interior cell
    # to its last).  dt: the CFL step the device slot holds.  Wall-clock time
    # of the synchronous calls.
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    off_np, sz_np = h_off.numpy(), h_sz.numpy()
    dt_e2e = fv.fv_read_dt(b.h)
    h_out.copy_(h_q)
    fv.fv_patch_update_host(b.h, h_out, h_out, off_np, sz_np, n, dx, dt_e2e)  # staging warm-up
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for _ in range(e2e_steps):
        fv.fv_patch_update_host(b.h, h_out, h_out, off_np, sz_np, n, dx, dt_e2e)
    ems = (time.perf_counter() - t_e2e) * 1e3
    if b.status() != fv.FV_OK:
        raise RuntimeError("end-to-end: " + fv.fv_last_error(b.h))
    if ws > 1:
        tt = torch.tensor([ems], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ems = float(tt.item())
    e2e_value = ws * cells_per_step * e2e_steps / (ems / 1e3)
    # one size, equal spacing: the span copies
    h2d = n * _copied_in(d, p, s) * itemsize + h_off.numel() * 8 + h_sz.numel() * 4
    d2h = n * _copied_back(d, p, s) * itemsize
    if not args.no_variants:
        # the same pipeline out of place (host_out != host_in): whole boxes back
        fv.fv_patch_update_host(b.h, h_q, h_out, off_np, sz_np, n, dx, dt_e2e)
        torch.cuda.synchronize()
        t_oop = time.perf_counter()
        for _ in range(e2e_steps):
            fv.fv_patch_update_host(b.h, h_q, h_out, off_np, sz_np, n, dx, dt_e2e)
        oms = (time.perf_counter() - t_oop) * 1e3
        variants["e2e_out_of_place"] = {
            "value": cells_per_step * e2e_steps / (oms / 1e3), "unit": UNIT,
            "ms_per_step": oms / e2e_steps,
            "h2d_bytes_per_step": h_q.numel() * itemsize + h_off.numel() * 8 + h_sz.numel() * 4,
            "d2h_bytes_per_step": h_out.numel() * itemsize,
            "what": "fv_patch_update_host from the pinned host batch into a second one: whole "
                    "boxes (halos included) copied both ways"}
    if not args.no_variants:
        # the device time step with serial copies around it (state and
        # metadata in, halo gather + CFL + update, state out)
        te0, te1 = _events(1)[0]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            te0.record(stream)
            for _ in range(e2e_steps):
                qa.copy_(h_q, non_blocking=True)
                toff.copy_(h_off, non_blocking=True)
                tsz.copy_(h_sz, non_blocking=True)
                tnbr.copy_(h_nbr, non_blocking=True)
                seed(qa)
                b.time_step(qa, qb, toff, tsz, tnbr, dx, cfl)
                h_out.copy_(qb, non_blocking=True)
            te1.record(stream)
        stream.synchronize()
        sms = te0.elapsed_time(te1)
        variants["e2e_serial_time_step"] = {
            "value": cells_per_step * e2e_steps / (sms / 1e3), "unit": UNIT,
            "ms_per_step": sms / e2e_steps,
            "what": "state + metadata host->device, halo fill + reduce + fv_time_step, state "
                    "device->host, one after the other"}

    if prec == "f64" and not args.no_variants:
        variants["fp32"] = fp32_variant(args, b, h_q, toff, tsz, tnbr, n, stride, p, d, s, dx,
                                        cfl, stream)
        del h_out
        variants["batching_uneven_fp64"] = batching_variant(args, "f64")
        variants["batching_uneven_fp32"] = batching_variant(args, "f32")
        variants["precision_2d_4095"] = precision_variant(args)
        variants["learned_correction_1024"] = learned_variant(args)
        variants["paper_shape_2d_p17_sweep"] = sweep_variant(args)
        variants["amr_3d_two_levels"] = amr_variant(args)

    peaks, peak_src = _peaks()
    if prec == "f64":
        ops = fp64_ops_per_patch(d, p, "carry") * n
        peak_ops = FP64_LANES_PER_SM * NUM_SMS * peaks.get("sm_max_mhz", 2070.0) * 1e6
        achieved = ops / (kern_ms / 1e3)
        roof = {"bound": "alu", "kernel": "step_kernel<double,3,gather,fused,carry>",
                "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "T FP64-pipe ops/s", "frac": achieved / peak_ops,
                "traffic": _traffic(args.workload),
                "ops_per_launch": ops,
                "peak_source": "derived: 2 FP64 lanes/SM x 152 SMs x max SM clock "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz"}
    else:
        roof = None
    alg_bytes = alg_bytes_per_patch(d, p, itemsize, carry=use_carry) * n
    hbm = {"achieved": alg_bytes / (kern_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
           "unit": "GB/s", "frac": alg_bytes / (kern_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
           "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peak_src}
    if roof is None:
        kname = ((("rows2d_kernel<5,step>" if d == 2 else "march3d_kernel<5,step>")
                  if fv.fv_batch_pairs_launches(b.h) > 0 else
                  f"step_kernel<float,{d},gather,fused>"))
        roof = {"bound": "hbm", "kernel": kname, **hbm,
                "traffic": _traffic(args.workload)}
    b.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.cpu_sample)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": args.workload, "d": d, "s": s, "patch": p,
                       "n_patches_per_gpu": n, "patch_grid": list(grid), "halo": 1,
                       "cfl": 0.4, "gamma": 1.4,
                       "step": ("fv_time_step_prim: halo gather + Rusanov update + "
                                "next-step CFL max in one kernel, primitives (u, p, c, E+p) "
                                "carried from step to step (initial CFL max seeded once)")
                               if use_carry else
                               ("fv_time_step: halo gather + Rusanov update + next-step "
                                "CFL max in one kernel (initial CFL max seeded once)"),
                       "l2": "inputs larger than L2 (2 x %.1f GB), no flush"
                             % (h_q.numel() * itemsize / 1e9),
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "what": "fv_patch_update_host in place on the pinned host batch (patches "
                            "with their halos): chunked host->device copies of each patch's "
                            "span from its first to its last face-halo cell (327 of 343 "
                            "cells), update, device->host copies of each interior plane (165 "
                            "cells), overlapped; wall clock"},
            # per step: the one-thread kernel that zeroes the next wave-speed
            # slot, then the time-step kernel
            "gpu_launches": 2 * args.steps,
            "step_kernel_ms": kern_ms,
            "roofline": roof,
            "hbm": hbm,
            "variants": variants,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


_UNEVEN_CACHE = {}


def _uneven_batch(n: int):
    """The uneven batch in FP64, laid out with 32-byte alignment so that the
    same offsets also serve its FP32 copy."""
    from paper_2302_09005_gb300 import inputs
    if n not in _UNEVEN_CACHE:
        sizes = inputs.uneven_sizes(n, seed=0)
        _UNEVEN_CACHE[n] = inputs.random_batch(n, sizes, 3, seed=0, align_bytes=32)
    return _UNEVEN_CACHE[n]


def batching_variant(args, prec: str, n: int = 200000, steps_per_graph: int = 20,
                     replays: int = 3):
    """Uneven patch sizes (50% 3^3, 30% 5^3, 20% 7^3, shuffled; self-periodic
    halos): plan + autotune of the per-size CTA size and the schedule, then
    CUDA graphs of
    `steps_per_graph` fused time steps (plus the halo fill and CFL reduce that
    seed the first step) replayed; cell-updates/s over the replays."""
    import torch
    from paper_2302_09005_gb300 import fv, inputs
    d = 3
    q64, off, sz = _uneven_batch(n)
    sizes = sz
    q = q64 if prec == "f64" else q64.astype(np.float32)
    nbr = inputs.self_periodic_neighbours(n, d)
    cells = int(np.sum(sizes.astype(np.int64) ** 3))
    stream = torch.cuda.Stream()
    b = fv.Batch(d, precision=fv.FV_FP64 if prec == "f64" else fv.FV_FP32, max_patch_size=7,
                 stream=stream)
    x = torch.from_numpy(q).cuda()
    y = x.clone()
    toff, tsz, tnbr = (torch.from_numpy(a).cuda() for a in (off, sz, nbr))
    dx, cfl = 1.0 / 64, 0.4
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
    chosen, ms_sched = fv.fv_batch_autotune(b.h, x, y, toff, tsz, tnbr, n, dx, cfl)
    class_threads = {f"{p}^3": fv.fv_batch_class_threads(b.h, p) for p in (3, 5, 7)}
    x0 = x.clone()
    with torch.cuda.stream(stream):  # capture + first run
        b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps_per_graph, use_graph=True)
    stream.synchronize()
    e0, e1 = _events(1)[0]
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(replays):
            b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps_per_graph, use_graph=True)
        e1.record(stream)
    stream.synchronize()
    ok = b.status() == fv.FV_OK
    ms = e0.elapsed_time(e1) / replays
    # end to end: state host -> device, one graph replay, state device -> host
    hq = torch.from_numpy(q).pin_memory()
    hout = torch.empty_like(hq).pin_memory()
    e2, e3 = _events(1)[0]
    with torch.cuda.stream(stream):
        e2.record(stream)
        x.copy_(hq, non_blocking=True)
        b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps_per_graph, use_graph=True)
        hout.copy_(x if steps_per_graph % 2 == 0 else y, non_blocking=True)
        e3.record(stream)
    stream.synchronize()
    ems = e2.elapsed_time(e3)

    # eager steps (fv_run_steps without a graph) under one schedule
    def eager_ms(sched, steps=steps_per_graph):
        fv.fv_batch_set_schedule(b.h, sched)
        with torch.cuda.stream(stream):
            b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, 2)
            a_, b_ = _events(1)[0]
            a_.record(stream)
            b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps)
            b_.record(stream)
        stream.synchronize()
        return a_.elapsed_time(b_) / steps
    queue_ms = eager_ms(fv.FV_SCHED_QUEUE)
    classes_ms = eager_ms(fv.FV_SCHED_CLASSES)
    # why one launch loses: the persistent kernel has one CTA size for every
    # patch (the largest patch's); the per-size launches at that same size
    pers_nt = fv.fv_batch_class_threads(b.h, 7)
    for p_ in (3, 5):
        fv.fv_batch_set_class_threads(b.h, p_, pers_nt)
    classes_one_nt_ms = eager_ms(fv.FV_SCHED_CLASSES)
    ok = ok and b.status() == fv.FV_OK
    b.close()
    del x0
    names = ["stride (persistent, index order)", "lpt (persistent, largest first)",
             "classes (one launch per size)"]
    return {"value": steps_per_graph * cells / (ms / 1e3), "unit": UNIT,
            "ms_per_graph": ms, "steps_per_graph": steps_per_graph, "status_ok": ok,
            "n_patches": n, "cells_per_step": cells, "dtype": prec,
            "schedule_chosen": names[chosen],
            "ms_per_step_by_schedule": dict(zip(names, ms_sched)),
            "class_threads_chosen": class_threads,
            "work_queue": {"ms_per_step": queue_ms, "classes_ms_per_step": classes_ms,
                           "classes_at_one_cta_size_ms_per_step": classes_one_nt_ms,
                           "one_cta_size": pers_nt,
                           "what": "eager steps: FV_SCHED_QUEUE (one persistent launch, CTAs "
                                   "pop patches largest first from a device counter) against "
                                   "one launch per size with the tuned CTA sizes, and with "
                                   "every size at the persistent launch's one CTA size"},
            "e2e": {"value": steps_per_graph * cells / (ems / 1e3), "unit": UNIT,
                    "h2d_bytes": q.nbytes, "d2h_bytes": q.nbytes}}


def sweep_variant(args, p: int = 17, ns=(1, 4, 16, 64, 256, 1024, 4096, 16384, 65536),
                  reps: int = 20):
    """The paper's own benchmark shape: 2D Euler, patches of 17 x 17, N patches
    per kernel invocation for a range of N; time per finite-volume (cell)
    update, with the host<->device transfers of the batch included (as in the
    paper's figure) and device-resident.  FP64, i.i.d. random states in every
    cell (halos included), one fv_patch_update_batch per invocation."""
    import torch
    from paper_2302_09005_gb300 import fv, inputs
    d = 2
    stream = torch.cuda.Stream()
    b = fv.Batch(d, max_patch_size=p, stream=stream)
    dx, dt = 1.0 / 1024, 1e-4
    rows = []
    for n in ns:
        q, off, sz = inputs.random_batch(n, p, d, seed=5)
        hq = torch.from_numpy(q).pin_memory()
        hout = torch.empty_like(hq).pin_memory()
        x = hq.to("cuda")
        y = x.clone()
        toff, tsz = torch.from_numpy(off).cuda(), torch.from_numpy(sz).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(3):
                x.copy_(hq, non_blocking=True)
                b.update(x, y, toff, tsz, dx, dt)
                hout.copy_(y, non_blocking=True)
        stream.synchronize()
        e = _events(2)
        with torch.cuda.stream(stream):
            e[0][0].record(stream)
            for _ in range(reps):
                x.copy_(hq, non_blocking=True)
                b.update(x, y, toff, tsz, dx, dt)
                hout.copy_(y, non_blocking=True)
            e[0][1].record(stream)
            e[1][0].record(stream)
            for _ in range(reps):
                b.update(x, y, toff, tsz, dx, dt)
            e[1][1].record(stream)
        stream.synchronize()
        cells = n * p ** d
        ms_x = e[0][0].elapsed_time(e[0][1]) / reps
        ms_d = e[1][0].elapsed_time(e[1][1]) / reps
        # the host-memory entry point: chunked copies overlapped with the update
        fv.fv_patch_update_host(b.h, hq, hout, off, sz, n, dx, dt)
        t0 = time.perf_counter()
        for _ in range(reps):
            fv.fv_patch_update_host(b.h, hq, hout, off, sz, n, dx, dt)
        ms_h = (time.perf_counter() - t0) * 1e3 / reps
        rows.append({"N": n, "ns_per_cell_update_with_transfers": ms_x * 1e6 / cells,
                     "ns_per_cell_update_host_pipeline": ms_h * 1e6 / cells,
                     "ns_per_cell_update_device": ms_d * 1e6 / cells,
                     "us_per_invocation_with_transfers": ms_x * 1e3,
                     "us_per_invocation_host_pipeline": ms_h * 1e3,
                     "us_per_invocation_device": ms_d * 1e3,
                     "bytes_each_way": int(q.nbytes)})
        del x, y, hq, hout
    ok = b.status() == fv.FV_OK
    b.close()
    return {"what": "2D Euler FP64, p = 17, N patches per invocation; time per cell update: "
                    "copy in + fv_patch_update_batch + copy out one after the other, "
                    "fv_patch_update_host (chunked copies overlapped with the update; wall "
                    "clock), and device-resident",
            "status_ok": ok, "rows": rows}


def amr_variant(args, d: int = 3, p: int = 5, base_level: int = 3, reps: int = 10):
    """A 3:1 refined 3D mesh: every tree cell of level 3 (27^3) carries a 5^3
    patch except a central 5^3 block of tree cells, refined into level-4
    patches; FP64.  Times the refined-mesh halo fill (copies, prolongation,
    restriction) and a refined-mesh step (halo fill + update with per-patch
    cell sizes and one dt)."""
    import torch
    from paper_2302_09005_gb300 import fv, inputs
    nb = 3 ** base_level
    mid = nb // 2
    refine = [(x, y, z) for x in range(mid - 2, mid + 3) for y in range(mid - 2, mid + 3)
              for z in range(mid - 2, mid + 3)]
    q, off, sz, level, coord = inputs.amr_mesh(d, p, base_level, refine, seed=9)
    n = len(off)
    stream = torch.cuda.Stream()
    b = fv.Batch(d, max_patch_size=p, stream=stream)
    plan = fv.AmrPlan(b.h, level, coord, off, p, 0)
    x = torch.from_numpy(q).cuda()
    y = x.clone()
    toff, tsz = torch.from_numpy(off).cuda(), torch.from_numpy(sz).cuda()
    dx = torch.from_numpy(1.0 / (3.0 ** level * p)).cuda()
    dt = torch.full((n,), 0.1 / (3.0 ** (base_level + 1) * p), dtype=torch.float64,
                    device="cuda")
    torch.cuda.synchronize()
    e = _events(2)
    with torch.cuda.stream(stream):
        for _ in range(3):
            plan.fill(x)
        e[0][0].record(stream)
        for _ in range(reps):
            plan.fill(x)
        e[0][1].record(stream)
        e[1][0].record(stream)
        for _ in range(reps):
            plan.fill(x)
            fv.fv_patch_update_local(b.h, x, y, toff, tsz, n, dx, dt)
        e[1][1].record(stream)
    stream.synchronize()
    ok = b.status() == fv.FV_OK
    ms_fill = e[0][0].elapsed_time(e[0][1]) / reps
    ms_step = e[1][0].elapsed_time(e[1][1]) / reps
    plan.close()
    b.close()
    halo_cells = n * 2 * d * p ** (d - 1)
    cells = n * p ** d
    n_fine = int(np.sum(level > base_level))
    # algorithmic bytes of the fill: every halo cell written, its sources read
    # (restriction: 27 fine cells for the coarse halo cells next to finer ones)
    return {"what": f"3D FP64, {n} patches of {p}^3 ({n - n_fine} of level {base_level}, "
                    f"{n_fine} of level {base_level + 1}), periodic",
            "status_ok": ok, "halo_cells": halo_cells,
            "ms_halo_fill": ms_fill, "halo_cells_per_s": halo_cells / (ms_fill / 1e3),
            "ms_step": ms_step, "value": cells / (ms_step / 1e3), "unit": UNIT}


def precision_variant(args, N: int = 4095, p: int = 5, steps: int = 100):
    """Periodic 2D Fourier-perturbed state (rho = 1 + drho, (u, v) random
    modes 1-16, amplitude 0.1, p = 1) on N^2 cells in p x p patches, `steps`
    fused time steps in FP64 and in FP32 (FP32 fluxes and update, FP64
    conservation sums and dt), each as one CUDA graph: time per step, relative
    L1 distance of FP32 to FP64, and the drift of the conserved totals."""
    import torch
    from paper_2302_09005_gb300 import fv, inputs
    U = inputs.fourier_perturbation(N, seed=0)
    q64, off, sz, grid = inputs.domain_to_patches(U, p, align_bytes=32)
    del U
    nbr = inputs.grid_neighbours(grid)
    n = len(off)
    toff, tsz, tnbr = (torch.from_numpy(a).cuda() for a in (off, sz, nbr))
    dx, cfl = 1.0 / N, 0.4
    stride = int(off[1] - off[0])
    out = {}
    finals = {}
    for prec in ("f64", "f32"):
        stream = torch.cuda.Stream()
        b = fv.Batch(2, precision=fv.FV_FP64 if prec == "f64" else fv.FV_FP32,
                     max_patch_size=p, stream=stream)
        if prec == "f32":  # one patch size: the FP32 kernel built for it
            fv.fv_batch_plan(b.h, tsz, n)
        q = q64 if prec == "f64" else q64.astype(np.float32)
        x0 = torch.from_numpy(q).cuda()
        x, y = x0.clone(), x0.clone()
        t0 = torch.zeros(4, dtype=torch.float64, device="cuda")
        t1 = torch.zeros(4, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            b.totals(x, toff, tsz, t0)
            b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps, use_graph=True)  # capture+run
        stream.synchronize()
        res = x if steps % 2 == 0 else y
        with torch.cuda.stream(stream):
            b.totals(res, toff, tsz, t1)
        stream.synchronize()
        finals[prec] = _interior_view(res, n, stride, p, 2, 4).double().clone()
        l1_scale = _interior_view(x0, n, stride, p, 2, 4).double().abs().reshape(-1, 4).sum(0)
        # timing: replay the graph from the initial state
        x.copy_(x0)
        torch.cuda.synchronize()
        e0, e1 = _events(1)[0]
        with torch.cuda.stream(stream):
            e0.record(stream)
            b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps, use_graph=True)
            e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        ok = b.status() == fv.FV_OK
        a0, a1 = t0.cpu().numpy(), t1.cpu().numpy()
        out[prec] = {"ms_per_step": ms / steps, "value": n * p * p * steps / (ms / 1e3),
                     "unit": UNIT, "status_ok": ok,
                     "conserved_totals_start": a0.tolist(),
                     "conserved_drift_rel_to_l1": (np.abs(a1 - a0) / l1_scale.cpu().numpy()
                                                   ).tolist()}
        if prec == "f32":
            out[prec]["one_size_kernel_used"] = fv.fv_batch_pairs_launches(b.h) > 0
            # HBM roofline of the FP32 step (one rows2d launch per step): read
            # the interior and face-halo cells, write the interior
            alg = n * ((p * p + 4 * p) * 4 + p * p * 4) * 4
            peaks, src = _peaks()
            gbs = alg / (ms / steps / 1e3) / 1e9
            out[prec]["roofline"] = {
                "bound": "hbm", "kernel": "rows2d_kernel<5,step>", "achieved": gbs,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                "algorithmic_bytes_per_step": alg,
                "traffic": _traffic("euler2d_fp32_670761x5") if n == 670761 else None,
                "peak_source": src}
            # the same steps on the general kernel (no plan)
            bg = fv.Batch(2, precision=fv.FV_FP32, max_patch_size=p, stream=stream)
            x.copy_(x0)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                bg.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps, use_graph=True)
            stream.synchronize()
            x.copy_(x0)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                e0.record(stream)
                bg.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps, use_graph=True)
                e1.record(stream)
            stream.synchronize()
            out[prec]["general_kernel_ms_per_step"] = e0.elapsed_time(e1) / steps
            bg.close()
        b.close()
        del x0, x, y
    d64, d32 = finals["f64"], finals["f32"]
    rel_l1 = ((d32 - d64).abs().reshape(-1, 4).sum(0) / d64.abs().reshape(-1, 4).sum(0)).tolist()
    del finals, d64, d32
    return {"domain": f"{N}x{N} periodic, {n} patches of {p}x{p}", "steps": steps, **out,
            "fp32_rel_l1_vs_fp64_after_steps": rel_l1}


def learned_variant(args, Nc: int = 1024, pc: int = 8, pf: int = 8, r: int = 4, steps: int = 8,
                    train_seeds=(1, 2), eval_seed: int = 3, train_steps: int = 2000,
                    batch: int = 32768):
    """Learned face-flux correction on a periodic shear layer: training data
    from 4x finer FP64 runs (two seeds), BF16 tensor-core training, then on a
    held-out seed the relative L1 distance to the restricted fine run of
    plain Rusanov at Nc, learned at Nc and plain Rusanov at 2 Nc (the
    equal-cost comparison), with the time per coarse step of each, and the
    throughput of the correction kernel against the BF16 roofline."""
    import torch
    from paper_2302_09005_gb300 import fv, inputs, learned
    st = torch.cuda.Stream()
    Xs, Ts = [], []
    for seed in train_seeds:
        X, T, _, _ = learned.generate(inputs.shear_layer(Nc * r, seed=seed), Nc, pc, pf, r,
                                      steps, 0.4, st)
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    del Xs, Ts
    nsamples = X.shape[0]
    norm = learned.normalisation(X, T, st)
    e0, e1 = _events(1)[0]
    e0.record(st)
    params, losses = learned.train(X, T, norm, steps=train_steps, batch=batch, lr=2e-3, seed=0,
                                   stream=st)
    e1.record(st)
    st.synchronize()
    train_ms = e0.elapsed_time(e1)
    steps_ms = learned.train.last_ms
    del X, T
    Uf = inputs.shear_layer(Nc * r, seed=eval_seed)
    _, _, dts, refs = learned.generate(Uf, Nc, pc, pf, r, steps, 0.4, st)
    l1_plain, l1_learned, ms = learned.evaluate(refs[0], refs, dts, pc, params, norm, st)
    # plain Rusanov at twice the resolution, two substeps per coarse step
    fine = learned.Mesh2D(Nc * r, pf, fv.FV_FP64, st, U=Uf)
    m2 = learned.Mesh2D(2 * Nc, pc, fv.FV_FP64, st)
    mc = learned.Mesh2D(Nc, pc, fv.FV_FP64, st)
    fv.fv_restrict_mesh(fine.b.h, fine.x, fine.off, *fine.grid, m2.b.h, m2.x, m2.off, *m2.grid,
                        r // 2)
    fine.close()
    l1_2x, ms_2x = [], 0.0
    for n, dt in enumerate(dts):
        a, b = _events(1)[0]
        with torch.cuda.stream(st):
            a.record(st)
            m2.step(dt / 2)
            m2.step(dt / 2)
            b.record(st)
            fv.fv_restrict_mesh(m2.b.h, m2.x, m2.off, *m2.grid, mc.b.h, mc.x, mc.off, *mc.grid,
                                2)
        st.synchronize()
        ms_2x += a.elapsed_time(b)
        D, ref = mc.domain(), refs[n + 1]
        l1_2x.append((np.abs(D - ref).sum(axis=(0, 1)) / np.abs(ref).sum(axis=(0, 1))).tolist())
    m2.close()
    mean = lambda rows: float(np.mean(rows[-1]))  # noqa: E731
    # equal cost: the plain method's cost per coarse step at N = 1024, 1448,
    # 2048 (N / Nc substeps of its own step), its error where measured (Nc,
    # 2 Nc), both interpolated log-log to the learned step's cost
    cost_n = {}
    for Nr in (Nc, int(round(Nc * 2 ** 0.5 / pc)) * pc, 2 * Nc):
        mr = learned.Mesh2D(Nr, pc, fv.FV_FP64, st, U=inputs.shear_layer(Nr, seed=eval_seed))
        with torch.cuda.stream(st):
            for _ in range(3):
                mr.step(dts[0] * Nc / Nr)
            a, b = _events(1)[0]
            a.record(st)
            for _ in range(10):
                mr.step(dts[0] * Nc / Nr)
            b.record(st)
        st.synchronize()
        cost_n[Nr] = a.elapsed_time(b) / 10 * (Nr / Nc)
        mr.close()
    # the learned step timed as the plain ones: correction (the halo fill on a
    # second stream beside it) + corrected update, ten back to back
    ml = learned.Mesh2D(Nc, pc, fv.FV_FP64, st, U=refs[0])
    cl = torch.zeros(ml.n * fv.fv_corr_stride(ml.b.h), dtype=torch.float32, device="cuda")

    def learned_step():
        ml.step_learned(dts[0], params, norm, cl)
    with torch.cuda.stream(st):
        for _ in range(3):
            learned_step()
        a, b = _events(1)[0]
        a.record(st)
        for _ in range(10):
            learned_step()
        b.record(st)
    st.synchronize()
    learned_ms = a.elapsed_time(b) / 10
    ml.close()
    eq = _equal_cost(cost_n, {Nc: mean(l1_plain), 2 * Nc: mean(l1_2x)}, learned_ms)
    eq["learned_ms"] = learned_ms
    eq["learned_mean_rel_l1"] = mean(l1_learned)
    eq["learned_beats_plain_at_equal_cost"] = bool(mean(l1_learned) < eq["plain_mean_rel_l1"])
    # the same network, FP32 state arithmetic
    l1_plain32, l1_learned32, ms32 = learned.evaluate(refs[0], refs, dts, pc, params, norm, st,
                                                      precision=fv.FV_FP32)
    # correction kernel alone: faces/s and BF16 TFLOP/s (10,752 flop per face)
    m = learned.Mesh2D(Nc, pc, fv.FV_FP32, st, U=refs[0])
    corr = torch.zeros(m.n * fv.fv_corr_stride(m.b.h), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(st):
        for _ in range(3):
            fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, params, norm, corr)
        a, b = _events(1)[0]
        a.record(st)
        for _ in range(10):
            fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, params, norm, corr)
        b.record(st)
    st.synchronize()
    kms = a.elapsed_time(b) / 10
    faces = m.n * 2 * pc * pc  # each face of the mesh once
    flops = faces * 2 * (16 * 64 + 64 * 64 + 64 * 4)
    m.close()
    mc.close()
    peaks, src = _peaks()
    tf = flops / (kms / 1e3) / 1e12
    tanh_rate = faces * 128 / (kms / 1e3)  # one hardware tanh per hidden unit
    return {
        "domain": f"{Nc}x{Nc} periodic shear layer, {pc}x{pc} patches; fine {Nc * r}^2 FP64",
        "train": {"samples": nsamples, "seeds": list(train_seeds), "steps": train_steps,
                  "batch": batch, "ms": train_ms, "adam_steps_ms": steps_ms,
                  "note": "ms: normalisation, one shuffle of the sample set and the Adam "
                          "steps; adam_steps_ms: the steps alone (tcgen05 network kernel "
                          "and the fixed-order reduction + Adam kernel, two launches a step)",
                  "loss_first_last": [losses[0][1], losses[-1][1]]},
        "eval_seed": eval_seed, "coarse_steps": steps,
        "rel_l1_after_steps": {"plain_Nc": l1_plain[-1], "learned_Nc": l1_learned[-1],
                               "plain_2Nc": l1_2x[-1]},
        "mean_rel_l1": {"plain_Nc": mean(l1_plain), "learned_Nc": mean(l1_learned),
                        "plain_2Nc": mean(l1_2x)},
        "ms_per_coarse_step": {"plain_Nc": ms[False], "learned_Nc": ms[True],
                               "plain_2Nc": ms_2x / len(dts)},
        "equal_cost": eq,
        "fp32_state": {"mean_rel_l1": {"plain_Nc": mean(l1_plain32),
                                       "learned_Nc": mean(l1_learned32)},
                       "ms_per_coarse_step": {"plain_Nc": ms32[False], "learned_Nc": ms32[True]}},
        "correction_kernel": {"ms": kms, "faces": faces, "gflop": flops / 1e9,
                              "roofline": {"bound": "tensor", "achieved": tf,
                                           "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                                           "frac": tf / peaks["bf16_tflops"],
                                           "peak_source": src + " (BF16 dense, burst)"},
                              "roofline_sfu": {"bound": "sfu", "achieved": tanh_rate / 1e12,
                                               "peak": SFU_TANH_PEAK / 1e12,
                                               "unit": "T tanh/s",
                                               "frac": tanh_rate / SFU_TANH_PEAK,
                                               "peak_source": "derived: 16 tanh per SM per "
                                                              "cycle x 152 SMs x 2.07 GHz"},
                              "roofline_issue": _issue_roofline(kms, Nc)},
    }


def correction_variant(args, Nc: int = 1024, pc: int = 8, reps: int = 20):
    """The correction kernel alone on the learned workload's mesh (the
    periodic shear layer, Nc^2 cells in pc x pc patches, FP32 state) with a
    seeded random network: time per call and its rooflines (for profiling
    the kernel without the training and evaluation around it)."""
    import torch
    from paper_2302_09005_gb300 import fv, inputs, learned
    st = torch.cuda.Stream()
    m = learned.Mesh2D(Nc, pc, fv.FV_FP32, st, U=inputs.shear_layer(Nc, seed=3))
    params = torch.from_numpy(learned.init_params(0)).cuda()
    norm = torch.tensor(np.concatenate([np.full(16, 0.5), np.ones(16), np.full(4, 0.05)]),
                        dtype=torch.float32, device="cuda")
    corr = torch.zeros(m.n * fv.fv_corr_stride(m.b.h), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(st):
        for _ in range(3):
            fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, params, norm, corr)
        a, b = _events(1)[0]
        a.record(st)
        for _ in range(reps):
            fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, params, norm, corr)
        b.record(st)
    st.synchronize()
    kms = a.elapsed_time(b) / reps
    ok = m.b.status() == fv.FV_OK
    faces = m.n * 2 * pc * pc
    flops = faces * 2 * (16 * 64 + 64 * 64 + 64 * 4)
    m.close()
    peaks, src = _peaks()
    tf = flops / (kms / 1e3) / 1e12
    tanh_rate = faces * 128 / (kms / 1e3)
    return {"domain": f"{Nc}x{Nc} periodic shear layer, {pc}x{pc} patches, FP32 state",
            "ms": kms, "faces": faces, "status_ok": ok,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": tf / peaks["bf16_tflops"],
                         "peak_source": src + " (BF16 dense, burst)"},
            "roofline_sfu": {"bound": "sfu", "achieved": tanh_rate / 1e12,
                             "peak": SFU_TANH_PEAK / 1e12, "unit": "T tanh/s",
                             "frac": tanh_rate / SFU_TANH_PEAK},
            "roofline_issue": _issue_roofline(kms, Nc)}


def _equal_cost(cost_n, err_n, target_ms):
    """The resolution N* at which the plain method costs target_ms per coarse
    step and its error there: cost(N) and err(N) interpolated piecewise
    linearly in log-log (extrapolated from the end segments outside the
    measured range)."""
    def interp(pts, x):
        pts = sorted(pts)
        lx = [math.log(a) for a, _ in pts]
        ly = [math.log(b) for _, b in pts]
        i = 0
        while i < len(lx) - 2 and x > lx[i + 1]:
            i += 1
        t = (x - lx[i]) / (lx[i + 1] - lx[i])
        return ly[i] + t * (ly[i + 1] - ly[i])
    # invert cost(N): N as a function of cost
    lnN = interp([(c, n) for n, c in cost_n.items()], math.log(target_ms))
    n_star = math.exp(lnN)
    err = math.exp(interp(list(err_n.items()), lnN))
    lo, hi = min(cost_n), max(cost_n)
    return {"cost_ms_by_N": {str(k): v for k, v in sorted(cost_n.items())},
            "N_at_learned_cost": n_star, "plain_mean_rel_l1": err,
            "plain_mean_rel_l1_by_N": {str(k): v for k, v in sorted(err_n.items())},
            "interpolated": bool(lo <= n_star <= hi),
            "how": "plain Rusanov cost per coarse step (N / Nc substeps) timed at each N; "
                   "error measured at Nc and 2 Nc against the restricted fine run; both "
                   "interpolated log-log to the learned step's cost"}


def fp32_variant(args, b64, h_q, toff, tsz, tnbr, n, stride, p, d, s, dx, cfl, stream):
    """FP32 arithmetic on the same workload (FP32-rounded initial state): timed
    fused steps, and the relative L1 distance to the FP64 path after one
    step from the same initial state."""
    import torch
    from paper_2302_09005_gb300 import fv
    b = fv.Batch(d, precision=fv.FV_FP32, max_patch_size=p, stream=stream)
    x64 = h_q.to("cuda")
    y64 = x64.clone()
    x = x64.float()
    y = x.clone()
    with torch.cuda.stream(stream):
        b64.halo_fill(x64, toff, tsz, tnbr)
        b64.max_eigenvalue(x64, toff, tsz, cfl, dx)
        b64.time_step(x64, y64, toff, tsz, tnbr, dx, cfl)
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
        b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
    stream.synchronize()
    i64 = _interior_view(y64, n, stride, p, d, s)
    i32 = _interior_view(y, n, stride, p, d, s).double()
    diff = (i32 - i64).abs().reshape(-1, s).sum(0)
    norm = i64.abs().reshape(-1, s).sum(0)
    rel_l1 = (diff / norm).tolist()
    max_rel = ((i32 - i64).abs().reshape(-1, s).amax(0) / i64.abs().reshape(-1, s).amax(0))
    del i64, i32, diff

    def timed_steps():
        nonlocal x, y
        for _ in range(args.warmup):
            with torch.cuda.stream(stream):
                b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
            x, y = y, x
        ev = _events(args.steps)
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[k][0].record(stream)
                b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
                ev[k][1].record(stream)
                x, y = y, x
        stream.synchronize()
        return sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps

    # the general kernel (no plan), then the kernel for one patch size (the
    # batch planned: all patches are 5^3)
    ms_general = timed_steps()
    fv.fv_batch_plan(b.h, tsz, n)
    ms = timed_steps()
    one_size_used = fv.fv_batch_pairs_launches(b.h) > 0
    # the same with the primitive carry
    prims = [torch.empty(n * b.prim_stride(), dtype=torch.float32, device="cuda")
             for _ in range(2)]
    ev = _events(args.steps)
    with torch.cuda.stream(stream):
        b.time_step_prim(x, y, None, prims[0], toff, tsz, tnbr, dx, cfl)
        x, y = y, x
        for k in range(args.steps):
            ev[k][0].record(stream)
            b.time_step_prim(x, y, prims[k & 1], prims[(k + 1) & 1], toff, tsz, tnbr, dx, cfl)
            ev[k][1].record(stream)
            x, y = y, x
    stream.synchronize()
    ms_carry = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    del prims
    ok = b.status() == fv.FV_OK
    peaks, peak_src = _peaks()
    alg = alg_bytes_per_patch(d, p, 4) * n
    alg_c = alg_bytes_per_patch(d, p, 4, carry=True) * n
    b.close()
    return {"value": n * p ** d / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "what": "fv_time_step in FP32 (no primitive carry), the batch planned: the "
                    "kernel for 5^3 patches (march3d_kernel<5>: a lane per row, the patch "
                    "swept plane by plane)",
            "one_size_kernel_used": one_size_used,
            "general_kernel": {"value": n * p ** d / (ms_general / 1e3),
                               "ms_per_step": ms_general,
                               "what": "the same step on the general kernel (no plan)"},
            "carry": {"value": n * p ** d / (ms_carry / 1e3), "ms_per_step": ms_carry,
                      "what": "fv_time_step_prim in FP32",
                      "hbm_frac": alg_c / (ms_carry / 1e3) / 1e9 / peaks["hbm_gbs"]},
            "status_ok": ok,
            "rel_l1_vs_fp64_one_step": rel_l1, "max_rel_err_vs_fp64_one_step":
                max_rel.tolist(),
            "roofline": {"bound": "hbm", "kernel": "march3d_kernel<5,step>",
                         "achieved": alg / (ms / 1e3) / 1e9,
                         "traffic": _traffic("euler3d_fp32_262144x5"),
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": alg / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                         "peak_source": peak_src}}


def _copied_in(d, p, s):
    """Elements of a patch box the in-place host update copies in: from its
    first to its last face-halo cell."""
    ne = p + 2
    tot, top = 0, 1
    for m in range(d):
        tot += top
        if m + 1 < d:
            top *= ne
    return s * (p * (tot - top) + (p + 1) * top + 1) - s * (tot - top)


def _copied_back(d, p, s):
    """Elements of a patch box the in-place host update copies back: 3D, each
    interior plane's (1, 1, z) .. (p, p, z); else from the first to the last
    interior cell."""
    ne = p + 2
    if d == 3:
        return s * p * ((p - 1) * ne + p)
    tot, pw = 0, 1
    for _ in range(d):
        tot += pw
        pw *= ne
    return s * (p * tot + 1) - s * tot


def _warp_instructions(key):
    """Warp instructions per launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            ent = json.load(f).get(key)
        from paper_2302_09005_gb300 import _build
        if ent and ent.get("kernel_hash") == _build.kernel_hash(ent.get("kernel", "step")):
            return ent.get("warp_instructions_per_launch")
    except Exception:
        return None
    return None


def _issue_roofline(kms, nc):
    """The correction kernel's instruction issue against one warp instruction
    per scheduler per clock (ncu's count of its full launch on the 1024^2
    mesh; None on another mesh or another source)."""
    winstr = _warp_instructions("corr_shear_1024") if nc == 1024 else None
    if winstr is None:
        return None
    rate = winstr / (kms / 1e3)
    return {"bound": "issue", "achieved": rate / 1e12, "peak": ISSUE_PEAK / 1e12,
            "unit": "T warp instructions/s", "frac": rate / ISSUE_PEAK,
            "warp_instructions_per_launch": winstr,
            "peak_source": "derived: 4 schedulers per SM x 152 SMs x 2.07 GHz",
            "count_source": "ncu smsp__inst_executed.sum of the same launch "
                            "(profiles/traffic.json)"}


def _traffic(workload):
    """DRAM bytes per update launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            t = json.load(f)
        from paper_2302_09005_gb300 import _build
        ent = t.get(workload)
        if ent and ent.get("kernel_hash") == _build.kernel_hash(ent.get("kernel", "step")):
            return ent["dram_bytes_per_launch"]
    except Exception:
        return None
    return None


def _oracle_step(q, off, sz, d, dx, cfl, threads: int):
    """One oracle step over the patches: halo fill (each patch's face halos
    from its own opposite faces, self-periodic: the same copies per patch as
    a neighbour on the mesh), max-eigenvalue reduce, CFL dt, update.  The
    patches are split into `threads` contiguous chunks run by host threads
    (the oracle's C calls release the interpreter lock); the oracle's code is
    the same for any split."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    from paper_2302_09005_gb300 import inputs
    n = len(off)
    bounds = [(n * k) // threads for k in range(threads + 1)]
    chunks = [(bounds[k], bounds[k + 1]) for k in range(threads) if bounds[k + 1] > bounds[k]]
    out = q.copy()
    with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
        list(ex.map(lambda c: oracle.halo_fill(
            q, off[c[0]:c[1]], sz[c[0]:c[1]], inputs.self_periodic_neighbours(c[1] - c[0], d),
            d, d + 2), chunks))
        lams = list(ex.map(lambda c: oracle.max_eigenvalue(q, off[c[0]:c[1]], sz[c[0]:c[1]],
                                                           d)[1], chunks))
        dt = oracle.cfl_dt(max(lams), cfl, dx, d)
        list(ex.map(lambda c: oracle.patch_update(q, off[c[0]:c[1]], sz[c[0]:c[1]], d, dx, dt,
                                                  q_out=out), chunks))
    return out


def cpu_baseline(workload: str, sample: int):
    """The oracle as it stands on the first ``sample`` patches of the same
    workload, one step (halo fill + CFL reduce + update, Eq. 3-5): on every
    host core (patches split across threads), and on one core."""
    d, p, n, grid, prec = WORKLOADS[workload]
    from paper_2302_09005_gb300 import inputs
    multi = min(n, 4 * sample)  # all cores: a larger sample
    q, off, sz = inputs.random_batch(multi, p, d, seed=0)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    _oracle_step(q, off, sz, d, dx, cfl, cores)
    el = time.perf_counter() - t
    single = max(1, sample // 2)
    t = time.perf_counter()
    _oracle_step(q, off[:single], sz[:single], d, dx, cfl, 1)
    el1 = time.perf_counter() - t
    return {"value": multi * p ** d / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{multi} of {n} patches ({p}^{d}, FP64): halo fill (self-periodic) + "
                      f"max-eigenvalue reduce + update, one step, {el:.2f} s on "
                      f"{cores} threads",
            "single_core": {"value": single * p ** d / el1, "patches": single,
                            "seconds": el1}}


def run_reference(args, ws, rank):
    """The oracle on the host cores, same metric and workload, each step a
    bounded sample of the patches."""
    if rank != 0:
        return
    import oracle
    from paper_2302_09005_gb300 import inputs
    oracle.build()
    d, p, n, grid, prec = WORKLOADS[args.workload]
    sample = args.cpu_sample
    q, off, sz = inputs.random_batch(sample, p, d, seed=0)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    cores = os.cpu_count() or 1

    def one():
        _oracle_step(q, off, sz, d, dx, cfl, cores)

    for _ in range(args.warmup):
        one()
    t = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t
    value = sample * p ** d * args.steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "d": d, "patch": p, "n_patches_per_gpu": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} of {n} patches per step (halo fill, "
                                       f"self-periodic + max-eigenvalue reduce + update), "
                                       f"patches split across {cores} host threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="euler3d_fp64_262144x5")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=32768)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variant", choices=["batching", "precision", "learned", "correction",
                                          "sweep", "amr"],
                    default=None,
                    help="run one variant on its own")
    ap.add_argument("--small", action="store_true", help="small case of --variant")
    ap.add_argument("--prec", choices=["f64", "f32"], default="f64",
                    help="precision of --variant batching")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    ws, rank, local = dist_setup()
    if args.variant:
        run_variant(args)
    elif args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


def run_variant(args):
    """One variant on its own (profiling captures, focused measurements);
    --small shrinks it to a case that an ncu capture finishes quickly."""
    import torch
    from paper_2302_09005_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    if args.variant == "batching":
        res = batching_variant(args, args.prec, n=20000 if args.small else 200000)
    elif args.variant == "precision":
        res = precision_variant(args, N=1020 if args.small else 4095,
                                steps=10 if args.small else 100)
    elif args.variant == "sweep":
        res = sweep_variant(args, ns=(1, 16, 256, 4096) if args.small else
                            (1, 4, 16, 64, 256, 1024, 4096, 16384, 65536))
    elif args.variant == "amr":
        res = amr_variant(args, base_level=2 if args.small else 3)
    elif args.variant == "correction":
        res = correction_variant(args, Nc=256 if args.small else 1024)
    elif args.variant == "learned":
        res = (learned_variant(args, Nc=256, steps=4, train_steps=200, batch=8192)
               if args.small else learned_variant(args))
    else:
        raise SystemExit(f"unknown variant {args.variant}")
    print(json.dumps({"variant": args.variant, "small": bool(args.small), **res}), flush=True)


if __name__ == "__main__":
    main()
