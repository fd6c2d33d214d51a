"""Benchmark of the PSATD step on GB300: one JSON line per run (rank 0).

Workload (the metric's configuration): 2D TE PSATD on a 2048 x 2048 periodic
grid in FP32, dx = lambda/64, c dt = dx/sqrt(2), J-form sources from the
prescribed oscillating current sheet J_y(x, t) = J0 exp(-(x - x0(t))^2/w^2),
x0(t) = a sin(w0 t)/w0, a = 0.9 c, w = 2 dx (a synthetic stand-in for the
plasma-mirror surface of the paper's harmonic-generation runs).  A step is one
psatd_step call with that step's J^(n+1/2); L2 is flushed (256 MiB write)
before every timed step and only the step itself is inside the CUDA events.

Arms:
  default            the CUDA path through the C ABI (device-resident inputs);
                     e2e: the same step fed from pinned host buffers (E, B, J
                     uploaded, E, B downloaded every step) through the C ABI.
  --impl reference   the FP64 CPU oracle on the host cores (rank 0 only).
Multi-GPU (torchrun, N > 1): independent replicas, one per GPU (the step has
no exchange on one patch); value = all ranks' cell-steps / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PSATD cell-steps/s on 1 GB300, mixed/batched vs plain FP32 at stated FP64 error"
NX = NY = 2048
LAM_CELLS = 64
WORKLOAD = ("2D TE PSATD 2048x2048 FP32, J-form current-sheet drive J_y(x,t), dx=lambda/64, "
            "c dt=dx/sqrt(2), a=0.9c, w=2dx")
# algorithmic bytes per cell and launch (2D TE J-form, FP32: 5 input components,
# 3 outputs, complex half spectrum of (nx/2+1) x ny 8-byte values per component,
# coefficient table of (nx/2+1) x (ny/2+1) 32-byte entries)
N_IN, N_OUT = 5, 3


def algorithmic_bytes():
    cells = NX * NY
    half = (NX // 2 + 1) * NY
    tab = (NX // 2 + 1) * (NY // 2 + 1) * 32
    return {
        "fwd_x_r2c": N_IN * cells * 4 + N_IN * half * 8,
        "line_fft_push": N_IN * half * 8 + N_OUT * half * 8 + tab,
        "inv_x_c2r": N_OUT * half * 8 + N_OUT * cells * 4,
    }


def sheet_profile(n, dt, dx):
    """J_y(x) of the current sheet at t = (n + 1/2) dt (length NX, float64)."""
    lam = LAM_CELLS * dx
    w0 = 2.0 * math.pi / lam
    t = (n + 0.5) * dt
    Lx = NX * dx
    x0 = 0.5 * Lx + 0.9 * math.sin(w0 * t) / w0
    x = np.arange(NX) * dx
    r = (x - x0 + 0.5 * Lx) % Lx - 0.5 * Lx
    return np.exp(-(r / (2.0 * dx)) ** 2)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The FP64 CPU oracle on the host cores (bounded sample of the workload)."""
    if rank != 0:
        return
    from oracle import psatd as orc
    dx = 1.0 / LAM_CELLS
    dt = dx / math.sqrt(2.0)
    shape = (NY, NX)
    E = np.zeros((3,) + shape)
    B = np.zeros((3,) + shape)
    J = np.zeros((3,) + shape)
    for n in range(min(args.warmup, 1)):
        J[1] = sheet_profile(n, dt, dx)[None, :]
        E, B = orc.psatd_step(E, B, J, d=(dx, dx), dt=dt, form="J")
    steps = 0
    t0 = time.perf_counter()
    while steps < args.steps:
        J[1] = sheet_profile(steps, dt, dx)[None, :]
        E, B = orc.psatd_step(E, B, J, d=(dx, dx), dt=dt, form="J")
        steps += 1
        if time.perf_counter() - t0 > args.ref_seconds:
            break
    el = time.perf_counter() - t0
    value = NX * NY * steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [NX, NY], "precision": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d oracle steps of the full 2048^2 workload (numpy FFT, 1 thread)" % steps},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(seconds):
    """Time the oracle as it stands on a bounded sample of the workload."""
    from oracle import psatd as orc
    dx = 1.0 / LAM_CELLS
    dt = dx / math.sqrt(2.0)
    shape = (NY, NX)
    E = np.zeros((3,) + shape)
    B = np.zeros((3,) + shape)
    J = np.zeros((3,) + shape)
    steps = 0
    t0 = time.perf_counter()
    while True:
        J[1] = sheet_profile(steps, dt, dx)[None, :]
        E, B = orc.psatd_step(E, B, J, d=(dx, dx), dt=dt, form="J")
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds or steps >= 50:
            break
    return {"value": NX * NY * steps / el, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d FP64 oracle steps of the 2048^2 TE workload (numpy pocketfft, one thread), %.1f s"
                      % (steps, el)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=30.0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1608_05739_gb300 import build as bld
    from paper_1608_05739_gb300 import capi

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or not os.path.exists(capi.LIB_PATH):
        bld.build()
    if world > 1:
        dist.barrier()
    capi.load()

    dev = torch.device("cuda", local)
    dx = 1.0 / LAM_CELLS
    dt = dx / math.sqrt(2.0)
    stream = torch.cuda.current_stream()
    plan = capi.Plan((NX, NY), (dx, dx), dt, layout="te", prec="fp32", src="J", stream=stream)
    Ex = torch.zeros(NY, NX, device=dev)
    Ey = torch.zeros(NY, NX, device=dev)
    Bz = torch.zeros(NY, NX, device=dev)
    Jx = torch.zeros(NY, NX, device=dev)
    total = args.warmup + args.steps
    prof = torch.from_numpy(np.stack([sheet_profile(n, dt, dx) for n in range(total)])).float().to(dev)
    Jy_all = [prof[n].expand(NY, NX).contiguous() for n in range(total)]  # resident before timing
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for n in range(args.warmup):
        plan.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy_all[n], None])
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    plan.set_timing(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for s in range(args.steps):
        flush.zero_()
        starts[s].record(stream)
        plan.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy_all[args.warmup + s], None])
        ends[s].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = sum(starts[s].elapsed_time(ends[s]) for s in range(args.steps))
    ktimes = plan.kernel_times()
    plan.set_timing(False)
    if not bool(torch.isfinite(Ey).all()):
        raise RuntimeError("non-finite field after the timed steps")

    # end to end through the C ABI from pinned host buffers
    hE = [torch.zeros(NY, NX).pin_memory() for _ in range(3)]
    hJ = [torch.zeros(NY, NX).pin_memory(), Jy_all[0].cpu().pin_memory()]
    dE = [torch.empty(NY, NX, device=dev) for _ in range(3)]
    dJ = [torch.empty(NY, NX, device=dev) for _ in range(2)]
    e2e_steps = max(10, min(args.steps, 50))
    for it in range(2):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(e2e_steps if it else 2):
            for h, d_ in zip(hE, dE):
                d_.copy_(h, non_blocking=True)
            for h, d_ in zip(hJ, dJ):
                d_.copy_(h, non_blocking=True)
            plan.step([dE[0], dE[1], None], [None, None, dE[2]], [dJ[0], dJ[1], None])
            for h, d_ in zip(hE, dE):
                h.copy_(d_, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = NX * NY * e2e_steps / (e2e_ms * 1e-3)

    t_local = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    t_max = float(t_local.item())
    cells = NX * NY
    value = world * cells * args.steps / (t_max * 1e-3)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_kind = "measured"
    if not hbm:
        hbm, peak_kind = 6800.0, "fallback"
    alg = algorithmic_bytes()
    dom = max(ktimes, key=lambda k: ktimes[k][1]) if ktimes else None
    roof = None
    if dom is not None:
        n_l, tot = ktimes[dom]
        achieved = alg[dom] / (tot / n_l * 1e-3) / 1e9
        traffic = None
        try:
            tr = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
            ent = tr.get(dom)
            if ent and ent.get("source_hash") == source_hash():
                traffic = ent["bytes_per_launch"]
        except Exception:
            pass
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": dom, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": alg[dom],
                "per_kernel_ms": {k: v[1] / v[0] for k, v in ktimes.items()}}
    launches = sum(v[0] for v in ktimes.values())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NX, NY], "precision": "fp32 (compensated twiddles and C, S)",
                       "l2": "flushed before every timed step (256 MiB write), step alone inside the events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": 5 * cells * 4,
                    "d2h_bytes_per_step": 3 * cells * 4},
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        dist.destroy_process_group()


def source_hash():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1608_05739_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
