"""Benchmark of the PSATD step on GB300: one JSON line per run (rank 0).

Default workload (the metric's configuration: mixed precision, batched): 512
independent periodic 2D TE patches -- the paper's local-FFT subdomains
(Sec. II.A.3) -- with interior sides U{64..512} and guards U{8..16} per axis,
each side widened to the next transform length (powers of two for the
tensor-core passes), J-form with a seeded random current held over the run.
The step runs with split-BF16 tensor-core radix-16 stages (FP32 accumulate);
the whole timed run is one psatd_batch_step(nsteps = --steps) call, i.e. a
CUDA graph of one step replayed.  Reported beside it: plain FP32 on the same
patches, the error of both against the FP64 oracle on sampled patches after the
same steps, the oracle's own speed on the host cores (cpu_baseline), the end to
end rate from pinned host arrays, and the single 2048^2 TE grid in FP32 as a
side key.  --workload selects the side measurements instead (te2048, 3D, FDTD,
local decomposition, cost comparison).

Arms:
  default            the CUDA path through the C ABI (device-resident inputs);
  --impl reference   the FP64 CPU oracle on the host cores (rank 0 only).
Multi-GPU (torchrun, N > 1): independent replicas, one per GPU (no exchange);
value = all ranks' cell-steps / max rank time.
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
# algorithmic bytes per launch of each PSATD pass: every input component read
# once and every output written once per pass, complex half spectra of
# (nx/2+1) ny nz values (8 B in FP32), plus the coefficient table (one 32-byte
# entry per (nx/2+1)(ny/2+1)(nz/2+1) octant point) read by the fused pass.
N_IN, N_OUT = 5, 3


PREC_NOTE = {
    "fp32": "fp32 (compensated twiddles and C, S)",
    "mixed_fp16": "mixed: radix-16 stages as tcgen05 DFT-matrix MMAs, split-FP16 operands, FP32 accumulate; "
                  "rest fp32 as the plain path",
    "mixed_bf16": "mixed: radix-16 stages as tcgen05 DFT-matrix MMAs, split-BF16 operands (3 pieces), FP32 "
                  "accumulate; rest fp32 as the plain path",
}
DTYPE = {"fp32": "f32", "mixed_fp16": "f16x2-split tensor + f32", "mixed_bf16": "bf16x3-split tensor + f32"}


def algorithmic_bytes(nx=NX, ny=NY, nz=1, n_in=N_IN, n_out=N_OUT, real=4):
    cells = nx * ny * nz
    half = (nx // 2 + 1) * ny * nz
    cplx = 2 * real
    tab = (nx // 2 + 1) * (ny // 2 + 1) * (nz // 2 + 1 if nz > 1 else 1) * 8 * real
    out = {
        "fwd_x_r2c": n_in * cells * real + n_in * half * cplx,
        "line_fft_push": n_in * half * cplx + n_out * half * cplx + tab,
        "inv_x_c2r": n_out * half * cplx + n_out * cells * real,
    }
    if nz > 1:
        out["fwd_y_c2c"] = 2 * n_in * half * cplx
        out["inv_y_c2c"] = 2 * n_out * half * cplx
    return out


def sheet_profile(n, dt, dx, nx=NX):
    """J_y(x) of the current sheet at t = (n + 1/2) dt (length nx, float64)."""
    lam = LAM_CELLS * dx
    w0 = 2.0 * math.pi / lam
    t = (n + 0.5) * dt
    Lx = nx * dx
    x0 = 0.5 * Lx + 0.9 * math.sin(w0 * t) / w0
    x = np.arange(nx) * dx
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


def replica_throughput(ms_local, cells, steps, world, device):
    """Whole-job cell-steps/s of `world` independent replicas: every rank advanced
    `cells` cells by `steps` steps; the job's time is the slowest rank's (max over
    ranks of the summed CUDA-event milliseconds).  Returns (value, max ms)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return world * cells * steps / (t_max * 1e-3), t_max


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------- the headline: batched patches
BATCH_SEED, BATCH_J_SEED, BATCH_J_SCALE = 1612, 1613, 0.01
BATCH_WORKLOAD = ("512 periodic 2D TE patches (the paper's local-FFT subdomains, Sec. II.A.3): interior "
                  "U{64..512}^2 and guards U{8..16} per axis (seed 1612), each side widened to the next "
                  "transform length; J-form, E = B = 0 at the start, J ~ N(0, 0.01^2) per patch (seed 1613 + i) "
                  "held over the run; dx = lambda/64, c dt = dx/sqrt(2)")
BATCH_DX = 1.0 / LAM_CELLS
BATCH_DT = BATCH_DX / math.sqrt(2.0)


def _oracle_patch(job):
    """Oracle worker (spawned process): `nsteps` FP64 oracle steps of batch patch
    `i` (nx x ny) from E = B = 0 with its seeded source; returns (i, seconds,
    Ex, Ey, Bz) or, with keep=False, (i, seconds) only."""
    i, nx, ny, nsteps, keep = job
    from oracle import psatd as orc
    from paper_1608_05739_gb300 import synth
    jx, jy = synth.batch_patch_source(i, nx, ny, BATCH_J_SEED, BATCH_J_SCALE)
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    J = np.zeros((3, ny, nx))
    J[0] = jx.astype(np.float64)
    J[1] = jy.astype(np.float64)
    t0 = time.perf_counter()
    E, B = orc.psatd_step(E, B, J, d=(BATCH_DX, BATCH_DX), dt=BATCH_DT, form="J", nsteps=nsteps)
    el = time.perf_counter() - t0
    return (i, el, E[0], E[1], B[2]) if keep else (i, el)


def _pool_ready(_):
    import oracle.psatd  # noqa: F401  (imports done before any timing)
    return os.getpid()


def oracle_pool():
    """Process pool for the oracle on every host core this process may use, started
    with spawn (before any CUDA call of the parent)."""
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0))
    pool = mp.get_context("spawn").Pool(n)
    pool.map(_pool_ready, range(4 * n))
    return pool, n


def batch_cpu_baseline(pool, ncores, sizes, stride=2, steps=1):
    """The oracle as it stands on a bounded sample of the batch: every `stride`-th
    patch, `steps` steps each, patches spread over the pool's processes."""
    jobs = [(i, nx, ny, steps, False) for i, (nx, ny) in enumerate(sizes) if i % stride == 0]
    cells = sum(sizes[j[0]][0] * sizes[j[0]][1] for j in jobs)
    t0 = time.perf_counter()
    res = pool.map(_oracle_patch, sorted(jobs, key=lambda j: -j[1] * j[2]), chunksize=1)
    el = time.perf_counter() - t0
    cpu = sum(r[1] for r in res)
    return {"value": cells * steps / el, "unit": "cell-steps/s", "cores": ncores, "kind": "oracle",
            "sample": "%d of the 512 patches (every %dth, %.3g cells), %d FP64 oracle step(s) each, one patch "
                      "per process on %d processes (numpy pocketfft): %.1f s wall, %.1f s of CPU work"
                      % (len(jobs), stride, cells, steps, ncores, el, cpu)}


def batch_sample(sizes, budget_cell_steps, nsteps, seed=1617, count=8):
    """Patches compared with the oracle after the timed run: the smallest, and
    seeded others whose oracle run (area x nsteps) fits the budget."""
    area = [a * b for a, b in sizes]
    small = [i for i in range(len(sizes)) if area[i] * nsteps <= budget_cell_steps]
    pick = {int(np.argmin(area))}
    if small:
        g = np.random.default_rng(seed)
        pick |= set(int(i) for i in g.choice(small, min(count - 1, len(small)), replace=False))
    return sorted(pick)


def patch_fields(fields, sizes, offsets, idx):
    """{i: [Ex, Ey, Bz] of patch i as float64 host arrays} from the packed fields."""
    out = {}
    for i in idx:
        o, m = int(offsets[i]), sizes[i][0] * sizes[i][1]
        out[i] = [np.asarray(f[o:o + m].cpu() if hasattr(f, "cpu") else f[o:o + m], dtype=np.float64)
                  for f in fields]
    return out


def rel_l2_patches(gpu_patches, oracle_res):
    """Relative L2 (Ex, Ey, c Bz together, over all sampled patches) and the
    largest per-patch value, GPU fields of the patches vs the oracle."""
    num = den = 0.0
    worst = 0.0
    for (i, _el, ex, ey, bz) in oracle_res:
        got = np.concatenate(gpu_patches[i])
        want = np.concatenate([ex.ravel(), ey.ravel(), bz.ravel()])
        n2, d2 = float(np.sum((got - want) ** 2)), float(np.sum(want ** 2))
        num += n2
        den += d2
        worst = max(worst, math.sqrt(n2 / d2))
    return math.sqrt(num / den), worst


def batch_algorithmic_bytes(sizes):
    """Algorithmic bytes of each pass over all patches (see algorithmic_bytes)."""
    tot = {}
    for nx, ny in sizes:
        for k, v in algorithmic_bytes(nx, ny, 1, N_IN, N_OUT).items():
            tot[k] = tot.get(k, 0) + v
    return tot


def time_batch(capi, torch, prec, sizes, Jhost, args, dev, stream, sample_clocks, nsteps=None, persistent=None,
               forked=True):
    """A batch at precision `prec`: W untimed steps (one call: the step graph is
    recorded and replayed), then one psatd_batch_step(nsteps = K) call between
    CUDA events on the batch's stream.  Per-kernel event pairs are recorded in the
    graph (their times are the last replay's).  The mixed-precision batch is
    autotuned per size class at creation (its shapes are then cached for the
    process); the FP32 batch keeps the built-in shapes, which ran faster for it
    (each class is tuned alone, while the batch runs the classes side by side).
    Returns (ms, kernel times, clocks, batch, (Ex, Ey, Bz, Jx, Jy))."""
    K = nsteps or args.steps
    b = capi.Batch(sizes, (BATCH_DX, BATCH_DX), BATCH_DT, layout="te", prec=prec, src="J", stream=stream,
                   autotune=(prec != "fp32"))
    if persistent is not None:
        b.set_persistent(persistent)
    if not forked:
        b.set_branches(False)
    tot = b.total
    Ex, Ey, Bz = (torch.zeros(tot, device=dev) for _ in range(3))
    Jx = torch.from_numpy(Jhost[0]).to(dev)
    Jy = torch.from_numpy(Jhost[1]).to(dev)
    b.set_timing(True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        b.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy, None], nsteps=args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
        time.sleep(0.3)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy, None], nsteps=K)
        e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    kt = b.kernel_times()
    kt["_launches_per_step"] = (b.launches_per_step(), 0.0)
    b.set_timing(False)
    b.sync()  # raises if a tensor-core pass reported an expired wait
    if not bool(torch.isfinite(Ey).all()):
        raise RuntimeError("non-finite field after the timed steps")
    return ms, kt, clk, b, (Ex, Ey, Bz, Jx, Jy)


def batch_e2e(torch, b, Jhost, stream, nsteps):
    """End to end through psatd_batch_step with E, B and J in pinned host memory:
    (a) the passes read the host arrays and write E, B back over the host link
    inside the step (the library's host-buffer mode, one call of nsteps steps);
    (b) staged: per step, copies of the five inputs to device arrays, the step,
    copies of the three outputs back.  Returns (value a, value b) in cell-steps/s."""
    tot = b.total
    hE = [torch.zeros(tot).pin_memory() for _ in range(3)]
    hJ = [torch.from_numpy(Jhost[0]).pin_memory(), torch.from_numpy(Jhost[1]).pin_memory()]
    dE = [torch.empty(tot, device="cuda") for _ in range(3)]
    dJ = [torch.empty(tot, device="cuda") for _ in range(2)]
    out = []
    for staged in (False, True):
        for it in range(2):
            n = nsteps if it else 1
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                if staged:
                    for _ in range(n):
                        for h, d_ in zip(hE + hJ, dE + dJ):
                            d_.copy_(h, non_blocking=True)
                        b.step([dE[0], dE[1], None], [None, None, dE[2]], [dJ[0], dJ[1], None])
                        for h, d_ in zip(hE, dE):
                            h.copy_(d_, non_blocking=True)
                else:
                    b.step([hE[0], hE[1], None], [None, None, hE[2]], [hJ[0], hJ[1], None], nsteps=n)
                e1.record(stream)
            torch.cuda.synchronize()
        out.append(tot * nsteps / (e0.elapsed_time(e1) * 1e-3))
    b.sync()
    return out[0], out[1]


def roofline_of(ktimes, bytes_of, hbm, peak_kind, traffic_lookup=True, note=None, traffic_prefix=""):
    """Roofline object of the kernel with the largest summed time: the algorithmic
    bytes of its timed launches (bytes_of(kernel, launches)) over their summed
    CUDA-event time, against `hbm`.  `traffic`: the stored ncu DRAM bytes per launch
    of that kernel (entry `traffic_prefix` + kernel name in profiles/dram_traffic.json)
    while the CUDA sources are unchanged since the capture, else null."""
    if not ktimes:
        return None
    dom = max(ktimes, key=lambda k: ktimes[k][1])
    n_l, tot = ktimes[dom]
    nbytes = bytes_of(dom, n_l)
    achieved = nbytes / (tot * 1e-3) / 1e9
    traffic = None
    if traffic_lookup:
        try:
            tr = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
            ent = tr.get(traffic_prefix + dom)
            if ent and ent.get("source_hash") == source_hash():
                traffic = ent["bytes_per_launch"]
        except Exception:
            pass
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
           "traffic": traffic, "kernel": dom, "peak_kind": peak_kind, "launches": n_l,
           "algorithmic_bytes_per_launch": nbytes / n_l,
           "per_kernel_ms": {k: v[1] / v[0] for k, v in ktimes.items()}}
    if note:
        out["note"] = note
    return out


def step_bytes(pass_bytes_per_step, cells, ms_per_step, hbm):
    """Whole-step byte rates: the pass model (every pass's algorithmic bytes) and
    the compulsory bytes (5 inputs read once, 3 outputs written once, 4 B each)."""
    s = ms_per_step * 1e-3
    out = {}
    for name, nb in (("pass_model", pass_bytes_per_step), ("compulsory", 32.0 * cells)):
        gbs = nb / s / 1e9
        out[name] = {"bytes_per_cell": nb / cells, "gbs": gbs, "frac": gbs / hbm}
    return out


def run_batch_line(args, world, rank, local):
    """The metric's own configuration: 512 batched TE patches at the mixed precision
    (split-BF16 tensor-core stages) against plain FP32 on the same patches."""
    pool = ncores = None
    if rank == 0:
        pool, ncores = oracle_pool()  # spawned before the first CUDA call
    import torch
    from paper_1608_05739_gb300 import build as bld
    from paper_1608_05739_gb300 import capi, synth

    npatch = args.patches
    sizes, interior = synth.batch_patch_sizes(npatch, BATCH_SEED, mixed_ok=False)
    sizes_fp32, _ = synth.batch_patch_sizes(npatch, BATCH_SEED, mixed_ok=True)
    requested = synth.batch_requested_cells(npatch, BATCH_SEED)
    cells, cells_fp32 = sum(a * b for a, b in sizes), sum(a * b for a, b in sizes_fp32)
    offs = np.concatenate([[0], np.cumsum([a * b for a, b in sizes])]).astype(np.int64)
    offs32 = np.concatenate([[0], np.cumsum([a * b for a, b in sizes_fp32])]).astype(np.int64)
    K, W = args.steps, args.warmup
    cb = None
    pend = pend32 = None
    samp = samp32 = []
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            cb = batch_cpu_baseline(pool, ncores, sizes)
        # oracle references of sampled patches after the W + K steps, computed while the GPU runs
        samp = batch_sample(sizes, 2.0e7, W + K)
        samp32 = batch_sample(sizes_fp32, 2.0e7, W + K, seed=1618)
        pend = pool.map_async(_oracle_patch, [(i, sizes[i][0], sizes[i][1], W + K, True) for i in samp])
        pend32 = pool.map_async(_oracle_patch, [(i, sizes_fp32[i][0], sizes_fp32[i][1], W + K, True)
                                                for i in samp32])

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
    stream = torch.cuda.Stream()
    J = synth.batch_source(sizes, BATCH_J_SEED, BATCH_J_SCALE)
    J32 = synth.batch_source(sizes_fp32, BATCH_J_SEED, BATCH_J_SCALE)

    prec = args.precision if args.precision != "fp32" else "mixed_bf16"
    if world > 1:
        dist.barrier()
    ms, kt, clk, b, F = time_batch(capi, torch, prec, sizes, J, args, dev, stream, sample_clocks=True)
    value, t_max = replica_throughput(ms, cells, K, world, dev)
    gpu_fields = patch_fields(F[:3], sizes, offs, samp)
    launches_per_step = kt.pop("_launches_per_step")[0]
    # the roofline's timed region: the same batch and call with the size classes one after
    # another on the batch's stream, so that each launch's event time is its own
    ms_s, kt_s, _, b_s, F_s = time_batch(capi, torch, prec, sizes, J, args, dev, stream, sample_clocks=False,
                                         forked=False)
    kt_s.pop("_launches_per_step")
    b_s.destroy()
    del F_s
    # a longer series of the same call with its own clock record (at least ~2 s of steps)
    long_series = None
    n_long = int(math.ceil(2000.0 / (ms / K)))
    if n_long > K and not args.no_long_series:
        ms_l, _, clk_l, b_l, _ = time_batch(capi, torch, prec, sizes, J, args, dev, stream, sample_clocks=True,
                                            nsteps=n_long)
        b_l.destroy()
        long_series = {"steps": n_long, "ms_per_step": ms_l / n_long, "value": cells * n_long / (ms_l * 1e-3),
                       "clocks": clk_l}
    # the same batch and precision with the other launch mode (persistent passes or per-class launches)
    other = None
    if not args.no_side_precision:
        persistent_now = launches_per_step <= 6
        ms_o, kt_o, _, b_o, F_o = time_batch(capi, torch, prec, sizes, J, args, dev, stream, sample_clocks=False,
                                             persistent=not persistent_now)
        lps_o = kt_o.pop("_launches_per_step")[0]
        b_o.destroy()
        del F_o
        other = {"mode": "per-class launches on branch streams" if persistent_now else "persistent passes",
                 "ms_per_step": ms_o / K, "value": cells * K / (ms_o * 1e-3), "launches_per_step": lps_o,
                 "per_kernel_ms_summed": {k: v[1] for k, v in kt_o.items()}}
    e2e_a = e2e_b = None
    e2e_steps = max(3, min(K, 20))
    if not args.no_e2e:
        e2e_a, e2e_b = batch_e2e(torch, b, J, stream, e2e_steps)
    b.destroy()
    # plain FP32 on the same patches (same transform sizes), and on the sizes FP32 itself takes
    ms32, kt32, _, b32, F32 = time_batch(capi, torch, "fp32", sizes, J, args, dev, stream, sample_clocks=False)
    lps32 = kt32.pop("_launches_per_step")[0]
    f32_fields = patch_fields(F32[:3], sizes, offs, samp)
    b32.destroy()
    del F32
    msb, ktb, _, bb, Fb = time_batch(capi, torch, "fp32", sizes_fp32, J32, args, dev, stream, sample_clocks=False)
    lpsb = ktb.pop("_launches_per_step")[0]
    fb_fields = patch_fields(Fb[:3], sizes_fp32, offs32, samp32)
    bb.destroy()
    del Fb, F

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_kind = "measured"
    if not hbm:
        hbm, peak_kind = 6800.0, "fallback"
    alg_b = batch_algorithmic_bytes(sizes)
    alg_fb = batch_algorithmic_bytes(sizes_fp32)
    concurrent = ("persistent passes: one launch per pass type (and length family) over every patch, so a "
                  "launch's bytes are the whole batch's for that pass" if launches_per_step <= 6 else
                  "the size classes' kernels run side by side on the batch's branch streams, so each launch's "
                  "duration includes time shared with other classes' kernels")
    roof = roofline_of(kt_s, lambda k, n: alg_b[k], hbm, peak_kind,
                       traffic_lookup=(prec == "mixed_bf16" and len(sizes) == 512),
                       traffic_prefix="batch_",
                       note="the size classes one after another (%.3f ms per step; %.3f forked, the line's value): each "
                            "launch's own duration; the pass's launches over every class of one step" % (ms_s / K, ms / K))
    roof["forked_per_kernel_ms_summed"] = {k: v[1] for k, v in kt.items()}

    side = None
    if not args.no_side_precision and rank == 0:
        side = te2048_side(capi, torch, args, dev, world, hbm, peak_kind)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "patches": npatch, "precision": PREC_NOTE[prec],
                       "patch_sides": "powers of two (the tensor-core passes' lengths)",
                       "cells": cells, "interior_cells": interior, "requested_domain_cells": requested,
                       "size_classes": len(set(sizes)),
                       "value_counts": "cells of the transformed patch domains (interior + widened guards)",
                       "run": "one psatd_batch_step(nsteps = steps) call: a CUDA graph of one step replayed",
                       "launch_shapes": ("autotuned per size class at batch creation (lines per CTA of every pass, "
                                         "component groups of the fused pass)" if prec != "fp32" else "built-in"),
                       "launches_per_step": launches_per_step,
                       "l2": "not flushed: the inputs (%.2f GB) are 15x the 129 MB L2" % (5 * cells * 4 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "interior_cell_steps_per_s": value * interior / cells,
            "gpu_launches": launches_per_step * K,
            "roofline": roof,
            "step_bytes": step_bytes(sum(alg_b.values()), cells, t_max / K, hbm),
            "clocks": clk,
        }
        if long_series:
            line["long_series"] = long_series
        line["config"]["mode"] = "persistent passes" if launches_per_step <= 6 else "per-class launches"
        if other is not None:
            line["other_mode"] = other
        line["vs_plain_fp32"] = {
            "same_patches": {"precision": PREC_NOTE["fp32"], "value": cells * K / (ms32 * 1e-3),
                             "ms_per_step": ms32 / K, "ratio": (cells * K / (ms * 1e-3)) / (cells * K / (ms32 * 1e-3)),
                             "what": "FP32 batch on the same power-of-two patch sides; ratio = mixed / FP32",
                             "launch_shapes": "built-in (faster for FP32 in this batch than per-class autotuned "
                                              "shapes, which are tuned with each class alone)",
                             "launches_per_step": lps32,
                             "roofline": roofline_of(kt32, lambda k, n: alg_b[k], hbm, peak_kind,
                                                     traffic_lookup=False, note=concurrent),
                             "step_bytes": step_bytes(sum(alg_b.values()), cells, ms32 / K, hbm)},
            "fp32_own_sides": {"value": cells_fp32 * K / (msb * 1e-3), "ms_per_step": msb / K, "cells": cells_fp32,
                               "interior_cell_steps_per_s": interior * K / (msb * 1e-3),
                               "interior_ratio": (interior * K / (ms * 1e-3)) / (interior * K / (msb * 1e-3)),
                               "what": "FP32 batch with the sides FP32 takes (2^k or 3 * 2^k); interior_ratio = "
                                       "mixed / FP32 interior cell-steps/s",
                               "launches_per_step": lpsb,
                               "roofline": roofline_of(ktb, lambda k, n: alg_fb[k], hbm, peak_kind,
                                                       traffic_lookup=False, note=concurrent),
                               "step_bytes": step_bytes(sum(alg_fb.values()), cells_fp32, msb / K, hbm)},
        }
        if not args.no_e2e:
            line["e2e"] = {"value": e2e_a, "unit": "cell-steps/s", "h2d_bytes_per_step": 5 * cells * 4,
                           "d2h_bytes_per_step": 3 * cells * 4, "steps": e2e_steps,
                           "how": "psatd_batch_step on pinned host arrays: the x passes read E, B, J and write E, B "
                                  "in host memory over the host link, every step",
                           "staged_value": e2e_b,
                           "staged_how": "per step: cudaMemcpyAsync of the five inputs to device arrays, the "
                                         "step, copies of the three outputs back"}
        if pend is not None:
            ref = pend.get()
            ref32 = pend32.get()
            r, worst = rel_l2_patches(gpu_fields, ref)
            r32, worst32 = rel_l2_patches(f32_fields, ref)
            rb, worstb = rel_l2_patches(fb_fields, ref32)
            line["rel_l2_vs_oracle"] = {
                "value": r, "max_patch": worst, "steps": W + K, "patches": samp,
                "what": "Ex, Ey, c Bz of the sampled patches after the warm-up and timed steps (E = B = 0 at the "
                        "start, the same J), the line's precision vs the FP64 oracle on each patch alone"}
            line["vs_plain_fp32"]["same_patches"]["rel_l2_vs_oracle"] = {"value": r32, "max_patch": worst32}
            line["vs_plain_fp32"]["fp32_own_sides"]["rel_l2_vs_oracle"] = {"value": rb, "max_patch": worstb,
                                                                           "patches": samp32}
        if cb is not None:
            line["cpu_baseline"] = cb
        if side is not None:
            line["side_te2048"] = side
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.close()
    if world > 1:
        dist.destroy_process_group()


def te2048_side(capi, torch, args, dev, world, hbm, peak_kind):
    """Side key of the headline line: the single 2048^2 TE grid in FP32 (the
    fused pass k_line_push at its largest), with its own roofline."""
    dx = 1.0 / LAM_CELLS
    dt = dx / math.sqrt(2.0)
    stream = torch.cuda.current_stream()
    total = args.warmup + args.steps
    prof = torch.from_numpy(np.stack([sheet_profile(n, dt, dx) for n in range(total)])).float().to(dev)
    Jy_all = [prof[n].expand(NY, NX).contiguous() for n in range(total)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ms, kt, clk, plan = time_te2048(capi, torch, "fp32", args, dev, dt, dx, Jy_all, flush, stream, 1,
                                    sample_clocks=True)
    plan.destroy()
    return {"workload": WORKLOAD, "precision": PREC_NOTE["fp32"], "value": NX * NY * args.steps / (ms * 1e-3),
            "ms_per_step": ms / args.steps, "unit": "cell-steps/s",
            "l2": "flushed before every timed step (256 MiB write)",
            "roofline": roofline_of(kt, lambda k, n: algorithmic_bytes()[k] * n, hbm, peak_kind),
            "step_bytes": step_bytes(sum(algorithmic_bytes().values()), NX * NY, ms / args.steps, hbm),
            "clocks": clk}


def run_reference_batch(args, world, rank):
    """The reference arm on the headline's workload: the FP64 oracle as it stands on
    the host cores.  A step = every patch of the batch advanced one oracle step
    (patches spread over the pool's processes); runs until --steps steps or
    --ref-seconds, whichever comes first (after one untimed warm-up step)."""
    if rank != 0:
        return
    from paper_1608_05739_gb300 import synth
    pool, ncores = oracle_pool()
    sizes, _ = synth.batch_patch_sizes(512, BATCH_SEED, mixed_ok=False)
    cells = sum(a * b for a, b in sizes)
    order = sorted(range(len(sizes)), key=lambda i: -sizes[i][0] * sizes[i][1])
    jobs = [(i, sizes[i][0], sizes[i][1], 1, False) for i in order]
    if args.warmup > 0:
        pool.map(_oracle_patch, jobs[len(jobs) // 2:], chunksize=1)  # warm-up on half the patches
    steps = 0
    t0 = time.perf_counter()
    while steps < args.steps:
        pool.map(_oracle_patch, jobs, chunksize=1)
        steps += 1
        if time.perf_counter() - t0 > args.ref_seconds:
            break
    el = time.perf_counter() - t0
    pool.close()
    value = cells * steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "patches": 512, "cells": cells,
                   "precision": "fp64 (oracle, each patch a periodic grid of its own)"},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": ncores, "kind": "oracle",
                         "sample": "%d step(s) of all 512 patches (the full workload per step), one patch per "
                                   "process on %d processes" % (steps, ncores)},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_te2048(args, world, rank):
    """The FP64 CPU oracle on the host cores (bounded sample of the 2048^2 workload)."""
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


def cpu_baseline(seconds, with_state=False):
    """Time the oracle as it stands on a bounded sample of the workload (the first
    steps of the run from zero fields); with_state: also return the oracle's fields
    after those steps and their count, for the accuracy check of the same steps."""
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
    out = {"value": NX * NY * steps / el, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
           "sample": "%d FP64 oracle steps of the 2048^2 TE workload (numpy pocketfft, one thread), %.1f s"
                     % (steps, el)}
    return (out, E, B, steps) if with_state else out


def time_te2048(capi, torch, prec, args, dev, dt, dx, Jy_all, flush, stream, world, sample_clocks):
    """W untimed + K timed steps of the 2048^2 TE workload at precision `prec`
    from zero fields, L2 flushed before every timed step; returns the summed
    CUDA-event ms of the K steps, the per-kernel times, the clock record and the
    plan (kept for the end-to-end leg)."""
    plan = capi.Plan((NX, NY), (dx, dx), dt, layout="te", prec=prec, src="J", stream=stream)
    Ex = torch.zeros(NY, NX, device=dev)
    Ey = torch.zeros(NY, NX, device=dev)
    Bz = torch.zeros(NY, NX, device=dev)
    Jx = torch.zeros(NY, NX, device=dev)
    for n in range(args.warmup):
        plan.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy_all[n], None])
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    plan.set_timing(True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    for s in range(args.steps):
        flush.zero_()
        starts[s].record(stream)
        plan.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy_all[args.warmup + s], None])
        ends[s].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms = sum(starts[s].elapsed_time(ends[s]) for s in range(args.steps))
    ktimes = plan.kernel_times()
    plan.set_timing(False)
    plan.sync()  # raises if a tensor-core pass reported an expired wait
    if not bool(torch.isfinite(Ey).all()):
        raise RuntimeError("non-finite field after the timed steps")
    return ms, ktimes, clk, plan


def cufft_comparator(torch, args, dev, dt, dx, Jy_all, flush, stream, plan):
    """The same 2048^2 TE J-form step written with library calls, for context
    (not the product path): torch.fft (cuFFT) rfft2 of the five inputs, the
    per-mode update of the collocated exact-k scheme as torch elementwise ops on
    FP32 coefficient arrays (computed in FP64, Nyquist k := 0, c = eps0 = 1),
    irfft2 of the three fields.  Timed like the step (L2 flushed, CUDA events),
    and compared once with the library's step from the same random state."""
    c, eps0 = 1.0, 1.0
    kx = 2.0 * math.pi * torch.fft.rfftfreq(NX, d=dx, dtype=torch.float64, device=dev)
    ky = 2.0 * math.pi * torch.fft.fftfreq(NY, d=dx, dtype=torch.float64, device=dev)
    kx[NX // 2] = 0.0
    ky[NY // 2] = 0.0
    KX = kx[None, :].expand(NY, -1)
    KY = ky[:, None].expand(-1, NX // 2 + 1)
    k = torch.sqrt(KX * KX + KY * KY)
    zero = k == 0
    ks = torch.where(zero, torch.ones_like(k), k)
    C = torch.cos(c * k * dt)
    S = torch.sin(c * k * dt)
    sck = torch.where(zero, torch.full_like(k, dt), S / (c * ks))
    f32 = lambda t: t.float().contiguous()
    co = {"C": f32(C), "a1": f32(1.0 - C), "cS": f32(c * S), "sck": f32(sck), "sJ": f32(sck / eps0),
          "aJL": f32(torch.where(zero, torch.zeros_like(k), (sck - dt) / eps0)),
          "bJ": f32(torch.where(zero, torch.zeros_like(k), (1.0 - C) / (eps0 * c * c * ks * ks))),
          "kapx": f32(KX / ks), "kapy": f32(KY / ks), "kx": f32(KX), "ky": f32(KY)}

    def step(Ex, Ey, Bz, Jx, Jy):
        ex, ey, bz, jx, jy = torch.fft.rfft2(torch.stack([Ex, Ey, Bz, Jx, Jy]))
        kE = co["kapx"] * ex + co["kapy"] * ey
        kJ = co["kapx"] * jx + co["kapy"] * jy
        ex1 = co["C"] * ex + co["a1"] * co["kapx"] * kE + 1j * co["cS"] * co["kapy"] * bz - co["sJ"] * jx \
            + co["aJL"] * co["kapx"] * kJ
        ey1 = co["C"] * ey + co["a1"] * co["kapy"] * kE - 1j * co["cS"] * co["kapx"] * bz - co["sJ"] * jy \
            + co["aJL"] * co["kapy"] * kJ
        bz1 = co["C"] * bz - 1j * co["sck"] * (co["kx"] * ey - co["ky"] * ex) \
            + 1j * co["bJ"] * (co["kx"] * jy - co["ky"] * jx)
        out = torch.fft.irfft2(torch.stack([ex1, ey1, bz1]), s=(NY, NX))
        Ex.copy_(out[0])
        Ey.copy_(out[1])
        Bz.copy_(out[2])

    # agreement with the library's step from one random state
    g = torch.Generator(device=dev).manual_seed(1615)
    st = [torch.randn(NY, NX, device=dev, generator=g) for _ in range(5)]
    a = [t.clone() for t in st]
    step(a[0], a[1], a[2], a[3], a[4])
    b = [t.clone() for t in st]
    plan.step([b[0], b[1], None], [None, None, b[2]], [b[3], b[4], None])
    torch.cuda.synchronize()
    num = sum(float(torch.sum((a[i].double() - b[i].double()) ** 2)) for i in range(3))
    den = sum(float(torch.sum(b[i].double() ** 2)) for i in range(3))
    Ex, Ey, Bz, Jx = (torch.zeros(NY, NX, device=dev) for _ in range(4))
    steps = min(args.steps, 50)
    ms, _ = timed_steps(lambda i: step(Ex, Ey, Bz, Jx, Jy_all[i % len(Jy_all)]), steps, max(args.warmup, 3),
                        flush, stream)
    return {"what": "torch.fft (cuFFT) rfft2 / irfft2 + torch elementwise push, FP32, same workload; "
                    "context only, not the product path",
            "ms_per_step": ms / steps, "value": NX * NY * steps / (ms * 1e-3), "unit": "cell-steps/s",
            "rel_l2_vs_library_step": math.sqrt(num / den)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default=None, choices=["fp32", "mixed_fp16", "mixed_bf16"],
                    help="batch512: the mixed precision of the headline (default mixed_bf16); te2048: the "
                         "headline precision (default fp32; the others are timed too, under 'other_precision')")
    ap.add_argument("--no-side-precision", action="store_true",
                    help="skip the side keys (other precisions, the te2048 side line)")
    ap.add_argument("--no-comparator", action="store_true", help="skip timing the cuFFT comparator")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end legs (profiling runs: only the timed steps' kernels)")
    ap.add_argument("--patches", type=int, default=512,
                    help="batch512: patches of the batch (the first N of the 512-patch recipe; profiling runs)")
    ap.add_argument("--no-long-series", action="store_true", help="batch512: skip the >= 2 s clock series")
    ap.add_argument("--workload", default="batch512",
                    choices=["batch512", "te2048", "3d256", "3d512", "fdtd-yee", "fdtd-ckc", "local", "cost3d",
                             "small128", "batch512-side"],
                    help="batch512 (default) is the metric's configuration; the others are side measurements")
    args = ap.parse_args()
    if args.warmup < 2:
        ap.error("--warmup must be >= 2 (the warm-up call records the step graph)")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if args.workload == "te2048":
            run_reference_te2048(args, world, rank)
        else:
            run_reference_batch(args, world, rank)
        return
    if args.workload == "batch512":
        args.precision = args.precision or "mixed_bf16"
        run_batch_line(args, world, rank, local)
        return
    args.precision = args.precision or "fp32"
    if args.workload != "te2048":
        if args.workload == "batch512-side":
            args.workload = "batch512"
        run_side_workload(args)
        return
    run_te2048_line(args, world, rank, local)


def run_te2048_line(args, world, rank, local):
    """Side line: the single 2048^2 TE grid (one psatd_step per step), all precisions."""
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
    total = args.warmup + args.steps
    prof = torch.from_numpy(np.stack([sheet_profile(n, dt, dx) for n in range(total)])).float().to(dev)
    Jy_all = [prof[n].expand(NY, NX).contiguous() for n in range(total)]  # resident before timing
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    side = None
    if not args.no_side_precision:
        side = []
        for other in (pr for pr in PREC_NOTE if pr != args.precision):
            side_ms, side_kt, _, side_plan = time_te2048(capi, torch, other, args, dev, dt, dx, Jy_all, flush,
                                                         stream, world, sample_clocks=False)
            side_plan.destroy()
            side.append({"precision": PREC_NOTE[other], "dtype": DTYPE[other],
                         "value": NX * NY * args.steps / (side_ms * 1e-3), "unit": "cell-steps/s",
                         "ms_per_step": side_ms / args.steps,
                         "per_kernel_ms": {k: v[1] / v[0] for k, v in side_kt.items()}})
    ms, ktimes, clk, plan = time_te2048(capi, torch, args.precision, args, dev, dt, dx, Jy_all, flush, stream,
                                        world, sample_clocks=True)

    # end to end through the C ABI with the fields and sources in pinned host memory: (a) the
    # passes read and write the host arrays in place over the host link (the library's
    # host-buffer mode), (b) staged: explicit copies to device arrays and back around each step
    hE = [torch.zeros(NY, NX).pin_memory() for _ in range(3)]
    hJ = [torch.zeros(NY, NX).pin_memory(), Jy_all[0].cpu().pin_memory()]
    dE = [torch.empty(NY, NX, device=dev) for _ in range(3)]
    dJ = [torch.empty(NY, NX, device=dev) for _ in range(2)]
    e2e_steps = max(10, min(args.steps, 50))

    def e2e_run(staged):
        for it in range(2):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s in range(e2e_steps if it else 2):
                if staged:
                    for h, d_ in zip(hE, dE):
                        d_.copy_(h, non_blocking=True)
                    for h, d_ in zip(hJ, dJ):
                        d_.copy_(h, non_blocking=True)
                    plan.step([dE[0], dE[1], None], [None, None, dE[2]], [dJ[0], dJ[1], None])
                    for h, d_ in zip(hE, dE):
                        h.copy_(d_, non_blocking=True)
                else:
                    plan.step([hE[0], hE[1], None], [None, None, hE[2]], [hJ[0], hJ[1], None])
            e1.record(stream)
            torch.cuda.synchronize()
        return NX * NY * e2e_steps / (e0.elapsed_time(e1) * 1e-3)

    plan.set_timing(False)
    e2e_value = e2e_staged = None
    if not args.no_e2e:
        e2e_value = e2e_run(False)
        e2e_staged = e2e_run(True)

    comparator = None
    if rank == 0 and not args.no_comparator:
        comparator = cufft_comparator(torch, args, dev, dt, dx, Jy_all, flush, stream, plan)

    cells = NX * NY
    value, t_max = replica_throughput(ms, cells, args.steps, world, dev)

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
            "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NX, NY], "precision": PREC_NOTE[args.precision],
                       "l2": "flushed before every timed step (256 MiB write), step alone inside the events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": 5 * cells * 4,
                    "d2h_bytes_per_step": 3 * cells * 4,
                    "how": "psatd_step on pinned host arrays: the x passes read E, B, J and write E, B in host "
                           "memory over the host link, each step",
                    "staged_value": e2e_staged,
                    "staged_how": "cudaMemcpyAsync of the five inputs to device arrays and of the three "
                                  "outputs back, around each step"},
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": clk,
        }
        # whole-step byte efficiency: compulsory (each input read once, each output written
        # once: 5 x 4 + 3 x 4 B per cell) and the three-pass model (sum of the passes' bytes)
        step_s = t_max / args.steps * 1e-3
        for name, bpc in (("compulsory", 32.0), ("pass_model", sum(alg.values()) / cells)):
            gbs = bpc * cells / step_s / 1e9
            line["step_bytes_" + name] = {"bytes_per_cell": bpc, "gbs": gbs, "frac": gbs / hbm}
        if comparator is not None:
            line["cufft_comparator"] = comparator
        if side is not None:
            line["other_precision"] = side
        if world == 1 and not args.no_cpu_baseline:
            cb, Eo, Bo, nst = cpu_baseline(args.cpu_seconds, with_state=True)
            line["cpu_baseline"] = cb
            # the same first steps on the GPU path at the headline precision, against the oracle
            p2 = capi.Plan((NX, NY), (dx, dx), dt, layout="te", prec=args.precision, src="J", stream=stream)
            G = [torch.zeros(NY, NX, device=dev) for _ in range(4)]
            for n in range(nst):
                Jn = torch.from_numpy(sheet_profile(n, dt, dx)).float().to(dev).expand(NY, NX).contiguous()
                p2.step([G[0], G[1], None], [None, None, G[2]], [G[3], Jn, None])
            p2.sync()
            p2.destroy()
            got = np.concatenate([G[i].double().cpu().numpy().ravel() for i in range(3)])
            want = np.concatenate([Eo[0].ravel(), Eo[1].ravel(), Bo[2].ravel()])
            line["rel_l2_vs_oracle"] = {
                "value": float(np.linalg.norm(got - want) / np.linalg.norm(want)), "steps": nst,
                "what": "E, B after the oracle sample's steps (same J, zero initial fields), GPU at the line's "
                        "precision vs the FP64 oracle; relative L2 over Ex, Ey, Bz"}
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        dist.destroy_process_group()


def timed_steps(step, steps, warmup, flush, stream):
    """Run ``warmup`` untimed steps, then ``steps`` steps each preceded by an L2
    flush and bracketed by CUDA events on ``stream``; returns total ms and clocks."""
    import torch
    for n in range(warmup):
        step(n)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    for s in range(steps):
        flush.zero_()
        starts[s].record(stream)
        step(warmup + s)
        ends[s].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return sum(starts[s].elapsed_time(ends[s]) for s in range(steps)), clk


def run_side_workload(args):
    """Side measurements (not the metric's line): the 3D step of the Gaussian-charge
    workload and the FDTD comparators on the 2048^2 TE grid."""
    import torch
    from paper_1608_05739_gb300 import build as bld
    from paper_1608_05739_gb300 import capi, synth
    bld.build()
    capi.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    line = {"metric": METRIC + " (side measurement)", "unit": "cell-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic"}
    if args.workload == "3d256":
        n = 256
        d = 1.0
        dt = 0.5 * d
        r0, r1, J, E = synth.gaussian_charges_torch((n, n, n), (d, d, d), dt, n_charges=64, seed=1610, device=dev)
        E = [E[i].contiguous() for i in range(3)]
        B = [torch.zeros(n, n, n, device=dev) for _ in range(3)]
        J = [J[i].contiguous() for i in range(3)]
        plan = capi.Plan((n, n, n), (d, d, d), dt, layout="3d6", prec="fp32", src="rho", stream=stream)
        plan.set_timing(True)
        ms, clk = timed_steps(lambda i: plan.step(E, B, J, r0, r1), args.steps, args.warmup, flush, stream)
        kt = plan.kernel_times()
        alg = algorithmic_bytes(n, n, n, 11, 6)
        cells = n ** 3
        per = {k: v[1] / v[0] for k, v in kt.items()}
        line.update({
            "value": cells * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
            "config": {"workload": "3D PSATD 256^3 FP32, rho-form, 64 moving Gaussian charges (sigma = 3 dx, "
                                   "|v| < 0.5c), c dt = 0.5 dx, sources held over the run",
                       "l2": "flushed before every timed step"},
            "per_kernel_ms": per,
            "per_kernel_gbs": {k: alg[k] / (per[k] * 1e-3) / 1e9 for k in per},
            "step_algorithmic_bytes_per_cell": sum(alg.values()) / cells,
            "hbm_gbs_peak": hbm, "clocks": clk, "gpu_launches": sum(v[0] for v in kt.values()),
        })
        plan.destroy()
    elif args.workload == "3d512":
        # the large 3D workload: 512 x 512 x 1024 cells, rho-form, divergence-free k^-2 fields plus
        # 1e5 moving Gaussian charges (sigma = 3 dx), c dt = 0.5 dx; FP32 and split-FP16 tensor-core
        # stages on the same inputs (each from the same initial state), L2 flushed before every step
        shape = (1024, 512, 512)
        d = (1.0, 1.0, 1.0)
        dt = 0.5
        E0, B0, J, r0, r1 = synth.large_3d_inputs_torch(shape, d, dt, seed=1614, device=dev)
        J = [J[i] for i in range(3)]
        cells = 512 * 512 * 1024
        alg = algorithmic_bytes(512, 512, 1024, 11, 6)
        res = {}
        clk = None
        for prec in ("fp32", "mixed_fp16"):
            E = [E0[i].clone() for i in range(3)]
            B = [B0[i].clone() for i in range(3)]
            plan = capi.Plan((512, 512, 1024), d, dt, layout="3d6", prec=prec, src="rho", stream=stream)
            plan.set_timing(True)
            ms, c_ = timed_steps(lambda i: plan.step(E, B, J, r0, r1), args.steps, args.warmup, flush, stream)
            kt = plan.kernel_times()
            plan.sync()
            plan.destroy()
            clk = clk or c_
            per = {k: v[1] / v[0] for k, v in kt.items()}
            res[prec] = {"ms_per_step": ms / args.steps, "value": cells * args.steps / (ms * 1e-3),
                         "per_kernel_ms": per, "gpu_launches": sum(v[0] for v in kt.values()),
                         "per_kernel_gbs": {k: alg[k] / (per[k] * 1e-3) / 1e9 for k in per}}
            del E, B
        line.update({
            "value": res["fp32"]["value"], "ms_per_step": res["fp32"]["ms_per_step"],
            "config": {"workload": "3D PSATD 512x512x1024, rho-form, divergence-free fields with |F(k)|^2 ~ k^-2 "
                                   "plus 1e5 moving Gaussian charges (sigma = 3 dx, |v| < 0.5c), c dt = 0.5 dx",
                       "l2": "flushed before every timed step", "state_gb": 11 * cells * 4 / 1e9},
            "fp32": res["fp32"], "mixed_fp16": res["mixed_fp16"],
            "step_algorithmic_bytes_per_cell": sum(alg.values()) / cells,
            "hbm_gbs_peak": hbm, "clocks": clk, "gpu_launches": res["fp32"]["gpu_launches"],
        })
    elif args.workload == "batch512":
        # 512 local-FFT patches (Sec. II.A.3): interior n ~ U{64..512} per side, guard g ~ U{8..16},
        # each patch a periodic domain whose side is the smallest transform length >= n + 2g: a power
        # of two, or (FP32) 3 * 2^k from 96 up; TE J-form, smooth random J; the whole run is one
        # psatd_batch_step call (a CUDA graph of one step replayed `steps` times)
        mixed_ok = args.precision == "fp32"
        sizes, interior = synth.batch_patch_sizes(512, 1612, mixed_ok=mixed_ok)
        dx = 1.0 / LAM_CELLS
        dt = dx / math.sqrt(2.0)
        side_stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        b = capi.Batch(sizes, (dx, dx), dt, layout="te", prec=args.precision, src="J", stream=side_stream)
        tot = b.total
        Ex, Ey, Bz = (torch.zeros(tot, device=dev) for _ in range(3))
        Jx = torch.randn(tot, device=dev, generator=torch.Generator(device=dev).manual_seed(1613)) * 0.01
        Jy = torch.randn(tot, device=dev, generator=torch.Generator(device=dev).manual_seed(1614)) * 0.01
        torch.cuda.synchronize()
        with torch.cuda.stream(side_stream):
            b.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy, None], nsteps=args.warmup)  # records the graph
            side_stream.synchronize()
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            clocks = ClockSampler(0)
            clocks.start()
            time.sleep(0.3)
            e0.record(side_stream)
            b.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy, None], nsteps=args.steps)
            e1.record(side_stream)
            side_stream.synchronize()
            clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        classes = len(set(sizes))
        alg = float(sum(sum(algorithmic_bytes(nx, ny, 1, 5, 3).values()) for (nx, ny) in sizes))
        line.update({
            "value": tot * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
            "interior_cell_steps_per_s": interior * args.steps / (ms * 1e-3),
            "dtype": DTYPE[args.precision],
            "config": {"workload": "512 2D TE patches, interior U{64..512}^2, guards U{8..16}, periodic domain "
                                   "of the smallest transform length >= n+2g per side (%s), J-form, one CUDA "
                                   "graph of one step replayed" % ("2^k or 3*2^k" if mixed_ok else "2^k"),
                       "precision": PREC_NOTE[args.precision],
                       "cells": tot, "interior_cells": interior, "size_classes": classes,
                       "l2": "inputs %.1f GB >> L2, flushed once before the run" % (tot * 5 * 4 / 1e9)},
            "step_gbs": alg / (ms / args.steps * 1e-3) / 1e9, "hbm_gbs_peak": hbm, "clocks": clk,
            "gpu_launches": 3 * classes * args.steps,
        })
        b.destroy()
    elif args.workload == "cost3d":
        # Table 2 (Sec. V) restated for the field solvers on this GPU: per cell-step cost of each
        # scheme on one 3D 256^3 grid (FP32, J-form, L2 flushed before every step), the field-solver
        # xi = t(PSATD-128) / t(Yee), and the paper's time factors with its resolution factor
        # A = 2.3 (FDTD, lambda/322 vs lambda/140) and its PSTD step ratio 9 (c dt 0.110 dx).
        n = 256
        d = 1.0
        cells = n ** 3
        r0, r1, J, E0 = synth.gaussian_charges_torch((n, n, n), (d, d, d), 0.5, n_charges=64, seed=1610, device=dev)
        J = [J[i].contiguous() for i in range(3)]
        E = [E0[i].contiguous() for i in range(3)]
        B = [torch.zeros(n, n, n, device=dev) for _ in range(3)]
        res = {}
        for name, kw, dtc in (("psatd_order128", dict(order=128), 0.99), ("psatd_exact_k", dict(order=0), 0.99),
                              ("pstd", dict(order=0, scheme="pstd"), 0.110)):
            plan = capi.Plan((n, n, n), (d, d, d), dtc * d, layout="3d6", prec=args.precision, src="J",
                             stream=stream, **kw)
            ms, _ = timed_steps(lambda i: plan.step(E, B, J), args.steps, args.warmup, flush, stream)
            plan.sync()
            plan.destroy()
            res[name] = ms / args.steps
        dty = d / math.sqrt(3.0) * 0.99
        ms, clk = timed_steps(lambda i: capi.fdtd_step((n, n, n), (d, d, d), dty, E, B, J, scheme="yee", layout="3d6",
                                                       prec="fp32", stream=stream), args.steps, args.warmup, flush,
                              stream)
        res["yee"] = ms / args.steps
        xi = res["psatd_order128"] / res["yee"]
        A = 2.3
        line.update({
            "value": cells / (res["psatd_order128"] * 1e-3), "ms_per_step": res["psatd_order128"],
            "config": {"workload": "3D 256^3 FP32 J-form: PSATD order 128 (staggered), PSATD exact k, PSTD, Yee FDTD; "
                                   "Table 2 time factors restated with this GPU's field-solver xi",
                       "precision": PREC_NOTE[args.precision], "l2": "flushed before every timed step"},
            "ns_per_cell_step": {k: v * 1e6 / cells for k, v in res.items()},
            "xi_field_solver": xi,
            "paper_xi_full_pic_mira": 1.8,
            "time_factor_vs_psatd128": {"yee (A^4/xi, A = 2.3)": A ** 4 / xi,
                                        "pstd (9 x step cost ratio)": 9.0 * res["pstd"] / res["psatd_order128"]},
            "paper_time_factors": {"ckc": 16, "yee": 28, "pstd": 9},
            "clocks": clk, "gpu_launches": None,
        })
    elif args.workload == "small128":
        # the small FP64 case: 2D 128^2, six components, vacuum, 8 on-grid plane waves, c dt = 0.5 dx,
        # PSATD and Yee; the whole state (3 MB) stays in L2, so these are L2-resident times, not an
        # HBM measurement (no flush between steps; the run is a sequence of steps, as in use)
        n = 128
        waves = synth.plane_waves((n, n), 8, seed=1608)
        E0, B0 = synth.plane_wave_fields(waves, (n, n), (1.0, 1.0))
        res = {}
        clk = None
        for scheme in ("psatd", "yee"):
            E = [torch.from_numpy(E0[i]).to(dev, torch.float64) for i in range(3)]
            B = [torch.from_numpy(B0[i]).to(dev, torch.float64) for i in range(3)]
            if scheme == "psatd":
                plan = capi.Plan((n, n), (1.0, 1.0), 0.5, layout="2d6", prec="fp64", src="none", stream=stream)
                step = lambda i: plan.step(E, B)
            else:
                step = lambda i: capi.fdtd_step((n, n), (1.0, 1.0), 0.5, E, B, scheme="yee", layout="2d6",
                                                prec="fp64", stream=stream)
            for i in range(args.warmup):
                step(i)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            clocks = ClockSampler(0)
            clocks.start()
            time.sleep(0.3)
            e0.record(stream)
            for i in range(args.steps):
                step(i)
            e1.record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
            res[scheme] = e0.elapsed_time(e1) / args.steps
            if scheme == "psatd":
                plan.destroy()
        line.update({
            "value": n * n / (res["psatd"] * 1e-3), "ms_per_step": res["psatd"], "dtype": "f64",
            "config": {"workload": "2D 128^2 FP64 six-component vacuum, 8 on-grid plane waves, c dt = 0.5 dx",
                       "l2": "L2-resident (3 MB of state): a latency/launch-bound time, not an HBM figure"},
            "ms_per_step_yee": res["yee"], "clocks": clk, "gpu_launches": 3 * args.steps,
        })
    elif args.workload == "local":
        # the paper's decomposition (Sec. II.A.3): a 3840 x 1920 TE grid as 16 x 8 patches of 240^2
        # interior cells with 8 guard cells (extended 256^2), guards refreshed from the neighbours every
        # step, each patch advanced by its own FFTs; staggered PSATD of order 16 (Table 1, PSATD-p)
        px, py, gd, order = 16, 8, 8, 16
        nx, ny = px * 240, py * 240
        dx = 1.0 / LAM_CELLS
        dt = dx / math.sqrt(2.0)
        L = capi.Local((nx, ny), (dx, dx), dt, px=px, py=py, guard=gd, layout="te", prec=args.precision, src="J",
                       order=order, stream=stream)
        Ex, Ey, Bz = (torch.zeros(ny, nx, device=dev) for _ in range(3))
        Jx = torch.zeros(ny, nx, device=dev)
        total = args.warmup + args.steps
        prof = torch.from_numpy(np.stack([sheet_profile(k, dt, dx, nx) for k in range(total)])).float().to(dev)
        Jy = [prof[k].expand(ny, nx).contiguous() for k in range(total)]
        ms, clk = timed_steps(lambda i: L.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy[i], None]), args.steps,
                              args.warmup, flush, stream)
        L.sync()
        cells = nx * ny
        ext = px * py * (240 + 2 * gd) ** 2
        alg = sum(algorithmic_bytes(256, 256, 1, 5, 3).values()) * px * py
        guard_bytes = 4 * (5 * ext + 5 * ext + 3 * cells + 3 * cells)  # gathers (read + write), scatter
        line.update({
            "value": cells * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
            "dtype": DTYPE[args.precision],
            "config": {"workload": "2D TE local-FFT decomposition: 3840x1920 grid, 16x8 patches of 240^2 + 8 guard "
                                   "cells (extended 256^2), staggered PSATD order 16, current-sheet J",
                       "precision": PREC_NOTE[args.precision], "cells": cells, "extended_cells": ext,
                       "l2": "flushed before every timed step"},
            "step_gbs": (alg + guard_bytes) / (ms / args.steps * 1e-3) / 1e9, "hbm_gbs_peak": hbm, "clocks": clk,
            "gpu_launches": 6 * args.steps,
        })
        L.destroy()
    else:
        scheme = args.workload.split("-")[1]
        dx = 1.0 / LAM_CELLS
        dt = dx / math.sqrt(2.0)
        Ex, Ey, Bz, Jx = (torch.zeros(NY, NX, device=dev) for _ in range(4))
        total = args.warmup + args.steps
        prof = torch.from_numpy(np.stack([sheet_profile(k, dt, dx) for k in range(total)])).float().to(dev)
        Jy = [prof[k].expand(NY, NX).contiguous() for k in range(total)]
        ms, clk = timed_steps(lambda i: capi.fdtd_step((NX, NY), (dx, dx), dt, [Ex, Ey, None], [None, None, Bz],
                                                       [Jx, Jy[i], None], scheme=scheme, layout="te", prec="fp32",
                                                       stream=stream), args.steps, args.warmup, flush, stream)
        cells = NX * NY
        # per step: two B half steps (read Ex, Ey, Bz, write Bz) and one E step
        # (read Ex, Ey, Bz, Jx, Jy, write Ex, Ey), 4-byte values, neighbours from cache
        bytes_step = cells * 4 * (2 * (3 + 1) + (5 + 2))
        line.update({
            "value": cells * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
            "config": {"workload": "2D TE %s FDTD 2048x2048 FP32, current-sheet J, dx=lambda/64, c dt=dx/sqrt(2)"
                                   % scheme.upper(), "l2": "flushed before every timed step"},
            "step_gbs": bytes_step / (ms / args.steps * 1e-3) / 1e9, "hbm_gbs_peak": hbm, "clocks": clk,
            "gpu_launches": 3 * args.steps,
        })
    print(json.dumps(line), flush=True)


def source_hash():
    """Hash of the CUDA sources with comments and blank space removed: changes to the
    code (not to its comments) invalidate the stored ncu DRAM figures."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1608_05739_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            text = open(os.path.join(csrc, f)).read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(f.encode())
            h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
