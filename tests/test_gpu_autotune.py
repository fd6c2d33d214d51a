"""GPU checks of the launch-shape autotuner (psatd_plan_autotune) and of every
launch shape it may choose (psatd_plan_set_launch): the radix schedule of the
fused pass (radix-8 or radix-16 stages) and the lines per CTA of every pass.

Lines per CTA change neither the arithmetic nor its order within a line, so all
shapes with the same radix schedule give bitwise identical fields; each radix
schedule is checked against the FP64 oracle at the precision's bound."""
import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, psatd_gpu, rel_l2_fields, rounded
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "mixed_fp16": 4e-6}


def _inputs(shape, layout, seed, prec):
    E = rounded(mask_layout(synth.random_fields(shape, 3, seed), layout, "E"), prec)
    B = rounded(mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B"), prec)
    J = rounded(mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J"), prec)
    return E, B, J


def _shapes(plan, ndim):
    """Every accepted launch configuration, one knob varied at a time."""
    out = []
    passes = [0, 3] if ndim == 2 else [0, 1, 2, 3]
    for k in passes:
        for lg in range(6):
            cfg = [-1] * 6
            cfg[k] = lg
            try:
                plan.set_launch(cfg)
            except capi.PsatdError:
                continue
            out.append(cfg)
    for ept in (8, 16):
        for tb in (1, 2, 4, 8, 16, 32, 64, 128):
            cfg = [-1, -1, -1, -1, tb, ept]
            try:
                plan.set_launch(cfg)
            except capi.PsatdError:
                continue
            out.append(cfg)
    return out


@pytest.mark.parametrize("prec,shape,layout", [
    ("fp32", (256, 512), "te"), ("fp64", (128, 64), "2d6"), ("fp32", (32, 64, 128), "3d6"),
    ("mixed_fp16", (256, 512), "te"),
])
def test_every_launch_shape_matches_oracle(prec, shape, layout):
    ensure_lib()
    d = (1.0, 0.8, 1.1)[:len(shape)]
    dt = 0.5
    E, B, J = _inputs(shape, layout, 31, prec)
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    Eo, Bo = mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")
    plan = capi.Plan(tuple(reversed(shape)), d, dt, layout=layout, prec=prec, src="J")
    shapes = _shapes(plan, len(shape))
    assert len(shapes) >= 4
    ref = {}
    for cfg in shapes:
        plan.set_launch(cfg)
        got = plan.get_launch()
        for i, v in enumerate(cfg):
            if v >= 0:
                assert got[i] == v
        Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout=layout, prec=prec, src="J", plan=plan)
        assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL[prec], cfg
        ept = got[5]
        if ept in ref:   # same radix schedule: bitwise identical
            assert np.array_equal(Eg, ref[ept][0]) and np.array_equal(Bg, ref[ept][1]), cfg
        else:
            ref[ept] = (Eg, Bg)
    if prec != "mixed_fp16":
        assert set(ref) == {8, 16}
    else:
        assert set(ref) == {16}
        with pytest.raises(capi.PsatdError):
            plan.set_launch([-1, -1, -1, -1, -1, 8])   # tensor-core stages are radix 16
    plan.destroy()


def test_autotune_report_and_choice():
    ensure_lib()
    shape, d, dt = (512, 512), (1.0, 1.0), 0.5
    E, B, J = _inputs(shape, "te", 7, "fp32")
    plan = capi.Plan((512, 512), d, dt, layout="te", prec="fp32", src="J")
    rep = plan.autotune(3)
    for key in ("fwd_x", "inv_x", "push"):
        assert key in rep
    assert rep.count("*") == 3
    cfg = plan.get_launch()
    assert cfg[5] in (8, 16) and cfg[4] >= 1
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", plan=plan)
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL["fp32"]
    plan.destroy()


def test_autotune_flag_uses_the_process_cache():
    import time
    ensure_lib()
    n, d, dt = (256, 128), (1.0, 1.0), 0.5
    capi.Plan(n, d, dt, layout="te", prec="fp32", src="J").destroy()   # one-time costs out of the timing
    t0 = time.perf_counter()
    p1 = capi.Plan(n, d, dt, layout="te", prec="fp32", src="J", autotune=True)
    t1 = time.perf_counter()
    p2 = capi.Plan(n, d, dt, layout="te", prec="fp32", src="J", autotune=True)
    t2 = time.perf_counter()
    assert p1.get_launch() == p2.get_launch()
    assert t2 - t1 < t1 - t0   # the second plan recalls the shapes instead of timing them
    p1.destroy()
    p2.destroy()


def test_autotuned_batch_matches_oracle():
    import torch
    ensure_lib()
    sizes = [(64, 64), (128, 32), (64, 64), (256, 128)]
    d, dt = (1.0, 1.0), 0.5
    per = [_inputs((ny, nx), "te", 50 + 10 * i, "fp32") for i, (nx, ny) in enumerate(sizes)]
    pe, pb, pj = capi.PRESENT["te"]

    def packed(arrs):
        return torch.from_numpy(np.concatenate([a.ravel() for a in arrs])).to(device="cuda", dtype=torch.float32)

    Et = [packed([p[0][i] for p in per]) if pe[i] else None for i in range(3)]
    Bt = [packed([p[1][i] for p in per]) if pb[i] else None for i in range(3)]
    Jt = [packed([p[2][i] for p in per]) if pj[i] else None for i in range(3)]
    b = capi.Batch(sizes, d, dt, layout="te", prec="fp32", src="J", autotune=True)
    b.step(Et, Bt, Jt)
    torch.cuda.synchronize()
    off = 0
    for (nx, ny), (E, B, J) in zip(sizes, per):
        n = nx * ny
        Eg = np.zeros((3, ny, nx))
        Bg = np.zeros((3, ny, nx))
        for i in range(3):
            if pe[i]:
                Eg[i] = Et[i][off:off + n].double().cpu().numpy().reshape(ny, nx)
            if pb[i]:
                Bg[i] = Bt[i][off:off + n].double().cpu().numpy().reshape(ny, nx)
        Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
        assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL["fp32"]
        off += n
    b.destroy()
