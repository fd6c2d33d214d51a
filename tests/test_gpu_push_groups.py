"""Component groups of the fused pass (psatd_plan_set_push_groups).

With G > 1 each line's input components are forward-transformed, and its
output components inverse-transformed, by G thread groups in turn, which meet
only for the per-mode push (tensor-core plans: two groups in lockstep, one
128-row MMA group each, sharing every tensor-core round).  Every transform and every mode's update runs the
same arithmetic in the same order as with one group, so the fields must be
bitwise identical for every valid G; one G > 1 case per shape is also checked
against the FP64 oracle.  Shapes: 2D TE (lines of 256 and 2048 points), 2D
six-component, 3D rho-form (eleven input components), TM vacuum, 3 * 2^k and
5 * 2^k lines, radix-16 stages, PSTD and the staggered order-p step.  Invalid
requests (FP64, tensor-core stages, lines of fewer than 32 threads) are refused
on the host."""
import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, psatd_gpu, rel_l2_fields, rounded
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _inputs(shape, layout, seed):
    E = rounded(mask_layout(synth.random_fields(shape, 3, seed), layout, "E"), "fp32")
    B = rounded(mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B"), "fp32")
    J = rounded(mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J"), "fp32")
    r0 = rounded(synth.random_fields(shape, 1, seed + 3)[0], "fp32")
    r1 = rounded(synth.random_fields(shape, 1, seed + 4)[0], "fp32")
    return E, B, J, r0, r1


# (array shape [.., ny, nx], layout, source form, extra plan kwargs, elements per thread or None)
CASES = [
    ((256, 128), "te", "J", {}, None),
    ((2048, 32), "te", "J", {}, None),
    ((512, 64), "2d6", "J", {}, None),
    ((256, 16, 32), "3d6", "rho", {}, None),
    ((512, 64), "tm", "none", {}, None),
    ((384, 64), "te", "J", {}, None),
    ((640, 32), "te", "J", {}, None),
    ((512, 64), "te", "J", {}, 16),
    ((256, 64), "te", "J", {"scheme": "pstd"}, None),
    ((256, 64), "te", "J", {"order": 8}, None),
]


def _oracle(shape, d, dt, E, B, J, r0, r1, layout, src, kw):
    if kw.get("scheme") == "pstd":
        Eo, Bo = orc.pstd_step(E, B, J, d=d, dt=dt)
    else:
        form = {"J": "J", "rho": "rho", "none": "none"}[src]
        Eo, Bo = orc.psatd_step(E, B, J if src != "none" else None, r0 if src == "rho" else None,
                                r1 if src == "rho" else None, d=d, dt=dt, form=form, order=kw.get("order", 0))
    return mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")


@pytest.mark.parametrize("shape,layout,src,kw,ept", CASES)
def test_groups_give_the_same_bits(shape, layout, src, kw, ept):
    ensure_lib()
    d = (1.0, 0.9, 1.1)[:len(shape)]
    dt = 0.4
    E, B, J, r0, r1 = _inputs(shape, layout, 211)
    plan = capi.Plan(tuple(reversed(shape)), d, dt, layout=layout, prec="fp32", src=src, **kw)
    if ept is not None:
        plan.set_launch([-1, -1, -1, -1, -1, ept])
    ref = None
    tried = []
    for G in (1, 2, 4):
        try:
            plan.set_push_groups(G)
        except capi.PsatdError:
            assert G > 1
            continue
        assert plan.get_push_groups() == G
        Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout=layout, prec="fp32", src=src, plan=plan)
        tried.append(G)
        if ref is None:
            ref = (Eg, Bg)
        else:
            assert np.array_equal(Eg, ref[0]) and np.array_equal(Bg, ref[1]), G
    assert 2 in tried, "every case here admits two groups"
    Eo, Bo = _oracle(shape, d, dt, E, B, J, r0, r1, layout, src, kw)
    assert rel_l2_fields(ref[0], ref[1], Eo, Bo) < 2e-6
    plan.set_push_groups(-1)
    assert plan.get_push_groups() in (1, 2, 4)
    plan.destroy()


def test_groups_over_many_steps_stay_bitwise():
    ensure_lib()
    shape, d, dt = (512, 128), (1.0, 1.0), 0.5
    E, B, J, _, _ = _inputs(shape, "te", 5)
    out = []
    for G in (1, 2):
        plan = capi.Plan(tuple(reversed(shape)), d, dt, layout="te", prec="fp32", src="J")
        plan.set_push_groups(G)
        out.append(psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", plan=plan, nsteps=50))
        plan.destroy()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec,shape,bad", [
    ("fp64", (256, 64), [2, 4]),          # FP64 plans keep one group
    ("mixed_bf16", (512, 128), [4]),      # tensor-core stages: pairs only
    ("fp32", (128, 64), [2, 4]),          # 128-point lines: 16 threads a line
    ("fp32", (384, 64), [4]),             # 12 elements per thread: no four groups (odd modes per thread)
])
def test_invalid_groups_are_refused(prec, shape, bad):
    ensure_lib()
    plan = capi.Plan(tuple(reversed(shape)), (1.0, 1.0), 0.5, layout="te", prec=prec, src="J")
    for G in bad:
        with pytest.raises(capi.PsatdError):
            plan.set_push_groups(G)
    for G in (0, 3, 8):
        with pytest.raises(capi.PsatdError):
            plan.set_push_groups(G)
    plan.set_push_groups(1)
    assert plan.get_push_groups() == 1
    # the one-group pass of these shapes (lines of 16 threads among them) still steps correctly
    d, dt = (1.0, 1.0), 0.5
    E, B, J, _, _ = _inputs(shape, "te", 17)
    if prec == "fp64":
        E, B, J = (np.asarray(x, dtype=np.float64) for x in (E, B, J))
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=prec, src="J", plan=plan)
    Eo, Bo = _oracle(shape, d, dt, E, B, J, None, None, "te", "J", {})
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < {"fp64": 1e-12, "fp32": 2e-6, "mixed_bf16": 2e-5}[prec]
    plan.destroy()


def test_autotuner_considers_groups():
    ensure_lib()
    plan = capi.Plan((128, 1024), (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
    rep = plan.autotune(2)
    assert " g=2 " in rep and " g=1 " in rep
    assert plan.get_push_groups() in (1, 2, 4)
    plan.destroy()


def test_batch_groups_give_the_same_bits():
    """A batch of power-of-two, 3 * 2^k and 5 * 2^k patches: each class takes the
    groups where its shape admits them; every class's fields are unchanged."""
    import torch
    ensure_lib()
    sizes = [(64, 256), (128, 384), (32, 640), (64, 128), (256, 512)]
    tot = sum(a * b for a, b in sizes)
    g = torch.Generator().manual_seed(3)
    J = [torch.randn(tot, generator=g).cuda() * 0.01 for _ in range(2)]
    E0 = [torch.randn(tot, generator=g).cuda() for _ in range(3)]
    res = []
    for G in (1, 2, 4):
        b = capi.Batch(sizes, (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
        b.set_push_groups(G)
        E = [x.clone() for x in E0]
        b.step([E[0], E[1], None], [None, None, E[2]], [J[0], J[1], None], nsteps=3)
        b.sync()
        res.append([x.cpu().numpy() for x in E])
        b.destroy()
    for r in res[1:]:
        for a, c in zip(res[0], r):
            assert np.array_equal(a, c)
    with pytest.raises(capi.PsatdError):
        capi.Batch(sizes, (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J").set_push_groups(3)


# tensor-core pairs: (array shape, layout, source form); odd and even component counts
TC_CASES = [
    ((512, 128), "te", "J"),       # 5 inputs, 3 outputs: the last pair of each has one component
    ((64, 128), "2d6", "rho"),     # 11 inputs, 6 outputs
    ((1024, 128), "tm", "none"),   # 3 inputs, 3 outputs
    ((128, 256), "te", "J"),       # 128-point lines: 8 threads a line, 16 lines per group
]


@pytest.mark.parametrize("prec", ["mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("shape,layout,src", TC_CASES)
def test_tensor_core_pairs_give_the_same_bits(shape, layout, src, prec):
    ensure_lib()
    d, dt = (1.0, 0.9), 0.4
    E, B, J, r0, r1 = _inputs(shape, layout, 311)
    out = []
    for G in (1, 2):
        plan = capi.Plan(tuple(reversed(shape)), d, dt, layout=layout, prec=prec, src=src)
        plan.set_push_groups(G)
        assert plan.get_push_groups() == G
        out.append(psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout=layout, prec=prec, src=src, plan=plan, nsteps=3))
        plan.destroy()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    Eo, Bo = orc.psatd_step(E, B, J if src != "none" else None, r0 if src == "rho" else None,
                            r1 if src == "rho" else None, d=d, dt=dt, form=src, nsteps=3)
    assert rel_l2_fields(out[1][0], out[1][1], mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")) < 2e-5


def test_tensor_core_pairs_in_a_batch():
    """Split-BF16 batch of mixed sizes (tensor-core sides): pairs in every class give the
    one-group bits over a multi-step graph replay."""
    import torch
    ensure_lib()
    sizes = [(256, 512), (128, 256), (512, 128), (128, 1024), (256, 512)]
    tot = sum(a * b for a, b in sizes)
    g = torch.Generator().manual_seed(9)
    J = [torch.randn(tot, generator=g).cuda() * 0.01 for _ in range(2)]
    E0 = [torch.randn(tot, generator=g).cuda() for _ in range(3)]
    stream = torch.cuda.Stream()
    res = []
    for G in (1, 2):
        b = capi.Batch(sizes, (1.0, 1.0), 0.5, layout="te", prec="mixed_bf16", src="J", stream=stream)
        b.set_push_groups(G)
        E = [x.clone() for x in E0]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            b.step([E[0], E[1], None], [None, None, E[2]], [J[0], J[1], None], nsteps=4)
        b.sync()
        res.append([x.cpu().numpy() for x in E])
        b.destroy()
    for a, c in zip(res[0], res[1]):
        assert np.array_equal(a, c)
