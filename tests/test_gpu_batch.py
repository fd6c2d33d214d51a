"""GPU parity of batched patches (psatd_batch_*): every patch of a batch of uneven
power-of-two sizes advanced in one launch per pass and size class must match the
FP64 oracle on that patch alone; a multi-step call (CUDA graph replay) must equal
the same number of single-step calls bitwise."""
import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, rel_l2_fields, rounded
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 64), (128, 32), (64, 64), (32, 128), (256, 256), (16, 8), (64, 64)]


def _packed(arrs, prec):
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.concatenate([a.ravel() for a in arrs])).to(device="cuda", dtype=dt)


def _make(layout, src, prec, seed):
    per = []
    for i, (nx, ny) in enumerate(SIZES):
        shape = (ny, nx)
        E = rounded(mask_layout(synth.random_fields(shape, 3, seed + 10 * i), layout, "E"), prec)
        B = rounded(mask_layout(synth.random_fields(shape, 3, seed + 10 * i + 1), layout, "B"), prec)
        J = rounded(mask_layout(synth.random_fields(shape, 3, seed + 10 * i + 2), layout, "J"), prec)
        per.append((E, B, J))
    return per


def _run(per, layout, src, prec, d, dt, nsteps=1, calls=1):
    ensure_lib()
    pe, pb, pj = capi.PRESENT[layout]
    Et = [_packed([p[0][i] for p in per], prec) if pe[i] else None for i in range(3)]
    Bt = [_packed([p[1][i] for p in per], prec) if pb[i] else None for i in range(3)]
    Jt = [_packed([p[2][i] for p in per], prec) if pj[i] else None for i in range(3)]
    import torch
    stream = torch.cuda.Stream()  # a non-default stream: multi-step calls replay a CUDA graph
    torch.cuda.synchronize()
    b = capi.Batch(SIZES, d, dt, layout=layout, prec=prec, src=src, stream=stream)
    assert b.cells() == sum(a * c for a, c in SIZES)
    with torch.cuda.stream(stream):
        for _ in range(calls):
            b.step(Et, Bt, Jt if src != "none" else None, nsteps=nsteps)
    torch.cuda.synchronize()
    b.destroy()
    E = [t.double().cpu().numpy() if t is not None else None for t in Et]
    B = [t.double().cpu().numpy() if t is not None else None for t in Bt]
    return E, B


def _patch(arrs, i):
    off = sum(a * c for a, c in SIZES[:i])
    nx, ny = SIZES[i]
    return np.stack([a[off:off + nx * ny].reshape(ny, nx) if a is not None else np.zeros((ny, nx))
                     for a in arrs])


@pytest.mark.parametrize("prec,layout,src", [("fp32", "te", "J"), ("fp64", "2d6", "none"), ("fp32", "tm", "J")])
def test_batch_patches_match_oracle(prec, layout, src):
    d, dt = (1.0, 1.0), 0.6
    per = _make(layout, src, prec, 77)
    E, B = _run(per, layout, src, prec, d, dt)
    tol = 1e-12 if prec == "fp64" else 2e-6
    for i in range(len(SIZES)):
        Eo, Bo = orc.psatd_step(per[i][0], per[i][1], per[i][2] if src != "none" else None, d=d, dt=dt,
                                form=src if src != "none" else "none")
        assert rel_l2_fields(_patch(E, i), _patch(B, i), mask_layout(Eo, layout, "E"),
                             mask_layout(Bo, layout, "B")) < tol, i


def test_batch_graph_replay_equals_single_calls():
    d, dt = (1.0, 1.0), 0.6
    per = _make("te", "J", "fp32", 5)
    E1, B1 = _run(per, "te", "J", "fp32", d, dt, nsteps=6)
    E2, B2 = _run(per, "te", "J", "fp32", d, dt, calls=6)
    for a, b in zip(E1 + B1, E2 + B2):
        if a is not None:
            assert np.array_equal(a, b)
    Eo, Bo = orc.psatd_step(per[4][0], per[4][1], per[4][2], d=d, dt=dt, form="J", nsteps=6)
    assert rel_l2_fields(_patch(E1, 4), _patch(B1, 4), mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < 1e-5


@pytest.mark.parametrize("prec,persistent", [("fp32", False), ("fp32", True), ("mixed_bf16", False),
                                             ("mixed_bf16", True)])
def test_batch_kernel_times_of_a_graph_replay(prec, persistent):
    """Batch timing with a multi-step call: the event pairs are recorded inside the
    step graph, each replay times the launches again, and the results stay those of
    an untimed run (bitwise)."""
    import torch
    ensure_lib()
    sizes = [(256, 128), (128, 128), (256, 128), (512, 256)]
    tot = sum(a * b for a, b in sizes)
    g = torch.Generator(device="cuda").manual_seed(9)
    init = [torch.randn(tot, device="cuda", generator=g) for _ in range(5)]
    out = []
    for timed in (False, True):
        F = [t.clone() for t in init]
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        b = capi.Batch(sizes, (1.0, 1.0), 0.5, layout="te", prec=prec, src="J", stream=stream)
        b.set_persistent(persistent)
        if timed:
            b.set_timing(True)
        with torch.cuda.stream(stream):
            b.step([F[0], F[1], None], [None, None, F[2]], [F[3], F[4], None], nsteps=4)
        b.sync()
        if timed:
            kt = b.kernel_times()
            assert set(kt) == {"fwd_x_r2c", "line_fft_push", "inv_x_c2r"}, kt
            # one step's launches (the last replay's): one per pass and class, or one per pass (persistent)
            assert all(v[0] >= 1 and v[1] > 0 for v in kt.values()), kt
            assert sum(v[0] for v in kt.values()) == b.launches_per_step() == (3 if persistent else 9), kt
            b.set_timing(False)
        b.sync()
        b.destroy()
        out.append(F[:3])
    for x, y in zip(*out):
        assert torch.equal(x, y)


PERSIST_SIZES = {
    "fp32": [(64, 64), (128, 96), (192, 128), (256, 256), (1024, 768), (96, 1024), (512, 384), (64, 64)],
    # (the per-class tensor-core path it is compared with needs nx/32 * min(32, ny) >= 128)
    "mixed_fp16": [(128, 64), (128, 128), (256, 512), (1024, 1024), (512, 64), (128, 128)],
    "mixed_bf16": [(128, 64), (128, 128), (256, 512), (1024, 1024), (512, 64), (128, 128)],
}


@pytest.mark.parametrize("prec,layout", [("fp32", "te"), ("fp32", "tm"), ("fp32", "2d6"), ("mixed_fp16", "te"),
                                         ("mixed_bf16", "te"), ("mixed_bf16", "2d6")])
def test_persistent_passes_equal_per_class_launches(prec, layout):
    """One persistent launch per pass type and length family over every patch (the
    default where the sizes allow) gives the bits of the per-class launches, in a
    graph replay of several steps, and matches the oracle on a patch of each family."""
    import torch
    ensure_lib()
    sizes = PERSIST_SIZES[prec]
    tot = sum(a * b for a, b in sizes)
    g = torch.Generator(device="cuda").manual_seed(21)
    pe, pb, pj = capi.PRESENT[layout]
    mk = lambda p: [torch.randn(tot, device="cuda", generator=g) if p[i] else None for i in range(3)]
    E0, B0, J = mk(pe), mk(pb), mk(pj)
    host0 = ([t.double().cpu().numpy() if t is not None else None for t in E0],
             [t.double().cpu().numpy() if t is not None else None for t in B0],
             [t.double().cpu().numpy() if t is not None else None for t in J])
    out = []
    for persistent in (True, False):
        E = [t.clone() if t is not None else None for t in E0]
        B = [t.clone() if t is not None else None for t in B0]
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        b = capi.Batch(sizes, (1.0, 1.0), 0.5, layout=layout, prec=prec, src="J", stream=stream)
        assert b.launches_per_step() == 3 * len(set(sizes))      # per-class launches by default
        b.set_persistent(persistent)
        if persistent:
            fams_x = len({(nx // 2) & (nx // 2 - 1) == 0 for nx, _ in sizes})
            fams_y = len({ny & (ny - 1) == 0 for _, ny in sizes})
            assert b.launches_per_step() == 2 * fams_x + fams_y
        with torch.cuda.stream(stream):
            b.step(E, B, J, nsteps=3)
        b.sync()
        b.destroy()
        out.append(E + B)
    for x, y in zip(*out):
        if x is not None:
            assert torch.equal(x, y)
    # the oracle on the first patch and the largest one
    offs = np.concatenate([[0], np.cumsum([a * c for a, c in sizes])])
    area = [a * c for a, c in sizes]
    for i in {0, int(np.argmax(area))}:
        nx, ny = sizes[i]
        cut = lambda arrs: np.stack([a[offs[i]:offs[i + 1]].reshape(ny, nx) if a is not None else np.zeros((ny, nx))
                                     for a in arrs])
        Eo, Bo = orc.psatd_step(cut(host0[0]), cut(host0[1]), cut(host0[2]), d=(1.0, 1.0), dt=0.5, form="J",
                                nsteps=3)
        Eg = cut([t.double().cpu().numpy() if t is not None else None for t in out[0][:3]])
        Bg = cut([t.double().cpu().numpy() if t is not None else None for t in out[0][3:]])
        tol = 4e-6 if prec == "fp32" else 8e-6
        assert rel_l2_fields(Eg, Bg, mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")) < tol, i


def test_serialised_classes_give_the_forked_bits():
    """psatd_batch_set_branches(0) runs the size classes one after another on the
    batch's stream (the bench's roofline run): the same bits as the forked default."""
    import torch
    ensure_lib()
    sizes = [(256, 128), (128, 96), (192, 256), (512, 64), (128, 96)]
    tot = sum(a * b for a, b in sizes)
    g = torch.Generator(device="cuda").manual_seed(31)
    init = [torch.randn(tot, device="cuda", generator=g) for _ in range(5)]
    out = []
    for forked in (True, False):
        F = [t.clone() for t in init]
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        b = capi.Batch(sizes, (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J", stream=stream)
        b.set_branches(forked)
        with torch.cuda.stream(stream):
            b.step([F[0], F[1], None], [None, None, F[2]], [F[3], F[4], None], nsteps=3)
        b.sync()
        b.destroy()
        out.append(F[:3])
    for x, y in zip(*out):
        assert torch.equal(x, y)
