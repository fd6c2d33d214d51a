"""GPU parity of the mixed-precision PSATD steps (PSATD_MIXED_FP16 and
PSATD_MIXED_BF16): every radix-16 FFT stage is a 16 x 16 DFT-matrix contraction
on the tensor cores (tcgen05, split-FP16 or split-BF16 operands with an exact
head, FP32 accumulation in TMEM), the rest as FP32.

Tolerances (relative L2 over all E and c*B components, vs the FP64 oracle on
the same float32-rounded inputs):
  per step 4e-6: a split operand keeps 22 bits (x_h + x_l, |x_l| <= 2^-11 |x_h|),
        the dropped x_l G_l product is below 2^-22 relative, so a radix-16 stage
        adds about 2^-22 = 2.4e-7 of rms error per element; a 2D step runs 4-6
        such stages per component (forward and inverse) on top of the FP32
        error budget of 2e-6, and 4e-6 bounds the sum with margin.
  after N steps 2e-5 (the stated bound for the mixed-precision path).
"""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, psatd_gpu, rel_l2_fields, rounded, torch_dev
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL_STEP = 4e-6
TOL_RUN = 2e-5
MIXED = ["mixed_fp16", "mixed_bf16"]


def _inputs(shape, layout, src, seed, P):
    E = mask_layout(synth.random_fields(shape, 3, seed), layout, "E")
    B = mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B")
    J = mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J") if src != "none" else None
    r0 = synth.random_fields(shape, 1, seed + 3)[0] if src == "rho" else None
    r1 = synth.random_fields(shape, 1, seed + 4)[0] if src == "rho" else None
    rd = (lambda a: rounded(a, P) if a is not None else None)
    return rd(E), rd(B), rd(J), rd(r0), rd(r1)


def _oracle(E, B, J, r0, r1, d, dt, src, nsteps=1):
    form = {"none": "none", "J": "J", "rho": "rho"}[src]
    return orc.psatd_step(E, B, J, r0, r1, d=d, dt=dt, form=form, nsteps=nsteps)


CASES_2D = [
    ((256, 512), "te", "J"), ((512, 256), "te", "rho"), ((128, 256), "tm", "J"),
    ((64, 128), "2d6", "none"), ((128, 128), "2d6", "J"), ((64, 128), "2d6", "rho"),
    ((16, 4096), "te", "J"), ((4096, 128), "te", "none"),
]


@pytest.mark.parametrize("P", MIXED)
@pytest.mark.parametrize("shape,layout,src", CASES_2D)
def test_mixed_2d_one_step_matches_oracle(shape, layout, src, P):
    d, dt = (1.0, 0.7), 0.45
    E, B, J, r0, r1 = _inputs(shape, layout, src, 4321, P)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout=layout, prec=P, src=src)
    Eo, Bo = _oracle(E, B, J, r0, r1, d, dt, src)
    Eo, Bo = mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL_STEP


@pytest.mark.parametrize("P", MIXED)
@pytest.mark.parametrize("shape,src", [((32, 64, 128), "J"), ((32, 64, 128), "rho"), ((32, 64, 256), "none")])
def test_mixed_3d_one_step_matches_oracle(shape, src, P):
    d, dt = (1.0, 0.8, 1.2), 0.6
    E, B, J, r0, r1 = _inputs(shape, "3d6", src, 77, P)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec=P, src=src)
    Eo, Bo = _oracle(E, B, J, r0, r1, d, dt, src)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL_STEP


@pytest.mark.parametrize("P", MIXED)
@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_mixed_rows_with_zeros_and_extreme_magnitudes(scale, P):
    """Inputs scaled by 1e-30 or 1e30 (the per-row power-of-two scale follows each
    row, so FP16's range does not limit the data) with some rows and one source
    component entirely zero (the row scale falls back to 1): same bound."""
    shape, d, dt = (256, 256), (1.0, 1.0), 0.5
    E, B, J, _, _ = _inputs(shape, "te", "J", 5, P)
    B[2][::3, :] = 0.0
    J[1][:, :] = 0.0
    E, B, J = (rounded(a * scale, P) for a in (E, B, J))
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=P, src="J")
    Eo, Bo = _oracle(E, B, J, None, None, d, dt, "J")
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL_STEP


def _sheet_J(shape, d, n, dt, lam):
    return synth.current_sheet(shape, d, (n + 0.5) * dt, lam=lam, a=0.9, w=2.0 * d[0])


@pytest.mark.parametrize("P", MIXED)
def test_mixed_config2_full_size_one_step(P):
    """2048^2 TE, dx = lambda/64, c dt = dx/sqrt(2), current-sheet J (the bench's workload)."""
    shape = (2048, 2048)
    d = (1.0 / 64, 1.0 / 64)
    dt = d[0] / math.sqrt(2.0)
    E = mask_layout(synth.random_fields(shape, 3, 5), "te", "E")
    B = mask_layout(synth.random_fields(shape, 3, 6), "te", "B")
    J = _sheet_J(shape, d, 17, dt, 1.0)
    E, B, J = (rounded(a, P) for a in (E, B, J))
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=P, src="J")
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL_STEP


@pytest.mark.parametrize("P", MIXED)
def test_mixed_sheet_long_run_within_2e5(P):
    """Current-sheet drive from zero fields on 512^2 (dx = lambda/64, c dt = dx/sqrt(2)),
    time-varying J one call per step: relative L2 vs the FP64 oracle below 2e-5 at
    100 steps (the batched workload's run length) and at 2000 steps (the FP32 test's)."""
    shape = (512, 512)
    d = (1.0 / 64, 1.0 / 64)
    dt = d[0] / math.sqrt(2.0)
    ensure_lib()
    plan = capi.Plan((512, 512), d, dt, layout="te", prec=P, src="J")
    Et = [torch_dev(np.zeros(shape), P) for _ in range(2)]
    Bz = torch_dev(np.zeros(shape), P)
    E = np.zeros((3,) + shape)
    B = np.zeros((3,) + shape)
    errs = {}
    for n in range(2000):
        J = rounded(_sheet_J(shape, d, n, dt, 1.0), P)
        Jt = [torch_dev(J[0], P), torch_dev(J[1], P), None]
        plan.step([Et[0], Et[1], None], [None, None, Bz], Jt)
        E, B = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
        if n + 1 in (100, 500, 2000):
            plan.sync()
            Eg = np.zeros_like(E)
            Bg = np.zeros_like(B)
            Eg[0], Eg[1], Bg[2] = (t.double().cpu().numpy() for t in (Et[0], Et[1], Bz))
            errs[n + 1] = rel_l2_fields(Eg, Bg, E, B)
    plan.destroy()
    print(P, "long-run rel L2:", errs)
    assert errs[100] < TOL_RUN and errs[2000] < TOL_RUN, errs


@pytest.mark.parametrize("P", MIXED)
def test_mixed_config3_full_size_one_step(P):
    """3D 256^3 rho-form, all five passes with tensor-core radix-16 stages."""
    shape = (256, 256, 256)
    d, dt = (1.0, 1.0, 1.0), 0.5
    E, B, J, r0, r1 = _inputs(shape, "3d6", "rho", 2024, P)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec=P, src="rho")
    Eo, Bo = _oracle(E, B, J, r0, r1, d, dt, "rho")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL_STEP


@pytest.mark.parametrize("P", MIXED)
def test_mixed_nsteps_equals_repeated_calls_bitwise(P):
    shape, d, dt = (128, 256), (1.0, 1.0), 0.4
    E, B, J, _, _ = _inputs(shape, "te", "J", 11, P)
    E1, B1 = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=P, src="J", nsteps=5)
    E2, B2 = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=P, src="J", calls=5)
    assert np.array_equal(E1, E2) and np.array_equal(B1, B2)
    Eo, Bo = _oracle(E, B, J, None, None, d, dt, "J", nsteps=5)
    assert rel_l2_fields(E1, B1, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL_RUN


@pytest.mark.parametrize("P", MIXED)
def test_mixed_batch_matches_oracle_per_patch(P):
    """A batch of uneven patches with tensor-core stages: each patch vs the oracle alone."""
    import torch
    ensure_lib()
    sizes = [(128, 128), (256, 128), (128, 128), (128, 256), (256, 256)]
    d, dt = (1.0, 1.0), 0.5
    per = []
    for i, (nx, ny) in enumerate(sizes):
        E, B, J, _, _ = _inputs((ny, nx), "te", "J", 300 + 10 * i, P)
        per.append((E, B, J))
    pe, pb, pj = capi.PRESENT["te"]

    def packed(arrs):
        return torch.from_numpy(np.concatenate([a.ravel() for a in arrs])).to(device="cuda", dtype=torch.float32)

    Et = [packed([p[0][i] for p in per]) if pe[i] else None for i in range(3)]
    Bt = [packed([p[1][i] for p in per]) if pb[i] else None for i in range(3)]
    Jt = [packed([p[2][i] for p in per]) if pj[i] else None for i in range(3)]
    stream = torch.cuda.Stream()
    b = capi.Batch(sizes, d, dt, layout="te", prec=P, src="J", stream=stream)
    with torch.cuda.stream(stream):
        b.step(Et, Bt, Jt, nsteps=3)
    stream.synchronize()
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
        Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J", nsteps=3)
        assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL_STEP * 3
        off += n
    b.destroy()
