"""GPU parity of the mixed-radix line lengths L = 3 * 2^k and 5 * 2^k (FP32):
every pass (R2C x rows of nx/2 points, C2C y lines in 3D, the fused last-axis
pass, the inverses) transforms such lines with a radix-3 first stage, then
radix-2/4 and radix-8 stages, or a radix-5 first stage, then radix-2 and
radix-4 stages.  The method does not restrict the grid to powers of two; these
lengths matter for the local FFTs of Sec. II.A.3, whose extended patches are
an interior plus two guard regions (e.g. 16 + 2 * 16 = 48 cells).

Each case is compared with the FP64 oracle on the same float-rounded inputs at
the FP32 bound: one step within 2e-6 (relative L2 over all field components),
N steps within 2e-6 * N."""
import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, psatd_gpu, rel_l2_fields, rounded, torch_dev
from oracle import local as loc
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _inputs(shape, layout, seed, src="J"):
    E = rounded(mask_layout(synth.random_fields(shape, 3, seed), layout, "E"), "fp32")
    B = rounded(mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B"), "fp32")
    J = rounded(mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J"), "fp32") if src != "none" else None
    r0 = rounded(synth.random_fields(shape, 1, seed + 3)[0], "fp32") if src == "rho" else None
    r1 = rounded(synth.random_fields(shape, 1, seed + 4)[0], "fp32") if src == "rho" else None
    return E, B, J, r0, r1


CASES_2D = [
    # (ny, nx): x rows of nx/2 points, y lines of ny points
    ((48, 96), "te", "J"),          # smallest mixed lengths on both axes (48, 48)
    ((384, 192), "2d6", "rho"),     # 96-point x rows, 384-point lines
    ((96, 1536), "tm", "J"),        # 768-point x rows
    ((3072, 64), "te", "J"),        # longest fused-pass line (3072)
    ((64, 3072), "te", "none"),     # longest x rows (1536 points, R2C)
    ((192, 256), "2d6", "J"),       # power-of-two x, mixed y
    ((128, 384), "tm", "none"),     # mixed x, power-of-two y
    ((80, 160), "te", "J"),         # smallest 5 * 2^k lengths on both axes (80, 80)
    ((320, 192), "2d6", "rho"),     # 96-point x rows, 320-point lines
    ((1280, 64), "te", "J"),        # longest 5 * 2^k fused-pass line
    ((64, 2560), "tm", "none"),     # longest 5 * 2^k x rows (1280 points, R2C)
    ((160, 384), "te", "J"),        # 3 * 2^k x rows, 5 * 2^k lines
]


@pytest.mark.parametrize("shape,layout,src", CASES_2D)
def test_mixed_lengths_2d_match_oracle(shape, layout, src):
    d, dt, n = (1.0, 0.8), 0.45, 3
    E, B, J, r0, r1 = _inputs(shape, layout, 900, src)
    form = {"none": "none", "J": "J", "rho": "rho"}[src]
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout=layout, prec="fp32", src=src, nsteps=n)
    Eo, Bo = orc.psatd_step(E, B, J, r0, r1, d=d, dt=dt, form=form, nsteps=n)
    Eo, Bo = mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL * n


@pytest.mark.parametrize("shape", [(48, 96, 192), (64, 48, 128), (96, 64, 96), (48, 48, 96), (80, 160, 64),
                                   (96, 80, 320)])
@pytest.mark.parametrize("src", ["J", "rho"])
def test_mixed_lengths_3d_match_oracle(shape, src):
    """(nz, ny, nx): the C2C y pass and the fused z pass on mixed and
    power-of-two lengths in every combination."""
    d, dt = (1.0, 0.9, 1.1), 0.4
    E, B, J, r0, r1 = _inputs(shape, "3d6", 930, src)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec="fp32", src=src, nsteps=2)
    Eo, Bo = orc.psatd_step(E, B, J, r0, r1, d=d, dt=dt, form=src, nsteps=2)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < 2 * TOL


def test_mixed_lengths_staggered_and_pstd():
    shape, d, dt = (96, 192), (1.0, 1.0), 0.4
    E, B, J, _, _ = _inputs(shape, "te", 960)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", order=8, nsteps=2)
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J", order=8, nsteps=2)
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < 2 * TOL
    ensure_lib()
    plan = capi.Plan((192, 96), d, 0.3, layout="te", prec="fp32", src="J", scheme="pstd")
    Eg, Bg = psatd_gpu(shape, d, 0.3, E, B, J, layout="te", prec="fp32", src="J", plan=plan, nsteps=4)
    plan.destroy()
    Eo, Bo = orc.pstd_step(E, B, J, d=d, dt=0.3, nsteps=4)
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < 4 * TOL


def test_largest_mixed_grid_one_step():
    """3072 x 3072 TE, J-form: x rows of 1536 points, lines of 3072."""
    shape, d, dt = (3072, 3072), (1.0, 1.0), 0.5
    E, B, J, _, _ = _inputs(shape, "te", 990)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J")
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL


def test_local_patches_of_96_by_48_cells():
    """Local FFTs with 64 x 16 interiors and 16 guard cells: extended patches of
    96 x 48 cells (x rows of 48 points, lines of 48), all mixed-radix."""
    shape, d, dt = (128, 256), (1.0, 1.0), 0.5
    E, B, J, _, _ = _inputs(shape, "te", 1000)
    ensure_lib()
    pe, pb, pj = capi.PRESENT["te"]
    L = capi.Local((256, 128), d, dt, px=4, py=8, guard=16, layout="te", prec="fp32", src="J")
    Et = [torch_dev(E[i], "fp32") if pe[i] else None for i in range(3)]
    Bt = [torch_dev(B[i], "fp32") if pb[i] else None for i in range(3)]
    Jt = [torch_dev(J[i], "fp32") if pj[i] else None for i in range(3)]
    L.step(Et, Bt, Jt, nsteps=2)
    L.sync()
    L.destroy()
    Eg = np.zeros((3,) + shape)
    Bg = np.zeros((3,) + shape)
    for i in range(3):
        if pe[i]:
            Eg[i] = Et[i].double().cpu().numpy()
        if pb[i]:
            Bg[i] = Bt[i].double().cpu().numpy()
    Eo, Bo = loc.local_step(E, B, J, d=d, dt=dt, px=4, py=8, guard=16, form="J", nsteps=2)
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < 2 * TOL


def test_batch_of_mixed_and_power_of_two_patches():
    import torch
    ensure_lib()
    sizes = [(96, 48), (64, 64), (192, 96), (96, 48), (128, 384), (160, 80), (320, 640), (192, 160)]
    d, dt = (1.0, 1.0), 0.5
    per = [_inputs((ny, nx), "te", 1100 + 10 * i)[:3] for i, (nx, ny) in enumerate(sizes)]
    pe, pb, pj = capi.PRESENT["te"]

    def packed(arrs):
        return torch.from_numpy(np.concatenate([a.ravel() for a in arrs])).to(device="cuda", dtype=torch.float32)

    Et = [packed([p[0][i] for p in per]) if pe[i] else None for i in range(3)]
    Bt = [packed([p[1][i] for p in per]) if pb[i] else None for i in range(3)]
    Jt = [packed([p[2][i] for p in per]) if pj[i] else None for i in range(3)]
    b = capi.Batch(sizes, d, dt, layout="te", prec="fp32", src="J")
    b.step(Et, Bt, Jt)
    torch.cuda.synchronize()
    b.destroy()
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
        assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL, (nx, ny)
        off += n


def test_every_launch_shape_of_a_mixed_plan():
    """Lines per CTA change no arithmetic: all accepted shapes give the same bits;
    the fused pass takes 12 elements per thread only (radix-8/16 schedules do
    not divide 3 * 2^k)."""
    shape, d, dt = (384, 768), (1.0, 0.8), 0.5
    E, B, J, _, _ = _inputs(shape, "te", 1200)
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    Eo, Bo = mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")
    ensure_lib()
    plan = capi.Plan((768, 384), d, dt, layout="te", prec="fp32", src="J")
    assert plan.get_launch()[5] == 12
    for ept in (8, 16, 24):
        with pytest.raises(capi.PsatdError):
            plan.set_launch([-1, -1, -1, -1, -1, ept])
    shapes = []
    for k in (0, 3):
        for lg in range(6):
            cfg = [-1] * 6
            cfg[k] = lg
            try:
                plan.set_launch(cfg)
            except capi.PsatdError:
                continue
            shapes.append(cfg)
    for tb in (1, 2, 4, 8, 16, 32):
        try:
            plan.set_launch([-1, -1, -1, -1, tb, 12])
        except capi.PsatdError:
            continue
        shapes.append([-1, -1, -1, -1, tb, 12])
    assert len(shapes) >= 6
    ref = None
    for cfg in shapes:
        plan.set_launch(cfg)
        Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", plan=plan)
        assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL, cfg
        if ref is None:
            ref = (Eg, Bg)
        else:
            assert np.array_equal(Eg, ref[0]) and np.array_equal(Bg, ref[1]), cfg
    rep = plan.autotune(2)
    assert "push" in rep and plan.get_launch()[5] == 12
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", plan=plan)
    assert np.array_equal(Eg, ref[0]) and np.array_equal(Bg, ref[1])
    plan.destroy()
