"""GPU parity of the local-FFT decomposition (psatd_local_*, Sec. II.A.3) with the
local-FFT oracle (``oracle/local.py``): the same patches, guard width and steps,
compared over the whole global grid at the precision's per-step bound; and the
truncation error against the global step falling with the guard width."""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, rel_l2_fields, rounded, torch_dev
from oracle import local as loc
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "mixed_fp16": 4e-6}


def _run_local(shape, d, dt, E, B, J, *, layout, prec, src, px, py, guard, nsteps=1):
    ensure_lib()
    pe, pb, pj = capi.PRESENT[layout]
    L = capi.Local(tuple(reversed(shape)), d, dt, px=px, py=py, guard=guard, layout=layout, prec=prec, src=src)
    Et = [torch_dev(E[i], prec) if pe[i] else None for i in range(3)]
    Bt = [torch_dev(B[i], prec) if pb[i] else None for i in range(3)]
    Jt = [torch_dev(J[i], prec) if (J is not None and pj[i]) else None for i in range(3)]
    L.step(Et, Bt, Jt if src != "none" else None, nsteps=nsteps)
    L.sync()
    Eo = np.zeros((3,) + tuple(shape))
    Bo = np.zeros((3,) + tuple(shape))
    for i in range(3):
        if pe[i]:
            Eo[i] = Et[i].double().cpu().numpy()
        if pb[i]:
            Bo[i] = Bt[i].double().cpu().numpy()
    L.destroy()
    return Eo, Bo


CASES = [
    # (ny, nx), layout, source form, px, py, guard: extended patches must be powers of two
    ((112, 224), "te", "J", 4, 2, 4),        # interior 56 x 56 + 2*4 = 64 x 64
    ((240, 120), "2d6", "none", 1, 2, 4),    # interior 120 x 120 + 8 = 128 x 128
    ((96, 192), "tm", "J", 6, 3, 16),        # interior 32 x 32 + 32 = 64 x 64
    ((128, 128), "te", "rho", 2, 2, 0),      # no guards: 64 x 64 periodic patches
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,layout,src,px,py,guard", CASES)
def test_local_step_matches_local_oracle(prec, shape, layout, src, px, py, guard):
    d, dt = (1.0, 0.8), 0.45
    E = rounded(mask_layout(synth.random_fields(shape, 3, 71), layout, "E"), prec)
    B = rounded(mask_layout(synth.random_fields(shape, 3, 72), layout, "B"), prec)
    J = rounded(mask_layout(synth.random_fields(shape, 3, 73), layout, "J"), prec) if src != "none" else None
    r0 = rounded(synth.random_fields(shape, 1, 74)[0], prec) if src == "rho" else None
    r1 = rounded(synth.random_fields(shape, 1, 75)[0], prec) if src == "rho" else None
    if src == "rho":
        ensure_lib()
        pe, pb, pj = capi.PRESENT[layout]
        L = capi.Local(tuple(reversed(shape)), d, dt, px=px, py=py, guard=guard, layout=layout, prec=prec, src=src)
        Et = [torch_dev(E[i], prec) if pe[i] else None for i in range(3)]
        Bt = [torch_dev(B[i], prec) if pb[i] else None for i in range(3)]
        Jt = [torch_dev(J[i], prec) if pj[i] else None for i in range(3)]
        L.step(Et, Bt, Jt, torch_dev(r0, prec), torch_dev(r1, prec), nsteps=2)
        L.sync()
        Eg = np.zeros((3,) + shape)
        Bg = np.zeros((3,) + shape)
        for i in range(3):
            if pe[i]:
                Eg[i] = Et[i].double().cpu().numpy()
            if pb[i]:
                Bg[i] = Bt[i].double().cpu().numpy()
        L.destroy()
    else:
        Eg, Bg = _run_local(shape, d, dt, E, B, J, layout=layout, prec=prec, src=src, px=px, py=py, guard=guard,
                            nsteps=2)
    Eo, Bo = loc.local_step(E, B, J, r0, r1, d=d, dt=dt, px=px, py=py, guard=guard,
                            form={"none": "none", "J": "J", "rho": "rho"}[src], nsteps=2)
    Eo, Bo = mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < 2 * TOL[prec]


def test_one_patch_without_guards_equals_the_global_plan_bitwise():
    shape, d, dt = (128, 256), (1.0, 1.0), 0.5
    E = rounded(mask_layout(synth.random_fields(shape, 3, 1), "te", "E"), "fp32")
    B = rounded(mask_layout(synth.random_fields(shape, 3, 2), "te", "B"), "fp32")
    J = rounded(mask_layout(synth.random_fields(shape, 3, 3), "te", "J"), "fp32")
    El, Bl = _run_local(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", px=1, py=1, guard=0, nsteps=3)
    from gpu_helpers import psatd_gpu
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", nsteps=3)
    assert np.array_equal(El, Eg) and np.array_equal(Bl, Bg)


def test_truncation_error_against_global_falls_with_guard_width():
    """Smooth random fields (power ~ k^-4) on 192^2 split into 4 x 4 patches of 48^2
    cells with g = 8, 40, 104 guard cells (extended patches 64, 128, 256): the GPU
    matches the local oracle, and the error against the global step falls with g."""
    n = 192
    shape, d, dt = (n, n), (1.0, 1.0), 1.0 / math.sqrt(2.0)
    rng = np.random.default_rng(5)
    ky = 2 * np.pi * np.fft.fftfreq(n)[:, None]
    kx = 2 * np.pi * np.fft.rfftfreq(n)[None, :]
    filt = 1.0 / (1.0 + 40.0 * (kx ** 2 + ky ** 2)) ** 2
    E = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal(shape)) * filt, s=shape) for _ in range(3)])
    B = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal(shape)) * filt, s=shape) for _ in range(3)])
    Eg, Bg = orc.psatd_step(E, B, d=d, dt=dt)
    errs = []
    for g in (8, 40, 104):
        El, Bl = _run_local(shape, d, dt, E, B, None, layout="2d6", prec="fp64", src="none", px=4, py=4, guard=g)
        Eo, Bo = loc.local_step(E, B, d=d, dt=dt, px=4, py=4, guard=g)
        assert rel_l2_fields(El, Bl, Eo, Bo) < 1e-12
        errs.append(rel_l2_fields(El, Bl, Eg, Bg))
    print("local-FFT truncation error vs guard (8, 40, 104):", errs)
    assert errs[0] > errs[1] > errs[2], errs
