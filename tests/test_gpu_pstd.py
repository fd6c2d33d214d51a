"""GPU parity of the PSTD step (PSATD_FLAG_PSTD; Table 1 row PSTD) with the FP64
oracle's ``pstd_step``: every layout, vacuum and J-form, on the nodes (order 0)
and staggered (order 8), one step and ten, below the Courant limit."""
import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, rel_l2_fields, rounded, torch_dev
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}


def _run(shape, d, dt, E, B, J, *, layout, prec, src, order, nsteps):
    ensure_lib()
    pe, pb, pj = capi.PRESENT[layout]
    plan = capi.Plan(tuple(reversed(shape)), d, dt, layout=layout, prec=prec, src=src, order=order, scheme="pstd")
    Et = [torch_dev(E[i], prec) if pe[i] else None for i in range(3)]
    Bt = [torch_dev(B[i], prec) if pb[i] else None for i in range(3)]
    Jt = [torch_dev(J[i], prec) if pj[i] else None for i in range(3)] if src == "J" else None
    plan.step(Et, Bt, Jt, nsteps=nsteps)
    plan.sync()
    Eo = np.zeros((3,) + tuple(shape))
    Bo = np.zeros((3,) + tuple(shape))
    for i in range(3):
        if pe[i]:
            Eo[i] = Et[i].double().cpu().numpy()
        if pb[i]:
            Bo[i] = Bt[i].double().cpu().numpy()
    plan.destroy()
    return Eo, Bo


CASES = [((32, 64), "te", "J"), ((64, 32), "tm", "J"), ((32, 32), "2d6", "none"), ((16, 64), "te", "none"),
         ((16, 16, 32), "3d6", "J")]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [0, 8])
@pytest.mark.parametrize("nsteps", [1, 10])
@pytest.mark.parametrize("shape,layout,src", CASES)
def test_pstd_matches_oracle(shape, layout, src, nsteps, order, prec):
    d = (1.0, 0.7, 1.2)[:len(shape)]
    dt = 0.3
    lay = layout
    E = rounded(mask_layout(synth.random_fields(shape, 3, 800), lay, "E"), prec)
    B = rounded(mask_layout(synth.random_fields(shape, 3, 801), lay, "B"), prec)
    J = rounded(mask_layout(synth.random_fields(shape, 3, 802), lay, "J"), prec) if src == "J" else None
    Eg, Bg = _run(shape, d, dt, E, B, J, layout=lay, prec=prec, src=src, order=order, nsteps=nsteps)
    Eo, Bo = orc.pstd_step(E, B, J, d=d, dt=dt, nsteps=nsteps, order=order)
    Eo, Bo = mask_layout(Eo, lay, "E"), mask_layout(Bo, lay, "B")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL[prec] * nsteps
