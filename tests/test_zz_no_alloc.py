"""psatd_step_noalloc (the allocation-free variant of the PSATD step) against
the plan-based psatd_step, through the C ABI.

Callers that cannot allocate device memory use this entry point; it must give
the same fields as the regular path.  This file is collected last so that a
run stopping at its first failure has already run every other test.
"""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, rel_l2_fields, rounded, torch_dev
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}   # the per-step tolerances of the parity tests


def _state(shape, layout, seed, prec):
    E = rounded(mask_layout(synth.random_fields(shape, 3, seed), layout, "E"), prec)
    B = rounded(mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B"), prec)
    J = rounded(mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J"), prec)
    pe, pb, pj = capi.PRESENT[layout]
    dev = lambda F, p: [torch_dev(F[i], prec) if p[i] else None for i in range(3)]
    return dev(E, pe), dev(B, pb), dev(J, pj)


def _np(ts):
    return np.stack([t.double().cpu().numpy() if t is not None else np.zeros(1) for t in ts if t is not None])


# (precision, layout, grid [nz,] ny, nx, steps per call, scheme): 2D TE and 2D6, a mixed-radix
# grid, a 3D grid (whose second spectrum is carved from the array after the first), calls
# of three steps, and the PSTD scheme
CASES = [("fp32", "te", (256, 256), 1, "psatd"), ("fp64", "2d6", (64, 128), 1, "psatd"),
         ("fp32", "te", (192, 96), 1, "psatd"), ("fp64", "3d6", (32, 32, 32), 1, "psatd"),
         ("fp32", "3d6", (16, 32, 64), 3, "psatd"), ("fp32", "te", (128, 256), 3, "psatd"),
         ("fp64", "te", (64, 64), 2, "pstd"),
         ("fp32", "te", (768, 768), 1, "psatd")]   # the largest square FP32 TE grid the array holds


@pytest.mark.parametrize("prec,layout,shape,nsteps,scheme", CASES)
def test_noalloc_matches_plan_step_on_two_calls(prec, layout, shape, nsteps, scheme):
    import torch
    ensure_lib()
    n = tuple(reversed(shape))
    d = tuple([1.0 / 64] * len(shape))
    dt = d[0] / math.sqrt(len(shape)) * (0.5 if scheme == "pstd" else 1.0)
    Ea, Ba, Ja = _state(shape, layout, 41, prec)
    Eb = [t.clone() if t is not None else None for t in Ea]
    Bb = [t.clone() if t is not None else None for t in Ba]
    plan = capi.Plan(n, d, dt, layout=layout, prec=prec, src="J", scheme=scheme)
    for call in range(2):
        plan.step(Ea, Ba, Ja, nsteps=nsteps)
        capi.step_noalloc(n, d, dt, Eb, Bb, Ja, layout=layout, prec=prec, src="J", nsteps=nsteps, scheme=scheme)
        torch.cuda.synchronize()
        err = rel_l2_fields(_np(Eb), _np(Bb), _np(Ea), _np(Ba))
        assert err < TOL[prec], (call, err)
    plan.destroy()


@pytest.mark.parametrize("n", [1024, 2048])
def test_noalloc_rejects_grids_beyond_its_array(n):
    ensure_lib()
    z = torch_dev(np.zeros((n, n)), "fp32")
    with pytest.raises(capi.PsatdError) as ei:
        capi.step_noalloc((n, n), (1.0, 1.0), 0.5, [z, z, None], [None, None, z], [z, z, None],
                          layout="te", prec="fp32", src="J")
    assert ei.value.status == 2 and "scratch" in str(ei.value)
