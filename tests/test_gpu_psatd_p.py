"""GPU parity of the staggered order-p PSATD step (desc.order = p; Table 1 row
PSATD-p) with the FP64 oracle's ``psatd_step(order=p)``: one step at every layout
and source form (white-noise inputs, so the Nyquist modes are exercised), a
staggered eigenmode over 100 steps against its closed form, and the local-FFT
decomposition reproducing the global step to rounding at finite order with a
moderate guard region (Sec. II.A.3)."""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, psatd_gpu, rel_l2_fields, rounded, torch_dev
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth
from test_oracle_psatd_p import _te_wave

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "mixed_fp16": 4e-6}


def _inputs(shape, layout, src, seed, prec):
    E = mask_layout(synth.random_fields(shape, 3, seed), layout, "E")
    B = mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B")
    J = mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J") if src != "none" else None
    r0 = synth.random_fields(shape, 1, seed + 3)[0] if src == "rho" else None
    r1 = synth.random_fields(shape, 1, seed + 4)[0] if src == "rho" else None
    rd = (lambda a: rounded(a, prec) if a is not None else None)
    return rd(E), rd(B), rd(J), rd(r0), rd(r1)


CASES = [((32, 64), "te", "J", 2), ((64, 32), "te", "rho", 8), ((64, 128), "tm", "J", 32),
         ((32, 32), "2d6", "none", 4), ((16, 64), "2d6", "rho", 16), ((256, 512), "te", "J", 128)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,layout,src,p", CASES)
def test_order_p_one_step_matches_oracle(shape, layout, src, p, prec):
    d, dt = (1.0, 0.7), 0.45
    E, B, J, r0, r1 = _inputs(shape, layout, src, 600, prec)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout=layout, prec=prec, src=src, order=p)
    Eo, Bo = orc.psatd_step(E, B, J, r0, r1, d=d, dt=dt, form={"none": "none", "J": "J", "rho": "rho"}[src],
                            order=p)
    Eo, Bo = mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,src,p", [((16, 16, 16), "J", 4), ((8, 32, 16), "rho", 16), ((32, 8, 16), "none", 2)])
def test_order_p_3d_one_step_matches_oracle(shape, src, p, prec):
    d, dt = (1.0, 0.8, 1.2), 0.6
    E, B, J, r0, r1 = _inputs(shape, "3d6", src, 610, prec)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec=prec, src=src, order=p)
    Eo, Bo = orc.psatd_step(E, B, J, r0, r1, d=d, dt=dt, form={"none": "none", "J": "J", "rho": "rho"}[src],
                            order=p)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL[prec]


def test_order_p_mixed_precision_one_step():
    shape, d, dt = (256, 512), (1.0, 1.0), 0.5
    E, B, J, _, _ = _inputs(shape, "te", "J", 620, "mixed_fp16")
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="mixed_fp16", src="J", order=16)
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J", order=16)
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL["mixed_fp16"]


def test_staggered_eigenmode_100_steps_fp64():
    shape, d, dt, p = (64, 128), (1.0, 0.8), 0.9, 8
    E0, B0 = _te_wave(shape, d, (9, -5), p, 1.0, 0.3, 0.0)
    Eg, Bg = psatd_gpu(shape, d, dt, E0, B0, layout="te", prec="fp64", src="none", nsteps=100, order=p)
    Ea, Ba = _te_wave(shape, d, (9, -5), p, 1.0, 0.3, 100 * dt)
    assert rel_l2_fields(Eg, Bg, Ea, Ba) < 1e-11


def test_local_decomposition_at_finite_order_equals_global_step():
    """128^2 grid, 4 x 4 patches of 32^2 with 16 guard cells (extended 64^2), order 8,
    FP64: the local-FFT result equals the global step to rounding, while the exact-k
    (order 0) decomposition differs by about 1e-2."""
    import torch
    ensure_lib()
    n, d, dt = 128, (1.0, 1.0), 1.0 / math.sqrt(2.0)
    rng = np.random.default_rng(5)
    ky = 2 * np.pi * np.fft.fftfreq(n)[:, None]
    kx = 2 * np.pi * np.fft.rfftfreq(n)[None, :]
    filt = 1.0 / (1.0 + 40.0 * (kx ** 2 + ky ** 2)) ** 2
    E = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal((n, n))) * filt, s=(n, n)) for _ in range(3)])
    B = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal((n, n))) * filt, s=(n, n)) for _ in range(3)])
    errs = {}
    for p in (0, 8):
        Eo, Bo = orc.psatd_step(E, B, d=d, dt=dt, order=p)   # the global step
        L = capi.Local((n, n), d, dt, px=4, py=4, guard=16, layout="2d6", prec="fp64", src="none", order=p)
        Et = [torch_dev(E[i], "fp64") for i in range(3)]
        Bt = [torch_dev(B[i], "fp64") for i in range(3)]
        L.step(Et, Bt)
        L.sync()
        Eg = np.stack([t.cpu().numpy() for t in Et])
        Bg = np.stack([t.cpu().numpy() for t in Bt])
        L.destroy()
        errs[p] = rel_l2_fields(Eg, Bg, Eo, Bo)
    print("local (4x4 patches, g = 16) vs global, order 0 / 8:", errs)
    assert errs[0] > 1e-3 and errs[8] < 1e-12, errs
