"""GPU parity of the Yee / CKC FDTD kernels with the FP64 oracle
(FP64: 1e-12 per step; FP32: 1e-6 per step, from FP32-rounded inputs)."""
import numpy as np
import pytest

from gpu_helpers import fdtd_gpu, mask_layout, rel_l2_fields, rounded
from oracle import fdtd as ofd
from paper_1608_05739_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("yee", "te", (64, 32), (1.0, 0.9), 0.6, True),
    ("yee", "tm", (32, 64), (1.0, 1.0), 0.7, True),
    ("yee", "2d6", (128, 128), (1.0, 1.0), 0.5, False),
    ("ckc", "te", (64, 64), (1.0, 1.0), 1.0, True),
    ("ckc", "2d6", (48, 40), (1.0, 1.0), 0.9, True),
    ("yee", "3d6", (16, 24, 20), (1.0, 1.0, 1.0), 0.5, True),
    ("yee", "te", (37, 53), (1.0, 1.0), 0.5, True),   # non-power-of-two
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme,layout,shape,d,dt,withJ", CASES)
def test_fdtd_one_step_matches_oracle(scheme, layout, shape, d, dt, withJ, prec):
    E = rounded(mask_layout(synth.random_fields(shape, 3, 21), layout, "E"), prec)
    B = rounded(mask_layout(synth.random_fields(shape, 3, 22), layout, "B"), prec)
    J = rounded(mask_layout(synth.random_fields(shape, 3, 23), layout, "J"), prec) if withJ else None
    Eg, Bg = fdtd_gpu(shape, d, dt, E, B, J, layout=layout, prec=prec, scheme=scheme)
    Eo, Bo = ofd.fdtd_step(E, B, J, d=d, dt=dt, scheme=scheme)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")) < tol


def test_yee_config1_200_steps_fp64():
    """The config-1 companion run: the same 8 plane waves advanced 200 Yee steps."""
    shape, d, dt = (128, 128), (1.0, 1.0), 0.5
    waves = synth.plane_waves(shape, 8, seed=1608)
    E, B = synth.plane_wave_fields(waves, shape, d)
    Eg, Bg = fdtd_gpu(shape, d, dt, E, B, layout="2d6", prec="fp64", scheme="yee", nsteps=200)
    Eo, Bo = ofd.fdtd_step(E, B, d=d, dt=dt, scheme="yee", nsteps=200)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < 1e-11
