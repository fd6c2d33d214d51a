"""GPU parity of the PSATD step (CUDA path through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over all E and c*B components):
  FP64: 1e-12 per step (the stated FP64 bound).
  FP32: 2e-6 per step: an FP32 forward + inverse FFT pair of N points carries a
        relative rounding error of a few u sqrt(log2 N) (u = 2^-24 = 6e-8, about
        3e-7 at N = 2048^2), the push a few u more; 2e-6 is ~30 u.
        After N steps: 1e-5 (the stated FP32 bound), from FP32-rounded inputs.
"""
import math

import numpy as np
import pytest

from analytic import plane_waves_at
from gpu_helpers import mask_layout, psatd_gpu, rel_l2_fields, rounded
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}


def _inputs(shape, layout, src, seed, d, dt, prec):
    E = mask_layout(synth.random_fields(shape, 3, seed), layout, "E")
    B = mask_layout(synth.random_fields(shape, 3, seed + 1), layout, "B")
    J = mask_layout(synth.random_fields(shape, 3, seed + 2), layout, "J") if src != "none" else None
    r0 = synth.random_fields(shape, 1, seed + 3)[0] if src == "rho" else None
    r1 = synth.random_fields(shape, 1, seed + 4)[0] if src == "rho" else None
    rd = (lambda a: rounded(a, prec) if a is not None else None)
    return rd(E), rd(B), rd(J), rd(r0), rd(r1)


def _oracle(E, B, J, r0, r1, d, dt, src, c=1.0, eps0=1.0, nsteps=1):
    form = {"none": "none", "J": "J", "rho": "rho"}[src]
    return orc.psatd_step(E, B, J, r0, r1, d=d, dt=dt, c=c, eps0=eps0, form=form, nsteps=nsteps)


CASES_2D = [
    ((32, 64), "te", "J"), ((64, 32), "te", "rho"), ((16, 16), "te", "none"),
    ((64, 128), "tm", "J"), ((32, 16), "tm", "none"),
    ((128, 64), "2d6", "none"), ((32, 32), "2d6", "J"), ((16, 64), "2d6", "rho"),
    ((8, 4096), "te", "J"), ((2048, 16), "te", "J"), ((256, 512), "te", "J"),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,layout,src", CASES_2D)
def test_psatd_2d_one_step_matches_oracle(shape, layout, src, prec):
    d, dt = (1.0, 0.7), 0.45
    E, B, J, r0, r1 = _inputs(shape, layout, src, 1234, d, dt, prec)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout=layout, prec=prec, src=src)
    Eo, Bo = _oracle(E, B, J, r0, r1, d, dt, src)
    Eo, Bo = mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL[prec]


CASES_3D = [((16, 16, 16), "none"), ((8, 32, 16), "J"), ((32, 8, 16), "rho"), ((16, 16, 64), "J")]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,src", CASES_3D)
def test_psatd_3d_one_step_matches_oracle(shape, src, prec):
    d, dt = (1.0, 0.8, 1.2), 0.6
    E, B, J, r0, r1 = _inputs(shape, "3d6", src, 99, d, dt, prec)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec=prec, src=src)
    Eo, Bo = _oracle(E, B, J, r0, r1, d, dt, src)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL[prec]


def test_psatd_physical_constants_and_large_dt():
    """c, eps0 != 1 and c dt = 2 dx (no Courant limit)."""
    shape, d, dt, c, eps0 = (32, 64), (0.5, 0.25), 1.0 / 3.0, 3.0, 0.7
    E, B, J, r0, r1 = _inputs(shape, "2d6", "J", 7, d, dt, "fp64")
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="2d6", prec="fp64", src="J", c=c, eps0=eps0)
    Eo, Bo = _oracle(E, B, J, None, None, d, dt, "J", c=c, eps0=eps0)
    assert rel_l2_fields(Eg, Bg, Eo, Bo, c=c) < 1e-12


def test_config1_vacuum_plane_waves_fp64():
    """128^2, dx = dy = 1, c dt = 0.5 dx, 8 seeded plane waves, 200 steps (FP64): per-step
    parity, and after 200 steps both the oracle and the exact solution (omega = c|k|)."""
    shape, d, dt = (128, 128), (1.0, 1.0), 0.5
    waves = synth.plane_waves(shape, 8, seed=1608)
    E, B = synth.plane_wave_fields(waves, shape, d)
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, layout="2d6", prec="fp64", src="none")
    Eo, Bo = orc.psatd_step(E, B, d=d, dt=dt)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < 1e-12
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, layout="2d6", prec="fp64", src="none", nsteps=200)
    Ea, Ba = plane_waves_at(waves, shape, d, 200 * dt)
    assert rel_l2_fields(Eg, Bg, Ea, Ba) < 1e-11
    Eo, Bo = orc.psatd_step(E, B, d=d, dt=dt, nsteps=200)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < 1e-11


def test_config1_fp32_plane_waves_200_steps():
    shape, d, dt = (128, 128), (1.0, 1.0), 0.5
    waves = synth.plane_waves(shape, 8, seed=1608)
    E, B = (rounded(a, "fp32") for a in synth.plane_wave_fields(waves, shape, d))
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, layout="2d6", prec="fp32", src="none", nsteps=200)
    Eo, Bo = orc.psatd_step(E, B, d=d, dt=dt, nsteps=200)
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < 1e-5


def _sheet_J(shape, d, n, dt, lam):
    return synth.current_sheet(shape, d, (n + 0.5) * dt, lam=lam, a=0.9, w=2.0 * d[0])


def test_config2_full_size_one_step_fp32():
    """2048^2 TE, dx = lambda/64, c dt = dx/sqrt(2), current-sheet J: one step from a
    non-trivial state, FP32 GPU vs FP64 oracle (the bench's launch configuration)."""
    shape = (2048, 2048)
    d = (1.0 / 64, 1.0 / 64)
    dt = d[0] / math.sqrt(2.0)
    E = mask_layout(synth.random_fields(shape, 3, 5), "te", "E")
    B = mask_layout(synth.random_fields(shape, 3, 6), "te", "B")
    J = _sheet_J(shape, d, 17, dt, 1.0)
    E, B, J = (rounded(a, "fp32") for a in (E, B, J))
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J")
    Eo, Bo = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < TOL["fp32"]


def test_sheet_fp32_many_steps_within_1e5():
    """Current-sheet drive from zero fields, 2000 FP32 steps on a 512^2 grid
    (dx = lambda/64, c dt = dx/sqrt(2)), one psatd_step call per step with the
    time-varying J: relative L2 vs the FP64 oracle <= 1e-5 (stated FP32 bound)."""
    shape = (512, 512)
    d = (1.0 / 64, 1.0 / 64)
    dt = d[0] / math.sqrt(2.0)
    nsteps = 2000
    from gpu_helpers import ensure_lib, torch_dev
    from paper_1608_05739_gb300 import capi
    ensure_lib()
    plan = capi.Plan((512, 512), d, dt, layout="te", prec="fp32", src="J")
    Et = [torch_dev(np.zeros(shape), "fp32") for _ in range(2)]
    Bz = torch_dev(np.zeros(shape), "fp32")
    E = np.zeros((3,) + shape)
    B = np.zeros((3,) + shape)
    k = orc.spectral_grid(shape, d)
    for n in range(nsteps):
        J = rounded(_sheet_J(shape, d, n, dt, 1.0), "fp32")
        Jt = [torch_dev(J[0], "fp32"), torch_dev(J[1], "fp32"), None]
        plan.step([Et[0], Et[1], None], [None, None, Bz], Jt)
        E, B = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    plan.sync()
    Eg = np.zeros_like(E)
    Bg = np.zeros_like(B)
    Eg[0], Eg[1], Bg[2] = (t.double().cpu().numpy() for t in (Et[0], Et[1], Bz))
    err = rel_l2_fields(Eg, Bg, E, B)
    plan.destroy()
    assert err < 1e-5, err


def test_rho_form_keeps_gauss_and_equals_J_form_on_gpu():
    shape, d, dt = (32, 32, 32), (1.0, 1.0, 1.0), 0.5
    r0, r1, J = synth.gaussian_charges(shape, d, dt, n_charges=16, seed=3)
    E = synth.coulomb_field(r0, d)
    B = np.zeros_like(E)
    Er, Br = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec="fp64", src="rho")
    Ej, Bj = psatd_gpu(shape, d, dt, E, B, J, layout="3d6", prec="fp64", src="J")
    assert rel_l2_fields(Er, Br, Ej, Bj) < 1e-12
    kx, ky, kz = orc.spectral_grid(shape, d)
    div = 1j * (kx * orc.forward(Er[0]) + ky * orc.forward(Er[1]) + kz * orc.forward(Er[2]))
    R = orc.forward(r1)
    assert np.linalg.norm(div - R) / np.linalg.norm(R) < 1e-12


def test_uniform_current_k0_mode():
    shape, d, dt = (16, 32), (1.0, 1.0), 0.3
    E = np.zeros((3,) + shape)
    B = np.zeros((3,) + shape)
    J = np.ones((3,) + shape) * np.array([0.5, -1.5, 2.0])[:, None, None]
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="2d6", prec="fp64", src="J", eps0=0.6)
    np.testing.assert_allclose(Eg, -dt / 0.6 * J, atol=1e-14)
    np.testing.assert_allclose(Bg, 0.0, atol=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nsteps_equals_repeated_calls_bitwise_and_deterministic(prec):
    shape, d, dt = (64, 64), (1.0, 1.0), 0.4
    E, B, J, _, _ = _inputs(shape, "te", "J", 11, d, dt, prec)
    E1, B1 = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=prec, src="J", nsteps=5)
    E2, B2 = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=prec, src="J", calls=5)
    E3, B3 = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec=prec, src="J", nsteps=5)
    assert np.array_equal(E1, E2) and np.array_equal(B1, B2)
    assert np.array_equal(E1, E3) and np.array_equal(B1, B3)


def test_step_argument_errors_raise():
    from gpu_helpers import ensure_lib, torch_dev
    from paper_1608_05739_gb300 import capi
    ensure_lib()
    plan = capi.Plan((32, 32), (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
    z = [torch_dev(np.zeros((32, 32)), "fp32") for _ in range(5)]
    with pytest.raises(capi.PsatdError):
        plan.step([z[0], z[1], None], [None, None, z[2]], None)           # J missing
    with pytest.raises(ValueError):
        plan.step([z[0], None, None], [None, None, z[2]], [z[3], z[4], None])  # Ey missing
    with pytest.raises(capi.PsatdError):
        plan.step([z[0], z[1], None], [None, None, z[2]], [z[3], z[4], None], nsteps=0)
    plan.set_timing(True)
    plan.step([z[0], z[1], None], [None, None, z[2]], [z[3], z[4], None], nsteps=3)
    t = plan.kernel_times()
    assert set(t) == {"fwd_x_r2c", "line_fft_push", "inv_x_c2r"}
    assert all(v[0] == 3 and v[1] > 0 for v in t.values())
    assert plan.workspace_bytes() > 5 * 17 * 32 * 8
    plan.destroy()


def test_config3_full_size_one_step_fp32():
    """3D 256^3 FP32 rho-form (all five passes at the size the 3D side bench times):
    one step from seeded white-noise fields and sources vs the FP64 oracle."""
    shape = (256, 256, 256)
    d, dt = (1.0, 1.0, 1.0), 0.5
    E, B, J, r0, r1 = _inputs(shape, "3d6", "rho", 2024, d, dt, "fp32")
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, r0, r1, layout="3d6", prec="fp32", src="rho")
    Eo, Bo = _oracle(E, B, J, r0, r1, d, dt, "rho")
    assert rel_l2_fields(Eg, Bg, Eo, Bo) < TOL["fp32"]


def test_longest_lines_fp32_and_the_fp64_shared_memory_limit():
    """4096-point fused-pass lines: FP32 TE J-form stages (5 + 1) x 4096 x 8 B = 192 KB
    per line and matches the oracle; FP64 would need 384 KB and is refused at plan
    creation (UNSUPPORTED, nothing allocated)."""
    shape, d, dt = (4096, 32), (1.0, 1.0), 0.5
    E, B, J, r0, r1 = _inputs(shape, "te", "J", 4096, d, dt, "fp32")
    Eg, Bg = psatd_gpu(shape, d, dt, E, B, J, layout="te", prec="fp32", src="J", nsteps=2)
    Eo, Bo = _oracle(E, B, J, None, None, d, dt, "J", nsteps=2)
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B")) < 2 * TOL["fp32"]
    with pytest.raises(capi.PsatdError) as ei:
        capi.Plan((32, 4096), d, dt, layout="te", prec="fp64", src="J")
    assert ei.value.status == 2 and "shared memory" in str(ei.value)
