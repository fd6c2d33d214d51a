"""Pins of the FP64 PSATD oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: the references are a brute-force
DFT, the matrix exponential of the per-mode ODE, the closed-form vacuum plane
waves (omega = c|k|, Table 1 row PSATD), energy and Gauss-law identities.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from analytic import plane_waves_at, rel_l2
from oracle import psatd
from paper_1608_05739_gb300 import synth


def _brute_dft(f):
    """O(N^2) DFT sum_x f(x) exp(-i k.x) over all axes (index space)."""
    out = f.astype(np.complex128)
    for ax in range(f.ndim):
        n = f.shape[ax]
        idx = np.arange(n)
        M = np.exp(-2j * np.pi * np.outer(idx, idx) / n)
        out = np.moveaxis(np.tensordot(M, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


@pytest.mark.parametrize("shape", [(6, 5), (4, 8), (3, 7), (4, 3, 6), (2, 5, 4)])
def test_forward_transform_is_the_dft(shape):
    f = synth.random_fields(shape, 1, seed=11)[0]
    full = _brute_dft(f)
    half = psatd.forward(f)
    np.testing.assert_allclose(half, full[..., : shape[-1] // 2 + 1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(psatd.inverse(half, shape), f, rtol=0, atol=1e-13)


def test_wavenumbers_nyquist_reading():
    k = psatd.wavenumbers(8, 0.5)
    assert k[4] == 0.0
    np.testing.assert_allclose(k[:4], 2 * np.pi * np.arange(4) / 4.0)
    np.testing.assert_allclose(k[5:], 2 * np.pi * np.arange(-3, 0) / 4.0)
    kh = psatd.wavenumbers(8, 0.5, half=True)
    assert kh.shape == (5,) and kh[4] == 0.0
    ko = psatd.wavenumbers(7, 1.0)
    assert np.all(ko[1:] != 0.0)


def _expm_push(k, E, B, J, dt, c, eps0):
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]], dtype=np.complex128)
    M = np.zeros((9, 9), dtype=np.complex128)
    M[0:3, 3:6] = 1j * c * c * K
    M[0:3, 6:9] = -np.eye(3) / eps0
    M[3:6, 0:3] = -1j * K
    s = sla.expm(M * dt) @ np.concatenate([E, B, J])
    return s[0:3], s[3:6]


def _one(v):
    return [np.array([x]) for x in v]


@pytest.mark.parametrize("seed", range(12))
def test_push_is_the_exact_solution_constant_J(seed):
    """J-form push == expm of the per-mode system dE/dt = i c^2 k x B - J/eps0, dB/dt = -i k x E."""
    g = np.random.default_rng(seed)
    k = g.normal(size=3) * 10.0 ** g.uniform(-6, 1.2)
    E, B, J = (g.normal(size=3) + 1j * g.normal(size=3) for _ in range(3))
    dt, c, eps0 = g.uniform(0.1, 2.0), g.uniform(0.5, 2.0), g.uniform(0.5, 2.0)
    Ee, Be = _expm_push(k, E, B, J, dt, c, eps0)
    En, Bn = psatd.push_modes(tuple(np.array([v]) for v in k), _one(E), _one(B), _one(J),
                              dt=dt, c=c, eps0=eps0, form="J")
    got = np.concatenate([np.ravel(En), np.ravel(Bn)])
    want = np.concatenate([Ee, Be])
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    En0, Bn0 = psatd.push_modes(tuple(np.array([v]) for v in k), _one(E), _one(B),
                                dt=dt, c=c, eps0=eps0, form="none")
    Ee0, Be0 = _expm_push(k, E, B, 0 * J, dt, c, eps0)
    want0 = np.concatenate([Ee0, Be0])
    assert np.max(np.abs(np.concatenate([np.ravel(En0), np.ravel(Bn0)]) - want0)) <= 1e-12 * np.max(np.abs(want0))


@pytest.mark.parametrize("seed", range(6))
def test_rho_form_is_the_exact_solution_when_gauss_and_continuity_hold(seed):
    g = np.random.default_rng(100 + seed)
    k = g.normal(size=3) * 10.0 ** g.uniform(-5, 1)
    E, B, J = (g.normal(size=3) + 1j * g.normal(size=3) for _ in range(3))
    dt, c, eps0 = g.uniform(0.1, 2.0), g.uniform(0.5, 2.0), g.uniform(0.5, 2.0)
    rho0 = 1j * eps0 * np.dot(k, E)                  # Gauss: i k.E = rho/eps0
    rho1 = rho0 - 1j * dt * np.dot(k, J)             # continuity
    Ee, Be = _expm_push(k, E, B, J, dt, c, eps0)
    En, Bn = psatd.push_modes(tuple(np.array([v]) for v in k), _one(E), _one(B), _one(J),
                              np.array([rho0]), np.array([rho1]), dt=dt, c=c, eps0=eps0, form="rho")
    got = np.concatenate([np.ravel(En), np.ravel(Bn)])
    want = np.concatenate([Ee, Be])
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def test_k0_mode():
    z = tuple(np.zeros(1) for _ in range(3))
    E, B, J = _one([1.0, 2.0, 3.0]), _one([4.0, 5.0, 6.0]), _one([0.5, -1.0, 2.0])
    En, Bn = psatd.push_modes(z, E, B, J, dt=0.3, c=2.0, eps0=0.5, form="J")
    np.testing.assert_allclose(np.ravel(En), [1.0 - 0.3, 2.0 + 0.6, 3.0 - 1.2])
    np.testing.assert_allclose(np.ravel(Bn), [4.0, 5.0, 6.0])


def test_series_branches_match_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for x in [1e-8, 1e-3, 0.1, 0.49, 0.5, 0.51, 1.0, 3.0, 10.0]:
        xm = mp.mpf(x)
        f1 = (mp.sin(xm) / xm - 1) / xm ** 2
        f2 = (mp.sin(xm) / xm - mp.cos(xm)) / xm ** 2
        assert abs(float(psatd.f1(x)) - float(f1)) <= 1e-15 * abs(float(f1)) + 1e-17
        assert abs(float(psatd.f2(x)) - float(f2)) <= 1e-15 * abs(float(f2)) + 1e-17


def test_config1_plane_waves_rotate_exactly():
    """128^2, dx=dy=1, c dt = 0.5 dx, 8 seeded on-grid plane waves, 200 steps: omega = c|k|."""
    shape, d, dt = (128, 128), (1.0, 1.0), 0.5
    waves = synth.plane_waves(shape, 8, seed=1608)
    E, B = synth.plane_wave_fields(waves, shape, d)
    E1, B1 = psatd.psatd_step(E, B, d=d, dt=dt, nsteps=200)
    Ea, Ba = plane_waves_at(waves, shape, d, 200 * dt)
    assert rel_l2(np.concatenate([E1, B1]), np.concatenate([Ea, Ba])) < 1e-11


def test_no_courant_limit_large_dt():
    """c dt = 2 dx (above every FDTD limit of Table 1): still exact."""
    shape, d, dt = (32, 64), (1.0, 0.5), 2.0
    waves = synth.plane_waves(shape, 4, seed=7)
    E, B = synth.plane_wave_fields(waves, shape, d)
    E1, B1 = psatd.psatd_step(E, B, d=d, dt=dt, nsteps=50)
    Ea, Ba = plane_waves_at(waves, shape, d, 50 * dt)
    assert rel_l2(np.concatenate([E1, B1]), np.concatenate([Ea, Ba])) < 1e-11


@pytest.mark.parametrize("shape,d", [((32, 48), (1.0, 0.7)), ((16, 12, 20), (1.0, 1.3, 0.8))])
def test_energy_conserved_without_sources(shape, d):
    E = synth.random_fields(shape, 3, seed=21)
    B = synth.random_fields(shape, 3, seed=22)
    W0 = psatd.field_energy(E, B, d, c=1.5, eps0=0.7)
    E1, B1 = psatd.psatd_step(E, B, d=d, dt=0.9, c=1.5, eps0=0.7, nsteps=20)
    assert abs(psatd.field_energy(E1, B1, d, c=1.5, eps0=0.7) / W0 - 1.0) < 1e-12


def _half_weights(shape):
    """Parseval weights of the rfft half spectrum (2 for columns with a mirror)."""
    nx = shape[-1]
    w = np.full(nx // 2 + 1, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    return w


def test_energy_balance_with_current():
    """W(n+1) - W(n) = -dV sum_x J . int_0^dt E dt (Poynting theorem, per-mode exact)."""
    shape, d, dt, c, eps0 = (24, 32), (1.0, 1.0), 0.6, 1.3, 0.9
    E = synth.random_fields(shape, 3, seed=31)
    B = synth.random_fields(shape, 3, seed=32)
    J = synth.random_fields(shape, 3, seed=33)
    E1, B1 = psatd.psatd_step(E, B, J, d=d, dt=dt, c=c, eps0=eps0, form="J")
    dW = psatd.field_energy(E1, B1, d, c, eps0) - psatd.field_energy(E, B, d, c, eps0)
    # time integral of E over the step, written independently of the push:
    # transverse part: (S/ck) E_T + ((1-C)/(c k)^2)(i c^2 k x B - J_T/eps0); longitudinal: E_L dt - J_L dt^2/(2 eps0)
    kx, ky, kz = psatd.spectral_grid(shape, d)
    kv = np.broadcast_arrays(kx, ky, kz)
    k2 = kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2
    kn = np.sqrt(k2)
    Eh = [psatd.forward(E[i]) for i in range(3)]
    Bh = [psatd.forward(B[i]) for i in range(3)]
    Jh = [psatd.forward(J[i]) for i in range(3)]
    I = []
    for i in range(3):
        I.append(np.zeros_like(Eh[0]))
    with np.errstate(divide="ignore", invalid="ignore"):
        kap = [np.where(kn > 0, v / kn, 0.0) for v in kv]
        x = c * kn * dt
        s_ck = np.where(kn > 0, np.sin(x) / (c * kn), dt)
        omc = np.where(kn > 0, (1 - np.cos(x)) / (c * kn) ** 2, dt * dt / 2)
    kE = sum(kap[i] * Eh[i] for i in range(3))
    kJ = sum(kap[i] * Jh[i] for i in range(3))
    kxB = [kv[1] * Bh[2] - kv[2] * Bh[1], kv[2] * Bh[0] - kv[0] * Bh[2], kv[0] * Bh[1] - kv[1] * Bh[0]]
    for i in range(3):
        EL, JL = kap[i] * kE, kap[i] * kJ
        ET, JT = Eh[i] - EL, Jh[i] - JL
        I[i] = s_ck * ET + omc * (1j * c * c * kxB[i] - JT / eps0) + EL * dt - JL * dt * dt / (2 * eps0)
    Ir = np.stack([psatd.inverse(I[i], shape) for i in range(3)])
    work = -float(np.prod(d)) * float(np.sum(J * Ir))
    assert abs(dW - work) <= 1e-11 * abs(work)


def _gauss_residual(E, rho, d, eps0):
    kx, ky, kz = psatd.spectral_grid(rho.shape, d)
    div = 1j * (kx * psatd.forward(E[0]) + ky * psatd.forward(E[1]) + kz * psatd.forward(E[2]))
    r = psatd.forward(rho) / eps0
    return float(np.linalg.norm(div - r) / np.linalg.norm(r))


@pytest.mark.parametrize("shape,d", [((16, 16, 16), (1.0, 1.0, 1.0)), ((32, 24), (1.0, 1.0))])
def test_rho_form_equals_J_form_and_keeps_gauss(shape, d):
    dt, c, eps0 = 0.5, 1.0, 1.0
    r0, r1, J = synth.gaussian_charges(shape, d, dt, n_charges=8, seed=5)
    # transverse noise plus the Coulomb field of rho^n, so Gauss holds at t_n
    E = 0.3 * synth.random_fields(shape, 3, seed=6)
    kx, ky, kz = psatd.spectral_grid(shape, d)
    kv = np.broadcast_arrays(kx, ky, kz)
    k2 = kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2
    Eh = [psatd.forward(E[i]) for i in range(3)]
    with np.errstate(divide="ignore", invalid="ignore"):
        proj = np.where(k2 > 0, (kv[0] * Eh[0] + kv[1] * Eh[1] + kv[2] * Eh[2]) / k2, 0.0)
    R0 = psatd.forward(r0)
    with np.errstate(divide="ignore", invalid="ignore"):
        EL = [np.where(k2 > 0, -1j * kv[i] * R0 / (eps0 * k2), 0.0) for i in range(3)]
    E = np.stack([psatd.inverse(Eh[i] - kv[i] * proj + EL[i], shape) for i in range(3)])
    B = synth.random_fields(shape, 3, seed=7) * 0.1
    Bh = [psatd.forward(B[i]) for i in range(3)]
    with np.errstate(divide="ignore", invalid="ignore"):
        pb = np.where(k2 > 0, (kv[0] * Bh[0] + kv[1] * Bh[1] + kv[2] * Bh[2]) / k2, 0.0)
    B = np.stack([psatd.inverse(Bh[i] - kv[i] * pb, shape) for i in range(3)])
    assert _gauss_residual(E, r0, d, eps0) < 1e-12
    Ej, Bj = psatd.psatd_step(E, B, J, d=d, dt=dt, c=c, eps0=eps0, form="J")
    Er, Br = psatd.psatd_step(E, B, J, r0, r1, d=d, dt=dt, c=c, eps0=eps0, form="rho")
    assert rel_l2(np.concatenate([Er, Br]), np.concatenate([Ej, Bj])) < 1e-12
    assert _gauss_residual(Er, r1, d, eps0) < 1e-12
    assert _gauss_residual(Ej, r1, d, eps0) < 1e-12


def test_nyquist_mode_is_left_unchanged_in_vacuum():
    """Reading of the paper's silence: k_i := 0 at the Nyquist index, so a pure
    Nyquist-x pattern is a k = 0 mode along x and the vacuum step leaves it."""
    shape, d = (8, 16), (1.0, 1.0)
    x = np.arange(16)
    E = np.zeros((3,) + shape)
    E[2] = np.cos(np.pi * x)[None, :]
    B = np.zeros_like(E)
    E1, B1 = psatd.psatd_step(E, B, d=d, dt=0.7)
    np.testing.assert_allclose(E1, E, atol=1e-14)
    np.testing.assert_allclose(B1, 0.0, atol=1e-14)
