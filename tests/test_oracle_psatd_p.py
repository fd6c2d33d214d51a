"""Pins of the staggered order-p PSATD step (``oracle.psatd.psatd_step(order=p)``;
Sec. III.B, Table 1 row PSATD-p).

The closed form: on the staggered (Yee) grid a plane wave sampled at each
component's own position is an eigenmode of the order-p scheme; its wavenumber
is k_p, the symbol of the order-p staggered difference, and it rotates at
omega = c |k_p| (refractive index |k|/|k_p|).  Here k_p is measured by applying
the stencil to the sampled wave (not from the sine sum the oracle uses), the
wave is built at its staggered positions by hand, and the oracle must carry it
for many steps to rounding (TE, TM, 3D, and the Nyquist mode, which the
staggered scheme propagates).  Also: energy conservation (the update is
unitary), the refractive index |k|/|k_p| at a printed-by-hand value, and the
local-FFT truncation error at finite order, the paper's reason for high-order
solvers with few guard cells (Sec. II.A.3)."""
import math

import numpy as np
import pytest

from oracle import dispersion as dsp
from oracle import local as loc
from oracle import psatd as orc


def _kp_by_stencil(k, dx, p):
    """i k_p from the order-p staggered difference applied to exp(i k x) at x = 0."""
    C = dsp.fornberg_staggered(p)
    l = np.arange(1, len(C) + 1)
    h = (2 * l - 1) * dx / 2.0
    val = np.sum(C * (np.exp(1j * k * h) - np.exp(-1j * k * h))) / dx
    assert abs(val.real) < 1e-14
    return val.imag


def _te_wave(shape, d, m, p, a, phi0, t, c=1.0):
    """TE (Ex, Ey, Bz) eigenmode of the order-p scheme, sampled at the Yee positions."""
    ny, nx = shape
    kx = 2 * math.pi * m[0] / (nx * d[0])
    ky = 2 * math.pi * m[1] / (ny * d[1])
    kpx, kpy = _kp_by_stencil(kx, d[0], p), _kp_by_stencil(ky, d[1], p)
    kn = math.hypot(kpx, kpy)
    w = c * kn
    x = np.arange(nx)[None, :] * d[0]
    y = np.arange(ny)[:, None] * d[1]
    hx, hy = d[0] / 2, d[1] / 2
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    E[0] = -a * (kpy / kn) * np.cos(kx * (x + hx) + ky * y - w * t + phi0)
    E[1] = a * (kpx / kn) * np.cos(kx * x + ky * (y + hy) - w * t + phi0)
    B[2] = (a / c) * np.cos(kx * (x + hx) + ky * (y + hy) - w * t + phi0)
    return E, B


def _tm_wave(shape, d, m, p, a, phi0, t, c=1.0):
    """TM (Ez, Bx, By) eigenmode: Ez on the nodes, Bx at y + dy/2, By at x + dx/2."""
    ny, nx = shape
    kx = 2 * math.pi * m[0] / (nx * d[0])
    ky = 2 * math.pi * m[1] / (ny * d[1])
    kpx, kpy = _kp_by_stencil(kx, d[0], p), _kp_by_stencil(ky, d[1], p)
    kn = math.hypot(kpx, kpy)
    w = c * kn
    x = np.arange(nx)[None, :] * d[0]
    y = np.arange(ny)[:, None] * d[1]
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    E[2] = a * np.cos(kx * x + ky * y - w * t + phi0)
    # B = kappa x E / c with kappa = k_p/|k_p|: (kappa_y Ez, -kappa_x Ez, 0) / c
    B[0] = (a / c) * (kpy / kn) * np.cos(kx * x + ky * (y + d[1] / 2) - w * t + phi0)
    B[1] = -(a / c) * (kpx / kn) * np.cos(kx * (x + d[0] / 2) + ky * y - w * t + phi0)
    return E, B


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("p", [2, 4, 16, 64])
@pytest.mark.parametrize("m", [(3, 5), (-7, 2), (13, -11)])
def test_staggered_plane_wave_rotates_at_c_kp(p, m):
    shape, d, dt, n = (32, 48), (1.0, 0.8), 0.9, 40
    E0, B0 = _te_wave(shape, d, m, p, 1.3, 0.4, 0.0)
    E1, B1 = orc.psatd_step(E0, B0, d=d, dt=dt, nsteps=n, order=p)
    Ea, Ba = _te_wave(shape, d, m, p, 1.3, 0.4, n * dt)
    assert _rel(np.concatenate([E1, B1]), np.concatenate([Ea, Ba])) < 1e-12
    E0, B0 = _tm_wave(shape, d, m, p, -0.7, 1.9, 0.0)
    E1, B1 = orc.psatd_step(E0, B0, d=d, dt=dt, nsteps=n, order=p)
    Ea, Ba = _tm_wave(shape, d, m, p, -0.7, 1.9, n * dt)
    assert _rel(np.concatenate([E1, B1]), np.concatenate([Ea, Ba])) < 1e-12


def test_order_p_refractive_index_is_k_over_kp():
    """Table 1 (PSATD-p): the phase advance per step of the eigenmode gives
    n = |k| / |k_p|; at p = 2 and k dx = pi/2 along x it is (pi/2)/(2 sin(pi/4))."""
    shape, d, dt = (16, 16), (1.0, 1.0), 0.3
    E0, B0 = _te_wave(shape, d, (4, 0), 2, 1.0, 0.0, 0.0)
    Eq, Bq = _te_wave(shape, d, (4, 0), 2, 1.0, -math.pi / 2, 0.0)   # the quadrature wave
    E1, B1 = orc.psatd_step(E0, B0, d=d, dt=dt, order=2)
    # E1 = cos(w dt) E0 + sin(w dt) Eq for the travelling wave
    cw = np.sum(E1 * E0) / np.sum(E0 * E0)
    sw = np.sum(E1 * Eq) / np.sum(Eq * Eq)
    w = math.atan2(sw, cw) / dt
    k = 2 * math.pi * 4 / 16
    assert abs(k / w - (math.pi / 2) / (2 * math.sin(math.pi / 4))) < 1e-12


def test_order_p_conserves_energy_without_sources():
    rng = np.random.default_rng(4)
    shape, d, dt = (24, 40), (1.0, 1.3), 2.5
    E = rng.standard_normal((3, *shape))
    B = rng.standard_normal((3, *shape))
    w0 = orc.field_energy(E, B, d)
    E1, B1 = orc.psatd_step(E, B, d=d, dt=dt, nsteps=7, order=8)
    assert abs(orc.field_energy(E1, B1, d) / w0 - 1.0) < 1e-13


def test_3d_order_p_plane_wave():
    """3D: a wave along (1, 2, -1) modes with E along k_p x z^, sampled at the Yee
    positions of every component, rotates at c |k_p|."""
    shape, d, dt, n, p = (16, 16, 16), (1.0, 1.0, 1.0), 0.7, 10, 4
    nz, ny, nx = shape
    m = (1, 2, -1)
    k = [2 * math.pi * m[i] / (shape[2 - i] * d[i]) for i in range(3)]
    kp = [_kp_by_stencil(k[i], d[i], p) for i in range(3)]
    kn = math.sqrt(sum(v * v for v in kp))
    kap = [v / kn for v in kp]
    e = np.cross(kap, [0.0, 0.0, 1.0])
    e = e / np.linalg.norm(e)
    b = np.cross(kap, e)
    X = [np.arange(nx)[None, None, :] * d[0], np.arange(ny)[None, :, None] * d[1],
         np.arange(nz)[:, None, None] * d[2]]

    def at(shift, t):
        ph = sum(k[i] * (X[i] + (d[i] / 2 if i in shift else 0.0)) for i in range(3))
        return np.cos(ph - kn * t + 0.3)

    def fields(t):
        E = np.stack([e[i] * at(orc.STAGGER_E[i], t) * np.ones(shape) for i in range(3)])
        B = np.stack([b[i] * at(orc.STAGGER_B[i], t) * np.ones(shape) for i in range(3)])
        return E, B

    E0, B0 = fields(0.0)
    E1, B1 = orc.psatd_step(E0, B0, d=d, dt=dt, nsteps=n, order=p)
    Ea, Ba = fields(n * dt)
    assert _rel(np.concatenate([E1, B1]), np.concatenate([Ea, Ba])) < 1e-12


def test_local_truncation_error_at_finite_order_reaches_rounding():
    """The paper's point (Sec. II.A.3): with a finite-order staggered stencil and a
    guard region somewhat wider than its reach, local FFTs give the global
    solution to machine precision; the exact-k scheme keeps an error of 1e-2."""
    n = 128
    shape, d, dt = (n, n), (1.0, 1.0), 1.0 / math.sqrt(2.0)
    rng = np.random.default_rng(5)
    ky = 2 * np.pi * np.fft.fftfreq(n)[:, None]
    kx = 2 * np.pi * np.fft.rfftfreq(n)[None, :]
    filt = 1.0 / (1.0 + 40.0 * (kx ** 2 + ky ** 2)) ** 2
    E = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal(shape)) * filt, s=shape) for _ in range(3)])
    B = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal(shape)) * filt, s=shape) for _ in range(3)])
    err = {}
    for p, g in ((0, 16), (2, 8), (8, 8), (8, 16), (32, 8), (32, 16)):
        Eg, Bg = orc.psatd_step(E, B, d=d, dt=dt, order=p)
        El, Bl = loc.local_step(E, B, d=d, dt=dt, px=4, py=4, guard=g, order=p)
        err[(p, g)] = _rel(np.concatenate([El, Bl]), np.concatenate([Eg, Bg]))
    assert err[(0, 16)] > 1e-3, err
    assert err[(2, 8)] < 1e-14 and err[(8, 16)] < 1e-14, err
    assert err[(8, 8)] > err[(8, 16)] and err[(32, 8)] > err[(32, 16)] > err[(8, 16)], err


def test_nyquist_mode_is_an_eigenmode_of_the_staggered_scheme():
    """A TE wave at the x Nyquist index (k dx = pi): k_p = (2/dx) sum_l C_l (-1)^(l+1)
    is non-zero on the staggered grid and the mode rotates at c|k_p| like any other."""
    for p in (2, 6):
        shape, d, dt, n = (8, 16), (1.0, 1.0), 0.4, 25
        E0, B0 = _te_wave(shape, d, (8, 3), p, 1.0, 0.2, 0.0)
        E1, B1 = orc.psatd_step(E0, B0, d=d, dt=dt, nsteps=n, order=p)
        Ea, Ba = _te_wave(shape, d, (8, 3), p, 1.0, 0.2, n * dt)
        assert _rel(np.concatenate([E1, B1]), np.concatenate([Ea, Ba])) < 1e-12
