"""Pins of the Fraunhofer far-field oracle (Sec. II.B diagnostic) against what
the mathematics fixes, independently of its own sum:

* the whole periodic grid without apodisation, at the grid's wavevectors
  2 pi m / (N d): the library DFT (numpy.fft.fft2) times the cell area;
* a plane wave in a Hann-apodised sub-window at arbitrary wavevectors: the
  closed form of the apodised geometric sum (Hann = 1/2 - cos/2 written as
  three exponentials, each summed as a geometric series);
* the direction of a plane wave: on the ring |k| = |q| the brightest angle is
  the wave's own angle (located to a small fraction of a degree).
"""
import math

import numpy as np
import pytest

from oracle import farfield as ff


def test_whole_grid_equals_library_dft():
    g = np.random.default_rng(5)
    ny, nx, d = 24, 40, (0.3, 0.7)
    F = g.standard_normal((ny, nx))
    X = np.fft.fft2(F)
    ms = [(0, 0), (1, 0), (0, 1), (3, -2), (-7, 5), (19, 11), (20, 12)]
    k = np.array([(2 * math.pi * mx / (nx * d[0]), 2 * math.pi * my / (ny * d[1])) for mx, my in ms])
    U = ff.fraunhofer(F, d, k)
    want = np.array([X[my % ny, mx % nx] for mx, my in ms]) * d[0] * d[1]
    np.testing.assert_allclose(U, want, rtol=0, atol=1e-11 * np.abs(X).max())


def _geom(a, n):
    """sum_{i<n} exp(i a i), closed form (n at a = 0 mod 2 pi)."""
    z = np.exp(1j * a)
    return n if abs(z - 1) < 1e-14 else (z ** n - 1) / (z - 1)


@pytest.mark.parametrize("window", ["x", "xy"])
def test_hann_windowed_plane_wave_closed_form(window):
    ny, nx, d = 48, 64, (1.0, 0.5)
    x0, x1, y0, y1 = 9, 55, 5, 42
    q = np.array([0.41, -0.93])
    yy, xx = np.meshgrid(np.arange(ny) * d[1], np.arange(nx) * d[0], indexing="ij")
    F = np.exp(1j * (q[0] * xx + q[1] * yy))
    k = np.array([(0.41, -0.93), (0.5, -0.9), (0.2, -1.1), (1.3, 0.4)])
    U = ff.fraunhofer(F, d, k, x_range=(x0, x1), y_range=(y0, y1), window=window)

    def apodised(delta, start, n, h, hann):
        # sum_{i<n} w_i exp(i delta (start + i) h), w_i = 1/2 - (e^{i phi_i} + e^{-i phi_i})/4
        a = delta * h
        ph = np.exp(1j * delta * start * h)
        if not hann:
            return ph * _geom(a, n)
        b = 2 * math.pi / n
        s = 0.5 * _geom(a, n) - 0.25 * np.exp(1j * b / 2) * _geom(a + b, n) - 0.25 * np.exp(-1j * b / 2) * _geom(a - b, n)
        return ph * s

    for j, (kx, ky) in enumerate(k):
        want = apodised(q[0] - kx, x0, x1 - x0, d[0], True) * \
            apodised(q[1] - ky, y0, y1 - y0, d[1], window == "xy") * d[0] * d[1]
        assert abs(U[j] - want) < 1e-10 * max(1.0, abs(want)), (j, U[j], want)


def test_ring_peak_is_the_wave_direction():
    n, d = 128, (1.0, 1.0)
    theta, kq = math.radians(37.0), 2 * math.pi / 8
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    F = np.cos(kq * (math.cos(theta) * xx + math.sin(theta) * yy))
    ang = np.radians(np.linspace(30.0, 44.0, 141))
    k = np.stack([kq * np.cos(ang), kq * np.sin(ang)], axis=1)
    P = np.abs(ff.fraunhofer(F, d, k, window="xy")) ** 2
    i = int(np.argmax(P))
    # parabolic refinement on log power
    a, b, c = np.log(P[i - 1:i + 2])
    off = 0.5 * (a - c) / (a - 2 * b + c)
    peak = ang[i] + off * (ang[1] - ang[0])
    assert abs(peak - theta) < math.radians(0.05), math.degrees(peak)
