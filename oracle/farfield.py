"""Fraunhofer far-field transform of a field snapshot -- TEST INFRASTRUCTURE ONLY.

Sec. II.B: the angularly resolved harmonic spectrum in the far field is obtained
by applying the Fraunhofer diffraction integral to the reflected field the
simulation gives.  In 2D, a field F(x, y) recorded over a window radiates to
the far-field direction u = (cos theta, sin theta) at wavenumber k with the
amplitude of its plane-wave component of wavevector k u:

    U(k u) = integral over the window of w(x, y) F(x, y) exp(-i k u . r) d^2r,

here as the sum over the window's cells (x = i dx, y = j dy, cell-centred on
the grid nodes) with an optional apodisation w (Hann along x and/or y) that
limits the leakage of a window edge.  This is the definition written out in
FP64, one wavevector at a time; nothing is blocked or reordered.  Each
harmonic n is a ring of radius |k| = n k0 (c |k| = n w0 in vacuum); the angle
of the ring's brightest point is the harmonic's direction theta_r, which the
Snell model of ``dispersion`` predicts.
"""
from __future__ import annotations

import numpy as np

__all__ = ["hann", "fraunhofer"]


def hann(n: int) -> np.ndarray:
    """Periodic Hann window of n points: w_i = sin^2(pi (i + 1/2) / n), i < n
    (symmetric about the window's centre, zero only outside it)."""
    i = np.arange(n, dtype=np.float64)
    return np.sin(np.pi * (i + 0.5) / n) ** 2


def fraunhofer(F, d, kvecs, *, x_range=None, y_range=None, window="none"):
    """U_j = sum_{i in x_range, j' in y_range} w F[j', i] exp(-i (kx_j i dx + ky_j j' dy)) dx dy.

    F: real or complex array [ny][nx] (float64 is used as given); d = (dx, dy);
    kvecs: array (M, 2) of (kx, ky); x_range / y_range: (start, stop) cell
    indices (default: the whole axis); window: "none", "x" (Hann along x) or
    "xy" (Hann along both).  Returns complex128 (M,)."""
    F = np.asarray(F)
    ny, nx = F.shape
    x0, x1 = x_range if x_range is not None else (0, nx)
    y0, y1 = y_range if y_range is not None else (0, ny)
    dx, dy = float(d[0]), float(d[1])
    sub = F[y0:y1, x0:x1].astype(np.complex128)
    wx = hann(x1 - x0) if window in ("x", "xy") else np.ones(x1 - x0)
    wy = hann(y1 - y0) if window == "xy" else np.ones(y1 - y0)
    sub = sub * wy[:, None] * wx[None, :]
    xs = np.arange(x0, x1, dtype=np.float64) * dx
    ys = np.arange(y0, y1, dtype=np.float64) * dy
    out = np.empty(len(kvecs), dtype=np.complex128)
    for j, (kx, ky) in enumerate(np.asarray(kvecs, dtype=np.float64)):
        phase = np.exp(-1j * (ky * ys[:, None] + kx * xs[None, :]))
        out[j] = np.sum(sub * phase) * dx * dy
    return out
