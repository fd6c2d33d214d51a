"""Closed-form solutions used as pins (independent of the oracle's update code)."""
import math

import numpy as np


def plane_waves_at(waves, shape, d, t, c=1.0):
    """Exact vacuum evolution of on-grid plane waves (omega = c|k|) at time t.

    Each wave E = e0 cos(k.x - c|k| t + phase), B = kappa x E / c, on the nodes
    of a 2D grid ``shape = (ny, nx)``.
    """
    ny, nx = shape
    x = np.arange(nx) * d[0]
    y = np.arange(ny) * d[1]
    X, Y = np.meshgrid(x, y)
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    for w in waves:
        kx = 2.0 * math.pi * w["m"][0] / (nx * d[0])
        ky = 2.0 * math.pi * w["m"][1] / (ny * d[1])
        kn = math.hypot(kx, ky)
        kap = np.array([kx / kn, ky / kn, 0.0])
        e0 = w["a_te"] * np.array([-kap[1], kap[0], 0.0]) + w["a_tm"] * np.array([0.0, 0.0, 1.0])
        b0 = np.cross(kap, e0) / c
        ph = np.cos(kx * X + ky * Y - c * kn * t + w["phase"])
        E += e0[:, None, None] * ph
        B += b0[:, None, None] * ph
    return E, B


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
