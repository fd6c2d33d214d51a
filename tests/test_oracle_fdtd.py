"""Pins of the FP64 Yee / CKC oracle.

The per-mode amplification matrix of one oracle step is extracted by stepping
single complex Fourier modes; its eigenvalues must be exp(+-i w dt) (and 1 for
the static modes) with w from the closed-form dispersion relations of Table 1
(written separately in ``oracle.dispersion``), |lambda| = 1 below the Courant
limits of Table 1 and |lambda| > 1 above them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import dispersion as disp
from oracle import fdtd

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _amplification(shape, d, dt, m, scheme, c=1.0):
    """6x6 per-mode matrix of one fdtd step for integer mode m on ``shape``."""
    ndim = len(shape)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    # grids[a] indexes numpy axis a: axis -1 is x
    phase = np.ones(shape, dtype=np.complex128)
    for ax in range(ndim):
        n = shape[ax]
        mi = m[ndim - 1 - ax]
        phase = phase * np.exp(2j * np.pi * mi * grids[ax] / n)
    M = np.zeros((6, 6), dtype=np.complex128)
    for col in range(6):
        F = np.zeros((6,) + tuple(shape), dtype=np.complex128)
        F[col] = phase
        E1, B1 = fdtd.fdtd_step(F[:3], F[3:], d=d, dt=dt, c=c, scheme=scheme)
        out = np.concatenate([E1, B1])
        for row in range(6):
            M[row, col] = np.vdot(phase, out[row]) / phase.size
    return M


def _closed_form_omega(m, shape, d, dt, scheme, c=1.0):
    ndim = len(shape)
    k = [2 * math.pi * m[i] / (shape[ndim - 1 - i] * d[i]) for i in range(ndim)]
    S = [math.sin(k[i] * d[i] / 2) for i in range(ndim)]
    if scheme == "yee":
        s2 = sum(S[i] ** 2 / d[i] ** 2 for i in range(ndim))
    else:
        b = 0.25
        Ax = (1 - b) + b * math.cos(k[1] * d[1])
        Ay = (1 - b) + b * math.cos(k[0] * d[0])
        s2 = Ax * S[0] ** 2 / d[0] ** 2 + Ay * S[1] ** 2 / d[1] ** 2
    return (2 / dt) * math.asin(c * dt * math.sqrt(s2))


CASES = [
    ("yee", (16, 16), (1.0, 1.0), 0.7, (3, 1)),
    ("yee", (16, 16), (1.0, 1.0), 0.5, (5, -7)),
    ("yee", (12, 20), (0.8, 1.1), 0.45, (-4, 2)),
    ("yee", (8, 8, 8), (1.0, 1.0, 1.0), 0.55, (1, 2, 3)),
    ("ckc", (16, 16), (1.0, 1.0), 1.0, (3, 5)),
    ("ckc", (16, 16), (1.0, 1.0), 0.9, (-6, 7)),
]


@pytest.mark.parametrize("scheme,shape,d,dt,m", CASES)
def test_eigenvalues_match_closed_form_dispersion(scheme, shape, d, dt, m):
    M = _amplification(shape, d, dt, m, scheme)
    lam = np.linalg.eigvals(M)
    np.testing.assert_allclose(np.abs(lam), 1.0, atol=1e-12)
    w = _closed_form_omega(m, shape, d, dt, scheme)
    phases = np.sort(np.abs(np.angle(lam)))
    # two wave pairs (+-w dt) and two static modes (phase 0)
    np.testing.assert_allclose(phases[:2], 0.0, atol=1e-7)
    np.testing.assert_allclose(phases[2:], w * dt, rtol=1e-12, atol=1e-13)


def test_dispersion_module_agrees_with_the_stencil():
    """The Table 1 index formula (oracle.dispersion) describes the same schemes."""
    for scheme, eta in (("yee", 0.7), ("ckc", 1.0)):
        shape, d, m = (16, 16), (1.0, 1.0), (3, 2)
        w_stencil = _closed_form_omega(m, shape, d, eta, scheme)
        kx, kz = 2 * math.pi * 3 / 16, 2 * math.pi * 2 / 16
        w_table = float(disp.omega_numeric(kx, kz, scheme, dt=eta, dx=1.0))
        assert abs(w_stencil - w_table) < 1e-13
        lam = np.linalg.eigvals(_amplification(shape, d, eta, m, scheme))
        assert abs(np.max(np.angle(lam)) - w_table * eta) < 1e-12


def test_ckc_is_dispersion_free_on_axis_at_courant_one():
    """Sec. III.A: CKC with dx = dz, beta = 1/4 allows c dt = dx and has no dispersion along x and z."""
    for m in [(1, 0), (5, 0), (0, 3), (7, 0)]:
        lam = np.linalg.eigvals(_amplification((16, 16), (1.0, 1.0), 1.0, m, "ckc"))
        k = 2 * math.pi * max(abs(m[0]), abs(m[1])) / 16
        assert abs(np.max(np.angle(lam)) - k * 1.0) < 1e-12


def _max_growth(scheme, eta, shape=(16, 16)):
    worst = 0.0
    for m in [(8, 8), (8, 0), (7, 7), (8, 4)]:
        lam = np.linalg.eigvals(_amplification(shape, (1.0, 1.0), eta, m, scheme))
        worst = max(worst, float(np.max(np.abs(lam))))
    return worst


def test_courant_limits_of_table1():
    lim = GOLD["courant_limits_2d"]
    assert _max_growth("yee", lim["yee"] * 0.999) < 1 + 1e-9
    assert _max_growth("yee", lim["yee"] * 1.01) > 1 + 1e-3
    assert _max_growth("ckc", lim["ckc"] * 0.999) < 1 + 1e-9
    assert _max_growth("ckc", lim["ckc"] * 1.01) > 1 + 1e-3
    assert abs(disp.courant_limit("yee") - lim["yee"]) < 1e-15
    assert abs(disp.courant_limit("pstd") - lim["pstd"]) < 1e-15


def test_uniform_current_drains_E():
    shape, d = (8, 8), (1.0, 1.0)
    E = np.zeros((3,) + shape)
    B = np.zeros((3,) + shape)
    J = np.ones((3,) + shape) * np.array([1.0, -2.0, 0.5])[:, None, None]
    E1, B1 = fdtd.fdtd_step(E, B, J, d=d, dt=0.3, eps0=0.6, scheme="yee")
    np.testing.assert_allclose(E1, -0.3 / 0.6 * J, atol=1e-15)
    np.testing.assert_allclose(B1, 0.0, atol=1e-15)
