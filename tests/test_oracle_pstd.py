"""Pins of the PSTD oracle (``oracle.psatd.pstd_step``; Table 1 row PSTD, the
pseudo-spectral solver of Sec. III.B that keeps the FDTD leapfrog in time).

Closed form: the per-mode amplification matrix of the leapfrog has the
eigenvalues exp(+-i w dt) with sin(w dt/2) = c dt |k|/2 (the dispersion relation
of Table 1's PSTD row, the Yee relation with exact derivatives) below the Courant
limit c dt |k| < 2, and grows above it.  The matrix is read off the oracle by
stepping single Fourier modes (brute force on a tiny grid)."""
import math

import numpy as np
import pytest

from oracle import psatd as orc


@pytest.mark.parametrize("m,cdt", [((3, 1), 0.4), ((5, -6), 0.5), ((1, 0), 1.3)])
def test_pstd_eigenvalues_follow_the_leapfrog_dispersion(m, cdt):
    shape, d = (16, 16), (1.0, 1.0)
    kx, ky = 2 * math.pi * m[0] / 16, 2 * math.pi * m[1] / 16
    kn = math.hypot(kx, ky)
    E = np.zeros((3, *shape))
    B = np.zeros((3, *shape))
    # single mode, complex amplitudes carried by cos/sin pairs: build the 3x3 matrix on
    # the complex amplitudes by stepping exp(i k.x) through its real and imaginary parts
    x = np.arange(16)[None, :]
    y = np.arange(16)[:, None]
    ph = kx * x + ky * y
    M = np.zeros((3, 3), dtype=complex)
    slots = [("E", 0), ("E", 1), ("B", 2)]
    for col, (fb, comp) in enumerate(slots):
        outs = []
        for part in (np.cos(ph), np.sin(ph)):
            E = np.zeros((3, *shape))
            B = np.zeros((3, *shape))
            (E if fb == "E" else B)[comp] = part
            outs.append(orc.pstd_step(E, B, d=d, dt=cdt))
        for row, (gb, rc) in enumerate(slots):
            fc = (outs[0][0] if gb == "E" else outs[0][1])[rc]
            fs = (outs[1][0] if gb == "E" else outs[1][1])[rc]
            # exp(i k.x) = cos + i sin, so its image is fc + i fs; project on exp(i k.x)
            img = fc + 1j * fs
            M[row, col] = np.sum(img * np.exp(-1j * ph)) / 256.0
    ev = np.linalg.eigvals(M)
    w = 2 * math.asin(cdt * kn / 2) / cdt
    want = sorted([1.0 + 0j, np.exp(1j * w * cdt), np.exp(-1j * w * cdt)], key=lambda z: np.angle(z))
    got = sorted(ev, key=lambda z: np.angle(z))
    assert np.allclose(got, want, atol=1e-12), (got, want)


def test_pstd_grows_above_its_courant_limit():
    """c dt |k| > 2 for the highest propagated mode (|m_i| = 7 on 16 cells; the Nyquist
    index is k = 0 on the nodes): unstable; just below the limit: stable."""
    shape, d = (16, 16), (1.0, 1.0)
    rng = np.random.default_rng(2)
    E = rng.standard_normal((3, *shape))
    B = rng.standard_normal((3, *shape))
    w0 = orc.field_energy(E, B, d)
    kmax = 2 * math.pi * 7 / 16 * math.sqrt(2.0)
    E1, B1 = orc.pstd_step(E, B, d=d, dt=2.2 / kmax, nsteps=50)    # c dt |k|max = 2.2
    assert orc.field_energy(E1, B1, d) > 1e3 * w0
    E1, B1 = orc.pstd_step(E, B, d=d, dt=1.95 / kmax, nsteps=50)   # 1.95 < 2: stable
    assert orc.field_energy(E1, B1, d) < 2 * w0


def test_pstd_agrees_with_psatd_as_dt_goes_to_zero():
    """Both integrate the same semi-discrete system; one step differs by O(dt^3)."""
    rng = np.random.default_rng(3)
    shape, d = (16, 24), (1.0, 1.0)
    E = rng.standard_normal((3, *shape))
    B = rng.standard_normal((3, *shape))
    J = rng.standard_normal((3, *shape))
    errs = []
    for dt in (0.1, 0.05, 0.025):
        Ep, Bp = orc.pstd_step(E, B, J, d=d, dt=dt)
        Ea, Ba = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
        errs.append(np.linalg.norm(np.concatenate([Ep - Ea, Bp - Ba])))
    assert 6.0 < errs[0] / errs[1] < 10.0 and 6.0 < errs[1] / errs[2] < 10.0, errs
