"""Pins of the local-FFT oracle (``oracle/local.py``, Sec. II.A.3): a grid split
into patches with guard cells, each advanced with its own FFT.

* one patch without guards is the global step (the definition reduces to it);
* an extended patch exactly one global period wide sees the global field as
  periodic on its own, so every patch reproduces the global step to rounding;
* plane waves whose period divides the extended patch width are periodic on
  every patch, so the local step is exact for them (closed form: the global
  step is the analytic rotation at omega = c|k|);
* for a generic field the truncation error against the global step falls as
  the guard region widens (the paper's statement of the error's dependence).
"""
import math

import numpy as np
import pytest

from analytic import plane_waves_at
from oracle import local as loc
from oracle import psatd as orc
from paper_1608_05739_gb300 import synth


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _fields(shape, seed):
    E = synth.random_fields(shape, 3, seed)
    B = synth.random_fields(shape, 3, seed + 1)
    J = synth.random_fields(shape, 3, seed + 2)
    return E, B, J


def test_one_patch_without_guards_is_the_global_step():
    shape, d, dt = (32, 48), (1.0, 0.7), 0.4
    E, B, J = _fields(shape, 3)
    El, Bl = loc.local_step(E, B, J, d=d, dt=dt, px=1, py=1, guard=0, form="J")
    Eg, Bg = orc.psatd_step(E, B, J, d=d, dt=dt, form="J")
    assert np.array_equal(El, Eg) and np.array_equal(Bl, Bg)


def test_extended_patch_one_period_wide_is_exact():
    """nx = 64, 2 x 2 patches of 32 interior cells, 16 guard cells: each extended
    patch is 64 wide, one full period of the global grid."""
    shape, d, dt = (64, 64), (1.0, 1.0), 0.5
    E, B, J = _fields(shape, 11)
    El, Bl = loc.local_step(E, B, J, d=d, dt=dt, px=2, py=2, guard=16, form="J", nsteps=3)
    Eg, Bg = orc.psatd_step(E, B, J, d=d, dt=dt, form="J", nsteps=3)
    assert _rel(np.concatenate([El, Bl]), np.concatenate([Eg, Bg])) < 1e-13


def test_plane_waves_periodic_on_each_patch_are_exact():
    """64 x 64 grid, 4 x 2 patches (16 x 32 interior) with 8 guard cells: extended
    patches 32 x 48.  Waves with x period 32 or 16 and y period 16 are periodic on
    every extended patch; after 20 local steps they match the analytic rotation."""
    shape, d, dt = (64, 64), (1.0, 1.0), 0.5
    waves = [dict(m=(2, 4), phase=0.3, a_te=1.0, a_tm=-0.5), dict(m=(-4, 4), phase=1.1, a_te=0.7, a_tm=0.2),
             dict(m=(2, -8), phase=2.0, a_te=-0.4, a_tm=0.9)]
    E, B = synth.plane_wave_fields(waves, shape, d)
    El, Bl = loc.local_step(E, B, d=d, dt=dt, px=4, py=2, guard=8, nsteps=20)
    Ea, Ba = plane_waves_at(waves, shape, d, 20 * dt)
    assert _rel(np.concatenate([El, Bl]), np.concatenate([Ea, Ba])) < 1e-12


def test_truncation_error_falls_with_guard_width():
    """A smooth random field (power ~ k^-4) on 128^2 split into 4 x 4 patches:
    the error of one local step against the global step decreases as g grows."""
    shape, d, dt = (128, 128), (1.0, 1.0), 1.0 / math.sqrt(2.0)
    rng = np.random.default_rng(5)
    ky = 2 * np.pi * np.fft.fftfreq(shape[0])[:, None]
    kx = 2 * np.pi * np.fft.rfftfreq(shape[1])[None, :]
    filt = 1.0 / (1.0 + 40.0 * (kx ** 2 + ky ** 2)) ** 2
    E = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal(shape)) * filt, s=shape) for _ in range(3)])
    B = np.stack([np.fft.irfft2(np.fft.rfft2(rng.standard_normal(shape)) * filt, s=shape) for _ in range(3)])
    Eg, Bg = orc.psatd_step(E, B, d=d, dt=dt)
    errs = []
    for g in (2, 4, 8, 16):
        El, Bl = loc.local_step(E, B, d=d, dt=dt, px=4, py=4, guard=g)
        errs.append(_rel(np.concatenate([El, Bl]), np.concatenate([Eg, Bg])))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[0] < 0.1


def test_patches_must_divide_the_grid():
    E = np.zeros((3, 30, 32))
    with pytest.raises(ValueError):
        loc.local_step(E, E, d=(1.0, 1.0), dt=0.5, px=3, py=4, guard=2)
