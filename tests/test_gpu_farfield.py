"""The far-field diagnostic on the GPU (Sec. II.B / Sec. IV).

* Parity: psatd_farfield against the oracle's Fraunhofer sum on seeded fields
  (FP32 and FP64 snapshots, sub-windows, Hann apodisation along x and along
  both axes, wavevectors on and off the grid).
* The harmonic deviation from simulation: the tilted multi-harmonic current
  sheet of Sec. IV's geometry (J_y(x0, y, t) = ramp(t) sum_n cos(n w0 t - n k0
  sin(theta_i) y), lambda0 = 64 cells, c dt = 0.5 dx, theta_i = asin(13/16)) is
  run with PSATD, Yee and CKC; one snapshot of E_y on the reflected side (a
  window of 512 x 1024 cells, whole periods along y, Hann along x) goes through
  the far-field transform along the wavevectors that share harmonic n's
  parallel wavenumber n k0 sin(theta_i); the brightest one gives the harmonic's
  direction theta_r = atan(k_par / k_perp), which must follow the refraction
  (Snell-Descartes) model: none for PSATD, the Table 1 dispersion for Yee/CKC.
"""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib
from oracle import dispersion as dsp
from oracle import farfield as off
from paper_1608_05739_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,window,tol", [("fp64", "none", 1e-12), ("fp64", "xy", 1e-12), ("fp32", "x", 2e-6),
                                             ("fp32", "xy", 2e-6)])
def test_farfield_matches_oracle(prec, window, tol):
    import torch
    ensure_lib()
    ny, nx, d = 200, 300, (0.5, 0.25)
    g = np.random.default_rng(7)
    F = g.standard_normal((ny, nx))
    if prec == "fp32":
        F = F.astype(np.float32).astype(np.float64)
    k = np.concatenate([g.uniform(-6.0, 6.0, (40, 2)),
                        [(2 * math.pi * 3 / (nx * d[0]), 2 * math.pi * 5 / (ny * d[1])), (0.0, 0.0)]])
    xr, yr = (17, 281), (3, 190)
    want = off.fraunhofer(F, d, k, x_range=xr, y_range=yr, window=window)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ft = torch.from_numpy(F).to("cuda", dt)
    kt = torch.from_numpy(k).to("cuda")
    got = capi.farfield((nx, ny), d, Ft, kt, x_range=xr, y_range=yr, window=window).cpu().numpy()
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < tol, err


def test_farfield_argument_errors():
    import torch
    ensure_lib()
    F = torch.zeros(32, 64, device="cuda")
    k = torch.zeros(4, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.PsatdError):
        capi.farfield((64, 32), (1.0, 1.0), F, k, x_range=(10, 70))          # outside the grid
    with pytest.raises(capi.PsatdError):
        capi.farfield((64, 32), (1.0, 1.0), F, k, y_range=(5, 5))            # empty


NX, NY = 4096, 1024
LAM = 64
M_PAR = 13                       # k0 sin(theta_i) = 2 pi 13 / 1024: sin(theta_i) = 13/16
X0 = 512                         # sheet column
WIN = (X0 + 64, X0 + 576)        # snapshot window along x (all y)
DT = 0.5
HARM = (1, 2, 3, 4, 5, 6, 8)
RAMP = 320.0
# Along x a harmonic's energy moves at the group velocity c cos(theta_i) = 0.58 c (its parallel
# wavenumber is fixed), so the turn-on tail leaves the window's far edge at t = RAMP + 576 / 0.58
# = 1306; the snapshot is taken at t = 1700, long before the sheet's wave going the other way
# comes round the periodic x axis (3520 cells at 0.58 c).
STEPS = 3400


def _snapshot(solver):
    import torch
    ensure_lib()
    dev = torch.device("cuda")
    w0 = 2 * math.pi / LAM
    kpar = 2 * math.pi * M_PAR / NY
    y = torch.arange(NY, device=dev, dtype=torch.float64)
    ysh = y + (0.5 if solver != "psatd" else 0.0)     # FDTD: J_y and E_y at y + 1/2
    Ex, Ey, Bz, Jx, Jy = (torch.zeros(NY, NX, device=dev) for _ in range(5))
    plan = capi.Plan((NX, NY), (1.0, 1.0), DT, layout="te", prec="fp32", src="J") if solver == "psatd" else None
    for s in range(STEPS):
        t = (s + 0.5) * DT
        r = min(1.0, t / RAMP)
        ramp = r * r * (3 - 2 * r)
        col = torch.zeros(NY, device=dev, dtype=torch.float64)
        for n in HARM:
            col += torch.cos(n * w0 * t - n * kpar * ysh)
        Jy[:, X0] = (ramp * col).float()
        if plan is not None:
            plan.step([Ex, Ey, None], [None, None, Bz], [Jx, Jy, None])
        else:
            capi.fdtd_step((NX, NY), (1.0, 1.0), DT, [Ex, Ey, None], [None, None, Bz], [Jx, Jy, None],
                           scheme=solver, layout="te", prec="fp32")
    torch.cuda.synchronize()
    if plan is not None:
        plan.sync()
        plan.destroy()
    return Ey


def _direction(Ey, n):
    """theta_r of harmonic n: the far-field amplitude along the wavevectors
    (kx, n k_par) for kx within +-12 % of the vacuum k_perp, its peak refined by a
    parabola through the three brightest samples (log power)."""
    import torch
    k0 = 2 * math.pi / LAM
    kp = n * 2 * math.pi * M_PAR / NY
    kperp0 = math.sqrt((n * k0) ** 2 - kp ** 2)
    kx = np.linspace(0.88 * kperp0, 1.12 * kperp0, 481)
    k = torch.from_numpy(np.stack([kx, np.full_like(kx, kp)], axis=1)).cuda()
    P = capi.farfield((NX, NY), (1.0, 1.0), Ey, k, x_range=WIN, window="x").abs().cpu().numpy() ** 2
    i = int(np.argmax(P))
    assert 0 < i < len(kx) - 1, "peak at the edge of the searched band"
    a, b, c = np.log(P[i - 1:i + 2])
    peak = kx[i] + 0.5 * (a - c) / (a - 2 * b + c) * (kx[1] - kx[0])
    return math.atan2(kp, peak)


@pytest.mark.parametrize("solver", ["psatd", "yee", "ckc"])
def test_far_field_harmonic_directions_follow_the_refraction_model(solver):
    ti = math.asin(M_PAR * LAM / NY)
    w0 = 2 * math.pi / LAM
    Ey = _snapshot(solver)
    rows = []
    for n in HARM:
        got = _direction(Ey, n)
        model = dsp.snell_theta_r(n * w0, ti, solver, dt=DT, dx=1.0)
        rows.append((n, 1e3 * (got - ti), 1e3 * (model - ti)))
        assert abs(got - model) < 0.05 * abs(model - ti) + 2e-4, (solver, n, got - ti, model - ti)
    print("%s far-field deviation theta_r - theta_i [mrad], harmonic: measured / model: %s" % (
        solver, "; ".join("%d: %+.2f / %+.2f" % r for r in rows)))
