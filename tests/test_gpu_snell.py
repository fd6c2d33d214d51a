"""The harmonic deviation of Sec. IV measured on the GPU solvers.

A current sheet J_y(x0, y, t) = ramp(t) sum_n cos(n w0 t - n k0 sin(theta_i) y)
radiates harmonics n w0 with the phase along the sheet of a surface driven at
incidence theta_i (the plasma-mirror geometry of Sec. IV.A, synthetic).  Each
harmonic leaves the sheet with the parallel wavenumber k_par = n k0 sin(theta_i)
it was given; its normal wavenumber k_perp is what the scheme's numerical
dispersion makes of the frequency n w0, so its direction
theta_r = atan(k_par / k_perp) obeys the refraction (Snell-Descartes) model
sin(theta_i) = n_r(w, theta_r) sin(theta_r) of the oracle's dispersion module.
k_perp is measured from the field: E_y is recorded along x at y = 0 over a
window of whole fundamental periods after the turn-on transient has passed and
before the periodic images arrive, each harmonic's complex amplitude is taken
by a lock-in at its frequency, and k_perp is the slope of its phase along x.

PSATD shows no deviation; Yee and CKC deviate as the model says (lambda0 = 64
cells, c dt = 0.5 dx, theta_i = asin(13/16) = 54.3 deg, harmonics 1..8)."""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib
from oracle import dispersion as dsp
from paper_1608_05739_gb300 import capi

pytestmark = pytest.mark.gpu

NX, NY = 4096, 1024
LAM = 64
M_PAR = 13                       # k0 sin(theta_i) = 2 pi 13 / 1024: sin(theta_i) = 13/16
X0 = 512                         # sheet column
XR = (X0 + 64, X0 + 576)         # recorded segment of the row y = 0
DT = 0.5
HARM = (1, 2, 3, 4, 5, 6, 8)
RAMP = 320.0                     # turn-on time (5 periods)
T_START, N_WIN = 3000, 2560      # window: steps [T_START, T_START + N_WIN) = 20 fundamental periods


def _run(solver):
    import torch
    ensure_lib()
    dev = torch.device("cuda")
    w0 = 2 * math.pi / LAM
    kpar = 2 * math.pi * M_PAR / NY
    y = torch.arange(NY, device=dev, dtype=torch.float64)
    ysh = y + (0.5 if solver != "psatd" else 0.0)     # FDTD: J_y and E_y at y + 1/2
    Ex, Ey, Bz, Jx, Jy = (torch.zeros(NY, NX, device=dev) for _ in range(5))
    rec = torch.empty(N_WIN, XR[1] - XR[0], device=dev)
    plan = None
    if solver == "psatd":
        plan = capi.Plan((NX, NY), (1.0, 1.0), DT, layout="te", prec="fp32", src="J")
    for s in range(T_START + N_WIN):
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
        if s >= T_START:
            rec[s - T_START] = Ey[0, XR[0]:XR[1]]
    torch.cuda.synchronize()
    if plan is not None:
        plan.sync()
        plan.destroy()
    E = rec.double().cpu().numpy()                      # [time, x]
    tt = (T_START + 1 + np.arange(N_WIN)) * DT          # time of the fields after each step
    x = np.arange(XR[0], XR[1], dtype=np.float64)
    out = {}
    for n in HARM:
        a = (E * np.exp(1j * n * w0 * tt)[:, None]).sum(axis=0)   # ~ A exp(i k_perp x)
        ph = np.unwrap(np.angle(a))
        kperp = np.polyfit(x, ph, 1)[0]
        out[n] = math.atan2(n * kpar, kperp)
    return out


@pytest.mark.parametrize("solver", ["psatd", "yee", "ckc"])
def test_harmonic_deviation_follows_the_refraction_model(solver):
    ti = math.asin(M_PAR * LAM / NY)
    w0 = 2 * math.pi / LAM
    got = _run(solver)
    rows = []
    for n in HARM:
        model = dsp.snell_theta_r(n * w0, ti, solver, dt=DT, dx=1.0)
        rows.append((n, 1e3 * (got[n] - ti), 1e3 * (model - ti)))
        assert abs(got[n] - model) < 0.05 * abs(model - ti) + 2e-4, (solver, n, got[n] - ti, model - ti)
    print("%s deviation theta_r - theta_i [mrad], harmonic: measured / model: %s" % (
        solver, "; ".join("%d: %+.2f / %+.2f" % r for r in rows)))
