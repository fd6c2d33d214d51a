"""Vacuum refractive index of each Maxwell solver, the Snell-Descartes toy model
and the Appendix A closed forms -- TEST INFRASTRUCTURE ONLY.

Table 1 of the paper gives, in 2D (x, z), the refractive index n = c / v_phi
and the Courant limit of each solver.  Readings taken where the printed
formulas are garbled:

* Yee / CKC / FDTD-p rows print c dt/2 inside the arcsin; the dispersion
  relation sin^2(w dt/2)/(c dt)^2 = sum_X A_X S_X^2/dX^2 (S_X = sin(k_X dX/2))
  gives n = (|k| c dt/2) / arcsin(c dt sqrt(sum_X A_X S_X^2/dX^2)), which tends
  to 1 as k -> 0 and equals the p = 2 case of the FDTD-p row.
* CKC weight: A_X = (1-beta) + beta cos(k_Y dY) (stencil weights 1-beta and
  beta/2, beta/2), beta = 1/4.
* p-order modified wavenumber (Sec. III.B; Table 1 caption): on the staggered
  grid k_{p,X} = (2/dX) sum_{l=1}^{p/2} C_l^p sin((2l-1) k_X dX/2), C_l^p the
  staggered Fornberg weights (sum_l (2l-1) C_l^p = 1).
* PSTD(-p): leapfrog in time, sin(w dt/2) = (c dt/2)|k_p|.
* PSATD(-p): w = c |k_p|, so n = |k|/|k_p| (1 for infinite order).

Snell model (Sec. IV.A, Eq. "Snell"): a harmonic of frequency w leaves the
plasma-vacuum interface from a non-dispersive medium (n_i = 1) at angle
theta_i into the numerical vacuum of index n_r[w, theta_r]; the refraction
angle solves n_i sin(theta_i) = n_r[w, theta_r] sin(theta_r), found by
Newton-Raphson.  The interface normal is taken along a grid axis, so theta_r
is also the propagation angle arctan(k_z/k_x) of Fig. 2.

Appendix A: eta (here c dt/dx; the appendix's "dx/(c dt)" is read as a typo,
the only reading consistent with its equations), beta' = -4 beta, the
angle-tuned coefficients and the Nyquist stability bound.

Parity unpinned: the PSTD cut-off harmonic at theta_i = 80 deg (Sec. IV.B).
The paper's PIC runs show it near harmonic 17; this model, at order 128 and a
time step the paper does not fix, only brackets it (the test checks a range,
not a value).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

__all__ = [
    "fornberg_staggered", "omega_numeric", "refractive_index", "k_of_omega",
    "snell_theta_r", "limit_angle", "courant_limit", "appendix_a_eta",
    "appendix_a_beta_prime", "appendix_a_eta_stable",
]


def fornberg_staggered(p: int, exact: bool = False):
    """Staggered-grid first-derivative weights C_l^p, l = 1..p/2.

    Returned as floats, or as exact ``Fraction``s with ``exact=True``.

    f'(0) ~ (1/h) sum_l C_l [f((l-1/2)h) - f(-(l-1/2)h)].  Closed form
    C_l = (-1)^(l+1) 16^(1-p/2) ((p-1)!)^2 /
          ((2l-1)^2 (p/2+l-1)! (p/2-l)! ((p/2-1)!)^2).
    """
    if p < 2 or p % 2:
        raise ValueError("p must be even and >= 2")
    h = p // 2
    f = math.factorial
    out = []
    for l in range(1, h + 1):
        num = (-1) ** (l + 1) * f(p - 1) ** 2
        den = (2 * l - 1) ** 2 * f(h + l - 1) * f(h - l) * f(h - 1) ** 2
        out.append(Fraction(num, den) * Fraction(16) ** (1 - h))
    if exact:
        return out
    return np.array([float(v) for v in out])


def _kp_axis(k, dX, p):
    """Modified wavenumber of the order-p staggered stencil along one axis."""
    if p is None:
        return np.asarray(k, dtype=np.float64)
    C = fornberg_staggered(p)
    l = np.arange(1, len(C) + 1)
    k = np.asarray(k, dtype=np.float64)
    return (2.0 / dX) * np.sum(C * np.sin(np.multiply.outer(k, (2 * l - 1)) * dX / 2.0), axis=-1)


def omega_numeric(kx, kz, solver, *, dt, dx, dz=None, c=1.0, p=None, beta=0.25):
    """Numerical angular frequency of a vacuum wave of wavevector (kx, kz) in 2D."""
    dz = dx if dz is None else dz
    kx = np.asarray(kx, dtype=np.float64)
    kz = np.asarray(kz, dtype=np.float64)
    if solver in ("yee", "ckc"):
        Sx = np.sin(kx * dx / 2.0)
        Sz = np.sin(kz * dz / 2.0)
        if solver == "yee":
            Ax = Az = 1.0
        else:
            Ax = (1.0 - beta) + beta * np.cos(kz * dz)
            Az = (1.0 - beta) + beta * np.cos(kx * dx)
        arg = c * dt * np.sqrt(Ax * Sx ** 2 / dx ** 2 + Az * Sz ** 2 / dz ** 2)
        return (2.0 / dt) * np.arcsin(arg)
    kpx = _kp_axis(kx, dx, p)
    kpz = _kp_axis(kz, dz, p)
    kp = np.sqrt(kpx ** 2 + kpz ** 2)
    if solver == "pstd":
        return (2.0 / dt) * np.arcsin(c * dt * kp / 2.0)
    if solver == "psatd":
        return c * kp
    raise ValueError("unknown solver %r" % solver)


def refractive_index(kdx, theta, solver, *, eta, c=1.0, p=None, beta=0.25):
    """n_r = c|k|/w as a function of |k| dx and theta = arctan(kz/kx), dx = dz = 1."""
    k = np.asarray(kdx, dtype=np.float64)
    kx, kz = k * np.cos(theta), k * np.sin(theta)
    w = omega_numeric(kx, kz, solver, dt=eta / c, dx=1.0, c=c, p=p, beta=beta)
    return c * k / w


def k_of_omega(omega, theta, solver, *, dt, dx, c=1.0, p=None, beta=0.25):
    """|k| of the numerical vacuum wave of frequency ``omega`` travelling at ``theta``.

    Solves omega_numeric(|k| cos theta, |k| sin theta) = omega by bisection on
    (0, k_max] where k_max is the first Nyquist crossing along the direction.
    """
    ct, st = abs(math.cos(theta)), abs(math.sin(theta))
    kmax = math.pi / dx / max(ct, st, 1e-300)

    def f(k):
        return float(omega_numeric(k * ct, k * st, solver, dt=dt, dx=dx, c=c, p=p, beta=beta)) - omega

    lo, hi = 0.0, kmax
    if f(hi) < 0:
        raise ValueError("frequency above the numerical band along this direction")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _n_of(omega, theta, solver, **kw):
    k = k_of_omega(omega, theta, solver, **kw)
    return kw.get("c", 1.0) * k / omega


def snell_theta_r(omega, theta_i, solver, *, dt, dx, c=1.0, p=None, beta=0.25,
                  tol=1e-13, maxit=60):
    """Refraction angle theta_r solving sin(theta_i) = n_r[omega, theta_r] sin(theta_r).

    Newton-Raphson on g(t) = n_r(omega, t) sin t - sin theta_i, started from
    theta_i, with a central-difference derivative.  Returns NaN when there is
    no solution (total reflection, sin theta_i > max n_r sin theta_r).
    """
    kw = dict(dt=dt, dx=dx, c=c, p=p, beta=beta)

    def g(t):
        return _n_of(omega, t, solver, **kw) * math.sin(t) - math.sin(theta_i)

    t = theta_i
    for _ in range(maxit):
        h = 1e-7
        try:
            gt = g(t)
            dg = (g(min(t + h, math.pi / 2)) - g(t - h)) / (min(t + h, math.pi / 2) - (t - h))
        except ValueError:
            return float("nan")
        if dg == 0:
            return float("nan")
        step = gt / dg
        t_new = min(max(t - step, 1e-9), math.pi / 2)
        if abs(t_new - t) < tol:
            t = t_new
            break
        t = t_new
    if abs(g(t)) > 1e-9:
        return float("nan")
    return t


def limit_angle(n_r):
    """Total-reflection limit angle theta_l = arcsin(n_r) (n_i = 1), in radians."""
    return math.asin(n_r)


def courant_limit(solver, ndim=2, p=None):
    """Courant limit on eta = c dt/dx (dx = dz) from Table 1 (inf for PSATD)."""
    if solver == "yee":
        return 1.0 / math.sqrt(ndim)
    if solver == "ckc":
        return 1.0
    if solver == "pstd":
        if p is None:
            return math.sqrt(2.0) / math.pi if ndim == 2 else 2.0 / (math.pi * math.sqrt(ndim))
        return 1.0 / (math.sqrt(ndim) * float(np.sum(np.abs(fornberg_staggered(p)))))
    if solver == "psatd":
        return math.inf
    raise ValueError(solver)


def appendix_a_eta(theta):
    """eta(theta) = (1/2) sqrt(5 - sqrt(1 + 32 cos^2 sin^2)) (Appendix A)."""
    cs2 = (math.cos(theta) * math.sin(theta)) ** 2
    return 0.5 * math.sqrt(5.0 - math.sqrt(1.0 + 32.0 * cs2))


def appendix_a_beta_prime(theta):
    """beta'(theta) = (1 - eta^2 - 2 cos^2 sin^2) / (3 cos^2 sin^2) (Appendix A)."""
    cs2 = (math.cos(theta) * math.sin(theta)) ** 2
    eta = appendix_a_eta(theta)
    return (1.0 - eta ** 2 - 2.0 * cs2) / (3.0 * cs2)


def appendix_a_eta_stable(beta_prime):
    """Nyquist stability bound eta_stable = 1/sqrt(2 + beta') (Appendix A)."""
    return 1.0 / math.sqrt(2.0 + beta_prime)
