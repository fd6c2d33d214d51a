"""FP64 PSATD step -- TEST INFRASTRUCTURE ONLY (see the ``oracle`` package doc).

What the paper fixes (Sec. III.B, item 2; Table 1, row "PSATD"): Maxwell's
equations are solved in (k, t) space and integrated analytically in time; the
only assumption is that the sources are constant during one time step Delta t.
The scheme is dispersion-free (refractive index 1 for every k) and has no
Courant condition.  The paper does not print the update equations, so this
module writes out the exact solution of the per-mode linear system that the
statement defines.

Conventions
-----------
* Grids: 2D arrays are ``[ny, nx]``, 3D arrays ``[nz, ny, nx]``; x is the last
  (contiguous) axis.  A 2D grid is uniform along z (k_z = 0).
* Vector fields are arrays of shape ``(3, *grid)`` holding (x, y, z) components.
* Fourier transform: f^(k) = sum_x f(x) exp(-i k.x) (unnormalised forward,
  inverse with 1/N), so grad -> i k.  numpy's ``rfftn`` / ``irfftn`` are used
  as the transform step (a library primitive; the half spectrum along x).
* Wavenumbers k_i = 2 pi m_i / (n_i d_i) with m_i the signed FFT index.  The
  paper is silent on the Nyquist index of an even-length axis; here k_i := 0 at
  m_i = n_i/2 in every coefficient and vector operation (keeps real fields
  real and the update Hermitian-consistent).

Per-mode update (sources constant over the step)
------------------------------------------------
For each k, Maxwell's equations in SI form with explicit c and eps0,

    dE^/dt = i c^2 k x B^ - J^/eps0 ,      dB^/dt = -i k x E^ ,

are integrated exactly over Delta t.  With kappa = k/|k|, x = c|k|dt,
C = cos x, S = sin x, splitting E^ into its part along kappa (which only sees
-J/eps0) and its transverse part (a harmonic oscillator of frequency c|k|):

  J-form
    E' = C E + (1-C) kappa(kappa.E) + i c S kappa x B - S/(eps0 c k) J
         + (S/(c k) - dt)/eps0 * kappa(kappa.J)
    B' = C B + (1-C) kappa(kappa.B) - i S/(c k) k x E
         + i (1-C)/(eps0 c^2 k^2) k x J

  (the kappa(kappa.B) term keeps the longitudinal part of B constant, as the
  equations do; it vanishes for physical, divergence-free B)

  rho-form (continuity rho1 - rho0 = -i dt k.J replaces kappa.J, Gauss's law
  i k.E = rho0/eps0 replaces kappa.E; it enforces Gauss's law at t + dt)
    E' = C E + i c S kappa x B - S/(eps0 c k) J
         + i k/(eps0 k^2) [ (S/x - 1) rho1 - (S/x - C) rho0 ]
    B' = as in the J-form

  k = 0: E' = E - dt J/eps0, B' = B (the limits of the above, with kappa := 0).

The factors that cancel near k = 0 are evaluated in stable forms:
  S/(c k) = dt sinc(x);  (1-C)/(c k)^2 = (dt^2/2) sinc(x/2)^2;
  S/(c k) - dt = dt x^2 f1(x);  (S/x - 1)/k^2 = (c dt)^2 f1(x);
  (S/x - C)/k^2 = (c dt)^2 f2(x);
with f1(x) = (sin x/x - 1)/x^2 and f2(x) = (sin x/x - cos x)/x^2 summed from
their Taylor series below x = 0.5.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "wavenumbers", "spectral_grid", "forward", "inverse", "sinc", "f1", "f2",
    "push_modes", "psatd_step", "field_energy",
]


def wavenumbers(n: int, d: float, half: bool = False) -> np.ndarray:
    """Signed wavenumbers of an axis of ``n`` cells of size ``d`` in FFT order.

    ``half=True`` gives the first n//2+1 entries (the R2C half axis).  The
    Nyquist entry of an even axis is set to 0 (reading of the paper's silence).
    """
    if half:
        m = np.arange(n // 2 + 1, dtype=np.float64)
    else:
        m = np.fft.fftfreq(n) * n
    k = 2.0 * math.pi * m / (n * d)
    if n % 2 == 0:
        k[np.abs(m) == n // 2] = 0.0
    return k


def spectral_grid(shape, d):
    """(kx, ky, kz) broadcastable to the ``rfftn`` spectrum of a grid ``shape``.

    ``shape`` is ``(ny, nx)`` or ``(nz, ny, nx)``; ``d`` is ``(dx, dy[, dz])``.
    """
    if len(shape) == 2:
        ny, nx = shape
        kx = wavenumbers(nx, d[0], half=True)[None, :]
        ky = wavenumbers(ny, d[1])[:, None]
        kz = np.zeros((1, 1))
        return kx, ky, kz
    nz, ny, nx = shape
    kx = wavenumbers(nx, d[0], half=True)[None, None, :]
    ky = wavenumbers(ny, d[1])[None, :, None]
    kz = wavenumbers(nz, d[2])[:, None, None]
    return kx, ky, kz


def _raw_grid(shape, d):
    """As :func:`spectral_grid` but with the Nyquist wavenumbers kept (+pi/d on the
    half x axis, -pi/d at index n/2 of a full axis, numpy's ``fftfreq`` order)."""
    def ax(n, dd, half):
        m = np.arange(n // 2 + 1, dtype=np.float64) if half else np.fft.fftfreq(n) * n
        return 2.0 * math.pi * m / (n * dd)
    if len(shape) == 2:
        ny, nx = shape
        return ax(nx, d[0], True)[None, :], ax(ny, d[1], False)[:, None], np.zeros((1, 1))
    nz, ny, nx = shape
    return (ax(nx, d[0], True)[None, None, :], ax(ny, d[1], False)[None, :, None],
            ax(nz, d[2], False)[:, None, None])


def forward(f: np.ndarray) -> np.ndarray:
    """Unnormalised forward DFT of a real grid array (half spectrum along x)."""
    return np.fft.rfftn(f, axes=tuple(range(f.ndim)))


def inverse(F: np.ndarray, shape) -> np.ndarray:
    """Inverse of :func:`forward` (includes the 1/N factor)."""
    return np.fft.irfftn(F, s=tuple(shape), axes=tuple(range(len(shape))))


def sinc(x):
    """sin(x)/x with sinc(0) = 1."""
    return np.sinc(np.asarray(x, dtype=np.float64) / math.pi)


def _series(x, coeffs):
    x2 = np.asarray(x, dtype=np.float64) ** 2
    acc = np.zeros_like(x2)
    for c in reversed(coeffs):
        acc = acc * x2 + c
    return acc


# Taylor coefficients (in x^2) of f1 = (sin x/x - 1)/x^2 = sum_{n>=1} (-1)^n x^(2n-2)/(2n+1)!
_F1 = [(-1) ** n / math.factorial(2 * n + 1) for n in range(1, 12)]
# and of f2 = (sin x/x - cos x)/x^2 = sum_{n>=1} (-1)^(n+1) 2n x^(2n-2)/(2n+1)!
_F2 = [(-1) ** (n + 1) * 2 * n / math.factorial(2 * n + 1) for n in range(1, 12)]
_SERIES_BELOW = 0.5


def f1(x):
    """(sin x / x - 1) / x^2, stable for all x >= 0 (limit -1/6)."""
    x = np.asarray(x, dtype=np.float64)
    small = x < _SERIES_BELOW
    xs = np.where(small, 1.0, x)
    direct = (np.sin(xs) / xs - 1.0) / xs ** 2
    return np.where(small, _series(x, _F1), direct)


def f2(x):
    """(sin x / x - cos x) / x^2, stable for all x >= 0 (limit 1/3)."""
    x = np.asarray(x, dtype=np.float64)
    small = x < _SERIES_BELOW
    xs = np.where(small, 1.0, x)
    direct = (np.sin(xs) / xs - np.cos(xs)) / xs ** 2
    return np.where(small, _series(x, _F2), direct)


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1],
            a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def push_modes(k, E, B, J=None, rho0=None, rho1=None, *, dt, c=1.0, eps0=1.0,
               form="none"):
    """Advance spectral fields by dt, mode by mode (the analytic PSATD push).

    ``k`` = (kx, ky, kz) arrays broadcastable against the spectral arrays;
    ``E``, ``B``, ``J`` = sequences of three complex spectral arrays.
    ``form`` is ``"none"`` (J = rho = 0), ``"J"`` or ``"rho"``.
    Returns the new (E, B) as lists of three complex arrays.
    """
    kx, ky, kz = (np.asarray(v, dtype=np.float64) for v in k)
    kn = np.sqrt(kx * kx + ky * ky + kz * kz)
    nz = kn > 0
    kn_safe = np.where(nz, kn, 1.0)
    kap = tuple(np.where(nz, v / kn_safe, 0.0) for v in (kx, ky, kz))
    kvec = (kx, ky, kz)
    x = c * kn * dt
    C = np.cos(x)
    S = np.sin(x)
    S_ck = dt * sinc(x)                            # S/(c k)      -> dt
    omC_c2k2 = 0.5 * dt * dt * sinc(0.5 * x) ** 2  # (1-C)/(c k)^2 -> dt^2/2
    omC = 2.0 * np.sin(0.5 * x) ** 2               # 1 - C

    kE = _dot(kap, E)
    kB = _dot(kap, B)
    kxB = _cross(kap, B)
    KxE = _cross(kvec, E)
    En = [C * E[i] + 1j * c * S * kxB[i] for i in range(3)]
    Bn = [C * B[i] + omC * kap[i] * kB - 1j * S_ck * KxE[i] for i in range(3)]
    if form == "none":
        for i in range(3):
            En[i] = En[i] + omC * kap[i] * kE
        return En, Bn
    if J is None:
        raise ValueError("form %r needs J" % form)
    KxJ = _cross(kvec, J)
    for i in range(3):
        En[i] = En[i] - (S_ck / eps0) * J[i]
        Bn[i] = Bn[i] + 1j * (omC_c2k2 / eps0) * KxJ[i]
    if form == "J":
        kJ = _dot(kap, J)
        dlong = dt * x * x * f1(x)                 # S/(c k) - dt
        for i in range(3):
            En[i] = En[i] + omC * kap[i] * kE + (dlong / eps0) * kap[i] * kJ
        return En, Bn
    if form == "rho":
        if rho0 is None or rho1 is None:
            raise ValueError("form 'rho' needs rho0 and rho1")
        cdt2 = (c * dt) ** 2
        g = (cdt2 / eps0) * (f1(x) * rho1 - f2(x) * rho0)
        for i in range(3):
            En[i] = En[i] + 1j * kvec[i] * g
        return En, Bn
    raise ValueError("unknown source form %r" % form)


# Staggered (Yee) positions: the axes along which each component sits half a
# cell from the nodes.  Ex(i+1/2, j, k) Ey(i, j+1/2, k) Ez(i, j, k+1/2),
# Bx(i, j+1/2, k+1/2) By(i+1/2, j, k+1/2) Bz(i+1/2, j+1/2, k); J as E; rho on nodes.
STAGGER_E = ((0,), (1,), (2,))
STAGGER_B = ((1, 2), (0, 2), (0, 1))


def staggered_operators(shape, d, order):
    """(k_p, phases) of the order-``order`` staggered scheme on the rfftn spectrum.

    Sec. III.B / Table 1 row PSATD-p: the exact wavenumber of PSATD is replaced by
    that of the order-p centred staggered difference,
    k_p,i = (2/d_i) sum_l C_l^p sin((2l-1) k_i d_i / 2)  (Fornberg weights).
    A component stored at index j but located at x_j + d_i/2 along axis i has the
    true-position spectrum exp(-i k_i d_i / 2) times its array spectrum; in those
    spectra the order-p difference is multiplication by i k_p,i, so the push is the
    collocated one with k -> k_p.  Every product the push forms of a k_p,i with the
    phases of the two components it couples is the staggered difference's own
    symbol, 2 pi/d_i-periodic in k_i, so the Nyquist index needs no special
    reading here: it keeps k_i = +-pi/d_i (unlike the collocated scheme, whose
    i k_i is not periodic there and is set to 0).
    """
    from . import dispersion
    k = _raw_grid(shape, d)
    kp = tuple(dispersion._kp_axis(k[i], d[i], order) if i < len(shape) else np.zeros_like(k[i])
               for i in range(3))
    dd = tuple(d) + (1.0,) * (3 - len(d))
    ph = tuple(np.exp(-0.5j * k[i] * dd[i]) for i in range(3))
    return kp, ph


def _shift(F, axes, ph, sign):
    for a in axes:
        F = F * (ph[a] if sign > 0 else np.conj(ph[a]))
    return F


def psatd_step(E, B, J=None, rho0=None, rho1=None, *, d, dt, c=1.0, eps0=1.0,
               form="none", nsteps=1, order=0):
    """``nsteps`` PSATD steps of real fields E, B (arrays ``(3, *grid)``).

    Sources (J at t+dt/2; rho at t and t+dt) are held constant over the
    ``nsteps`` steps, each step being: forward DFT of every component, the
    per-mode push of :func:`push_modes`, inverse DFT.  Returns new (E, B).

    ``order`` = 0: all components on the nodes, exact wavenumbers.  ``order`` = p
    (even, >= 2): components at their staggered (Yee) positions and the order-p
    wavenumbers of :func:`staggered_operators`; each step shifts the spectra to
    true positions, pushes with k_p, and shifts back.
    """
    E = np.asarray(E, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    shape = E.shape[1:]
    if order:
        k, ph = staggered_operators(shape, d, order)
    else:
        k, ph = spectral_grid(shape, d), None
    sE = STAGGER_E if order else ((), (), ())
    sB = STAGGER_B if order else ((), (), ())
    Jh = [_shift(forward(np.asarray(J[i], dtype=np.float64)), sE[i], ph, +1) for i in range(3)] \
        if J is not None else None
    r0 = forward(np.asarray(rho0, dtype=np.float64)) if rho0 is not None else None
    r1 = forward(np.asarray(rho1, dtype=np.float64)) if rho1 is not None else None
    for _ in range(nsteps):
        Eh = [_shift(forward(E[i]), sE[i], ph, +1) for i in range(3)]
        Bh = [_shift(forward(B[i]), sB[i], ph, +1) for i in range(3)]
        Eh, Bh = push_modes(k, Eh, Bh, Jh, r0, r1, dt=dt, c=c, eps0=eps0, form=form)
        E = np.stack([inverse(_shift(Eh[i], sE[i], ph, -1), shape) for i in range(3)])
        B = np.stack([inverse(_shift(Bh[i], sB[i], ph, -1), shape) for i in range(3)])
    return E, B


def pstd_modes(k, E, B, J=None, *, dt, c=1.0, eps0=1.0):
    """One pseudo-spectral time-domain (PSTD, Table 1) step of spectral fields, mode by
    mode: the leapfrog of the FDTD schemes with spectral derivatives, for co-temporal
    E, B: B half step, E full step, B half step,
        B' = B - (dt/2) i k x E,  E'' = E + c^2 dt i k x B' - dt J/eps0,
        B'' = B' - (dt/2) i k x E''.
    Its vacuum dispersion relation is sin(w dt/2) = c dt |k| / 2."""
    kvec = tuple(np.asarray(v, dtype=np.float64) for v in k)
    h = 0.5 * dt
    kxE = _cross(kvec, E)
    Bh = [B[i] - h * 1j * kxE[i] for i in range(3)]
    kxB = _cross(kvec, Bh)
    En = [E[i] + c * c * dt * 1j * kxB[i] - (dt / eps0 * J[i] if J is not None else 0.0) for i in range(3)]
    kxE = _cross(kvec, En)
    Bn = [Bh[i] - h * 1j * kxE[i] for i in range(3)]
    return En, Bn


def pstd_step(E, B, J=None, *, d, dt, c=1.0, eps0=1.0, nsteps=1, order=0):
    """``nsteps`` PSTD steps (J held constant): forward DFT, :func:`pstd_modes`, inverse
    DFT; ``order`` as in :func:`psatd_step` (0 nodes and exact k, p staggered order p)."""
    E = np.asarray(E, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    shape = E.shape[1:]
    if order:
        k, ph = staggered_operators(shape, d, order)
    else:
        k, ph = spectral_grid(shape, d), None
    sE = STAGGER_E if order else ((), (), ())
    sB = STAGGER_B if order else ((), (), ())
    Jh = [_shift(forward(np.asarray(J[i], dtype=np.float64)), sE[i], ph, +1) for i in range(3)] \
        if J is not None else None
    for _ in range(nsteps):
        Eh = [_shift(forward(E[i]), sE[i], ph, +1) for i in range(3)]
        Bh = [_shift(forward(B[i]), sB[i], ph, +1) for i in range(3)]
        Eh, Bh = pstd_modes(k, Eh, Bh, Jh, dt=dt, c=c, eps0=eps0)
        E = np.stack([inverse(_shift(Eh[i], sE[i], ph, -1), shape) for i in range(3)])
        B = np.stack([inverse(_shift(Bh[i], sB[i], ph, -1), shape) for i in range(3)])
    return E, B


def field_energy(E, B, d, c=1.0, eps0=1.0):
    """Electromagnetic energy sum (eps0 |E|^2 + |B|^2/mu0)/2 dV, mu0 = 1/(eps0 c^2)."""
    dV = float(np.prod(d))
    mu0 = 1.0 / (eps0 * c * c)
    return 0.5 * dV * (eps0 * np.sum(np.asarray(E) ** 2) + np.sum(np.asarray(B) ** 2) / mu0)
