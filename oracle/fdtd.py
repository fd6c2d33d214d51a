"""FP64 Yee and Cole-Karkkainen FDTD steps -- TEST INFRASTRUCTURE ONLY.

Paper: Sec. III.A and Table 1 (rows "Yee" and "CKC").  Yee: staggered
second-order differences in space and time, 2D Courant limit c dt/dx <= 1/sqrt(2).
CKC: the Faraday-law differences are widened transversally with a coefficient
beta; the paper uses dx = dz and beta = 1/4, which gives Courant limit 1 and
no dispersion along the grid axes.  Table 1 writes the CKC weight as
A_X = (1-beta) + (beta/2) cos(k_Y dY); the reading taken here is the stencil
with weight (1-beta) on the centre row and beta/2 on each neighbour row, whose
symbol is (1-beta) + beta cos(k_Y dY) (with beta = 1/4 it reproduces the
Appendix A dispersion relation with beta' = -4 beta = -1).

Staggering (index [k][j][i] of each component sits at):
  Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
  Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
J is co-located with E.  A 2D grid ``[ny, nx]`` is uniform along z.

One step advances co-temporal (E, B) from t to t + dt as
  B -= (dt/2) curl E;   E += dt (c^2 curl B - J/eps0);   B -= (dt/2) curl E
(the leapfrog split symmetrically; it has the leapfrog dispersion relation
sin^2(w dt/2)/(c dt)^2 = sum_i A_i sin^2(k_i d_i/2)/d_i^2, A_i = 1 for Yee).
"""
from __future__ import annotations

import numpy as np

__all__ = ["fdtd_step", "curl_E", "curl_B", "CKC_BETA"]

CKC_BETA = 0.25


def _dp(f, axis, h):
    """Forward difference (f[i+1] - f[i]) / h along ``axis`` (periodic)."""
    return (np.roll(f, -1, axis=axis) - f) / h


def _dm(f, axis, h):
    """Backward difference (f[i] - f[i-1]) / h along ``axis`` (periodic)."""
    return (f - np.roll(f, 1, axis=axis)) / h


def _smooth(f, axis, beta):
    """Transverse CKC weighting: (1-beta) f[j] + beta/2 (f[j-1] + f[j+1])."""
    return (1.0 - beta) * f + 0.5 * beta * (np.roll(f, 1, axis=axis) + np.roll(f, -1, axis=axis))


def curl_E(E, d, scheme="yee", beta=CKC_BETA):
    """Faraday curl of E at the B positions (forward differences)."""
    ndim = E.ndim - 1
    ax = {"x": -1, "y": -2, "z": -3}
    Ex, Ey, Ez = E
    zero = np.zeros_like(Ex)
    dxEy, dxEz = _dp(Ey, ax["x"], d[0]), _dp(Ez, ax["x"], d[0])
    dyEx, dyEz = _dp(Ex, ax["y"], d[1]), _dp(Ez, ax["y"], d[1])
    if ndim == 3:
        dzEx, dzEy = _dp(Ex, ax["z"], d[2]), _dp(Ey, ax["z"], d[2])
    else:
        dzEx = dzEy = zero
    if scheme == "ckc":
        if ndim != 2:
            raise ValueError("the CKC scheme is provided in 2D only")
        # each x-difference is averaged over y-neighbours and vice versa
        dxEy, dxEz = _smooth(dxEy, ax["y"], beta), _smooth(dxEz, ax["y"], beta)
        dyEx, dyEz = _smooth(dyEx, ax["x"], beta), _smooth(dyEz, ax["x"], beta)
    elif scheme != "yee":
        raise ValueError("unknown scheme %r" % scheme)
    return np.stack([dyEz - dzEy, dzEx - dxEz, dxEy - dyEx])


def curl_B(B, d):
    """Ampere curl of B at the E positions (backward differences)."""
    ndim = B.ndim - 1
    Bx, By, Bz = B
    zero = np.zeros_like(Bx)
    dxBy, dxBz = _dm(By, -1, d[0]), _dm(Bz, -1, d[0])
    dyBx, dyBz = _dm(Bx, -2, d[1]), _dm(Bz, -2, d[1])
    if ndim == 3:
        dzBx, dzBy = _dm(Bx, -3, d[2]), _dm(By, -3, d[2])
    else:
        dzBx = dzBy = zero
    return np.stack([dyBz - dzBy, dzBx - dxBz, dxBy - dyBx])


def fdtd_step(E, B, J=None, *, d, dt, c=1.0, eps0=1.0, scheme="yee", nsteps=1):
    """``nsteps`` FDTD steps of co-temporal (E, B) (arrays ``(3, *grid)``).

    J (at t + dt/2, co-located with E) is held constant over the steps.
    Works on real or complex arrays (complex input is used to probe the
    per-mode amplification matrix in tests).
    """
    E = np.array(E, copy=True)
    B = np.array(B, copy=True)
    for _ in range(nsteps):
        B = B - 0.5 * dt * curl_E(E, d, scheme)
        E = E + dt * (c * c * curl_B(B, d))
        if J is not None:
            E = E - (dt / eps0) * np.asarray(J)
        B = B - 0.5 * dt * curl_E(E, d, scheme)
    return E, B
