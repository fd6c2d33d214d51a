"""FP64 local-FFT PSATD step on a decomposed 2D grid -- TEST INFRASTRUCTURE ONLY
(see the ``oracle`` package doc).

What the paper fixes (Sec. II.A.3): the global grid is split into subdomains;
each subdomain keeps guard regions holding copies of its neighbours' cells,
Maxwell's equations are advanced in the spectral domain with local FFTs over
the subdomain plus its guards, and the guards are refreshed from the
neighbours every step.  The local transform makes the extended subdomain
periodic on its own, which is the (small) truncation error the paper mentions
(it depends on the stencil order, the guard width and the resolution).

One step here, for a periodic global grid of nx x ny cells split into px x py
patches of ix = nx/px by iy = ny/py interior cells with g guard cells on every
side:

  1. fill: every patch takes the global cells
     ((x0 - g + i) mod nx, (y0 - g + j) mod ny), 0 <= i < ix + 2g,
     0 <= j < iy + 2g, for every field and source component (the guard refresh);
  2. advance each extended patch by one PSATD step as a periodic domain of its
     own (``psatd.psatd_step``, any stencil order);
  3. keep the interior of every patch (the guards are discarded).

With one patch and g = 0 this is the global step.
"""
import numpy as np

from . import psatd


def extract(f, px, py, g, p, q):
    """Extended block of patch (p, q) of a 2D array ``f`` [ny, nx] (periodic wrap)."""
    ny, nx = f.shape
    ix, iy = nx // px, ny // py
    xs = (p * ix - g + np.arange(ix + 2 * g)) % nx
    ys = (q * iy - g + np.arange(iy + 2 * g)) % ny
    return f[np.ix_(ys, xs)]


def local_step(E, B, J=None, rho0=None, rho1=None, *, d, dt, px, py, guard, c=1.0, eps0=1.0,
               form="none", nsteps=1, order=0):
    """``nsteps`` local-FFT PSATD steps of the 2D fields E, B (arrays ``(3, ny, nx)``)
    on px x py patches with ``guard`` cells; sources held constant over the steps."""
    E = np.array(E, dtype=np.float64)
    B = np.array(B, dtype=np.float64)
    _, ny, nx = E.shape
    if nx % px or ny % py:
        raise ValueError("patches must divide the grid")
    ix, iy = nx // px, ny // py
    g = guard
    for _ in range(nsteps):
        En = np.empty_like(E)
        Bn = np.empty_like(B)
        for q in range(py):
            for p in range(px):
                ext = lambda f: extract(f, px, py, g, p, q)
                Ep = np.stack([ext(E[i]) for i in range(3)])
                Bp = np.stack([ext(B[i]) for i in range(3)])
                Jp = np.stack([ext(J[i]) for i in range(3)]) if J is not None else None
                r0 = ext(rho0) if rho0 is not None else None
                r1 = ext(rho1) if rho1 is not None else None
                Eo, Bo = psatd.psatd_step(Ep, Bp, Jp, r0, r1, d=d, dt=dt, c=c, eps0=eps0, form=form,
                                          order=order)
                En[:, q * iy:(q + 1) * iy, p * ix:(p + 1) * ix] = Eo[:, g:g + iy, g:g + ix]
                Bn[:, q * iy:(q + 1) * iy, p * ix:(p + 1) * ix] = Bo[:, g:g + iy, g:g + ix]
        E, B = En, Bn
    return E, B
