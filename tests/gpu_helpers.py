"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
numpy inputs and compare with the FP64 oracle on the same (rounded) inputs."""
import math

import numpy as np

from paper_1608_05739_gb300 import build as bld
from paper_1608_05739_gb300 import capi

_built = False


def ensure_lib():
    global _built
    if not _built:
        bld.build()
        capi.load()
        _built = True


def torch_dev(a, prec):
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device="cuda", dtype=dt)


def rounded(a, prec):
    """Inputs as the GPU sees them (FP32 paths read float32-rounded arrays)."""
    a = np.asarray(a, dtype=np.float64)
    return a.astype(np.float32).astype(np.float64) if prec != "fp64" else a


def grid_n(shape):
    return tuple(reversed(shape))  # (nx, ny[, nz]) from [.., ny, nx]


def psatd_gpu(shape, d, dt, E, B, J=None, r0=None, r1=None, *, layout, prec, src, nsteps=1, c=1.0,
              eps0=1.0, plan=None, calls=1, order=0):
    """Run ``calls`` x psatd_step(nsteps) on the GPU; returns numpy (E, B), absent components 0."""
    ensure_lib()
    pe, pb, pj = capi.PRESENT[layout]
    own = plan is None
    if own:
        plan = capi.Plan(grid_n(shape), d, dt, layout=layout, prec=prec, src=src, c=c, eps0=eps0, order=order)
    Et = [torch_dev(E[i], prec) if pe[i] else None for i in range(3)]
    Bt = [torch_dev(B[i], prec) if pb[i] else None for i in range(3)]
    Jt = [torch_dev(J[i], prec) if (J is not None and pj[i] and src != "none") else None for i in range(3)]
    r0t = torch_dev(r0, prec) if (src == "rho") else None
    r1t = torch_dev(r1, prec) if (src == "rho") else None
    for _ in range(calls):
        plan.step(Et, Bt, Jt if src != "none" else None, r0t, r1t, nsteps=nsteps)
    plan.sync()
    Eo = np.zeros((3,) + tuple(shape))
    Bo = np.zeros((3,) + tuple(shape))
    for i in range(3):
        if pe[i]:
            Eo[i] = Et[i].double().cpu().numpy()
        if pb[i]:
            Bo[i] = Bt[i].double().cpu().numpy()
    if own:
        plan.destroy()
    return Eo, Bo


def fdtd_gpu(shape, d, dt, E, B, J=None, *, layout, prec, scheme, nsteps=1, c=1.0, eps0=1.0):
    ensure_lib()
    pe, pb, pj = capi.PRESENT[layout]
    Et = [torch_dev(E[i], prec) if pe[i] else None for i in range(3)]
    Bt = [torch_dev(B[i], prec) if pb[i] else None for i in range(3)]
    Jt = [torch_dev(J[i], prec) if pj[i] else None for i in range(3)] if J is not None else None
    capi.fdtd_step(grid_n(shape), d, dt, Et, Bt, Jt, scheme=scheme, layout=layout, prec=prec, c=c,
                   eps0=eps0, nsteps=nsteps)
    import torch
    torch.cuda.synchronize()
    Eo = np.zeros((3,) + tuple(shape))
    Bo = np.zeros((3,) + tuple(shape))
    for i in range(3):
        if pe[i]:
            Eo[i] = Et[i].double().cpu().numpy()
        if pb[i]:
            Bo[i] = Bt[i].double().cpu().numpy()
    return Eo, Bo


def mask_layout(F, layout, which):
    """Zero the components of F (shape (3, ...)) absent from ``layout``."""
    pe, pb, pj = capi.PRESENT[layout]
    p = {"E": pe, "B": pb, "J": pj}[which]
    F = np.array(F, copy=True)
    for i in range(3):
        if not p[i]:
            F[i] = 0.0
    return F


# Largest element error allowed, in units of (tolerance x rms of the reference):
# an error spread like noise over N elements peaks at a few times its rms
# (about sqrt(2 ln N) < 6 for N < 1e8), while an error confined to one line of a
# 2048^2 grid peaks at sqrt(2048) = 45 times its rms and fails.
PEAK_K = 30.0


class ParityErr(float):
    """Relative L2 error of a parity comparison that also carries its peak: the
    largest |a - b| over the rms of the reference b.  `err < tol` (tol a plain
    number) holds when both rel-L2 < tol and peak <= PEAK_K * tol; between two
    errors, and for every other operator, it is the plain rel-L2 float."""

    def __new__(cls, rel, peak):
        obj = float.__new__(cls, rel)
        obj.peak = peak
        return obj

    def __lt__(self, other):
        if isinstance(other, ParityErr) or not isinstance(other, (int, float)):
            return float(self) < other
        return float(self) < other and self.peak <= PEAK_K * other

    def __le__(self, other):
        if isinstance(other, ParityErr) or not isinstance(other, (int, float)):
            return float(self) <= other
        return float(self) <= other and self.peak <= PEAK_K * other

    def __repr__(self):
        return "%r (peak %.3g x rms)" % (float(self), self.peak)


def rel_l2_fields(E1, B1, E2, B2, c=1.0):
    """Relative L2 over all E and c B components, with the per-element peak (ParityErr)."""
    a = np.concatenate([np.ravel(E1), c * np.ravel(B1)])
    b = np.concatenate([np.ravel(E2), c * np.ravel(B2)])
    nb = float(np.linalg.norm(b))
    rms = nb / math.sqrt(b.size)
    return ParityErr(float(np.linalg.norm(a - b)) / nb, float(np.max(np.abs(a - b))) / rms)
