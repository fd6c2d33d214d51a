"""Seeded synthetic inputs shaped like the paper's plasma-mirror workloads.

This module only *generates inputs* (numpy, FP64, seeded with PCG64); it holds
none of the PSATD or FDTD update arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.  Every generator is deterministic in its seed.

Workloads (the paper's simulations, Fig. 1 and Sec. II.B, need a PIC code and
a plasma; these prescribed fields and sources stand in for them):

* ``plane_waves``   -- a sum of on-grid vacuum plane waves (integer mode
                       numbers, unit-normal amplitudes, random phases,
                       transverse polarisation so div E = div B = 0).
* ``current_sheet`` -- the oscillating plasma-mirror surface as a prescribed
                       current sheet J_y(x, t) = J0 exp(-(x - x0(t))^2 / w^2),
                       x0(t) = a sin(w0 t)/w0 around the box centre.
* ``gaussian_charges`` -- moving Gaussian macro-charges whose rho^n, rho^(n+1)
                       and J^(n+1/2) satisfy discrete continuity exactly.
* ``random_fields`` -- white-noise component arrays for parity tests.
* ``batch_patch_sizes`` -- the batched workload's 512 patch domains (interior
                       plus guards, rounded up to a transform length).
* ``large_3d_inputs_torch`` -- the large 3D workload (512 x 512 x 1024): k^-2
                       divergence-free fields plus 1e5 Gaussian charges.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng", "plane_waves", "plane_wave_fields", "current_sheet", "random_fields",
    "gaussian_charges", "coulomb_field", "batch_patch_sizes", "large_3d_inputs_torch",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def plane_waves(shape, nwaves=8, seed=1608, polarisations="both"):
    """Draw ``nwaves`` on-grid plane waves for a 2D grid ``shape = (ny, nx)``.

    Each wave: integer mode numbers (mx, my) with 1 <= |m| < n/2 on at least
    one axis and |m_i| < n_i/2 on every axis, a random phase, and amplitudes
    a1 (in-plane, TE: Ex, Ey, Bz) and a2 (out-of-plane, TM: Ez, Bx, By) drawn
    from N(0, 1).  ``polarisations`` is "both", "te" or "tm".
    Returns a list of dicts with keys m, phase, a_te, a_tm.
    """
    ny, nx = shape
    g = rng(seed)
    waves = []
    while len(waves) < nwaves:
        mx = int(g.integers(-(nx // 2) + 1, nx // 2))
        my = int(g.integers(-(ny // 2) + 1, ny // 2))
        if mx == 0 and my == 0:
            continue
        phase = float(g.uniform(0.0, 2.0 * math.pi))
        a_te, a_tm = (float(v) for v in g.standard_normal(2))
        if polarisations == "te":
            a_tm = 0.0
        elif polarisations == "tm":
            a_te = 0.0
        waves.append(dict(m=(mx, my), phase=phase, a_te=a_te, a_tm=a_tm))
    return waves


def plane_wave_fields(waves, shape, d, c=1.0):
    """Real fields E, B (arrays ``(3, ny, nx)``) of ``waves`` at t = 0, on the nodes.

    Wave: E = (a_te e_te + a_tm z) cos(k.x + phase), B = kappa x E / c,
    e_te = z x kappa (in-plane, transverse), kappa = k/|k|.
    """
    ny, nx = shape
    x = np.arange(nx) * d[0]
    y = np.arange(ny) * d[1]
    X, Y = np.meshgrid(x, y)
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    for w in waves:
        kx = 2.0 * math.pi * w["m"][0] / (nx * d[0])
        ky = 2.0 * math.pi * w["m"][1] / (ny * d[1])
        kn = math.hypot(kx, ky)
        kap = np.array([kx / kn, ky / kn, 0.0])
        e_te = np.array([-kap[1], kap[0], 0.0])
        e0 = w["a_te"] * e_te + w["a_tm"] * np.array([0.0, 0.0, 1.0])
        b0 = np.cross(kap, e0) / c
        ph = np.cos(kx * X + ky * Y + w["phase"])
        E += e0[:, None, None] * ph
        B += b0[:, None, None] * ph
    return E, B


def current_sheet(shape, d, t, *, lam, a, w, J0=1.0, c=1.0):
    """J = (0, J_y, 0) of the oscillating current sheet at time ``t`` (2D, ``(ny, nx)``).

    J_y(x) = J0 exp(-(x - x0(t))^2 / w^2), x0(t) = xc + a sin(w0 t)/w0,
    w0 = 2 pi c / lam, xc the box centre; the distance is taken to the nearest
    periodic image.  Uniform in y, so div J = 0 (rho = 0).
    """
    ny, nx = shape
    Lx = nx * d[0]
    w0 = 2.0 * math.pi * c / lam
    x0 = 0.5 * Lx + a * math.sin(w0 * t) / w0
    x = np.arange(nx) * d[0]
    dx = (x - x0 + 0.5 * Lx) % Lx - 0.5 * Lx
    prof = J0 * np.exp(-(dx / w) ** 2)
    J = np.zeros((3, ny, nx))
    J[1] = prof[None, :]
    return J


def random_fields(shape, ncomp, seed, scale=1.0):
    """``ncomp`` white-noise arrays of ``shape`` drawn from N(0, scale^2)."""
    return scale * rng(seed).standard_normal((ncomp,) + tuple(shape))


def _kaxes(shape, d, keep_nyquist=False):
    """Signed discrete wavenumbers per axis (Nyquist entry 0 unless ``keep_nyquist``),
    rfft half along x."""
    ks = []
    for ax, n in enumerate(shape):
        h = d[len(shape) - 1 - ax]
        if ax == len(shape) - 1:
            m = np.arange(n // 2 + 1, dtype=np.float64)
        else:
            m = np.fft.fftfreq(n) * n
        k = 2.0 * math.pi * m / (n * h)
        if n % 2 == 0 and not keep_nyquist:
            k[np.abs(m) == n // 2] = 0.0
        sh = [1] * len(shape)
        sh[ax] = k.size
        ks.append(k.reshape(sh))
    return ks[::-1]  # (kx, ky[, kz])


def gaussian_charges(shape, d, dt, *, n_charges=64, sigma=None, vmax=0.5, c=1.0,
                     seed=1610, step=0):
    """rho^n, rho^(n+1) and J^(n+1/2) of moving Gaussian macro-charges.

    Charges q = +1, -1 alternating (net zero), uniform positions, velocities
    uniform in the ball |v| < vmax c, Gaussian width ``sigma`` (default 3 dx).
    Built in Fourier space on the discrete wavenumbers (Nyquist entry 0):
      rho^(k, t)  = (N/V) sum_j q_j exp(-sigma^2 k^2/2) exp(-i k.x_j(t)),
      J^(k)       = (N/V) sum_j q_j v_j exp(-sigma^2 k^2/2) exp(-i k.x_j(t_n))
                    * (exp(-i k.v_j dt) - 1)/(-i k.v_j dt),
    the exact time average of the current over [t_n, t_n+1], so that
    rho^(n+1) - rho^n = -i dt k.J^ holds to rounding on the discrete k.
    Returns (rho_n, rho_np1, J) as real arrays (J has shape ``(3, *shape)``).
    """
    ndim = len(shape)
    g = rng(seed)
    Ls = [shape[ndim - 1 - i] * d[i] for i in range(ndim)]  # (Lx, Ly[, Lz])
    pos = np.stack([g.uniform(0.0, L, n_charges) for L in Ls], axis=1)
    dirs = g.standard_normal((n_charges, ndim))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    speed = vmax * c * g.uniform(0.0, 1.0, n_charges) ** (1.0 / ndim)
    vel = dirs * speed[:, None]
    q = np.where(np.arange(n_charges) % 2 == 0, 1.0, -1.0)
    sigma = 3.0 * d[0] if sigma is None else sigma
    ks = _kaxes(shape, d)
    k2 = sum(k * k for k in ks)
    N = float(np.prod(shape))
    V = float(np.prod(Ls))
    G = (N / V) * np.exp(-0.5 * sigma * sigma * k2)
    tn = step * dt
    rho0 = np.zeros(k2.shape, dtype=np.complex128)
    rho1 = np.zeros_like(rho0)
    Jh = [np.zeros_like(rho0) for _ in range(3)]
    for j in range(n_charges):
        xn = pos[j] + vel[j] * tn
        phase = np.exp(-1j * sum(ks[a] * xn[a] for a in range(ndim)))
        kv = sum(ks[a] * vel[j][a] for a in range(ndim)) * dt
        e = np.exp(-1j * kv)
        small = np.abs(kv) < 1e-12
        kv_safe = np.where(small, 1.0, kv)
        avg = np.where(small, 1.0 - 0.5j * kv, (e - 1.0) / (-1j * kv_safe))
        rho0 += q[j] * G * phase
        rho1 += q[j] * G * phase * e
        for a in range(ndim):
            Jh[a] += q[j] * vel[j][a] * G * phase * avg
    axes = tuple(range(ndim))
    r0 = np.fft.irfftn(rho0, s=shape, axes=axes)
    r1 = np.fft.irfftn(rho1, s=shape, axes=axes)
    J = np.zeros((3,) + tuple(shape))
    for a in range(ndim):
        J[a] = np.fft.irfftn(Jh[a], s=shape, axes=axes)
    return r0, r1, J


def coulomb_field(rho, d, eps0=1.0):
    """Longitudinal E with i k.E^ = rho^/eps0 (Nyquist entries 0), as ``(3, *shape)``."""
    shape = rho.shape
    ndim = len(shape)
    ks = _kaxes(shape, d)
    k2 = sum(k * k for k in ks)
    R = np.fft.rfftn(rho, axes=tuple(range(ndim)))
    k2s = np.where(k2 > 0, k2, 1.0)
    E = np.zeros((3,) + tuple(shape))
    for a in range(ndim):
        Eh = np.where(k2 > 0, -1j * ks[a] * R / (eps0 * k2s), 0.0)
        E[a] = np.fft.irfftn(Eh, s=shape, axes=tuple(range(ndim)))
    return E


def gaussian_charges_torch(shape, d, dt, *, n_charges=64, sigma=None, vmax=0.5, c=1.0, seed=1610,
                           step=0, device="cuda", double=False):
    """GPU twin of :func:`gaussian_charges` (same seeded draws and formulas, evaluated with
    torch on ``device``; for large grids).  Returns float32 (``double``: float64) CUDA
    tensors (rho_n, rho_np1, J) with J of shape ``(3, *shape)``, and the Coulomb field E
    of rho_n."""
    import torch

    ndim = len(shape)
    g = rng(seed)
    Ls = [shape[ndim - 1 - i] * d[i] for i in range(ndim)]
    pos = np.stack([g.uniform(0.0, L, n_charges) for L in Ls], axis=1)
    dirs = g.standard_normal((n_charges, ndim))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    speed = vmax * c * g.uniform(0.0, 1.0, n_charges) ** (1.0 / ndim)
    vel = dirs * speed[:, None]
    q = np.where(np.arange(n_charges) % 2 == 0, 1.0, -1.0)
    sigma = 3.0 * d[0] if sigma is None else sigma
    ks = [torch.from_numpy(np.ascontiguousarray(k)).to(device) for k in _kaxes(shape, d)]
    k2 = sum(k * k for k in ks)
    N = float(np.prod(shape))
    V = float(np.prod(Ls))
    G = (N / V) * torch.exp(-0.5 * sigma * sigma * k2)
    tn = step * dt
    rho0 = torch.zeros(k2.shape, dtype=torch.complex128, device=device)
    rho1 = torch.zeros_like(rho0)
    Jh = [torch.zeros_like(rho0) for _ in range(3)]
    for j in range(n_charges):
        xn = pos[j] + vel[j] * tn
        phase = torch.exp(-1j * sum(ks[a] * float(xn[a]) for a in range(ndim)))
        kv = sum(ks[a] * float(vel[j][a]) for a in range(ndim)) * dt
        e = torch.exp(-1j * kv)
        small = kv.abs() < 1e-12
        kv_safe = torch.where(small, torch.ones_like(kv), kv)
        avg = torch.where(small, 1.0 - 0.5j * kv, (e - 1.0) / (-1j * kv_safe))
        base = q[j] * G * phase
        rho0 += base
        rho1 += base * e
        for a in range(ndim):
            Jh[a] += float(vel[j][a]) * base * avg
    dims = tuple(range(ndim))
    r0 = torch.fft.irfftn(rho0, s=shape, dim=dims)
    r1 = torch.fft.irfftn(rho1, s=shape, dim=dims)
    J = torch.zeros((3,) + tuple(shape), dtype=torch.float64, device=device)
    for a in range(ndim):
        J[a] = torch.fft.irfftn(Jh[a], s=shape, dim=dims)
    k2s = torch.where(k2 > 0, k2, torch.ones_like(k2))
    E = torch.zeros_like(J)
    for a in range(ndim):
        Eh = torch.where(k2 > 0, -1j * ks[a] * rho0 / k2s, torch.zeros_like(rho0))
        E[a] = torch.fft.irfftn(Eh, s=shape, dim=dims)
    if double:
        return r0, r1, J, E
    return r0.float(), r1.float(), J.float(), E.float()


def batch_patch_domains(npatch=512, seed=1612):
    """Patch domains of the batched local-FFT workload (Sec. II.A.3): per patch an
    interior n ~ U{64..512} and a guard width g ~ U{8..16}, drawn independently per
    axis (x first).  Returns [((nx_int, gx), (ny_int, gy)), ...]."""
    g = rng(seed)
    out = []
    for _ in range(npatch):
        n = g.integers(64, 513, size=2)
        gg = g.integers(8, 17, size=2)
        out.append(((int(n[0]), int(gg[0])), (int(n[1]), int(gg[1]))))
    return out


def transform_lengths(mixed_ok=True, five=False):
    """Transform lengths of the batch's patch sides: powers of two, and with
    ``mixed_ok`` also 3 * 2^k from 96 up, with ``five`` also 5 * 2^k from 160 up
    (lengths the FP32 passes take on both axes: x lines of n/2 points, y lines
    of n).  The workload uses 2^k and 3 * 2^k: adding 5 * 2^k cuts the 512-patch
    batch's transformed cells by 10 % but measured 7 % slower per step (74
    smaller size classes instead of 46)."""
    return sorted([1 << k for k in range(4, 13)] + ([3 << k for k in range(5, 11)] if mixed_ok else []) +
                  ([5 << k for k in range(5, 9)] if mixed_ok and five else []))


def batch_patch_sizes(npatch=512, seed=1612, mixed_ok=True, lengths=None, five=False):
    """Periodic patch sides of the batched workload: each side is the smallest
    transform length >= n + 2g (``lengths``, default transform_lengths(mixed_ok)),
    i.e. the guard region is widened to the next length the FFT takes.  Returns
    ([(nx, ny), ...], interior cells)."""
    cand = sorted(lengths) if lengths is not None else transform_lengths(mixed_ok, five)

    def side(v):
        return min(x for x in cand if x >= v)

    sizes, interior = [], 0
    for (nx, gx), (ny, gy) in batch_patch_domains(npatch, seed):
        sizes.append((side(nx + 2 * gx), side(ny + 2 * gy)))
        interior += nx * ny
    return sizes, interior


def batch_requested_cells(npatch=512, seed=1612):
    """Cells of the requested patch domains (n + 2g per side), summed over patches."""
    return sum((nx + 2 * gx) * (ny + 2 * gy) for (nx, gx), (ny, gy) in batch_patch_domains(npatch, seed))


def batch_source(sizes, seed=1613, scale=0.01):
    """Seeded source of the batched workload: per patch i, (Jx, Jy) of shape
    (ny_i, nx_i) drawn N(0, scale^2) in float32 from rng(seed + i), packed per
    component patch after patch.  Returns (Jx, Jy) float32 arrays; any patch can
    be regenerated alone with batch_patch_source."""
    parts = [batch_patch_source(i, nx, ny, seed, scale) for i, (nx, ny) in enumerate(sizes)]
    return (np.concatenate([p[0].ravel() for p in parts]), np.concatenate([p[1].ravel() for p in parts]))


def batch_patch_source(i, nx, ny, seed=1613, scale=0.01):
    g = rng(seed + i)
    J = g.standard_normal((2, ny, nx), dtype=np.float32)
    J *= np.float32(scale)
    return J[0], J[1]


def large_3d_inputs_torch(shape, d, dt, *, n_charges=100000, sigma=None, vmax=0.5, c=1.0, eps0=1.0,
                          seed=1614, device="cuda"):
    """Inputs of the large 3D workload (``shape`` = (nz, ny, nx), e.g. 1024 x 512 x 512),
    built with torch on ``device`` in FP64 and returned as float32 tensors
    (E, B, J each ``(3, *shape)``, rho_n, rho_np1).

    * Sources: ``n_charges`` Gaussian macro-charges (sigma = 3 dx, q = +1/-1
      alternating, velocities uniform in the ball |v| < vmax c) centred on grid
      nodes, so that the sum over charges is the transform of a node deposit:
      rho^n(k) = G(k) FFT(sum_j q_j (N/V) delta_j), J(k) likewise with q_j v_j,
      G = exp(-sigma^2 |k|^2 / 2) on the true wavenumbers (Nyquist pi/d, where G
      is below 1e-19 at sigma = 3 dx); rho^(n+1) = rho^n - i dt k.J imposes
      discrete continuity exactly.
    * Fields: E = the Coulomb field of rho^n plus a divergence-free random field,
      B a divergence-free random field, the random parts with per-mode power
      |F(k)|^2 ~ |k|^-2 (complex Gaussian modes from the transform of real white
      noise, divided by |k|, projected transverse, scaled to unit rms).
    Wavenumbers: the discrete ones with the Nyquist entries 0."""
    import torch

    nz, ny, nx = shape
    g = rng(seed)
    ix = [torch.from_numpy(g.integers(0, n, n_charges)).to(device) for n in (nx, ny, nz)]
    dirs = g.standard_normal((n_charges, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    speed = vmax * c * g.uniform(0.0, 1.0, n_charges) ** (1.0 / 3.0)
    vel = torch.from_numpy(dirs * speed[:, None]).to(device)
    q = torch.from_numpy(np.where(np.arange(n_charges) % 2 == 0, 1.0, -1.0)).to(device)
    sigma = 3.0 * d[0] if sigma is None else sigma
    kx, ky, kz = (torch.from_numpy(np.ascontiguousarray(k)).to(device) for k in _kaxes(shape, d))
    k2 = kx * kx + ky * ky + kz * kz
    N = float(nx * ny * nz)
    V = N * d[0] * d[1] * d[2]
    G = torch.exp(-0.5 * sigma * sigma * sum(
        k * k for k in (torch.from_numpy(np.ascontiguousarray(v)).to(device)
                        for v in _kaxes(shape, d, keep_nyquist=True))))
    flat = (ix[2] * ny + ix[1]) * nx + ix[0]
    dims = (0, 1, 2)

    def deposited(w):
        a = torch.zeros(nz * ny * nx, dtype=torch.float64, device=device)
        a.index_add_(0, flat, w * (N / V))
        return torch.fft.rfftn(a.view(shape), dim=dims) * G

    R0 = deposited(q)
    kJ = torch.zeros_like(R0)
    J = torch.empty((3,) + tuple(shape), dtype=torch.float32, device=device)
    for a, ka in enumerate((kx, ky, kz)):
        Jh = deposited(q * vel[:, a])
        kJ += ka * Jh
        J[a] = torch.fft.irfftn(Jh, s=shape, dim=dims).float()
        del Jh
    r0 = torch.fft.irfftn(R0, s=shape, dim=dims).float()
    r1 = torch.fft.irfftn(R0 - 1j * dt * kJ, s=shape, dim=dims).float()
    del kJ
    nzk = k2 > 0
    k2s = torch.where(nzk, k2, torch.ones_like(k2))
    gen = torch.Generator(device=device).manual_seed(seed + 1)

    def transverse_random():
        W = [torch.fft.rfftn(torch.randn(shape, dtype=torch.float64, device=device, generator=gen), dim=dims)
             for _ in range(3)]
        kw = (kx * W[0] + ky * W[1] + kz * W[2]) / k2s
        out = []
        for a, ka in enumerate((kx, ky, kz)):
            F = torch.where(nzk, (W[a] - ka * kw) / torch.sqrt(k2s), torch.zeros_like(W[a]))
            out.append(torch.fft.irfftn(F, s=shape, dim=dims))
        rms = math.sqrt(sum(float(torch.mean(f * f)) for f in out) / 3.0)
        return [f / rms for f in out]

    E = torch.empty((3,) + tuple(shape), dtype=torch.float32, device=device)
    ET = transverse_random()
    for a, ka in enumerate((kx, ky, kz)):
        EL = torch.where(nzk, -1j * ka * R0 / (eps0 * k2s), torch.zeros_like(R0))
        E[a] = (ET[a] + torch.fft.irfftn(EL, s=shape, dim=dims)).float()
    del ET
    B = torch.empty_like(E)
    BT = transverse_random()
    for a in range(3):
        B[a] = BT[a].float()
    return E, B, J, r0, r1
