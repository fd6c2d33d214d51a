"""The seeded input recipes hold what their documentation states (CPU):

* the batched workload's patch sides are transform lengths at least n + 2g,
  drawn reproducibly (same seed, same list);
* the large 3D workload's generator (run here with torch on the CPU at a small
  size) gives discrete continuity rho^(n+1) - rho^n = -i dt k.J exactly in
  k-space, Gauss's law for E on rho^n, divergence-free B, unit-rms random parts;
* the pass model of the bench's byte accounting is 104 B per cell for the 2D TE
  J-form step (the figure the roofline uses).
"""
import math

import numpy as np
import pytest

from paper_1608_05739_gb300 import synth


def test_batch_patch_sizes_are_transform_lengths_covering_the_patch():
    sizes, interior = synth.batch_patch_sizes(512, 1612, mixed_ok=True)
    again, interior2 = synth.batch_patch_sizes(512, 1612, mixed_ok=True)
    assert sizes == again and interior == interior2 and len(sizes) == 512
    ok = {1 << k for k in range(4, 13)} | {3 << k for k in range(5, 11)}
    g = synth.rng(1612)
    for nx, ny in sizes:
        n = g.integers(64, 513, size=2)
        gg = g.integers(8, 17, size=2)
        need = [int(n[0]) + 2 * int(gg[0]), int(n[1]) + 2 * int(gg[1])]
        assert nx in ok and ny in ok
        assert nx >= need[0] and ny >= need[1]
        assert min(v for v in ok if v >= need[0]) == nx and min(v for v in ok if v >= need[1]) == ny
    pow2, _ = synth.batch_patch_sizes(512, 1612, mixed_ok=False)
    assert all(a & (a - 1) == 0 and b & (b - 1) == 0 for a, b in pow2)
    assert sum(a * b for a, b in sizes) < sum(a * b for a, b in pow2)
    five, _ = synth.batch_patch_sizes(512, 1612, mixed_ok=True, five=True)
    assert any(a % 5 == 0 or b % 5 == 0 for a, b in five)
    assert sum(a * b for a, b in five) < sum(a * b for a, b in sizes)


def test_large_3d_inputs_continuity_gauss_and_divergence():
    torch = pytest.importorskip("torch")
    shape, d, dt = (16, 12, 20), (1.0, 0.9, 1.1), 0.4
    E, B, J, r0, r1 = synth.large_3d_inputs_torch(shape, d, dt, n_charges=300, seed=7, device="cpu")
    kx, ky, kz = (torch.from_numpy(np.ascontiguousarray(k)) for k in synth._kaxes(shape, d))
    F = lambda f: torch.fft.rfftn(f.double(), dim=(0, 1, 2))
    R0, R1 = F(r0), F(r1)
    kJ = kx * F(J[0]) + ky * F(J[1]) + kz * F(J[2])
    scale = float(R0.abs().max())
    # continuity, imposed in k-space (float32 storage rounding only)
    assert float((R1 - R0 + 1j * dt * kJ).abs().max()) < 1e-5 * scale
    # Gauss's law i k.E = rho^n / eps0 (eps0 = 1)
    kE = kx * F(E[0]) + ky * F(E[1]) + kz * F(E[2])
    assert float((1j * kE - R0).abs().max()) < 1e-5 * max(scale, float(kE.abs().max()))
    # B divergence-free, unit rms
    kB = kx * F(B[0]) + ky * F(B[1]) + kz * F(B[2])
    assert float(kB.abs().max()) < 1e-5 * float(F(B[0]).abs().max())
    assert abs(float(torch.sqrt(torch.mean(B.double() ** 2))) - 1.0) < 1e-3
    # net charge zero (even number of alternating charges)
    assert abs(float(R0[0, 0, 0].real)) < 1e-6 * scale


def test_pass_model_bytes_per_cell():
    import bench
    alg = bench.algorithmic_bytes(2048, 2048, 1, 5, 3)
    per_cell = sum(v for k, v in alg.items()) / (2048 * 2048)
    assert abs(per_cell - 104.08) < 0.01
    assert abs(alg["line_fft_push"] - 167968800) < 1
