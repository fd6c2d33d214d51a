"""Checkpoint and resume: the state of a PSATD run is the caller's field arrays
(the sources are recomputed from their seed and step index), so N steps equal k
steps, a save of the fields to a file, a new plan and N - k more steps, bit for
bit (the kernels are deterministic: no data-path atomics)."""
import math

import numpy as np
import pytest

from gpu_helpers import ensure_lib
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _sheet(nx, ny, dx, dt, n):
    """J_y of the current-sheet workload at t = (n + 1/2) dt (seeded, uniform in y)."""
    J = synth.current_sheet((ny, nx), (dx, dx), (n + 0.5) * dt, lam=64 * dx, a=0.9, w=2 * dx)
    return J[1]


@pytest.mark.parametrize("prec", ["fp32", "fp64", "mixed_fp16"])
def test_save_and_resume_is_bitwise(prec, tmp_path):
    import torch
    ensure_lib()
    nx = ny = 256
    dx = 1.0 / 64
    dt = dx / math.sqrt(2.0)
    N, k = 12, 5
    dtype = torch.float64 if prec == "fp64" else torch.float32
    Js = [torch.from_numpy(_sheet(nx, ny, dx, dt, n)).to("cuda", dtype) for n in range(N)]
    zero = lambda: torch.zeros(ny, nx, device="cuda", dtype=dtype)

    def run(plan, E, n0, n1):
        Jx = zero()
        for n in range(n0, n1):
            plan.step([E[0], E[1], None], [None, None, E[2]], [Jx, Js[n], None])
        plan.sync()

    plan = capi.Plan((nx, ny), (dx, dx), dt, layout="te", prec=prec, src="J")
    A = [zero() for _ in range(3)]
    run(plan, A, 0, N)
    plan.destroy()

    plan = capi.Plan((nx, ny), (dx, dx), dt, layout="te", prec=prec, src="J")
    B = [zero() for _ in range(3)]
    run(plan, B, 0, k)
    plan.destroy()
    path = tmp_path / "fields.npz"
    np.savez(path, step=k, Ex=B[0].cpu().numpy(), Ey=B[1].cpu().numpy(), Bz=B[2].cpu().numpy())
    del B
    ck = np.load(path)
    C = [torch.from_numpy(ck[name]).to("cuda") for name in ("Ex", "Ey", "Bz")]
    plan = capi.Plan((nx, ny), (dx, dx), dt, layout="te", prec=prec, src="J")
    run(plan, C, int(ck["step"]), N)
    plan.destroy()
    for a, c in zip(A, C):
        assert torch.equal(a, c)
    assert float(A[1].abs().max()) > 0
