"""PSATD_FLAG_CHECKED: every step's output arrays are scanned for NaN / Inf and
a hit is reported by the next sync as PSATD_ERR_NONFINITE (host-made failure:
a NaN placed in an input; nothing faults on the GPU).  A checked plan computes
the same bits as an unchecked one, the word is cleared by the sync that reports
it, and the plan stays usable."""
import numpy as np
import pytest
import torch

from gpu_helpers import ensure_lib
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu

NONFINITE = 6


def _te(shape, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return [torch.randn(shape, device="cuda", generator=g) for _ in range(5)]


def test_checked_plan_same_bits_and_reports_nan():
    ensure_lib()
    n, shape = (256, 128), (128, 256)
    a = _te(shape, 1)
    b = [t.clone() for t in a]
    p0 = capi.Plan(n, (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
    p1 = capi.Plan(n, (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J", checked=True)
    p0.step([a[0], a[1], None], [None, None, a[2]], [a[3], a[4], None], nsteps=3)
    p1.step([b[0], b[1], None], [None, None, b[2]], [b[3], b[4], None], nsteps=3)
    p0.sync()
    p1.sync()
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    b[3][7, 11] = float("nan")          # a NaN in Jx spreads to every output mode
    p1.step([b[0], b[1], None], [None, None, b[2]], [b[3], b[4], None])
    with pytest.raises(capi.PsatdError) as ei:
        p1.sync()
    assert ei.value.status == NONFINITE
    p1.sync()                           # reported once, then cleared
    c = _te(shape, 2)
    p1.step([c[0], c[1], None], [None, None, c[2]], [c[3], c[4], None])
    p1.sync()
    assert all(bool(torch.isfinite(t).all()) for t in c[:3])
    p0.destroy()
    p1.destroy()


def test_checked_batch_reports_the_bad_patch_class():
    ensure_lib()
    sizes = [(64, 64), (128, 32), (64, 64)]
    total = sum(x * y for x, y in sizes)
    g = torch.Generator(device="cuda").manual_seed(3)
    E = [torch.randn(total, device="cuda", generator=g) for _ in range(5)]
    b = capi.Batch(sizes, (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J", checked=True)
    b.step([E[0], E[1], None], [None, None, E[2]], [E[3], E[4], None])
    b.sync()
    E[2][64 * 64 + 5] = float("inf")     # Bz of the 128 x 32 patch
    b.step([E[0], E[1], None], [None, None, E[2]], [E[3], E[4], None])
    with pytest.raises(capi.PsatdError) as ei:
        b.sync()
    assert ei.value.status == NONFINITE
    b.destroy()


def test_allocation_failure_is_reported_and_leaves_no_plan():
    """A plan whose spectral scratch cannot fit in HBM (4096^3 cells, about 1.6 TB)
    fails at plan creation with PSATD_ERR_OOM (a host-side failure: cudaMalloc
    returns an error, nothing is launched), and a normal plan works afterwards."""
    ensure_lib()
    with pytest.raises(capi.PsatdError) as ei:
        capi.Plan((4096, 4096, 4096), (1.0, 1.0, 1.0), 0.5, layout="3d6", prec="fp32", src="none")
    assert ei.value.status == 3 and "cudaMalloc" in str(ei.value)
    free0 = torch.cuda.mem_get_info()[0]
    a = _te((64, 128), 9)
    p = capi.Plan((128, 64), (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
    p.step([a[0], a[1], None], [None, None, a[2]], [a[3], a[4], None])
    p.sync()
    p.destroy()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)   # nothing of the failed plan is held
