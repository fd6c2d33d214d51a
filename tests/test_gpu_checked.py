"""PSATD_FLAG_CHECKED: every step's output arrays are scanned for NaN / Inf and
a hit is reported by the next sync as PSATD_ERR_NONFINITE (host-made failure:
a NaN placed in an input; nothing faults on the GPU).  A checked plan computes
the same bits as an unchecked one, the word is cleared by the sync that reports
it, and the plan stays usable.

The bounded MMA-completion wait of the tensor-core passes: with the test hook
PSATD_FLAG_TEST_STALL_MMA nothing is committed to the mbarrier, so every CTA's
first wait runs out (a short poll limit), the CTA stops using the tensor cores
and frees its TMEM, and the sync reports PSATD_ERR_TIMEOUT; a normal plan run
afterwards (whose CTAs allocate TMEM again on the same SMs) is correct."""
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


TIMEOUT = 5


@pytest.mark.parametrize("prec", ["mixed_fp16", "mixed_bf16"])
def test_expired_mma_wait_reports_timeout_and_frees_tmem(prec):
    from gpu_helpers import mask_layout, rel_l2_fields, rounded
    from oracle import psatd as orc
    ensure_lib()
    n, shape = (256, 256), (256, 256)
    a = _te(shape, 3)
    stalled = capi.Plan(n, (1.0, 1.0), 0.5, layout="te", prec=prec, src="J", test_stall_mma=True)
    stalled.step([a[0], a[1], None], [None, None, a[2]], [a[3], a[4], None])
    with pytest.raises(capi.PsatdError) as ei:
        stalled.sync()
    assert ei.value.status == TIMEOUT
    stalled.sync()                      # reported once, then cleared
    stalled.destroy()
    # the same kind of plan without the hook, on fresh inputs, against the oracle
    b = _te(shape, 4)
    host = [t.double().cpu().numpy() for t in b]
    good = capi.Plan(n, (1.0, 1.0), 0.5, layout="te", prec=prec, src="J")
    good.step([b[0], b[1], None], [None, None, b[2]], [b[3], b[4], None], nsteps=2)
    good.sync()
    good.destroy()
    z = np.zeros(shape)
    E = np.stack([host[0], host[1], z])
    B = np.stack([z, z, host[2]])
    J = np.stack([host[3], host[4], z])
    Eo, Bo = orc.psatd_step(E, B, J, d=(1.0, 1.0), dt=0.5, form="J", nsteps=2)
    Eg = np.stack([b[0].double().cpu().numpy(), b[1].double().cpu().numpy(), z])
    Bg = np.stack([z, z, b[2].double().cpu().numpy()])
    err = rel_l2_fields(Eg, Bg, mask_layout(Eo, "te", "E"), mask_layout(Bo, "te", "B"))
    assert err < 4e-6, err


BOUNDS = 7


@pytest.mark.parametrize("prec,layout,shape", [("fp32", "te", (128, 256)), ("mixed_bf16", "te", (256, 256)),
                                               ("fp64", "3d6", (16, 32, 32))])
def test_index_checks_trip_on_short_extents_and_pass_otherwise(prec, layout, shape):
    """The checked mode's index checks: told that every array is one element shorter
    (the test hook), the CTAs reaching the last element skip their accesses and the
    sync reports PSATD_ERR_BOUNDS; with the true extents the checked plan gives the
    unchecked plan's bits."""
    ensure_lib()
    n = tuple(reversed(shape))
    d = tuple([1.0] * len(shape))
    dt = 0.4
    g = torch.Generator(device="cuda").manual_seed(11)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    pe, pb, pj = capi.PRESENT[layout]
    mk = lambda p: [torch.randn(shape, device="cuda", generator=g, dtype=dtype) if p[i] else None for i in range(3)]
    E, B, J = mk(pe), mk(pb), mk(pj)
    clone = lambda F: [t.clone() if t is not None else None for t in F]
    E1, B1, E2, B2 = clone(E), clone(B), clone(E), clone(B)
    p0 = capi.Plan(n, d, dt, layout=layout, prec=prec, src="J")
    p1 = capi.Plan(n, d, dt, layout=layout, prec=prec, src="J", checked=True)
    p0.step(E1, B1, J, nsteps=2)
    p1.step(E2, B2, J, nsteps=2)
    p0.sync()
    p1.sync()
    for x, y in zip(E1 + B1, E2 + B2):
        if x is not None:
            assert torch.equal(x, y)
    p2 = capi.Plan(n, d, dt, layout=layout, prec=prec, src="J", checked=True, test_short_extent=True)
    p2.step(clone(E), clone(B), J)
    with pytest.raises(capi.PsatdError) as ei:
        p2.sync()
    assert ei.value.status == BOUNDS
    p2.sync()                            # reported once, then cleared
    for p in (p0, p1, p2):
        p.destroy()
