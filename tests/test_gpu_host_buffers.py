"""Host-resident field arrays through the C ABI: pinned host memory is accepted
and read / written by the passes in place (no separate copies), giving the same
bits as the same step on device arrays; pageable host memory is refused before
any launch (INVALID_ARG, nothing launched, the plan stays usable)."""
import ctypes as ct

import numpy as np
import pytest

from gpu_helpers import ensure_lib, mask_layout, rel_l2_fields
from oracle import psatd as orc
from paper_1608_05739_gb300 import capi, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout,shape,src", [("te", (256, 512), "J"), ("3d6", (32, 64, 128), "rho")])
def test_pinned_host_arrays_equal_device_arrays_bitwise(layout, shape, src):
    import torch
    ensure_lib()
    pe, pb, pj = capi.PRESENT[layout]
    n = tuple(reversed(shape))
    d = (1.0, 0.9, 1.1)[:len(shape)]
    dt = 0.4
    comps = [synth.random_fields(shape, 3, 40 + i) for i in range(3)]
    r0, r1 = synth.random_fields(shape, 2, 50)
    plan = capi.Plan(n, d, dt, layout=layout, prec="fp32", src=src)

    def tensors(dev):
        mk = lambda a: (torch.from_numpy(a).float().to(dev) if dev == "cuda"
                        else torch.from_numpy(a).float().pin_memory())
        E = [mk(comps[0][i]) if pe[i] else None for i in range(3)]
        B = [mk(comps[1][i]) if pb[i] else None for i in range(3)]
        J = [mk(comps[2][i]) if pj[i] else None for i in range(3)]
        rr = (mk(r0), mk(r1)) if src == "rho" else (None, None)
        return E, B, J, rr

    Ed, Bd, Jd, rd = tensors("cuda")
    Eh, Bh, Jh, rh = tensors("cpu")
    plan.step(Ed, Bd, Jd, *rd, nsteps=3)
    plan.step(Eh, Bh, Jh, *rh, nsteps=3)
    plan.sync()
    for a, b in zip(Ed + Bd, Eh + Bh):
        if a is not None:
            assert torch.equal(a.cpu(), b)
    # and the oracle agrees at the FP32 bound
    E0 = np.stack([comps[0][i] if pe[i] else np.zeros(shape) for i in range(3)]).astype(np.float32).astype(float)
    B0 = np.stack([comps[1][i] if pb[i] else np.zeros(shape) for i in range(3)]).astype(np.float32).astype(float)
    J0 = np.stack([comps[2][i] if pj[i] else np.zeros(shape) for i in range(3)]).astype(np.float32).astype(float)
    rr = (r0.astype(np.float32).astype(float), r1.astype(np.float32).astype(float)) if src == "rho" else (None, None)
    Eo, Bo = orc.psatd_step(E0, B0, J0, *rr, d=d, dt=dt, form=src, nsteps=3)
    Eg = np.stack([Eh[i].double().numpy() if pe[i] else np.zeros(shape) for i in range(3)])
    Bg = np.stack([Bh[i].double().numpy() if pb[i] else np.zeros(shape) for i in range(3)])
    assert rel_l2_fields(Eg, Bg, mask_layout(Eo, layout, "E"), mask_layout(Bo, layout, "B")) < 6e-6
    plan.destroy()


def test_pageable_host_memory_is_refused_before_launch():
    import torch
    ensure_lib()
    lib = capi.load()
    plan = capi.Plan((64, 32), (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
    dev = [torch.zeros(32, 64, device="cuda") for _ in range(5)]
    pageable = np.zeros((32, 64), dtype=np.float32)   # ordinary host memory
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    f.E[0] = pageable.ctypes.data
    f.E[1] = dev[1].data_ptr()
    f.B[2] = dev[2].data_ptr()
    s.J[0] = dev[3].data_ptr()
    s.J[1] = dev[4].data_ptr()
    st = lib.psatd_step(plan.handle, ct.byref(f), ct.byref(s), 1)
    assert st == 1   # PSATD_ERR_INVALID_ARG
    assert b"not accessible" in lib.psatd_last_error(plan.handle)
    # the plan stays usable
    plan.step([dev[0], dev[1], None], [None, None, dev[2]], [dev[3], dev[4], None])
    plan.sync()
    plan.destroy()
