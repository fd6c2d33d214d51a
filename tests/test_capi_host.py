"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function declared in include/psatd.h, and rejects invalid
arguments before any CUDA call."""
import ctypes as ct
import os
import re

import pytest

from paper_1608_05739_gb300 import build as bld
from paper_1608_05739_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return capi.load()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "psatd_step" in names and "fdtd_step" in names and len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert lib.psatd_abi_version() == 1


def test_desc_struct_layout_matches_c():
    assert ct.sizeof(capi.psatd_desc) == 96
    assert capi.psatd_desc.n.offset == 8 and capi.psatd_desc.d.offset == 32
    assert capi.psatd_desc.prec.offset == 80
    assert ct.sizeof(capi.psatd_fields) == 48 and ct.sizeof(capi.psatd_sources) == 40


def _create(lib, desc):
    h = ct.c_void_p()
    st = lib.psatd_plan_create(ct.byref(desc) if desc is not None else None, None, ct.byref(h))
    return st, h


@pytest.mark.parametrize("mutate,expect", [
    (lambda d: setattr(d, "ndim", 3), 1),                  # ndim does not match a 2D layout
    (lambda d: d.n.__setitem__(0, 100), 2),                # not a power of two
    (lambda d: d.n.__setitem__(0, 8192), 2),               # too long
    (lambda d: d.n.__setitem__(2, 4), 1),                  # n[2] != 1 in 2D
    (lambda d: setattr(d, "dt", 0.0), 1),
    (lambda d: setattr(d, "c", -1.0), 1),
    (lambda d: setattr(d, "eps0", float("nan")), 1),
    (lambda d: d.d.__setitem__(1, 0.0), 1),
    (lambda d: setattr(d, "prec", 2), 2),                  # split-BF16: 64 threads, no 128-row group
    (lambda d: setattr(d, "prec", 9), 1),
    (lambda d: setattr(d, "src", 7), 1),
    (lambda d: setattr(d, "flags", 16), 1),                # unknown flag bit
    (lambda d: setattr(d, "flags", 8), 1),                 # the MMA-stall test hook on an FP32 plan
    (lambda d: (setattr(d, "layout", 3), setattr(d, "src", 2)), 1),  # TM has no rho-form
    (lambda d: setattr(d, "layout", 9), 1),
])
def test_plan_create_rejects_invalid_descriptors(lib, mutate, expect):
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J")
    mutate(d)
    st, h = _create(lib, d)
    assert st == expect
    assert h.value is None
    assert len(lib.psatd_last_error(None)) > 0


def test_null_arguments(lib):
    h = ct.c_void_p()
    assert lib.psatd_plan_create(None, None, ct.byref(h)) == 1
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5)
    assert lib.psatd_plan_create(ct.byref(d), None, None) == 1
    assert lib.psatd_step(None, None, None, 1) == 1
    assert lib.psatd_coeffs_init(None) == 1
    assert lib.psatd_plan_destroy(None) == 0
    assert lib.psatd_plan_workspace_bytes(None) == 0
    assert b"NULL" in lib.psatd_last_error(None)


def test_fdtd_rejects_invalid_arguments(lib):
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="J")
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    assert lib.fdtd_step(ct.byref(d), 5, ct.byref(f), ct.byref(s), 1, None) == 1       # scheme
    d3 = capi.make_desc((16, 16, 16), (1.0, 1.0, 1.0), 0.5, layout="3d6", src="none")
    assert lib.fdtd_step(ct.byref(d3), 1, ct.byref(f), None, 1, None) == 2             # CKC 3D
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 0, None) == 1       # nsteps
    assert lib.fdtd_step(ct.byref(d), 0, None, ct.byref(s), 1, None) == 1              # fields NULL
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 1       # E missing
    f.E[0] = 0x1000
    f.E[1] = 0x2004                                                                     # misaligned
    f.B[2] = 0x3000
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 1
    dr = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="rho")
    assert lib.fdtd_step(ct.byref(dr), 0, ct.byref(f), ct.byref(s), 1, None) == 1      # rho-form


def test_batch_create_rejects_invalid_arguments(lib):
    d = capi.make_desc((64, 64), (1.0, 1.0), 0.5, layout="te", src="J")
    h = ct.c_void_p()
    n = (ct.c_int64 * 4)(64, 64, 100, 64)
    assert lib.psatd_batch_create(ct.byref(d), 2, n, None, ct.byref(h)) == 2       # 100 not a power of two
    assert b"patch 1" in lib.psatd_last_error(None)
    assert lib.psatd_batch_create(ct.byref(d), 0, n, None, ct.byref(h)) == 1       # no patch
    assert lib.psatd_batch_create(ct.byref(d), 1, None, None, ct.byref(h)) == 1
    d3 = capi.make_desc((16, 16, 16), (1.0, 1.0, 1.0), 0.5, layout="3d6", src="J")
    assert lib.psatd_batch_create(ct.byref(d3), 1, n, None, ct.byref(h)) == 1      # 3D
    assert lib.psatd_batch_step(None, None, None, 1) == 1
    assert lib.psatd_batch_destroy(None) == 0
    assert lib.psatd_batch_cells(None) == 0


@pytest.mark.parametrize("n,why", [((64, 32), b"128 threads"), ((16, 64), b"nx >= 32"), ((64, 8), b"ny, nz >= 16")])
def test_mixed_fp16_shape_limits(lib, n, why):
    """The tensor-core passes need one MMA row per thread in groups of 128:
    grids too small for that are refused before any allocation."""
    d = capi.make_desc(n, (1.0, 1.0), 0.5, layout="te", prec="mixed_fp16", src="J")
    st, h = _create(lib, d)
    assert st == 2 and h.value is None
    assert why in lib.psatd_last_error(None)


@pytest.mark.parametrize("n,prec", [
    ((96, 64), "fp64"), ((64, 48), "mixed_fp16"), ((96, 96), "mixed_bf16"),   # 3 * 2^k lengths: FP32 only
    ((160, 64), "fp64"), ((64, 80), "mixed_bf16"),                            # 5 * 2^k lengths: FP32 only
    ((6144, 64), "fp32"),                    # x rows of 3072 points: the R2C pass stops at 1536
    ((64, 6144), "fp32"), ((64, 24), "fp32"), ((72, 64), "fp32"), ((64, 112), "fp32"),
    ((64, 2560), "fp32"), ((64, 40), "fp32"),  # 5 * 2^k lines: 80 to 1280 points
])
def test_mixed_radix_length_limits(lib, n, prec):
    """Lines of 3 * 2^k points (48 to 3072) and 5 * 2^k points (80 to 1280; x rows
    are nx/2 points) are FP32-only; other lengths and other precisions are refused
    before any allocation."""
    d = capi.make_desc(n, (1.0, 1.0), 0.5, layout="te", prec=prec, src="J")
    st, h = _create(lib, d)
    assert st == 2 and h.value is None
    assert b"power of two" in lib.psatd_last_error(None)


def test_mixed_fp16_only_for_the_psatd_step(lib):
    d = capi.make_desc((64, 64), (1.0, 1.0), 0.5, layout="te", prec="mixed_fp16", src="J")
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 2
    assert lib.psatd_step_noalloc(ct.byref(d), ct.byref(f), ct.byref(s), 1, None) == 2
    assert b"FP32" in lib.psatd_last_error(None)


def test_autotune_argument_errors(lib):
    buf = ct.create_string_buffer(64)
    assert lib.psatd_plan_autotune(None, 5, buf, 64) == 1
    assert b"NULL" in lib.psatd_last_error(None)


def test_autotune_flag_is_psatd_only(lib):
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="J", autotune=True)
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 1
    assert b"flags" in lib.psatd_last_error(None)


def test_local_create_rejects_invalid_arguments(lib):
    h = ct.c_void_p()
    d = capi.make_desc((240, 120), (1.0, 1.0), 0.5, layout="te", src="J")
    assert lib.psatd_local_create(None, 2, 2, 8, None, ct.byref(h)) == 1
    assert lib.psatd_local_create(ct.byref(d), 7, 2, 8, None, ct.byref(h)) == 1       # 7 does not divide 240
    assert b"divide" in lib.psatd_last_error(None)
    assert lib.psatd_local_create(ct.byref(d), 2, 2, -1, None, ct.byref(h)) == 1      # guard < 0
    assert lib.psatd_local_create(ct.byref(d), 2, 2, 4, None, ct.byref(h)) == 2       # 128 x 68: not a power of two
    assert b"extended patch 128 x 68" in lib.psatd_last_error(None)
    d3 = capi.make_desc((64, 64, 64), (1.0, 1.0, 1.0), 0.5, layout="3d6", src="J")
    assert lib.psatd_local_create(ct.byref(d3), 2, 2, 8, None, ct.byref(h)) == 2
    assert lib.psatd_local_create(ct.byref(d), 2, 2, 8, None, None) == 1
    assert lib.psatd_local_step(None, None, None, 1) == 1
    assert lib.psatd_local_destroy(None) == 0
    assert lib.psatd_local_plan(None) is None


@pytest.mark.parametrize("order,expect", [(3, 1), (258, 1), (-2, 1), (1, 1)])
def test_invalid_orders(lib, order, expect):
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="J", order=order)
    st, h = _create(lib, d)
    assert st == expect and h.value is None
    assert b"order" in lib.psatd_last_error(None)


def test_order_is_psatd_only(lib):
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="J", order=4)
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 1
    assert lib.psatd_step_noalloc(ct.byref(d), ct.byref(f), ct.byref(s), 1, None) == 2


def test_pstd_flag_rules(lib):
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="rho", scheme="pstd")
    st, h = _create(lib, d)
    assert st == 1 and b"PSTD" in lib.psatd_last_error(None)
    d = capi.make_desc((64, 32), (1.0, 1.0), 0.5, layout="te", src="J", scheme="pstd")
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 1
    with pytest.raises(ValueError):
        capi.make_desc((64, 32), (1.0, 1.0), 0.5, scheme="leapfrog")


def test_checked_flag_limits(lib):
    """PSATD_FLAG_CHECKED is a plan flag: fdtd_step refuses any flag, the
    allocation-free step has no error word for it; batch sync needs a batch."""
    d = capi.make_desc((64, 64), (1.0, 1.0), 0.5, layout="te", prec="fp32", src="J", checked=True)
    f = capi.psatd_fields()
    s = capi.psatd_sources()
    assert lib.fdtd_step(ct.byref(d), 0, ct.byref(f), ct.byref(s), 1, None) == 1
    assert lib.psatd_step_noalloc(ct.byref(d), ct.byref(f), ct.byref(s), 1, None) == 2
    assert b"CHECKED" in lib.psatd_last_error(None)
    assert lib.psatd_batch_sync(None) == 1
