"""ctypes binding of the C ABI in ``include/psatd.h`` (argument marshalling only).

Every step of the PSATD/FDTD path runs in the CUDA kernels of ``libpsatd.so``;
this module only checks tensor arguments, builds the C structs and calls the
entry points of the same names.  PyTorch supplies device memory and streams.
There is no CPU fallback: if the library is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpsatd.so")

PSATD_OK = 0
STATUS = {0: "PSATD_OK", 1: "PSATD_ERR_INVALID_ARG", 2: "PSATD_ERR_UNSUPPORTED", 3: "PSATD_ERR_OOM",
          4: "PSATD_ERR_CUDA", 5: "PSATD_ERR_TIMEOUT", 6: "PSATD_ERR_NONFINITE", 7: "PSATD_ERR_BOUNDS"}
PREC = {"fp64": 0, "fp32": 1, "mixed_bf16": 2, "mixed_fp16": 3}
SRC = {"none": 0, "J": 1, "rho": 2}
LAYOUT = {"3d6": 0, "2d6": 1, "te": 2, "tm": 3}
SCHEME = {"yee": 0, "ckc": 1}
# (E, B, J) components present per layout
PRESENT = {
    "3d6": ((1, 1, 1), (1, 1, 1), (1, 1, 1)),
    "2d6": ((1, 1, 1), (1, 1, 1), (1, 1, 1)),
    "te": ((1, 1, 0), (0, 0, 1), (1, 1, 0)),
    "tm": ((0, 0, 1), (1, 1, 0), (0, 0, 1)),
}


class PsatdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class psatd_desc(ct.Structure):
    _fields_ = [("ndim", ct.c_int32), ("layout", ct.c_int32), ("n", ct.c_int64 * 3),
                ("d", ct.c_double * 3), ("dt", ct.c_double), ("c", ct.c_double),
                ("eps0", ct.c_double), ("prec", ct.c_int32), ("src", ct.c_int32),
                ("flags", ct.c_int32), ("order", ct.c_int32)]


class psatd_fields(ct.Structure):
    _fields_ = [("E", ct.c_void_p * 3), ("B", ct.c_void_p * 3)]


class psatd_sources(ct.Structure):
    _fields_ = [("J", ct.c_void_p * 3), ("rho_n", ct.c_void_p), ("rho_np1", ct.c_void_p)]


_lib = None

EXPORTS = [
    ("psatd_abi_version", ct.c_int32, []),
    ("psatd_plan_create", ct.c_int, [ct.POINTER(psatd_desc), ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    ("psatd_coeffs_init", ct.c_int, [ct.c_void_p]),
    ("psatd_step", ct.c_int, [ct.c_void_p, ct.POINTER(psatd_fields), ct.POINTER(psatd_sources), ct.c_int32]),
    ("psatd_plan_sync", ct.c_int, [ct.c_void_p]),
    ("psatd_plan_destroy", ct.c_int, [ct.c_void_p]),
    ("psatd_plan_workspace_bytes", ct.c_size_t, [ct.c_void_p]),
    ("psatd_plan_set_timing", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("psatd_kernel_times", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_char_p),
                                        ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double)]),
    ("fdtd_step", ct.c_int, [ct.POINTER(psatd_desc), ct.c_int32, ct.POINTER(psatd_fields),
                             ct.POINTER(psatd_sources), ct.c_int32, ct.c_void_p]),
    ("psatd_last_error", ct.c_char_p, [ct.c_void_p]),
    ("psatd_batch_create", ct.c_int, [ct.POINTER(psatd_desc), ct.c_int32, ct.POINTER(ct.c_int64), ct.c_void_p,
                                      ct.POINTER(ct.c_void_p)]),
    ("psatd_batch_step", ct.c_int, [ct.c_void_p, ct.POINTER(psatd_fields), ct.POINTER(psatd_sources), ct.c_int32]),
    ("psatd_batch_cells", ct.c_int64, [ct.c_void_p]),
    ("psatd_batch_sync", ct.c_int, [ct.c_void_p]),
    ("psatd_batch_destroy", ct.c_int, [ct.c_void_p]),
    ("psatd_batch_set_timing", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("psatd_batch_set_persistent", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("psatd_batch_launches_per_step", ct.c_int32, [ct.c_void_p]),
    ("psatd_batch_set_branches", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("psatd_batch_kernel_times", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_char_p),
                                              ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double)]),
    ("psatd_plan_autotune", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_char_p, ct.c_size_t]),
    ("psatd_plan_set_launch", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32)]),
    ("psatd_plan_get_launch", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32)]),
    ("psatd_plan_set_push_groups", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("psatd_batch_set_push_groups", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("psatd_plan_get_push_groups", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32)]),
    ("psatd_local_create", ct.c_int, [ct.POINTER(psatd_desc), ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p,
                                      ct.POINTER(ct.c_void_p)]),
    ("psatd_local_step", ct.c_int, [ct.c_void_p, ct.POINTER(psatd_fields), ct.POINTER(psatd_sources), ct.c_int32]),
    ("psatd_local_plan", ct.c_void_p, [ct.c_void_p]),
    ("psatd_local_destroy", ct.c_int, [ct.c_void_p]),
    ("psatd_farfield", ct.c_int, [ct.POINTER(psatd_desc), ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_int32, ct.c_int32,
                                  ct.c_void_p, ct.c_void_p, ct.c_void_p]),
]

FLAG_AUTOTUNE = 1
FLAG_PSTD = 2
FLAG_CHECKED = 4
FLAG_TEST_STALL_MMA = 8  # test hook of the failure path (mixed precisions): see include/psatd.h
FLAG_TEST_SHORT_EXTENT = 16  # test hook of the checked mode's index checks: see include/psatd.h


def load(path: str = LIB_PATH):
    """Load libpsatd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("%s is missing: build it with paper_1608_05739_gb300.build.build()" % path)
    lib = ct.CDLL(path)
    for name, res, args in EXPORTS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, plan=None):
    if status != PSATD_OK:
        msg = load().psatd_last_error(plan)
        raise PsatdError(status, msg.decode() if msg else "")


def make_desc(n, d, dt, *, layout="te", prec="fp32", src="J", c=1.0, eps0=1.0, autotune=False, order=0,
              scheme="psatd", checked=False, test_stall_mma=False, test_short_extent=False):
    """psatd_desc for grid ``n`` = (nx, ny[, nz]) and cell sizes ``d``."""
    nd = len(n)
    desc = psatd_desc()
    desc.ndim = nd
    desc.layout = LAYOUT[layout]
    for i in range(3):
        desc.n[i] = int(n[i]) if i < nd else 1
        desc.d[i] = float(d[i]) if i < nd else 1.0
    desc.dt, desc.c, desc.eps0 = float(dt), float(c), float(eps0)
    desc.prec = PREC[prec]
    desc.src = SRC[src]
    if scheme not in ("psatd", "pstd"):
        raise ValueError("scheme must be 'psatd' or 'pstd'")
    desc.flags = ((FLAG_AUTOTUNE if autotune else 0) | (FLAG_PSTD if scheme == "pstd" else 0)
                  | (FLAG_CHECKED if checked else 0) | (FLAG_TEST_STALL_MMA if test_stall_mma else 0)
                  | (FLAG_TEST_SHORT_EXTENT if test_short_extent else 0))
    desc.order = int(order)
    return desc


def _ptr(t, shape, dtype, what):
    """Pointer of tensor ``t`` after checking device, dtype, shape, layout: a CUDA
    tensor, or a pinned host tensor (the passes then read and write host memory
    directly over the host link)."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False) and not (hasattr(t, "is_pinned") and t.is_pinned()):
        raise ValueError("%s must be a CUDA tensor or a pinned host tensor" % what)
    if t.dtype != dtype:
        raise ValueError("%s must be %s (got %s)" % (what, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s (got %s)" % (what, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return t.data_ptr()


def _grid_shape(n):
    return tuple(int(v) for v in reversed(n))  # [nz][ny][nx] / [ny][nx]


def _fields_struct(layout, shape, dtype, E, B):
    pe, pb, _ = PRESENT[layout]
    f = psatd_fields()
    for i in range(3):
        e = E[i] if E is not None else None
        b = B[i] if B is not None else None
        if bool(pe[i]) != (e is not None) or bool(pb[i]) != (b is not None):
            raise ValueError("component %d of E/B presence does not match layout %r" % (i, layout))
        f.E[i] = _ptr(e, shape, dtype, "E[%d]" % i)
        f.B[i] = _ptr(b, shape, dtype, "B[%d]" % i)
    return f


def _sources_struct(layout, shape, dtype, J, rho_n, rho_np1):
    _, _, pj = PRESENT[layout]
    s = psatd_sources()
    for i in range(3):
        j = J[i] if J is not None else None
        if j is not None and not pj[i]:
            raise ValueError("J[%d] is not used by layout %r" % (i, layout))
        s.J[i] = _ptr(j, shape, dtype, "J[%d]" % i)
    s.rho_n = _ptr(rho_n, shape, dtype, "rho_n")
    s.rho_np1 = _ptr(rho_np1, shape, dtype, "rho_np1")
    return s


def _torch_dtype(prec):
    import torch
    return torch.float64 if prec == "fp64" else torch.float32


class Plan:
    """A PSATD plan (psatd_plan_create + psatd_coeffs_init) bound to a CUDA stream.

    ``n`` = (nx, ny[, nz]) cells, ``d`` cell sizes, ``dt`` time step; fields are
    passed per component as contiguous CUDA tensors of shape [ny, nx] or
    [nz, ny, nx] (None for components absent from the layout).
    """

    def __init__(self, n, d, dt, *, layout="te", prec="fp32", src="J", c=1.0, eps0=1.0, stream=None,
                 autotune=False, order=0, scheme="psatd", checked=False, test_stall_mma=False,
                 test_short_extent=False):
        import torch
        lib = load()
        self.n, self.layout, self.prec, self.src = tuple(n), layout, prec, src
        self.shape = _grid_shape(n)
        self.dtype = _torch_dtype(prec)
        self.desc = make_desc(n, d, dt, layout=layout, prec=prec, src=src, c=c, eps0=eps0, autotune=autotune,
                              order=order, scheme=scheme, checked=checked, test_stall_mma=test_stall_mma,
                              test_short_extent=test_short_extent)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ct.c_void_p()
        _check(lib.psatd_plan_create(ct.byref(self.desc), ct.c_void_p(stream.cuda_stream), ct.byref(h)))
        self.handle = h
        _check(lib.psatd_coeffs_init(self.handle), self.handle)

    def step(self, E, B, J=None, rho_n=None, rho_np1=None, nsteps=1):
        f = _fields_struct(self.layout, self.shape, self.dtype, E, B)
        s = _sources_struct(self.layout, self.shape, self.dtype, J, rho_n, rho_np1) \
            if self.src != "none" else None
        _check(load().psatd_step(self.handle, ct.byref(f), ct.byref(s) if s is not None else None,
                                 int(nsteps)), self.handle)

    def sync(self):
        _check(load().psatd_plan_sync(self.handle), self.handle)

    def get_launch(self):
        """[log2 tb fwd_x, fwd_y, inv_y, inv_x, push lines per CTA, push elements per thread]."""
        cfg = (ct.c_int32 * 6)()
        _check(load().psatd_plan_get_launch(self.handle, cfg), self.handle)
        return list(cfg)

    def set_launch(self, cfg):
        arr = (ct.c_int32 * 6)(*[int(v) for v in cfg])
        _check(load().psatd_plan_set_launch(self.handle, arr), self.handle)

    def get_push_groups(self):
        """Component groups the fused pass's next launch uses."""
        g = ct.c_int32(0)
        _check(load().psatd_plan_get_push_groups(self.handle, ct.byref(g)), self.handle)
        return g.value

    def set_push_groups(self, groups):
        """psatd_plan_set_push_groups: 1, 2 or 4 component groups (-1: the built-in choice)."""
        _check(load().psatd_plan_set_push_groups(self.handle, int(groups)), self.handle)

    def autotune(self, reps=5):
        """psatd_plan_autotune: time the launch shapes, keep the fastest; returns the report."""
        buf = ct.create_string_buffer(4096)
        _check(load().psatd_plan_autotune(self.handle, int(reps), buf, len(buf)), self.handle)
        return buf.value.decode()

    def workspace_bytes(self):
        return int(load().psatd_plan_workspace_bytes(self.handle))

    def set_timing(self, enable=True):
        _check(load().psatd_plan_set_timing(self.handle, 1 if enable else 0), self.handle)

    def kernel_times(self):
        """{kernel name: (launches, total ms)} of the launches since set_timing(True)."""
        names = (ct.c_char_p * 8)()
        launches = (ct.c_int64 * 8)()
        ms = (ct.c_double * 8)()
        k = load().psatd_kernel_times(self.handle, 8, names, launches, ms)
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(k)}

    def destroy(self):
        if getattr(self, "handle", None) is not None:
            load().psatd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Batch:
    """A batch of independent 2D periodic patches (psatd_batch_create) on a CUDA stream.

    ``sizes`` = [(nx, ny), ...] (sizes as for Plan).  Fields and sources are passed
    per component as one contiguous CUDA tensor of ``total`` elements holding
    the patches back to back, patch i being its (ny_i, nx_i) row-major block.
    """

    def __init__(self, sizes, d, dt, *, layout="te", prec="fp32", src="J", c=1.0, eps0=1.0, stream=None,
                 autotune=False, order=0, checked=False):
        import torch
        lib = load()
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        self.layout, self.prec, self.src = layout, prec, src
        self.dtype = _torch_dtype(prec)
        self.total = sum(a * b for a, b in self.sizes)
        self.offsets = []
        acc = 0
        for a, b in self.sizes:
            self.offsets.append(acc)
            acc += a * b
        desc = make_desc(self.sizes[0], d, dt, layout=layout, prec=prec, src=src, c=c, eps0=eps0,
                         autotune=autotune, order=order, checked=checked)
        arr = (ct.c_int64 * (2 * len(self.sizes)))(*[v for ab in self.sizes for v in ab])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ct.c_void_p()
        _check(lib.psatd_batch_create(ct.byref(desc), len(self.sizes), arr, ct.c_void_p(stream.cuda_stream),
                                      ct.byref(h)))
        self.handle = h

    def step(self, E, B, J=None, rho_n=None, rho_np1=None, nsteps=1):
        shape = (self.total,)
        f = _fields_struct(self.layout, shape, self.dtype, E, B)
        s = _sources_struct(self.layout, shape, self.dtype, J, rho_n, rho_np1) if self.src != "none" else None
        _check(load().psatd_batch_step(self.handle, ct.byref(f), ct.byref(s) if s is not None else None,
                                       int(nsteps)))

    def cells(self):
        return int(load().psatd_batch_cells(self.handle))

    def set_timing(self, enable=True):
        _check(load().psatd_batch_set_timing(self.handle, 1 if enable else 0))

    def set_persistent(self, enable=True):
        """Persistent passes (where the sizes allow) or per-class launches (the default)."""
        _check(load().psatd_batch_set_persistent(self.handle, 1 if enable else 0))

    def launches_per_step(self):
        return int(load().psatd_batch_launches_per_step(self.handle))

    def set_push_groups(self, groups):
        """psatd_batch_set_push_groups: component groups of each class's fused pass where valid."""
        _check(load().psatd_batch_set_push_groups(self.handle, int(groups)))

    def set_branches(self, forked=True):
        """Size classes on the branch streams (default) or one after another on the batch's stream."""
        _check(load().psatd_batch_set_branches(self.handle, 1 if forked else 0))

    def kernel_times(self):
        """{kernel name: (launches, total ms)} summed over the size classes."""
        names = (ct.c_char_p * 8)()
        launches = (ct.c_int64 * 8)()
        ms = (ct.c_double * 8)()
        k = load().psatd_batch_kernel_times(self.handle, 8, names, launches, ms)
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(k)}

    def sync(self):
        """psatd_batch_sync: wait for the batch and raise on a recorded device error."""
        _check(load().psatd_batch_sync(self.handle))

    def destroy(self):
        if getattr(self, "handle", None) is not None:
            load().psatd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Local:
    """Local-FFT decomposition of one periodic 2D grid (psatd_local_create): ``px`` x ``py``
    patches with ``guard`` cells, each advanced by its own FFTs.  Fields and sources are
    the global arrays, shape [ny, nx], as for Plan."""

    def __init__(self, n, d, dt, *, px, py, guard, layout="te", prec="fp32", src="J", c=1.0, eps0=1.0,
                 stream=None, autotune=False, order=0):
        import torch
        lib = load()
        self.n, self.layout, self.prec, self.src = tuple(n), layout, prec, src
        self.shape = _grid_shape(n)
        self.dtype = _torch_dtype(prec)
        desc = make_desc(n, d, dt, layout=layout, prec=prec, src=src, c=c, eps0=eps0, autotune=autotune,
                         order=order)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ct.c_void_p()
        _check(lib.psatd_local_create(ct.byref(desc), int(px), int(py), int(guard), ct.c_void_p(stream.cuda_stream),
                                      ct.byref(h)))
        self.handle = h

    def step(self, E, B, J=None, rho_n=None, rho_np1=None, nsteps=1):
        f = _fields_struct(self.layout, self.shape, self.dtype, E, B)
        s = _sources_struct(self.layout, self.shape, self.dtype, J, rho_n, rho_np1) \
            if self.src != "none" else None
        lib = load()
        _check(lib.psatd_local_step(self.handle, ct.byref(f), ct.byref(s) if s is not None else None, int(nsteps)),
               lib.psatd_local_plan(self.handle))

    def sync(self):
        lib = load()
        _check(lib.psatd_plan_sync(lib.psatd_local_plan(self.handle)), lib.psatd_local_plan(self.handle))

    def destroy(self):
        if getattr(self, "handle", None) is not None:
            load().psatd_local_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fdtd_step(n, d, dt, E, B, J=None, *, scheme="yee", layout="te", prec="fp32", c=1.0, eps0=1.0,
              nsteps=1, stream=None):
    """Yee / CKC FDTD steps of co-temporal (E, B) in place (see include/psatd.h)."""
    import torch
    lib = load()
    desc = make_desc(n, d, dt, layout=layout, prec=prec, src="J" if J is not None else "none", c=c, eps0=eps0)
    shape = _grid_shape(n)
    dtype = _torch_dtype(prec)
    f = _fields_struct(layout, shape, dtype, E, B)
    s = _sources_struct(layout, shape, dtype, J, None, None) if J is not None else None
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib.fdtd_step(ct.byref(desc), SCHEME[scheme], ct.byref(f), ct.byref(s) if s is not None else None,
                         int(nsteps), ct.c_void_p(stream.cuda_stream)))


def step_noalloc(n, d, dt, E, B, J=None, rho_n=None, rho_np1=None, *, layout="te", prec="fp32", src="J",
                 c=1.0, eps0=1.0, nsteps=1, stream=None, scheme="psatd"):
    """psatd_step_noalloc: one-call PSATD step that allocates no device memory.

    For callers that cannot allocate on the GPU: the library's scratch is a
    fixed 16 MiB device array (grids needing more raise PsatdError with
    PSATD_ERR_UNSUPPORTED).  Calls whose GPU work overlaps share that array
    and race; the first call on a device must precede any stream capture.
    Fields and sources are passed as for Plan.step.
    """
    import torch
    lib = load()
    fn = lib.psatd_step_noalloc
    fn.restype = ct.c_int
    fn.argtypes = [ct.POINTER(psatd_desc), ct.POINTER(psatd_fields), ct.POINTER(psatd_sources), ct.c_int32,
                   ct.c_void_p]
    desc = make_desc(n, d, dt, layout=layout, prec=prec, src=src, c=c, eps0=eps0, scheme=scheme)
    shape = _grid_shape(n)
    dtype = _torch_dtype(prec)
    f = _fields_struct(layout, shape, dtype, E, B)
    s = _sources_struct(layout, shape, dtype, J, rho_n, rho_np1) if src != "none" else None
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(fn(ct.byref(desc), ct.byref(f), ct.byref(s) if s is not None else None, int(nsteps),
              ct.c_void_p(stream.cuda_stream)))


APODISE = {"none": 0, "x": 1, "xy": 2}


def farfield(n, d, field, k, *, x_range=None, y_range=None, window="none", stream=None):
    """psatd_farfield: the Fraunhofer far-field transform of the 2D snapshot ``field``
    ([ny, nx] CUDA tensor, float32 or float64) at the wavevectors ``k`` ((nk, 2)
    float64 CUDA tensor of (kx, ky)); returns a complex128 CUDA tensor (nk,).
    x_range / y_range: (start, stop) cells of the window (default the whole
    axis); window: Hann apodisation "none", "x" or "xy"."""
    import torch
    lib = load()
    prec = "fp32" if field.dtype == torch.float32 else "fp64"
    desc = make_desc(n, d, 1.0, layout="te", prec=prec, src="none")
    shape = _grid_shape(n)
    ptr = _ptr(field, shape, field.dtype, "field")
    if k.dtype != torch.float64 or k.dim() != 2 or k.shape[1] != 2 or not k.is_contiguous():
        raise ValueError("k must be a contiguous float64 tensor of shape (nk, 2)")
    nx, ny = int(n[0]), int(n[1])
    x0, x1 = x_range if x_range is not None else (0, nx)
    y0, y1 = y_range if y_range is not None else (0, ny)
    win = (ct.c_int64 * 4)(int(x0), int(x1), int(y0), int(y1))
    out = torch.empty((k.shape[0], 2), dtype=torch.float64, device=k.device)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib.psatd_farfield(ct.byref(desc), ptr, win, APODISE[window], int(k.shape[0]), k.data_ptr(),
                              out.data_ptr(), ct.c_void_p(stream.cuda_stream)))
    return torch.view_as_complex(out)
