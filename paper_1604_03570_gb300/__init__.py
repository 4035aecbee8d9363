"""GB300 MultiFab time-step sweep: Python binding of libmf.so (include/mf.h).

Argument marshalling only: every step of the sweep (ghost fill, stencil, interpolation,
average-down, reductions, dtype conversion) runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams (``MultiFab``).  Importing this package fails if
libmf.so has not been built (``python -m paper_1604_03570_gb300.build``); there is no CPU
fallback.

Function names mirror the C ABI; errors raise ``MFError`` with the library's message.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_F64, MF_F32, MF_BF16 = 0, 1, 2
DTYPES = {"f64": MF_F64, "f32": MF_F32, "bf16": MF_BF16}
MF_LAP2_7PT, MF_LAP4_13PT, MF_LAP8_25PT = 1, 2, 4
MF_FP64_DIFF, MF_PLAIN_PER_BOX, MF_REFLUX, MF_FIXED_DIFF = 1, 2, 4, 8
MF_KERNEL_TMA, MF_KERNEL_GLOBAL = 0, 1
MF_RED_SUM, MF_RED_MAX, MF_RED_MIN, MF_RED_NORM0, MF_RED_NORM1, MF_RED_NORM2 = 0, 1, 2, 3, 4, 5
REDUCTIONS = {"sum": MF_RED_SUM, "max": MF_RED_MAX, "min": MF_RED_MIN, "norm0": MF_RED_NORM0,
              "norm1": MF_RED_NORM1, "norm2": MF_RED_NORM2}
MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_EUNSTABLE, MF_EALIGN, MF_ESTATE = -1, -2, -3, -4, -5, -6

EXPORTS = [
    "mf_create", "mf_create_boxes", "mf_destroy", "mf_nboxes", "mf_get_boxes", "mf_bytes", "mf_fb_regions",
    "mf_get_fb_regions", "mf_attach", "mf_set_tile", "mf_get_tile", "mf_copy_from_host", "mf_copy_to_host",
    "mf_copy_fab_to_host", "mf_copy_fab_from_host", "mf_fill_boundary", "mf_interp_cf", "mf_average_down",
    "mf_advance", "mf_amr_advance", "mf_sum", "mf_step_bytes", "mf_current", "mf_last_error", "mf_set_timing",
    "mf_phase_ms", "mf_set_kernel", "mf_sum_strided_noalloc", "mf_get_schedule", "mf_launch_count",
    "mf_fp64_fma_rate", "mf_set_schedule", "mf_reduce", "mf_stage_bytes", "mf_attach_stage",
    "mf_rk3_advance", "mf_interp_cells", "mf_reflux_faces", "mf_avgdown_cells", "mf_create_regional",
    "mf_box_regions", "mf_nregions", "mf_get_regions", "mf_set_class_tile", "mf_get_class_tiles",
    "mf_autotune_cache_reset",
]


class MFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libmf error %d: %s" % (code, msg))
        self.code = code


class mf_stencil(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("diffusivity", ctypes.POINTER(ctypes.c_double)), ("flags", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmf.so is not built (run `python -m paper_1604_03570_gb300.build` or "
                          "__graft_entry__.build()); this package has no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    I, P, D, LL, SZ = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mf_create": (I, [PP, P, P, I, I, I, I]),
        "mf_create_boxes": (I, [PP, P, P, P, I, I, I, I]),
        "mf_destroy": (None, [P]),
        "mf_nboxes": (I, [P]),
        "mf_get_boxes": (I, [P, P]),
        "mf_bytes": (SZ, [P]),
        "mf_fb_regions": (LL, [P, ctypes.POINTER(LL)]),
        "mf_get_fb_regions": (LL, [P, P, LL]),
        "mf_attach": (I, [P, P, SZ, P]),
        "mf_set_tile": (I, [P, P]),
        "mf_get_tile": (I, [P, P]),
        "mf_copy_from_host": (I, [P, P]),
        "mf_copy_to_host": (I, [P, P]),
        "mf_copy_fab_to_host": (I, [P, I, P]),
        "mf_copy_fab_from_host": (I, [P, I, P]),
        "mf_fill_boundary": (I, [P]),
        "mf_interp_cf": (I, [P, P, P, D, I]),
        "mf_average_down": (I, [P, P, I]),
        "mf_advance": (I, [P, ctypes.POINTER(mf_stencil), D, I]),
        "mf_amr_advance": (I, [P, P, ctypes.POINTER(mf_stencil), D, I, I, I]),
        "mf_sum": (I, [P, I, ctypes.POINTER(D)]),
        "mf_step_bytes": (D, [P, I]),
        "mf_current": (I, [P]),
        "mf_last_error": (ctypes.c_char_p, []),
        "mf_set_timing": (I, [P, I]),
        "mf_phase_ms": (I, [P, P]),
        "mf_set_kernel": (I, [P, I]),
        "mf_get_schedule": (I, [P, P]),
        "mf_launch_count": (I, [P, P]),
        "mf_fp64_fma_rate": (I, [ctypes.POINTER(D), P]),
        "mf_set_schedule": (I, [P, P]),
        "mf_reduce": (I, [P, I, I, ctypes.POINTER(D)]),
        "mf_stage_bytes": (SZ, [P]),
        "mf_attach_stage": (I, [P, P, SZ]),
        "mf_rk3_advance": (I, [P, ctypes.POINTER(mf_stencil), D, I]),
        "mf_interp_cells": (LL, [P, P, I, ctypes.POINTER(LL)]),
        "mf_reflux_faces": (LL, [P, P, I, ctypes.POINTER(LL)]),
        "mf_avgdown_cells": (LL, [P, P, I, ctypes.POINTER(LL)]),
        "mf_sum_strided_noalloc": (I, [P, I, I, I, I, LL, LL, ctypes.POINTER(D), P]),
        "mf_create_regional": (I, [PP, P, P, P, I, I, I, I, I]),
        "mf_box_regions": (I, [P, I, I, P, P]),
        "mf_nregions": (I, [P]),
        "mf_get_regions": (I, [P, P, P]),
        "mf_set_class_tile": (I, [P, I, I, I]),
        "mf_get_class_tiles": (I, [P, P]),
        "mf_autotune_cache_reset": (I, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def _check(rc):
    if rc < 0:
        raise MFError(rc, lib.mf_last_error().decode(errors="replace"))
    return rc


def _i3(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))
    return a


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _dtype_code(dtype):
    return DTYPES[dtype] if isinstance(dtype, str) else int(dtype)


# ------------------------------------------------------------------ C ABI, same names

def mf_create(domain_lo, domain_hi, max_grid_size, ncomp, ngrow, dtype):
    h = ctypes.c_void_p()
    lo, hi = _i3(domain_lo), _i3(domain_hi)
    _check(lib.mf_create(ctypes.byref(h), _ptr(lo), _ptr(hi), int(max_grid_size), int(ncomp), int(ngrow),
                         _dtype_code(dtype)))
    return h


def mf_create_boxes(domain_lo, domain_hi, boxes, ncomp, ngrow, dtype):
    h = ctypes.c_void_p()
    lo, hi = _i3(domain_lo), _i3(domain_hi)
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 6))
    _check(lib.mf_create_boxes(ctypes.byref(h), _ptr(lo), _ptr(hi), _ptr(b), b.shape[0], int(ncomp), int(ngrow),
                               _dtype_code(dtype)))
    return h


def mf_create_regional(domain_lo, domain_hi, boxes, ncomp, ngrow, dtype, max_region):
    h = ctypes.c_void_p()
    lo, hi = _i3(domain_lo), _i3(domain_hi)
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 6))
    _check(lib.mf_create_regional(ctypes.byref(h), _ptr(lo), _ptr(hi), _ptr(b), b.shape[0], int(ncomp), int(ngrow),
                                  _dtype_code(dtype), int(max_region)))
    return h


def mf_box_regions(boxes, max_region):
    """(regions (n, 6) int32, region of each box) that mf_create_regional makes from a box list."""
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 6))
    regs = np.zeros((b.shape[0], 6), dtype=np.int32)
    of = np.zeros(b.shape[0], dtype=np.int32)
    n = _check(lib.mf_box_regions(_ptr(b), b.shape[0], int(max_region), _ptr(regs), _ptr(of)))
    return regs[:n].copy(), of


def mf_nregions(h):
    return _check(lib.mf_nregions(h))


def mf_get_regions(h):
    """(regions (n, 6) int32, FArrayBox of each box) of a level's storage."""
    regs = np.zeros((mf_nregions(h), 6), dtype=np.int32)
    of = np.zeros(mf_nboxes(h), dtype=np.int32)
    _check(lib.mf_get_regions(h, _ptr(regs), _ptr(of)))
    return regs, of


def mf_set_class_tile(h, cls, ty, tz):
    _check(lib.mf_set_class_tile(h, int(cls), int(ty), int(tz)))


def mf_get_class_tiles(h):
    """{class: (ty, tz)} for the box-size classes present on the level (-1: the level's shape)."""
    out = np.zeros(15, dtype=np.int32)
    _check(lib.mf_get_class_tiles(h, _ptr(out)))
    return {k: (int(out[3 * k + 1]), int(out[3 * k + 2])) for k in range(5) if out[3 * k]}


def mf_autotune_cache_reset():
    _check(lib.mf_autotune_cache_reset())


def mf_destroy(h):
    lib.mf_destroy(h)


def mf_nboxes(h):
    return _check(lib.mf_nboxes(h))


def mf_get_boxes(h):
    out = np.zeros((mf_nboxes(h), 6), dtype=np.int32)
    _check(lib.mf_get_boxes(h, _ptr(out)))
    return out


def mf_bytes(h):
    return int(lib.mf_bytes(h))


def mf_fb_regions(h):
    g = ctypes.c_longlong()
    n = _check(lib.mf_fb_regions(h, ctypes.byref(g)))
    return int(n), int(g.value)


def mf_interp_cells(fine, crse, ratio):
    """(interpolated fine ghost cells per component, runs of the work list); host lists only."""
    runs = ctypes.c_longlong()
    n = _check(lib.mf_interp_cells(fine, crse, int(ratio), ctypes.byref(runs)))
    return int(n), int(runs.value)


def mf_avgdown_cells(fine, crse, ratio):
    """(coarse cells the average-down writes, regions of its work list); host lists only."""
    regs = ctypes.c_longlong()
    n = _check(lib.mf_avgdown_cells(fine, crse, int(ratio), ctypes.byref(regs)))
    return int(n), int(regs.value)


def mf_reflux_faces(fine, crse, ratio):
    """(coarse faces of the coarse-fine interface, coarse cells corrected); host lists only."""
    cells = ctypes.c_longlong()
    n = _check(lib.mf_reflux_faces(fine, crse, int(ratio), ctypes.byref(cells)))
    return int(n), int(cells.value)


def mf_get_fb_regions(h):
    n, _ = mf_fb_regions(h)
    out = np.zeros((n, 11), dtype=np.int32)
    _check(lib.mf_get_fb_regions(h, _ptr(out), n))
    return out


def mf_attach(h, dev_ptr, nbytes, stream):
    _check(lib.mf_attach(h, ctypes.c_void_p(int(dev_ptr)), int(nbytes), ctypes.c_void_p(int(stream or 0))))


def mf_set_tile(h, tile):
    if tile is None:
        _check(lib.mf_set_tile(h, None))
    else:
        _check(lib.mf_set_tile(h, _ptr(_i3(tile))))


def mf_get_tile(h):
    t = np.zeros(3, dtype=np.int32)
    auto = _check(lib.mf_get_tile(h, _ptr(t)))
    return tuple(int(v) for v in t), bool(auto)


def mf_copy_from_host(h, dense):
    """dense: float64 (C, Nz, Ny, Nx), numpy array or (pinned) CPU torch tensor."""
    if not hasattr(dense, "data_ptr"):
        dense = np.ascontiguousarray(dense, dtype=np.float64)
    _check(lib.mf_copy_from_host(h, _ptr(dense)))


def mf_copy_to_host(h, out):
    """Fills out: float64 (C, Nz, Ny, Nx) (numpy array or CPU torch tensor)."""
    _check(lib.mf_copy_to_host(h, _ptr(out)))
    return out


def mf_copy_fab_to_host(h, box, out):
    _check(lib.mf_copy_fab_to_host(h, int(box), _ptr(out)))
    return out


def mf_copy_fab_from_host(h, box, arr):
    arr = np.ascontiguousarray(arr, dtype=np.float64)
    _check(lib.mf_copy_fab_from_host(h, int(box), _ptr(arr)))


def mf_fill_boundary(h):
    _check(lib.mf_fill_boundary(h))


def mf_interp_cf(fine, crse_old, crse_new, alpha, ratio=2):
    _check(lib.mf_interp_cf(fine, crse_old, crse_new, float(alpha), int(ratio)))


def mf_average_down(fine, crse, ratio=2):
    _check(lib.mf_average_down(fine, crse, int(ratio)))


def _stencil(kind, diffusivity, flags):
    d = np.ascontiguousarray(np.asarray(diffusivity, dtype=np.float64).reshape(-1))
    st = mf_stencil(int(kind), d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(flags))
    return st, d


def mf_advance(h, kind, diffusivity, dt, nsteps, flags=0):
    st, keep = _stencil(kind, diffusivity, flags)
    _check(lib.mf_advance(h, ctypes.byref(st), float(dt), int(nsteps)))
    del keep


def mf_stage_bytes(h):
    return int(lib.mf_stage_bytes(h))


def mf_attach_stage(h, dev_ptr, nbytes):
    _check(lib.mf_attach_stage(h, ctypes.c_void_p(int(dev_ptr)), ctypes.c_size_t(int(nbytes))))


def mf_rk3_advance(h, kind, diffusivity, dt, nsteps, flags=0):
    st, keep = _stencil(kind, diffusivity, flags)
    _check(lib.mf_rk3_advance(h, ctypes.byref(st), float(dt), int(nsteps)))
    del keep


def mf_amr_advance(crse, fine, kind, diffusivity, dt_crse, ncrse_steps, nsub=2, ratio=2, flags=0):
    st, keep = _stencil(kind, diffusivity, flags)
    _check(lib.mf_amr_advance(crse, fine, ctypes.byref(st), float(dt_crse), int(ncrse_steps), int(nsub), int(ratio)))
    del keep


def mf_sum(h, comp=0):
    out = ctypes.c_double()
    _check(lib.mf_sum(h, int(comp), ctypes.byref(out)))
    return out.value


def mf_step_bytes(h, R):
    return float(lib.mf_step_bytes(h, int(R)))


def mf_current(h):
    return _check(lib.mf_current(h))


def mf_set_kernel(h, variant):
    _check(lib.mf_set_kernel(h, int(variant)))


def mf_set_schedule(h, rows=0, stages=0, group_bytes=0):
    _check(lib.mf_set_schedule(h, _ptr(np.array([rows, stages, group_bytes], dtype=np.int32))))


def mf_get_schedule(h):
    out = np.zeros(7, dtype=np.int32)
    _check(lib.mf_get_schedule(h, _ptr(out)))
    return {"tile": tuple(int(v) for v in out[:3]), "rows": int(out[3]), "stages": int(out[4]),
            "kernel": "tma" if out[5] == MF_KERNEL_TMA else "global", "group_bytes": int(out[6]),
            "class_tiles": {k: v for k, v in mf_get_class_tiles(h).items() if v != (-1, -1)}}


def mf_set_timing(h, on):
    _check(lib.mf_set_timing(h, int(bool(on))))


def mf_phase_ms(h):
    out = np.zeros(2, dtype=np.float64)
    _check(lib.mf_phase_ms(h, _ptr(out)))
    return float(out[0]), float(out[1])


def mf_reduce(h, comp, op):
    """Whole-level reduction of one component; op is a name of REDUCTIONS or an MF_RED_* code."""
    out = ctypes.c_double()
    code = REDUCTIONS[op] if isinstance(op, str) else int(op)
    _check(lib.mf_reduce(h, int(comp), code, ctypes.byref(out)))
    return out.value


def mf_launch_count(h):
    """Kernel launches of the last advance: fill, stencil, interp, average-down."""
    out = np.zeros(4, dtype=np.int32)
    _check(lib.mf_launch_count(h, _ptr(out)))
    return {"fill": int(out[0]), "stencil": int(out[1]), "interp": int(out[2]), "avgdown": int(out[3])}


def mf_fp64_fma_rate(stream=0):
    """Measured FP64 FMA throughput (TFLOP/s) of the current GPU."""
    out = ctypes.c_double()
    _check(lib.mf_fp64_fma_rate(ctypes.byref(out), ctypes.c_void_p(int(stream or 0))))
    return out.value


def mf_sum_strided_noalloc(data_ptr, dtype, nx, ny, nz, sy, sz, stream=0):
    """Compensated FP64 sum of a strided device array (element strides sy, sz), allocating
    nothing (scratch in a fixed device array of the library)."""
    out = ctypes.c_double()
    _check(lib.mf_sum_strided_noalloc(ctypes.c_void_p(int(data_ptr)), _dtype_code(dtype), int(nx), int(ny), int(nz),
                                      int(sy), int(sz), ctypes.byref(out), ctypes.c_void_p(int(stream or 0))))
    return out.value


def mf_last_error():
    return lib.mf_last_error().decode(errors="replace")


# ------------------------------------------------------------------ convenience: torch-backed level

def _chop(domain_lo, domain_hi, mgs):
    """The boxes mf_create makes: the domain chopped into max_grid_size blocks, x fastest."""
    lo, hi = _i3(domain_lo), _i3(domain_hi)
    n = (hi - lo + mgs) // mgs
    out = []
    for bz in range(n[2]):
        for by in range(n[1]):
            for bx in range(n[0]):
                a = lo + np.array([bx, by, bz]) * mgs
                out.append(list(a) + list(np.minimum(a + mgs - 1, hi)))
    return np.asarray(out, dtype=np.int32)


class MultiFab:
    """One level on the current CUDA device: a libmf handle plus its torch-allocated field
    memory, attached to the current torch stream."""

    def __init__(self, domain_lo, domain_hi, max_grid_size=None, boxes=None, ncomp=1, ngrow=1, dtype="f64",
                 stream=None, max_region=None):
        """max_region: store the boxes in regions of at most that many cells per side
        (mf_create_regional); boxes=None with max_region chops the domain by max_grid_size
        first."""
        import torch
        if max_region:
            if boxes is None:
                boxes = _chop(domain_lo, domain_hi, max_grid_size)
            self.h = mf_create_regional(domain_lo, domain_hi, boxes, ncomp, ngrow, dtype, max_region)
        elif boxes is None:
            self.h = mf_create(domain_lo, domain_hi, max_grid_size, ncomp, ngrow, dtype)
        else:
            self.h = mf_create_boxes(domain_lo, domain_hi, boxes, ncomp, ngrow, dtype)
        self.domain_lo, self.domain_hi = _i3(domain_lo), _i3(domain_hi)
        self.ncomp, self.ngrow, self.dtype = ncomp, ngrow, dtype
        self.nbytes = mf_bytes(self.h)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        mf_attach(self.h, self.buf.data_ptr(), self.nbytes, self.stream.cuda_stream)

    @property
    def shape(self):
        n = self.domain_hi - self.domain_lo + 1
        return (self.ncomp, int(n[2]), int(n[1]), int(n[0]))

    @property
    def boxes(self):
        return mf_get_boxes(self.h)

    @property
    def regions(self):
        return mf_get_regions(self.h)[0]

    def fab_shape(self, b):
        B = self.boxes[b]
        g = self.ngrow
        return (self.ncomp,) + tuple(int(B[3 + d] - B[d] + 1 + 2 * g) for d in (2, 1, 0))

    def from_host(self, dense):
        mf_copy_from_host(self.h, dense)

    def to_host(self):
        out = np.empty(self.shape, dtype=np.float64)
        return mf_copy_to_host(self.h, out)

    def fab_to_host(self, b):
        out = np.empty(self.fab_shape(b), dtype=np.float64)
        return mf_copy_fab_to_host(self.h, b, out)

    def fab_from_host(self, b, arr):
        mf_copy_fab_from_host(self.h, b, arr)

    def fill_boundary(self):
        mf_fill_boundary(self.h)

    def advance(self, kind, diffusivity, dt, nsteps, flags=0):
        mf_advance(self.h, kind, diffusivity, dt, nsteps, flags)

    def rk3_advance(self, kind, diffusivity, dt, nsteps, flags=0):
        """Third-order SSP Runge-Kutta steps; allocates and attaches the stage level once."""
        if getattr(self, "stage_buf", None) is None:
            import torch
            nb = mf_stage_bytes(self.h)
            self.stage_buf = torch.empty(nb, dtype=torch.uint8, device=self.buf.device)
            mf_attach_stage(self.h, self.stage_buf.data_ptr(), nb)
        mf_rk3_advance(self.h, kind, diffusivity, dt, nsteps, flags)

    def sum(self, comp=0):
        return mf_sum(self.h, comp)

    def reduce(self, op, comp=0):
        return mf_reduce(self.h, comp, op)

    def set_tile(self, tile):
        mf_set_tile(self.h, tile)

    def step_bytes(self, R):
        return mf_step_bytes(self.h, R)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and lib is not None:
            lib.mf_destroy(h)
            self.h = None
