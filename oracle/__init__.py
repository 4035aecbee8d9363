"""Plain FP64 CPU oracle for the MultiFab time-step sweep of "BoxLib with Tiling".

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.  The product
library never imports, links or calls it, and it imports nothing from the product.

What each function follows (section of arXiv 1604.03570):

* ``chop``            -- a level is a set of non-intersecting Boxes (Sec. 3); the domain is
                         cut into boxes of at most max_grid_size cells per side.
* ``Level``           -- FArrayBoxes over grown boxes, x fastest then y, z, component (Sec. 3.1).
* ``fill_boundary``   -- mf.FillBoundary() (Sec. 3.1): every ghost cell takes the value of
                         the valid cell owning the same point of the periodic domain.
* ``stencil``         -- the heat-equation kernel of Sec. 4.1: face fluxes in one loop per
                         direction, then the divergence, forward Euler, out of place; R = 1
                         is the paper's second-order scheme, R = 4 the 9-cell-wide 8th-order
                         stencil of Sec. 4.2.  ``form="direct"`` is a cross-check only.
* ``advance``         -- nsteps x (FillBoundary, stencil, swap) (Sec. 4.1).
* ``rk3_advance``     -- the third-order Runge-Kutta integration of Sec. 4.2 (SMC), read as the
                         three-stage SSP scheme: each stage a FillBoundary and a forward-Euler
                         stencil step, combined with the state at the start of the step.
* ``domain_sum``      -- the whole-level reduction (Sec. 3.1, mf.max(0) is the example), here
                         the sum of one component over the valid cells, correctly rounded
                         (Shewchuk's exact summation as implemented by ``math.fsum``).
* ``reduce``          -- the other MultiFab reductions of Sec. 3.1 by their definitions: max,
                         min, max |u|, sum |u| (correctly rounded), and the 2-norm.
* ``interp_cf`` / ``average_down`` / ``amr_advance`` -- the inter-level operations of a
                         refined level (Sec. 3, ratio 2 or 4); the paper gives no formula, the
                         readings are trilinear space / linear time interpolation of uncovered
                         fine ghosts, the mean of the children, and a coarse step followed by
                         ``nsub`` fine substeps and an average-down.

The C part (``mf_oracle.c``) is compiled with ``gcc -O2 -ffp-contract=off`` on first use.
"""
import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import coeffs

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB = os.path.join(_HERE, "_liborc.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C oracle (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            I, P, D, LNG = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_long
            L.orc_fab_offset.restype = LNG
            L.orc_fab_offset.argtypes = [I, P, I, I, I]
            L.orc_level_size.restype = LNG
            L.orc_level_size.argtypes = [I, P, I, I]
            L.orc_chop.restype = I
            L.orc_chop.argtypes = [P, P, I, P, I]
            L.orc_fabs_from_dense.argtypes = [I, P, P, P, I, I, P, P]
            L.orc_dense_from_fabs.argtypes = [I, P, P, P, I, I, P, P]
            L.orc_fill_boundary.restype = LNG
            L.orc_fill_boundary.argtypes = [I, P, P, P, I, I, P]
            L.orc_stencil_flux.argtypes = [I, P, I, I, I, P, P, P, P]
            L.orc_stencil_direct.argtypes = [I, P, I, I, I, P, P, P, P]
            L.orc_advance.restype = I
            L.orc_advance.argtypes = [I, P, P, P, I, I, I, P, P, I, P, P]
            L.orc_interp_cf.restype = LNG
            L.orc_interp_cf.argtypes = [I, P, P, P, I, I, P, P, P, I, I, I, D, P, P, P]
            L.orc_average_down.restype = LNG
            L.orc_average_down.argtypes = [I, P, I, I, P, I, I, I, P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))


def chop(domain_lo, domain_hi, max_grid_size):
    """Boxes (n, 6) int32 {lo, hi} inclusive; the last box per direction takes the remainder,
    box index x fastest, then y, then z."""
    dlo, dhi = _i3(domain_lo), _i3(domain_hi)
    n = lib().orc_chop(_p(dlo), _p(dhi), int(max_grid_size), None, 0)
    out = np.zeros((n, 6), dtype=np.int32)
    lib().orc_chop(_p(dlo), _p(dhi), int(max_grid_size), _p(out), n)
    return out


class Level:
    """Box layout of one MultiFab: boxes, periodic domain, ghost width, components."""

    def __init__(self, boxes, domain_lo, domain_hi, ngrow, ncomp):
        self.boxes = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 6))
        self.dlo, self.dhi = _i3(domain_lo), _i3(domain_hi)
        self.g, self.C = int(ngrow), int(ncomp)
        self.nbox = self.boxes.shape[0]
        self.size = lib().orc_level_size(self.nbox, _p(self.boxes), self.g, self.C)

    @property
    def shape(self):
        return tuple(int(h - l + 1) for l, h in zip(self.dlo[::-1], self.dhi[::-1]))

    def alloc(self):
        return np.full(self.size, np.nan, dtype=np.float64)

    def from_dense(self, dense):
        dense = np.ascontiguousarray(dense, dtype=np.float64)
        assert dense.size == self.C * int(np.prod(self.shape))
        out = np.empty(self.size, dtype=np.float64)
        lib().orc_fabs_from_dense(self.nbox, _p(self.boxes), _p(self.dlo), _p(self.dhi), self.g, self.C,
                                  _p(dense), _p(out))
        return out

    def to_dense(self, data, fill=np.nan):
        dense = np.full((self.C,) + self.shape, fill, dtype=np.float64)
        lib().orc_dense_from_fabs(self.nbox, _p(self.boxes), _p(self.dlo), _p(self.dhi), self.g, self.C,
                                  _p(np.ascontiguousarray(data)), _p(dense))
        return dense

    def fab(self, data, b):
        """View of FArrayBox b as (C, nz+2g, ny+2g, nx+2g)."""
        off = lib().orc_fab_offset(self.nbox, _p(self.boxes), self.g, self.C, int(b))
        lo, hi = self.boxes[b, :3], self.boxes[b, 3:]
        n = [int(h - l + 1 + 2 * self.g) for l, h in zip(lo, hi)]
        cnt = self.C * n[0] * n[1] * n[2]
        return data[off:off + cnt].reshape(self.C, n[2], n[1], n[0])


def fill_boundary(level, data):
    """FillBoundary in place; returns ghost cells written per component."""
    assert data.dtype == np.float64 and data.size == level.size
    return lib().orc_fill_boundary(level.nbox, _p(level.boxes), _p(level.dlo), _p(level.dhi), level.g, level.C,
                                   _p(data))


def _lam_array(level, lam):
    lam = np.asarray(lam, dtype=np.float64).reshape(-1)
    if lam.size == 1:
        lam = np.repeat(lam, level.C)
    assert lam.size == level.C
    return np.ascontiguousarray(lam)


def stencil(level, R, lam, src, dst, form="flux"):
    """One forward-Euler stencil application src -> dst on the valid cells (lam = D_c dt/dx^2)."""
    lam = _lam_array(level, lam)
    if form == "flux":
        b = np.array([float(x) for x in coeffs.flux_coefficients(R)], dtype=np.float64)
        lib().orc_stencil_flux(level.nbox, _p(level.boxes), level.g, level.C, int(R), _p(b), _p(lam), _p(src), _p(dst))
    elif form == "direct":
        c = np.array([float(x) for x in coeffs.laplacian_coefficients(R)], dtype=np.float64)
        lib().orc_stencil_direct(level.nbox, _p(level.boxes), level.g, level.C, int(R), _p(c), _p(lam), _p(src), _p(dst))
    else:
        raise ValueError(form)
    return dst


def advance(level, data, R, lam, nsteps):
    """nsteps x (FillBoundary, flux-form stencil, swap); returns the new FArrayBox storage."""
    lam = _lam_array(level, lam)
    b = np.array([float(x) for x in coeffs.flux_coefficients(R)], dtype=np.float64)
    a = np.array(data, dtype=np.float64, copy=True)
    other = level.alloc()
    which = lib().orc_advance(level.nbox, _p(level.boxes), _p(level.dlo), _p(level.dhi), level.g, level.C, int(R),
                              _p(b), _p(lam), int(nsteps), _p(a), _p(other))
    return a if which == 0 else other


# Stage weights of the three-stage SSP Runge-Kutta scheme: stage s returns
# a_s * u + b_s * E(v_s), E the forward-Euler step, u the state at the start of the step.
RK3_STAGES = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def rk3_advance(level, data, R, lam, nsteps):
    """nsteps of the third-order Runge-Kutta time integration of Sec. 4.2, read as the
    three-stage strong-stability-preserving scheme of Shu and Osher (1988):
        u1 = E(u),  u2 = 3/4 u + 1/4 E(u1),  u_new = 1/3 u + 2/3 E(u2),
    where E(v) = v + lam * div F(v) is one forward-Euler flux-form step (``stencil``) after a
    FillBoundary of v.  Returns the new FArrayBox storage (valid cells defined)."""
    u = np.array(data, dtype=np.float64, copy=True)
    e = level.alloc()
    for _ in range(nsteps):
        v = u
        for a, b in RK3_STAGES:
            fill_boundary(level, v)
            stencil(level, R, lam, v, e)
            v = e.copy() if a == 0.0 else a * u + b * e
        u = v
    return u


def domain_sum(level, data, comp=0):
    """Correctly rounded sum of component comp over all valid cells (math.fsum)."""
    g = level.g
    parts = []
    for b in range(level.nbox):
        f = level.fab(data, b)[comp]
        nz, ny, nx = f.shape
        parts.append(f[g:nz - g, g:ny - g, g:nx - g].ravel())
    return math.fsum(np.concatenate(parts).tolist()) if parts else 0.0


def _valid_cells(level, data, comp):
    g = level.g
    parts = []
    for b in range(level.nbox):
        f = level.fab(data, b)[comp]
        nz, ny, nx = f.shape
        parts.append(f[g:nz - g, g:ny - g, g:nx - g].ravel())
    return np.concatenate(parts)


def reduce(level, data, op, comp=0):
    """The MultiFab reductions of Sec. 3.1 (mf.max(0) is the paper's example) over the valid
    cells of component comp, each by its definition: "sum" (correctly rounded, math.fsum),
    "max", "min", "norm0" (max |u|), "norm1" (sum |u|, correctly rounded) and "norm2"
    (square root of the correctly rounded sum of the FP64 squares).  NaN values are skipped by
    the max-type reductions."""
    v = _valid_cells(level, data, comp)
    if op == "sum":
        return math.fsum(v.tolist())
    if op == "norm1":
        return math.fsum(np.abs(v).tolist())
    if op == "norm2":
        return math.sqrt(math.fsum((v * v).tolist()))
    v = v[~np.isnan(v)]
    if op == "max":
        return float(np.max(v))
    if op == "min":
        return float(np.min(v))
    if op == "norm0":
        return float(np.max(np.abs(v)))
    raise ValueError("unknown reduction %r" % (op,))


def interp_cf(fine, crse, ratio, alpha, c_old, c_new, fdata):
    """Fill the fine ghost cells no fine box covers by trilinear-in-space, linear-in-time
    interpolation of the coarse level (in place); returns cells written per component."""
    assert fine.C == crse.C
    n = lib().orc_interp_cf(fine.nbox, _p(fine.boxes), _p(fine.dlo), _p(fine.dhi), fine.g,
                            crse.nbox, _p(crse.boxes), _p(crse.dlo), _p(crse.dhi), crse.g,
                            fine.C, int(ratio), float(alpha), _p(c_old), _p(c_new), _p(fdata))
    if n < 0:
        raise ValueError("coarse level does not cover its domain")
    return n


def average_down(fine, crse, ratio, fdata, cdata):
    """Coarse cells covered by fine boxes become the mean of their children (in place)."""
    return lib().orc_average_down(fine.nbox, _p(fine.boxes), fine.g, crse.nbox, _p(crse.boxes), crse.g,
                                  fine.C, int(ratio), _p(fdata), _p(cdata))


def amr_advance(crse, fine, R, lam_c, cdata, fdata, ncrse_steps, nsub=2, ratio=2):
    """Two-level step (reading of Sec. 3's subcycling): per coarse step, FillBoundary and
    stencil on the coarse level (lam_c); then nsub fine substeps, each FillBoundary, coarse-fine
    interpolation at alpha = s/nsub between the coarse old and new data, and the fine stencil
    with lam_f = lam_c * ratio^2 / nsub; then average-down onto the new coarse data.
    No refluxing.  Returns (cdata, fdata) new arrays."""
    lam_c = _lam_array(crse, lam_c)
    lam_f = lam_c * (ratio * ratio) / nsub
    c_cur = np.array(cdata, dtype=np.float64, copy=True)
    f_cur = np.array(fdata, dtype=np.float64, copy=True)
    c_new, f_new = crse.alloc(), fine.alloc()
    for _ in range(ncrse_steps):
        fill_boundary(crse, c_cur)
        stencil(crse, R, lam_c, c_cur, c_new)
        for s in range(nsub):
            fill_boundary(fine, f_cur)
            interp_cf(fine, crse, ratio, s / nsub, c_cur, c_new, f_cur)
            stencil(fine, R, lam_f, f_cur, f_new)
            f_cur, f_new = f_new, f_cur
        average_down(fine, crse, ratio, f_cur, c_new)
        c_cur, c_new = c_new, c_cur
    return c_cur, f_cur
