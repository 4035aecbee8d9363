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
* ``CFFaces`` / ``cf_coarse_flux`` / ``cf_fine_flux`` / ``reflux`` -- flux correction at the
                         coarse-fine interface of the subcycled two-level step (the paper names
                         it without a formula; read as Berger-Colella): the coarse faces of
                         uncovered cells next to the fine region, their coarse flux and the sum of
                         their r^2 fine face fluxes, and the correction of the coarse cell.

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
    """Compile the C oracle (plain gcc, no CUDA; with OpenMP for orc_advance_omp where gcc has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
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
            L.orc_advance_omp.restype = I
            L.orc_advance_omp.argtypes = [I, P, P, P, I, I, I, P, P, I, P, P]
            L.orc_omp_threads.restype = I
            L.orc_omp_threads.argtypes = []
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


def advance_omp(level, data, R, lam, nsteps):
    """advance with the paper's threaded loop (Sec. 3.3): the boxes of each phase shared among
    OpenMP threads; the same bits as advance.  A CPU baseline, not part of the compared method."""
    lam = _lam_array(level, lam)
    b = np.array([float(x) for x in coeffs.flux_coefficients(R)], dtype=np.float64)
    a = np.array(data, dtype=np.float64, copy=True)
    other = level.alloc()
    which = lib().orc_advance_omp(level.nbox, _p(level.boxes), _p(level.dlo), _p(level.dhi), level.g, level.C,
                                  int(R), _p(b), _p(lam), int(nsteps), _p(a), _p(other))
    return a if which == 0 else other


def omp_threads():
    """Threads advance_omp uses (1 without OpenMP)."""
    return int(lib().orc_omp_threads())


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


class CFFaces:
    """The coarse-fine faces of a refined level, for refluxing (reading of the paper's
    subcycling: Berger-Colella flux correction).  A fine face is a coarse-fine face when the
    fine cell on its outside (periodic images included) lies in no fine box; the r^2 fine faces
    on one face of an uncovered coarse cell C form one coarse face.  Fine boxes must consist of
    whole coarse cells.

    For each coarse face: the coarse cell C (global index), the direction d and sc = +1 when the
    fine region is on C's high side in d (-1 on its low side).  For each fine box face: the
    coarse-face id of every fine face (-1 where the outside is another fine box)."""

    def __init__(self, crse, fine, ratio):
        r = int(ratio)
        flo, fhi = fine.dlo.astype(int), fine.dhi.astype(int)
        Lf = fhi - flo + 1
        clo = crse.dlo.astype(int)
        cov = np.zeros((Lf[2], Lf[1], Lf[0]), dtype=bool)  # fine domain coverage, (z, y, x)
        for b in fine.boxes:
            if any((b[d] - flo[d]) % r or (b[3 + d] - flo[d] + 1) % r for d in range(3)):
                raise ValueError("fine boxes must consist of whole coarse cells")
            cov[b[2] - flo[2]:b[5] - flo[2] + 1, b[1] - flo[1]:b[4] - flo[1] + 1, b[0] - flo[0]:b[3] - flo[0] + 1] = True
        keys = {}
        self.slabs = []
        for bi, b in enumerate(fine.boxes):
            lo, hi = np.array(b[:3]), np.array(b[3:])
            for d in range(3):
                e = [a for a in range(3) if a != d]  # the two in-face directions, increasing
                for s in (-1, 1):
                    inside = hi[d] if s > 0 else lo[d]
                    out = inside + s
                    ga = np.arange(lo[e[0]], hi[e[0]] + 1)
                    gb = np.arange(lo[e[1]], hi[e[1]] + 1)
                    A, B = np.meshgrid(ga, gb, indexing="ij")  # (n_a, n_b) fine indices in the face
                    P = [None, None, None]
                    P[d] = np.full(A.shape, out)
                    P[e[0]], P[e[1]] = A, B
                    W = [(P[k] - flo[k]) % Lf[k] for k in range(3)]  # wrapped outside cell
                    unc = ~cov[W[2], W[1], W[0]]
                    cid = np.full(A.shape, -1, dtype=np.int64)
                    if unc.any():
                        Cg = [(W[k] // r) + clo[k] for k in range(3)]  # coarse cell outside (wrapped)
                        for ia, ib in zip(*np.nonzero(unc)):
                            key = (int(Cg[0][ia, ib]), int(Cg[1][ia, ib]), int(Cg[2][ia, ib]), d, -s)
                            if key not in keys:
                                keys[key] = len(keys)
                            cid[ia, ib] = keys[key]
                    self.slabs.append((bi, d, s, e, cid))
        self.faces = np.array(sorted(keys, key=keys.get), dtype=np.int64).reshape(-1, 5)
        self.r = r

    @property
    def n(self):
        return self.faces.shape[0]


def _line_flux(vals, b):
    """F = sum_m b_m (v[R-1+m] - v[R-m]) over a line of 2R values (axis 0) across a face."""
    R = len(b)
    f = np.zeros(vals.shape[1:])
    for m in range(1, R + 1):
        f = f + b[m - 1] * (vals[R - 1 + m] - vals[R - m])
    return f


def cf_fine_flux(fine, cf, R, fdata):
    """Per coarse face and component: the sum of the face fluxes F of its r^2 fine faces, each
    from the fine box inside (its ghost cells hold the outside values); shape (C, nfaces)."""
    b = [float(x) for x in coeffs.flux_coefficients(R)]
    acc = np.zeros((fine.C, cf.n))
    g = fine.g
    for bi, d, s, e, cid in cf.slabs:
        if not (cid >= 0).any():
            continue
        lo, hi = fine.boxes[bi, :3], fine.boxes[bi, 3:]
        F = fine.fab(fdata, bi)  # (C, z, y, x) with ghosts
        inside = (hi[d] if s > 0 else lo[d]) - lo[d] + g  # local index along d
        low = inside if s > 0 else inside - 1  # lower cell of the face
        vals = []
        for k in range(-R + 1, R + 1):
            sl = [slice(None)] * 4
            sl[3 - d] = low + k
            for a in e:
                sl[3 - a] = slice(g, g + hi[a] - lo[a] + 1)
            v = F[tuple(sl)]  # (C, n_e1, n_e0) in (z, y, x) order without the d axis
            vals.append(np.transpose(v, (0, 2, 1)))  # (C, n_e0, n_e1) = (C, n_a, n_b)
        fl = _line_flux(np.stack(vals), b)  # (C, n_a, n_b)
        m = cid >= 0
        for c in range(fine.C):
            np.add.at(acc[c], cid[m], fl[c][m])
    return acc


def cf_coarse_flux(crse, cf, R, cdata):
    """Per coarse face and component: the coarse face flux F, from the (periodic) coarse level."""
    b = [float(x) for x in coeffs.flux_coefficients(R)]
    dense = crse.to_dense(cdata)  # (C, z, y, x)
    L = crse.dhi.astype(int) - crse.dlo.astype(int) + 1
    clo = crse.dlo.astype(int)
    out = np.zeros((crse.C, cf.n))
    for i, (x, y, z, d, sc) in enumerate(cf.faces):
        low = np.array([x, y, z]) - clo
        if sc < 0:
            low[d] -= 1
        vals = []
        for k in range(-R + 1, R + 1):
            p = low.copy()
            p[d] += k
            p = p % L
            vals.append(dense[:, p[2], p[1], p[0]])
        out[:, i] = _line_flux(np.stack(vals), b)
    return out


def reflux(crse, cf, corr, cdata):
    """Add corr[c, face] to the coarse cell of each coarse face (in place, valid cells)."""
    dense = crse.to_dense(cdata)
    clo = crse.dlo.astype(int)
    for i, (x, y, z, d, sc) in enumerate(cf.faces):
        dense[:, z - clo[2], y - clo[1], x - clo[0]] += corr[:, i]
    cdata[:] = crse.from_dense(dense)


def amr_advance(crse, fine, R, lam_c, cdata, fdata, ncrse_steps, nsub=2, ratio=2, reflux_faces=False):
    """Two-level step (reading of Sec. 3's subcycling): per coarse step, FillBoundary and
    stencil on the coarse level (lam_c); then nsub fine substeps, each FillBoundary, coarse-fine
    interpolation at alpha = s/nsub between the coarse old and new data, and the fine stencil
    with lam_f = lam_c * ratio^2 / nsub; then average-down onto the new coarse data.
    With reflux_faces, every uncovered coarse cell next to a coarse-fine face then trades the
    coarse face flux for the time- and area-average of the fine ones (Berger-Colella):
    u_C += sc * (lam_f / r^3 * sum over substeps and the r^2 fine faces of F_f - lam_c * F_c).
    Returns (cdata, fdata) new arrays."""
    lam_c = _lam_array(crse, lam_c)
    lam_f = lam_c * (ratio * ratio) / nsub
    c_cur = np.array(cdata, dtype=np.float64, copy=True)
    f_cur = np.array(fdata, dtype=np.float64, copy=True)
    c_new, f_new = crse.alloc(), fine.alloc()
    cf = CFFaces(crse, fine, ratio) if reflux_faces else None
    for _ in range(ncrse_steps):
        fill_boundary(crse, c_cur)
        if cf is not None:
            fc = lam_c[:, None] * cf_coarse_flux(crse, cf, R, c_cur)
            ff = np.zeros_like(fc)
        stencil(crse, R, lam_c, c_cur, c_new)
        for s in range(nsub):
            fill_boundary(fine, f_cur)
            interp_cf(fine, crse, ratio, s / nsub, c_cur, c_new, f_cur)
            if cf is not None:
                ff += (lam_f / ratio ** 3)[:, None] * cf_fine_flux(fine, cf, R, f_cur)
            stencil(fine, R, lam_f, f_cur, f_new)
            f_cur, f_new = f_new, f_cur
        average_down(fine, crse, ratio, f_cur, c_new)
        if cf is not None:
            reflux(crse, cf, cf.faces[:, 4][None, :] * (ff - fc), c_new)
        c_cur, c_new = c_new, c_cur
    return c_cur, f_cur
