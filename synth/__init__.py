"""Seeded synthetic inputs for the MultiFab sweep: initial fields, box lists, workload table.

This module holds none of the method's arithmetic (no ghost fill, no stencil, no
interpolation).  It only draws numbers and lays out problems, and it serves both the
product tests/benchmark and the oracle, so that both sides see identical inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator: the value for
(seed, stream, index) is the SplitMix64 output function applied to a key derived from the
seed and stream plus (index + 1) times the golden-ratio increment.  Fields are therefore
independent of the box layout.

The workloads stand in for the paper's heat-equation test (Sec. 4.1, one periodic 128^3
grid) and its 8th-order SMC stencil (Sec. 4.2), scaled to one GB300; no dataset is used.
"""
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

FIELD_SEED = 1604
BOX_SEED = 3570


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed) * GOLDEN + np.uint64(stream) * _M2 + GOLDEN)


def splitmix64(seed, stream, index):
    """uint64 draws for integer indices (array-like) under (seed, stream)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed, stream) + (idx + np.uint64(1)) * GOLDEN)


def uniform(seed, stream, index, lo=0.0, hi=1.0):
    """Doubles in [lo, hi) from the top 53 bits of each draw."""
    u = (splitmix64(seed, stream, index) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


class Rng:
    """Sequential draws on one (seed, stream) counter, for box generators."""

    def __init__(self, seed, stream):
        self.seed, self.stream, self.n = seed, stream, 0

    def u(self):
        v = float(uniform(self.seed, self.stream, [self.n])[0])
        self.n += 1
        return v

    def randint(self, lo, hi):
        """Integer in [lo, hi] inclusive."""
        return lo + min(int(self.u() * (hi - lo + 1)), hi - lo)


# ------------------------------------------------------------------ fields

def sine_modes(seed, stream, nmodes, kmax):
    """nmodes random Fourier modes: wavevector components uniform in +-{1..kmax},
    amplitudes U(0.5, 1)/nmodes, phases U(0, 2 pi)."""
    draws = uniform(seed, stream, np.arange(nmodes * 8))
    modes = []
    for m in range(nmodes):
        d = draws[8 * m: 8 * m + 8]
        k = []
        for j in range(3):
            mag = 1 + min(int(d[j] * kmax), kmax - 1)
            sign = -1 if d[3 + j] < 0.5 else 1
            k.append(sign * mag)
        amp = (0.5 + 0.5 * d[6]) / nmodes
        phase = 2.0 * math.pi * d[7]
        modes.append((tuple(k), amp, phase))
    return modes


def eval_modes(shape, modes, scale=None):
    """Sum_m a_m sin(2 pi k_m . x + phi_m) at cell centres x_d = (i + 1/2) / N_d of a periodic
    unit cube of the given (Nz, Ny, Nx) shape; returns float64 (Nz, Ny, Nx)."""
    Nz, Ny, Nx = shape
    out = np.zeros(shape, dtype=np.float64)
    xs = [(np.arange(n) + 0.5) / n for n in (Nx, Ny, Nz)]
    for k, a, ph in modes:
        ex = np.exp(2j * math.pi * k[0] * xs[0])
        ey = np.exp(2j * math.pi * k[1] * xs[1])
        ez = np.exp(2j * math.pi * k[2] * xs[2]) * np.exp(1j * ph)
        for z0 in range(0, Nz, 32):
            z1 = min(Nz, z0 + 32)
            blk = ez[z0:z1, None, None] * (ey[None, :, None] * ex[None, None, :])
            out[z0:z1] += a * blk.imag
    return out


def eval_modes_box(N, lo, shape, modes):
    """eval_modes restricted to the cells lo .. lo + shape - 1 (x, y, z lower corner; shape in
    (nz, ny, nx) order) of a periodic N^3 grid: the same values as the matching block of
    eval_modes((N, N, N), modes)."""
    nz, ny, nx = shape
    out = np.zeros(shape, dtype=np.float64)
    xs = [(lo[0] + np.arange(nx) + 0.5) / N, (lo[1] + np.arange(ny) + 0.5) / N, (lo[2] + np.arange(nz) + 0.5) / N]
    for k, a, ph in modes:
        ex = np.exp(2j * math.pi * k[0] * xs[0])
        ey = np.exp(2j * math.pi * k[1] * xs[1])
        ez = np.exp(2j * math.pi * k[2] * xs[2]) * np.exp(1j * ph)
        for z0 in range(0, nz, 32):
            z1 = min(nz, z0 + 32)
            blk = ez[z0:z1, None, None] * (ey[None, :, None] * ex[None, None, :])
            out[z0:z1] += a * blk.imag
    return out


def single_mode(shape, k, phase=0.3):
    """sin(2 pi k . x + phase) on the cell centres (the pure mode of the decay test)."""
    return eval_modes(shape, [(tuple(k), 1.0, phase)])


def noise(seed, stream, shape, amp):
    """Uniform noise in [-amp, amp), keyed by the global linear index."""
    n = int(np.prod(shape))
    return uniform(seed, stream, np.arange(n), -amp, amp).reshape(shape)


def gaussian_plus_noise(N, seed=FIELD_SEED):
    """exp(-r^2 / 0.01) about the domain centre (non-periodic r) plus U(-1e-3, 1e-3) noise."""
    x = (np.arange(N) + 0.5) / N - 0.5
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    return np.exp(-r2 / 0.01) + noise(seed, 1, (N, N, N), 1e-3)


# ------------------------------------------------------------------ box lists

def uneven_boxes(N, target, seed=BOX_SEED, base=32, quantum=8):
    """Many-small-box layout: cut the periodic N^3 domain into base^3 boxes, then keep
    splitting seeded boxes that have a side >= 2*quantum, along their longest side at a
    seeded multiple of quantum, until there are `target` boxes.  Sides end up in
    {quantum, ..., base}.  Returns int32 (target, 6) {lo, hi} inclusive."""
    nb = N // base
    boxes = []
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                lo = (bx * base, by * base, bz * base)
                boxes.append([lo[0], lo[1], lo[2], lo[0] + base - 1, lo[1] + base - 1, lo[2] + base - 1])
    if target < len(boxes):
        raise ValueError("target below the base box count")
    rng = Rng(seed, 7)

    def can_split(bb):
        return max(bb[3] - bb[0], bb[4] - bb[1], bb[5] - bb[2]) + 1 >= 2 * quantum

    # indices of the splittable boxes in increasing order: a split changes box i in place (it
    # stays at its position or leaves the list) and appends the new box (largest index)
    splittable = [i for i, b in enumerate(boxes) if can_split(b)]
    while len(boxes) < target:
        if not splittable:
            raise ValueError("cannot reach target")
        pick = rng.randint(0, len(splittable) - 1)
        i = splittable[pick]
        b = boxes[i]
        ext = [b[3] - b[0] + 1, b[4] - b[1] + 1, b[5] - b[2] + 1]
        d = max(range(3), key=lambda e: (ext[e], -e))
        npieces = ext[d] // quantum
        cut = rng.randint(1, npieces - 1) * quantum
        a = list(b)
        c = list(b)
        a[3 + d] = b[d] + cut - 1
        c[d] = b[d] + cut
        boxes[i] = a
        boxes.append(c)
        if not can_split(a):
            splittable.pop(pick)
        if can_split(c):
            splittable.append(len(boxes) - 1)
    return np.asarray(boxes, dtype=np.int32)


def sphere_fine_boxes(Nc, ratio=2, radius=0.25, seed=BOX_SEED, blocking=8, min_side=16, max_side=64):
    """Fine-level boxes covering a tagged sphere.  Coarse cells whose centre lies within
    `radius` of the domain centre are tagged; fine blocks of `blocking`^3 cells containing a
    tagged cell are marked; the fine bounding box is split recursively along its longest side
    at seeded multiples of `blocking` (both halves >= min_side) until every side is
    <= max_side; each leaf shrinks to the bounding box of its marked blocks, re-grown to
    >= min_side inside the leaf; empty leaves are dropped.  Returns fine-index boxes
    int32 (n, 6) inside [0, Nc*ratio)^3."""
    Nf = Nc * ratio
    x = (np.arange(Nc) + 0.5) / Nc - 0.5
    tag = (x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2) <= radius * radius
    cpb = blocking // ratio  # coarse cells per block side
    nbk = Nf // blocking
    blk = tag.reshape(nbk, cpb, nbk, cpb, nbk, cpb).any(axis=(1, 3, 5))  # (z, y, x) blocks
    zz, yy, xx = np.nonzero(blk)
    lo = [int(xx.min()), int(yy.min()), int(zz.min())]
    hi = [int(xx.max()), int(yy.max()), int(zz.max())]
    minb, maxb = min_side // blocking, max_side // blocking
    rng = Rng(seed, 11)
    leaves = []
    stack = [(lo, hi)]
    while stack:
        l, h = stack.pop()
        ext = [h[d] - l[d] + 1 for d in range(3)]
        d = max(range(3), key=lambda e: (ext[e], -e))
        if ext[d] <= maxb:
            leaves.append((l, h))
            continue
        cut = rng.randint(minb, ext[d] - minb)
        h1 = list(h)
        h1[d] = l[d] + cut - 1
        l2 = list(l)
        l2[d] = l[d] + cut
        stack.append((l2, h))
        stack.append((l, h1))
    out = []
    for l, h in leaves:
        sub = blk[l[2]:h[2] + 1, l[1]:h[1] + 1, l[0]:h[0] + 1]
        if not sub.any():
            continue
        z, y, xq = np.nonzero(sub)
        sl = [int(xq.min()) + l[0], int(y.min()) + l[1], int(z.min()) + l[2]]
        sh = [int(xq.max()) + l[0], int(y.max()) + l[1], int(z.max()) + l[2]]
        for d in range(3):
            while sh[d] - sl[d] + 1 < minb:
                if sh[d] < h[d]:
                    sh[d] += 1
                else:
                    sl[d] -= 1
        out.append([sl[0] * blocking, sl[1] * blocking, sl[2] * blocking,
                    (sh[0] + 1) * blocking - 1, (sh[1] + 1) * blocking - 1, (sh[2] + 1) * blocking - 1])
    return np.asarray(out, dtype=np.int32)


# ------------------------------------------------------------------ workload table

def heat_dt(N, R, D_max=1.0, safety=0.9):
    """Forward-Euler step at `safety` times the stability limit lam * 3 * |sigma_R(pi)| <= 2
    with |sigma_1(pi)| = 4, |sigma_2(pi)| = 16/3, |sigma_4(pi)| = 2048/315."""
    smax = {1: 4.0, 2: 16.0 / 3.0, 4: 2048.0 / 315.0}[R]
    dx = 1.0 / N
    return safety * 2.0 * dx * dx / (3.0 * smax * D_max)


WORKLOADS = {
    "c1": dict(name="heat64_fp64_8x32", N=64, max_grid_size=32, ngrow=1, ncomp=1, R=1,
               dtypes=("f64",), nsteps=10, init="gaussian"),
    "c2": dict(name="heat256_64x64", N=256, max_grid_size=64, ngrow=1, ncomp=1, R=1,
               dtypes=("f64", "f32"), nsteps=100, init="modes", nmodes=8, kmax=16, tile=(64, 8, 8)),
    "c3": dict(name="diff8th512_c5", N=512, max_grid_size=128, ngrow=4, ncomp=5, R=4,
               dtypes=("f64", "f32"), nsteps=20, init="modes+noise", nmodes=8, kmax=8, noise=1e-6),
    "c4": dict(name="amr2lev256_sphere", N=256, max_grid_size=64, ngrow=1, ncomp=1, R=1,
               dtypes=("f32",), nsteps=50, nsub=2, ratio=2, init="modes", nmodes=8, kmax=16),
    "c5": dict(name="manybox512_c2", N=512, ngrow=2, ncomp=2, R=2, dtypes=("f32", "f64"), nsteps=50,
               init="modes", nmodes=8, kmax=16, targets=(4096, 8192, 16384, 32768)),
}


def diffusivities(cfg, seed=FIELD_SEED):
    """Per-component diffusivity: 1, except the 8th-order workload draws U(0.5, 2)."""
    C = cfg["ncomp"]
    if cfg.get("R") == 4:
        return uniform(seed, 5, np.arange(C), 0.5, 2.0)
    return np.ones(C)


def dt_for(cfg, N=None):
    """Time step: c1/c2 use 0.9 dx^2/6 (lam = 0.15); the 8th-order workload uses the bound
    for D = 2; the AMR workload halves the coarse dt so that two fine substeps at ratio 2
    stay at lam_f = 0.15."""
    N = N or cfg["N"]
    if cfg.get("nsub"):
        return 0.5 * heat_dt(N, cfg["R"])
    if cfg["R"] == 4:
        return heat_dt(N, 4, D_max=2.0)
    return heat_dt(N, cfg["R"])


def initial_field(cfg, N=None, seed=FIELD_SEED):
    """Dense float64 (C, N, N, N) initial data for a workload (optionally at another N)."""
    N = N or cfg["N"]
    C = cfg["ncomp"]
    shape = (N, N, N)
    if cfg["init"] == "gaussian":
        return gaussian_plus_noise(N, seed)[None]
    out = np.empty((C,) + shape, dtype=np.float64)
    for c in range(C):
        out[c] = eval_modes(shape, sine_modes(seed, 100 + c, cfg["nmodes"], cfg["kmax"]))
        if "noise" in cfg["init"]:
            out[c] += noise(seed, 200 + c, shape, cfg["noise"])
    return out


# ------------------------------------------------------------------ the same fields on a device

def _u64(v):
    """A uint64 constant as the int64 with the same bits (torch has no uint64 arithmetic)."""
    v = int(v) & 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _torch_mix(z):
    """The SplitMix64 output function on int64 tensors holding uint64 bits (wrapping products,
    logical right shifts)."""
    def shr(x, s):
        return (x >> s) & ((1 << (64 - s)) - 1)
    z = (z ^ shr(z, 30)) * _u64(_M1)
    z = (z ^ shr(z, 27)) * _u64(_M2)
    return z ^ shr(z, 31)


def initial_field_device(cfg, device, N=None, seed=FIELD_SEED, comps=None):
    """initial_field evaluated with torch on `device` (float64 (C, N, N, N)): the same modes and
    the same counter-based noise draws, for workloads too large to generate on the host in a
    benchmark.  Agrees with initial_field to rounding (the sines are evaluated in a different
    order of operations)."""
    import torch
    N = N or cfg["N"]
    C = cfg["ncomp"]
    comps = range(C) if comps is None else comps
    out = torch.empty((len(comps), N, N, N), dtype=torch.float64, device=device)
    x = (torch.arange(N, dtype=torch.float64, device=device) + 0.5) / N
    for i, c in enumerate(comps):
        acc = out[i]
        acc.zero_()
        for k, a, ph in sine_modes(seed, 100 + c, cfg["nmodes"], cfg["kmax"]):
            # sin(2 pi k.x + ph) = Im(e^{i ph} e^{2 pi i kx x} e^{2 pi i ky y} e^{2 pi i kz z})
            ex = torch.polar(torch.ones_like(x), 2.0 * math.pi * k[0] * x)
            ey = torch.polar(torch.ones_like(x), 2.0 * math.pi * k[1] * x)
            ez = torch.polar(torch.ones_like(x), 2.0 * math.pi * k[2] * x) * complex(math.cos(ph), math.sin(ph))
            for z0 in range(0, N, 32):
                z1 = min(N, z0 + 32)
                blk = ez[z0:z1, None, None] * (ey[None, :, None] * ex[None, None, :])
                acc[z0:z1] += a * blk.imag
        if "noise" in cfg["init"]:
            key = int(_key(seed, 200 + c))
            lo, hi = -cfg["noise"], cfg["noise"]
            for z0 in range(0, N, 32):
                z1 = min(N, z0 + 32)
                idx = torch.arange(z0 * N * N, z1 * N * N, dtype=torch.int64, device=device)
                z = _torch_mix(_u64(key) + (idx + 1) * _u64(GOLDEN))
                u = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (1.0 / 9007199254740992.0)
                acc[z0:z1] += (lo + (hi - lo) * u).reshape(z1 - z0, N, N)
    return out
