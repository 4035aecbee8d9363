"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a published coefficient table, a library
routine (numpy.pad wrap mode), the exact Fourier-mode decay factor of the discrete
operator, telescoping of the flux form (conservation), exact rational arithmetic on tiny
grids, exactness of linear interpolation on linear data, and layout invariance (Sec. 3.2:
tiling and the box layout change the access pattern, not the data or the result).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import coeffs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def whole_domain(N):
    return [0, 0, 0], [N[0] - 1, N[1] - 1, N[2] - 1]


# --------------------------------------------------------------------------- coefficients

def _read_golden_coeffs():
    rows = {}
    with open(os.path.join(GOLDEN, "fd_laplacian_coefficients.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[int(parts[0])] = [Fraction(p) for p in parts[1:]]
    return rows


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_coefficients_match_published_table(R):
    """Fornberg (1988) Table 1, second-derivative rows: the moment-system solution agrees."""
    gold = _read_golden_coeffs()[R]
    c = coeffs.laplacian_coefficients(R)
    mine = [c[m] for m in range(R, 0, -1)] + [c[0]] + [c[m] for m in range(1, R + 1)]
    assert mine == gold


@pytest.mark.parametrize("R", [1, 2, 4])
def test_flux_coefficients_telescoping(R):
    """b_m = sum_{j>=m} c_j, summed by hand from the classical weights for R = 2 and 4."""
    b = coeffs.flux_coefficients(R)
    expected = {1: [Fraction(1)], 2: [Fraction(15, 12), Fraction(-1, 12)],
                4: [Fraction(205, 144), Fraction(-127, 720), Fraction(17, 720), Fraction(-1, 560)]}[R]
    assert b == expected


@pytest.mark.parametrize("R", [1, 2, 4])
def test_symbol_order_of_accuracy(R):
    """sigma_R(theta) = -theta^2 + O(theta^(2R+2)): the error shrinks by 2^(2R+2) when theta halves."""
    e1 = abs(coeffs.symbol(R, 0.2) + 0.04)
    e2 = abs(coeffs.symbol(R, 0.1) + 0.01)
    ratio = e1 / e2
    assert abs(math.log2(ratio) - (2 * R + 2)) < 0.2, ratio


# --------------------------------------------------------------------------- chop

def test_chop_even_and_remainder():
    b = oracle.chop([0, 0, 0], [63, 63, 63], 32)
    assert b.shape == (8, 6)
    assert b[0].tolist() == [0, 0, 0, 31, 31, 31] and b[1].tolist() == [32, 0, 0, 63, 31, 31]
    assert b[2].tolist() == [0, 32, 0, 31, 63, 31] and b[7].tolist() == [32, 32, 32, 63, 63, 63]
    b = oracle.chop([0, 0, 0], [9, 3, 4], 4)
    sides_x = sorted(set((r[3] - r[0] + 1) for r in b.tolist()))
    assert sides_x == [2, 4] and b.shape[0] == 3 * 1 * 2
    cells = sum((r[3] - r[0] + 1) * (r[4] - r[1] + 1) * (r[5] - r[2] + 1) for r in b.tolist())
    assert cells == 10 * 4 * 5


# --------------------------------------------------------------------------- FillBoundary

def _rand(shape, seed=7):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("g", [1, 2, 3])
def test_fill_single_box_equals_numpy_wrap(g):
    """One box = the whole periodic domain: FillBoundary is numpy.pad(mode='wrap')."""
    N = (6, 5, 7)  # Nx, Ny, Nz
    lo, hi = whole_domain(N)
    L = oracle.Level([lo + hi], lo, hi, g, 2)
    dense = _rand((2, N[2], N[1], N[0]))
    u = L.from_dense(dense)
    oracle.fill_boundary(L, u)
    fab = L.fab(u, 0)
    for c in range(2):
        np.testing.assert_array_equal(fab[c], np.pad(dense[c], g, mode="wrap"))


def _boxes_uneven():
    # a 12 x 8 x 10 domain cut into 7 unequal boxes that tile it
    return np.array([
        [0, 0, 0, 4, 7, 3], [5, 0, 0, 11, 2, 3], [5, 3, 0, 11, 7, 3],
        [0, 0, 4, 2, 7, 9], [3, 0, 4, 11, 4, 6], [3, 5, 4, 11, 7, 6], [3, 0, 7, 11, 7, 9]], dtype=np.int32)


@pytest.mark.parametrize("g", [1, 2])
def test_fill_multibox_equals_carved_padded_array(g):
    """Many boxes: every grown FArrayBox equals its window of the wrap-padded global array."""
    boxes = _boxes_uneven()
    N = (12, 8, 10)
    lo, hi = whole_domain(N)
    L = oracle.Level(boxes, lo, hi, g, 1)
    dense = _rand((1, N[2], N[1], N[0]), seed=3)
    u = L.from_dense(dense)
    oracle.fill_boundary(L, u)
    padded = np.pad(dense[0], g, mode="wrap")
    for b, B in enumerate(boxes):
        win = padded[B[2]:B[5] + 1 + 2 * g, B[1]:B[4] + 1 + 2 * g, B[0]:B[3] + 1 + 2 * g]
        np.testing.assert_array_equal(L.fab(u, b)[0], win)


def test_fill_partial_level_leaves_unowned_ghosts():
    """A level that does not cover the domain: ghosts owned by no box stay untouched."""
    N = (16, 16, 16)
    lo, hi = whole_domain(N)
    boxes = np.array([[0, 0, 0, 3, 3, 3], [4, 0, 0, 7, 3, 3]], dtype=np.int32)
    L = oracle.Level(boxes, lo, hi, 1, 1)
    u = L.from_dense(_rand((1, 16, 16, 16)))
    n = oracle.fill_boundary(L, u)
    # box 0's +x face (4 x 4 cells) comes from box 1 and vice versa; the x-periodic wrap of
    # box 0's -x face is x = 15: unowned.  Edges/corners within the pair: +-y, +-z are unowned.
    assert n == 2 * 16
    f0 = L.fab(u, 0)[0]
    assert np.isnan(f0[0, 0, 0]) and not np.isnan(f0[1, 1, 5])


# --------------------------------------------------------------------------- stencil forms

@pytest.mark.parametrize("R", [1, 2, 4])
def test_flux_form_equals_direct_form(R):
    N = (16, 16, 16)
    lo, hi = whole_domain(N)
    L = oracle.Level(oracle.chop(lo, hi, 8), lo, hi, R, 1)
    u = L.from_dense(_rand((1, 16, 16, 16), seed=R))
    oracle.fill_boundary(L, u)
    a, b = L.alloc(), L.alloc()
    oracle.stencil(L, R, 0.05, u, a, "flux")
    oracle.stencil(L, R, 0.05, u, b, "direct")
    da, db = L.to_dense(a), L.to_dense(b)
    assert rel_err(da, db) < 1e-13


# --------------------------------------------------------------------------- Fourier decay

@pytest.mark.parametrize("R,k", [(1, (1, 2, 3)), (1, (8, 8, 8)), (2, (3, -1, 5)), (2, (8, 1, 8)),
                                 (4, (2, 5, -7)), (4, (8, 8, 1))])
def test_single_mode_decays_by_exact_factor(R, k):
    """u0 = sin(2 pi k.x + phi) at cell centres: after n steps u_n = g^n u0 exactly, with
    g = 1 + lam * sum_d sigma_R(2 pi k_d / N); k_d = N/2 is the Nyquist mode."""
    N = 16
    lo, hi = whole_domain((N, N, N))
    L = oracle.Level(oracle.chop(lo, hi, 8), lo, hi, R, 1)
    u0 = synth.single_mode((N, N, N), k)
    lam = {1: 0.15, 2: 0.1125, 4: 0.09}[R]
    g = 1.0 + lam * sum(coeffs.symbol(R, 2 * math.pi * kd / N) for kd in k)
    assert abs(g) <= 1.0
    # as many steps (<= 40) as keep |g|^n >= 1e-2, so the comparison stays relative to a
    # solution that has not decayed into rounding noise
    nsteps = max(1, min(40, int(math.log(1e-2) / math.log(abs(g)))))
    out = L.to_dense(oracle.advance(L, L.from_dense(u0[None]), R, lam, nsteps))[0]
    exact = (g ** nsteps) * u0
    assert rel_err(out, exact) <= 1e-12


# --------------------------------------------------------------------------- conservation

@pytest.mark.parametrize("R", [1, 2, 4])
def test_domain_sum_conserved(R):
    """Flux form on a periodic level telescopes: the domain sum is invariant up to rounding."""
    N = 16
    lo, hi = whole_domain((N, N, N))
    boxes = oracle.chop(lo, hi, 8)
    L = oracle.Level(boxes, lo, hi, R, 1)
    dense = 1.0 + _rand((1, N, N, N), seed=11)
    u = L.from_dense(dense)
    s0 = oracle.domain_sum(L, u)
    nsteps = 30
    out = oracle.advance(L, u, R, 0.05, nsteps)
    s1 = oracle.domain_sum(L, out)
    mass = math.fsum(np.abs(dense).ravel().tolist())
    assert abs(s1 - s0) <= nsteps * 1e-15 * mass


def test_domain_sum_is_correctly_rounded():
    """fsum cancels exactly where naive summation does not."""
    L = oracle.Level([[0, 0, 0, 3, 0, 0]], [0, 0, 0], [3, 0, 0], 1, 1)
    u = L.from_dense(np.array([1e16, 1.0, -1e16, 1.0]).reshape(1, 1, 1, 4))
    assert oracle.domain_sum(L, u) == 2.0


# --------------------------------------------------------------------------- RK3 (Sec. 4.2)

@pytest.mark.parametrize("R,k", [(1, (1, 2, 1)), (2, (3, 1, 2)), (4, (2, 2, 3))])
def test_rk3_single_mode_decays_by_the_stability_polynomial(R, k):
    """For the linear operator one SSP-RK3 step maps a Fourier mode to P(z) times itself,
    P(z) = 1 + z + z^2/2 + z^3/6, z = lam * sum_d sigma_R(2 pi k_d / N) (the scheme is exact
    for linear autonomous problems up to third order)."""
    N = (12, 10, 8)
    lo, hi = whole_domain(N)
    L = oracle.Level(oracle.chop(lo, hi, 5), lo, hi, R, 1)
    u0 = synth.single_mode((N[2], N[1], N[0]), k)[None]
    lam = 0.12
    z = lam * sum(coeffs.symbol(R, 2 * math.pi * kd / n) for kd, n in zip(k, N))
    P = 1 + z + z * z / 2 + z ** 3 / 6
    nsteps = 4
    out = L.to_dense(oracle.rk3_advance(L, L.from_dense(u0), R, lam, nsteps))
    assert rel_err(out, P ** nsteps * u0) <= 1e-12


def test_rk3_conserves_the_sum():
    lo, hi = whole_domain((16, 12, 10))
    boxes = [[0, 0, 0, 9, 11, 9], [10, 0, 0, 15, 5, 9], [10, 6, 0, 15, 11, 9]]
    L = oracle.Level(boxes, lo, hi, 2, 1)
    u0 = np.random.default_rng(7).random((1, 10, 12, 16))
    u = oracle.rk3_advance(L, L.from_dense(u0), 2, 0.1, 3)
    s0, s1 = math.fsum(u0.ravel().tolist()), oracle.domain_sum(L, u)
    assert abs(s1 - s0) <= 3 * 3 * 1e-15 * float(np.sum(np.abs(u0)))


# --------------------------------------------------------------------------- other reductions

def _uneven_16():
    lo, hi = [0, 0, 0], [15, 15, 15]
    boxes = [[0, 0, 0, 9, 15, 15], [10, 0, 0, 15, 6, 15], [10, 7, 0, 15, 15, 15]]
    return oracle.Level(boxes, lo, hi, 2, 2)


def test_reductions_see_valid_cells_only_planted_extremes():
    """max / min / max|u| of a field in [0, 1) with a planted 2.5 and -3.25; the ghost cells
    hold +-100, which must not show (a reduction over the grown boxes would see them)."""
    L = _uneven_16()
    dense = np.random.default_rng(3).random((2, 16, 16, 16))
    dense[1, 3, 12, 14] = 2.5
    dense[1, 9, 1, 2] = -3.25
    u = L.from_dense(dense)
    for b in range(L.nbox):  # ghosts: +-100
        f = L.fab(u, b)
        g = L.g
        inner = f[:, g:-g, g:-g, g:-g].copy()
        f[:, :, :, :] = np.where(np.arange(f.shape[3]) % 2 == 0, 100.0, -100.0)
        f[:, g:-g, g:-g, g:-g] = inner
    assert oracle.reduce(L, u, "max", 1) == 2.5
    assert oracle.reduce(L, u, "min", 1) == -3.25
    assert oracle.reduce(L, u, "norm0", 1) == 3.25
    assert 0.0 <= oracle.reduce(L, u, "min", 0) and oracle.reduce(L, u, "max", 0) < 1.0


def test_norms_of_closed_form_fields():
    """2-norm of a constant c on 16^3 cells is 64 |c| exactly; the +-1 checkerboard has
    1-norm 4096, 2-norm 64, sum 0; a single nonzero cell v has every norm |v|."""
    L = _uneven_16()
    i = np.arange(16)
    cb = (-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :])
    dense = np.stack([np.full((16, 16, 16), -0.375), cb])
    u = L.from_dense(dense)
    assert oracle.reduce(L, u, "norm2", 0) == 24.0
    assert oracle.reduce(L, u, "norm1", 0) == 1536.0
    assert oracle.reduce(L, u, "sum", 0) == -1536.0
    assert oracle.reduce(L, u, "norm1", 1) == 4096.0
    assert oracle.reduce(L, u, "norm2", 1) == 64.0
    assert oracle.reduce(L, u, "sum", 1) == 0.0
    one = np.zeros((2, 16, 16, 16))
    one[0, 5, 11, 13] = -7.5
    u1 = L.from_dense(one)
    for op in ("norm0", "norm1", "norm2"):
        assert oracle.reduce(L, u1, op, 0) == 7.5
    assert oracle.reduce(L, u1, "min", 0) == -7.5 and oracle.reduce(L, u1, "max", 0) == 0.0


def test_max_type_reductions_skip_nan():
    L = _uneven_16()
    dense = np.zeros((2, 16, 16, 16))
    dense[0, 0, 0, 0] = np.nan
    dense[0, 15, 15, 15] = 1.25
    u = L.from_dense(dense)
    assert oracle.reduce(L, u, "max", 0) == 1.25 and oracle.reduce(L, u, "norm0", 0) == 1.25


# --------------------------------------------------------------------------- layout invariance

@pytest.mark.parametrize("R", [1, 2])
def test_layout_invariance_bitwise(R):
    """The same domain under 1 box, 8 boxes and uneven boxes gives identical bits."""
    N = (12, 8, 10)
    lo, hi = whole_domain(N)
    dense = _rand((2, N[2], N[1], N[0]), seed=5)
    results = []
    for boxes in ([lo + hi], oracle.chop(lo, hi, 4), _boxes_uneven()):
        L = oracle.Level(boxes, lo, hi, R, 2)
        out = oracle.advance(L, L.from_dense(dense), R, [0.08, 0.03], 7)
        results.append(L.to_dense(out))
    for r in results[1:]:
        np.testing.assert_array_equal(r, results[0])


# --------------------------------------------------------------------------- brute force

def _exact_evolve(u, R, lam, nsteps):
    """Exact rational evolution of the periodic direct-form operator on a global array."""
    c = coeffs.laplacian_coefficients(R)
    for _ in range(nsteps):
        lap = np.zeros_like(u)
        for ax in range(3):
            lap = lap + c[0] * u
            for m in range(1, R + 1):
                lap = lap + c[m] * (np.roll(u, m, axis=ax) + np.roll(u, -m, axis=ax))
        u = u + lam * lap
    return u


@pytest.mark.parametrize("N,R,mgs,nsteps", [(4, 1, 2, 4), (6, 1, 3, 3), (6, 2, 3, 3), (8, 4, 4, 2), (8, 2, 8, 3)])
def test_bruteforce_exact_rational(N, R, mgs, nsteps):
    """Tiny grids: the FP64 oracle (boxwise, flux form, FillBoundary) against exact rational
    arithmetic of (I + lam A)^n applied to dyadic data on one periodic array."""
    rng = np.random.default_rng(N * 10 + R)
    ints = rng.integers(-64, 64, size=(N, N, N))
    u0 = np.vectorize(lambda v: Fraction(int(v), 16))(ints).astype(object)
    lam = Fraction(1, 16)
    exact = _exact_evolve(u0, R, lam, nsteps)
    exact_f = np.vectorize(float)(exact).astype(np.float64)
    lo, hi = whole_domain((N, N, N))
    L = oracle.Level(oracle.chop(lo, hi, mgs), lo, hi, R, 1)
    out = L.to_dense(oracle.advance(L, L.from_dense(ints[None] / 16.0), R, float(lam), nsteps))[0]
    assert float(np.max(np.abs(out - exact_f))) <= 1e-14 * float(np.max(np.abs(exact_f)))


# --------------------------------------------------------------------------- AMR pieces

# Fine boxes of the two-box setup at ratio 2 (coarse cells 2..3 x 2..5 x 2..3 and 4..5 x 2..3 x
# 2..4); at ratio r the same coarse cells, refined by r.
_FINE_COARSE_CELLS = [[2, 2, 2, 3, 5, 3], [4, 2, 2, 5, 3, 4]]


def _fine_setup(Nc=8, gf=1, ratio=2):
    crse = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 4), [0, 0, 0], [Nc - 1] * 3, 1, 1)
    fboxes = np.array([[ratio * b[d] for d in range(3)] + [ratio * (b[3 + d] + 1) - 1 for d in range(3)]
                       for b in _FINE_COARSE_CELLS], dtype=np.int32)
    fine = oracle.Level(fboxes, [0, 0, 0], [ratio * Nc - 1] * 3, gf, 1)
    return crse, fine


def _level_from_fn(level, N, fn):
    x = (np.arange(N) + 0.5) / N
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    return level.from_dense(fn(xx, y, z)[None])


@pytest.mark.parametrize("ratio", [2, 4])
@pytest.mark.parametrize("alpha", [0.5, 0.25, 0.75])
def test_interp_reproduces_linear_field_exactly(alpha, ratio):
    """Trilinear interpolation is exact on linear data: every interpolated fine ghost equals
    the linear function at the fine cell centre, bit for bit (dyadic coefficients and
    centres; the weights are multiples of 1/4 at ratio 2 and of 1/8 at ratio 4), and the time
    blend of two linear fields is (1 - alpha) old + alpha new (at alpha != 1/2 a swap of the
    two levels shows).  A wrong weight offset at one ratio fails here."""
    Nc = 8
    crse, fine = _fine_setup(Nc, ratio=ratio)
    f_old = lambda x, y, z: 0.5 + 0.25 * x - 0.75 * y + 0.125 * z
    # no blend (alpha = 0, 1/4, 1/2, 3/4) has gradient components summing to zero, so a
    # position error common to the three directions cannot cancel
    f_new = lambda x, y, z: 1.5 - 0.5 * x + 0.25 * y + 0.875 * z
    c_old, c_new = _level_from_fn(crse, Nc, f_old), _level_from_fn(crse, Nc, f_new)
    fd = fine.alloc()
    n = oracle.interp_cf(fine, crse, ratio, alpha, c_old, c_new, fd)
    xf = (np.arange(ratio * Nc) + 0.5) / (ratio * Nc)
    checked = 0
    for b, B in enumerate(fine.boxes):
        fab = fine.fab(fd, b)[0]
        for k in range(B[2] - 1, B[5] + 2):
            for j in range(B[1] - 1, B[4] + 2):
                for i in range(B[0] - 1, B[3] + 2):
                    v = fab[k - B[2] + 1, j - B[1] + 1, i - B[0] + 1]
                    if np.isnan(v):
                        continue
                    x, y, z = xf[i], xf[j], xf[k]
                    assert v == (1 - alpha) * f_old(x, y, z) + alpha * f_new(x, y, z)
                    checked += 1
    assert checked == n > 0


@pytest.mark.parametrize("ratio", [2, 4])
def test_interp_fills_exactly_the_uncovered_ghosts(ratio):
    """Brute-force coverage count: fine ghosts whose periodic point lies in no fine box."""
    Nc = 8
    Nf = ratio * Nc
    crse, fine = _fine_setup(Nc, ratio=ratio)
    ones = crse.from_dense(np.ones((1, Nc, Nc, Nc)))
    fd = fine.alloc()
    n = oracle.interp_cf(fine, crse, ratio, 0.0, ones, ones, fd)
    expect = 0
    for B in fine.boxes:
        for k in range(B[2] - 1, B[5] + 2):
            for j in range(B[1] - 1, B[4] + 2):
                for i in range(B[0] - 1, B[3] + 2):
                    inside = B[0] <= i <= B[3] and B[1] <= j <= B[4] and B[2] <= k <= B[5]
                    if inside:
                        continue
                    p = (i % Nf, j % Nf, k % Nf)
                    covered = any(o[0] <= p[0] <= o[3] and o[1] <= p[1] <= o[4] and o[2] <= p[2] <= o[5]
                                  for o in fine.boxes)
                    expect += 0 if covered else 1
    assert n == expect
    vals = np.concatenate([fine.fab(fd, b)[0].ravel() for b in range(fine.nbox)])
    vals = vals[~np.isnan(vals)]
    assert vals.size == n and np.all(vals == 1.0)


@pytest.mark.parametrize("ratio", [2, 4])
def test_interp_weights_at_periodic_wrap(ratio):
    """Near the domain edge the coarse index wraps.  A fine box at the corner of the domain
    interpolates a coarse field that is constant along each periodic line: every ghost gets
    the constant.  Then a coarse field that is linear in y and constant in x and z (so the
    wrap in x and z cannot change it): the ghosts on the x and z sides, which stay inside the
    domain in y (fine rows j >= r/2, whose coarse rows k0 = floor((2j + 1 - r) / 2r) and
    k0 + 1 do not wrap), get the linear function at their centre exactly."""
    Nc = 8
    Nf = ratio * Nc
    s = 2 * ratio  # box side: two coarse cells
    crse = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 4), [0, 0, 0], [Nc - 1] * 3, 1, 1)
    fine = oracle.Level([[0, 0, 0, s - 1, s - 1, s - 1]], [0, 0, 0], [Nf - 1] * 3, 2, 1)
    c = crse.from_dense(np.full((1, Nc, Nc, Nc), 3.25))
    fd = fine.alloc()
    n = oracle.interp_cf(fine, crse, ratio, 0.25, c, c, fd)
    assert n == (s + 4) ** 3 - s ** 3
    vals = fine.fab(fd, 0)[0]
    assert np.all(vals[~np.isnan(vals)] == 3.25)
    fn = lambda x, y, z: 0.75 + 0.5 * y
    cl = _level_from_fn(crse, Nc, fn)
    fd = fine.alloc()
    oracle.interp_cf(fine, crse, ratio, 0.0, cl, cl, fd)
    fab = fine.fab(fd, 0)[0]
    yf = (np.arange(Nf) + 0.5) / Nf
    checked = 0
    for k in range(-2, s + 2):
        for j in range(ratio // 2, s):  # the coarse y rows of these fine rows do not wrap
            for i in range(-2, s + 2):
                if 0 <= i < s and 0 <= k < s:
                    continue
                assert fab[k + 2, j + 2, i + 2] == fn(0.0, yf[j], 0.0)
                checked += 1
    assert checked > 0


@pytest.mark.parametrize("ratio", [2, 4])
def test_average_down_of_constant_refinement_is_identity(ratio):
    """Each coarse value copied into its r^3 children averages back to itself (a 1/r^2 or a
    wrong child count at one ratio fails here)."""
    Nc = 8
    crse, fine = _fine_setup(Nc, ratio=ratio)
    # dyadic values with few significant bits, so that the r^3-term sum is exact
    dense_c = np.random.default_rng(2).integers(-512, 512, size=(1, Nc, Nc, Nc)) / 64.0
    dense_f = dense_c
    for ax in (1, 2, 3):
        dense_f = np.repeat(dense_f, ratio, axis=ax)
    fd = fine.from_dense(dense_f)
    cd = crse.from_dense(dense_c)
    before = crse.to_dense(cd)
    n = oracle.average_down(fine, crse, ratio, fd, cd)
    assert n == (2 * 4 * 2) + (2 * 2 * 3)
    np.testing.assert_array_equal(crse.to_dense(cd), before)


@pytest.mark.parametrize("ratio", [2, 4])
def test_average_down_of_linear_field(ratio):
    """The mean of the r^3 children of a linear field is its value at the coarse centre."""
    Nc = 8
    crse, fine = _fine_setup(Nc, ratio=ratio)
    fn = lambda x, y, z: 0.25 + 0.5 * x - 0.25 * y + 0.75 * z
    fd = _level_from_fn(fine, ratio * Nc, fn)
    cd = crse.from_dense(np.zeros((1, Nc, Nc, Nc)))
    oracle.average_down(fine, crse, ratio, fd, cd)
    xc = (np.arange(Nc) + 0.5) / Nc
    dense = crse.to_dense(cd)[0]
    for B in fine.boxes:
        for k in range(B[2] // ratio, B[5] // ratio + 1):
            for j in range(B[1] // ratio, B[4] // ratio + 1):
                for i in range(B[0] // ratio, B[3] // ratio + 1):
                    assert dense[k, j, i] == fn(xc[i], xc[j], xc[k])


@pytest.mark.parametrize("ratio,nsub,lam_c", [(2, 2, 0.075), (4, 4, 0.0375)])
def test_amr_with_full_fine_cover_equals_fine_single_level(ratio, nsub, lam_c):
    """A fine level covering the whole domain needs no interpolation: after n coarse steps
    the fine data equal n * nsub single-level fine steps with lam_f = lam_c r^2 / nsub
    (= 0.15 here), bit for bit, and the coarse data equal the average-down of that fine
    result."""
    Nc = 8
    Nf = ratio * Nc
    crse = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 4), [0, 0, 0], [Nc - 1] * 3, 1, 1)
    fine = oracle.Level(oracle.chop([0, 0, 0], [Nf - 1] * 3, 8), [0, 0, 0], [Nf - 1] * 3, 1, 1)
    dense_f = _rand((1, Nf, Nf, Nf), seed=9)
    fd = fine.from_dense(dense_f)
    cd = crse.from_dense(np.zeros((1, Nc, Nc, Nc)))
    oracle.average_down(fine, crse, ratio, fd, cd)
    ncrse = 3
    c_out, f_out = oracle.amr_advance(crse, fine, 1, lam_c, cd, fd, ncrse, nsub=nsub, ratio=ratio)
    f_ref = oracle.advance(fine, fd, 1, 0.15, ncrse * nsub)
    np.testing.assert_array_equal(fine.to_dense(f_out), fine.to_dense(f_ref))
    c_ref = crse.from_dense(np.zeros((1, Nc, Nc, Nc)))
    oracle.average_down(fine, crse, ratio, f_ref, c_ref)
    np.testing.assert_array_equal(crse.to_dense(c_out), crse.to_dense(c_ref))


@pytest.mark.parametrize("ratio,nsub,lam_c", [(2, 2, 0.075), (4, 4, 0.0375)])
def test_amr_partial_cover_keeps_constant_and_conserves_with_reflux(ratio, nsub, lam_c):
    """A fine level covering part of the domain at ratio r with nsub substeps: a constant
    state stays constant (interpolation weights sum to one at every substep time, the
    average-down is a mean), and with refluxing the composite sum is conserved to rounding."""
    Nc = 8
    crse, fine = _fine_setup(Nc, ratio=ratio)
    cd = crse.from_dense(np.full((1, Nc, Nc, Nc), 2.0))
    fd = fine.from_dense(np.full((1, ratio * Nc, ratio * Nc, ratio * Nc), 2.0))
    c_out, f_out = oracle.amr_advance(crse, fine, 1, lam_c, cd, fd, 2, nsub=nsub, ratio=ratio)
    assert np.all(crse.to_dense(c_out) == 2.0)
    fo = fine.to_dense(f_out)
    assert np.all(fo[~np.isnan(fo)] == 2.0)
    fd = fine.from_dense(_rand((1, ratio * Nc, ratio * Nc, ratio * Nc), seed=31))
    cd = crse.from_dense(_rand((1, Nc, Nc, Nc), seed=32))
    oracle.average_down(fine, crse, ratio, fd, cd)
    s0, a0 = _composite_sum(crse, fine, cd, fd, ratio=ratio)
    c1, f1 = oracle.amr_advance(crse, fine, 1, lam_c, cd, fd, 2, nsub=nsub, ratio=ratio, reflux_faces=True)
    s1, _ = _composite_sum(crse, fine, c1, f1, ratio=ratio)
    assert abs(s1 - s0) <= 2 * nsub * 1e-15 * a0, s1 - s0
    c2, f2 = oracle.amr_advance(crse, fine, 1, lam_c, cd, fd, 2, nsub=nsub, ratio=ratio)
    s2, _ = _composite_sum(crse, fine, c2, f2, ratio=ratio)
    assert abs(s2 - s0) > 1e-6 * a0  # no refluxing, no conservation


def _composite_sum(crse, fine, cdata, fdata, ratio=2, comp=0):
    """sum of the fine cells plus r^3 times the coarse cells no fine box covers (fine-cell units)."""
    cd, fd = crse.to_dense(cdata)[comp], fine.to_dense(fdata)[comp]
    covered = np.zeros(cd.shape, dtype=bool)
    for b in fine.boxes:
        covered[b[2] // ratio:b[5] // ratio + 1, b[1] // ratio:b[4] // ratio + 1, b[0] // ratio:b[3] // ratio + 1] = True
    vals = (ratio ** 3 * cd[~covered]).tolist() + fd[~np.isnan(fd)].tolist()
    return math.fsum(vals), math.fsum(np.abs(vals).tolist())


def _two_level_case(R, g):
    Nc = 16
    crse = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 8), [0, 0, 0], [Nc - 1] * 3, g, 2)
    fboxes = [[8, 8, 4, 15, 23, 19], [16, 8, 4, 23, 15, 11], [0, 24, 26, 5, 31, 31], [26, 24, 26, 31, 31, 31]]
    fine = oracle.Level(fboxes, [0, 0, 0], [2 * Nc - 1] * 3, g, 2)
    dense_f = _rand((2, 2 * Nc, 2 * Nc, 2 * Nc), seed=21)
    fd = fine.from_dense(dense_f)
    cd = crse.from_dense(_rand((2, Nc, Nc, Nc), seed=22))
    oracle.average_down(fine, crse, 2, fd, cd)
    return crse, fine, cd, fd


@pytest.mark.parametrize("R,g", [(1, 1), (2, 2)])
def test_reflux_conserves_the_composite_sum(R, g):
    """With refluxing, the coarse flux at every coarse-fine face is replaced by the fine fluxes
    through it, so the composite sum (fine cells plus r^3 times the uncovered coarse cells) is
    invariant up to rounding; without it, it is not.  The fine boxes include a pair that meets
    across the periodic boundary and one with a face on it."""
    crse, fine, cd, fd = _two_level_case(R, g)
    lam_c = {1: 0.075, 2: 0.05}[R]
    for comp in range(2):
        s0, a0 = _composite_sum(crse, fine, cd, fd, comp=comp)
        c1, f1 = oracle.amr_advance(crse, fine, R, lam_c, cd, fd, 3, reflux_faces=True)
        s1, _ = _composite_sum(crse, fine, c1, f1, comp=comp)
        assert abs(s1 - s0) <= 3 * 2 * 1e-15 * a0, (comp, s1 - s0)
        c2, f2 = oracle.amr_advance(crse, fine, R, lam_c, cd, fd, 3)
        s2, _ = _composite_sum(crse, fine, c2, f2, comp=comp)
        assert abs(s2 - s0) > 1e-6 * a0  # the test has teeth: no refluxing, no conservation


def test_reflux_without_coarse_fine_faces_changes_nothing():
    """A fine level covering the whole domain has no coarse-fine face."""
    Nc = 8
    crse = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 4), [0, 0, 0], [Nc - 1] * 3, 1, 1)
    fine = oracle.Level(oracle.chop([0, 0, 0], [2 * Nc - 1] * 3, 8), [0, 0, 0], [2 * Nc - 1] * 3, 1, 1)
    fd = fine.from_dense(_rand((1, 2 * Nc, 2 * Nc, 2 * Nc), seed=23))
    cd = crse.from_dense(np.zeros((1, Nc, Nc, Nc)))
    oracle.average_down(fine, crse, 2, fd, cd)
    assert oracle.CFFaces(crse, fine, 2).n == 0
    a = oracle.amr_advance(crse, fine, 1, 0.075, cd, fd, 2, reflux_faces=True)
    b = oracle.amr_advance(crse, fine, 1, 0.075, cd, fd, 2)
    np.testing.assert_array_equal(crse.to_dense(a[0]), crse.to_dense(b[0]))


def test_cf_faces_of_a_single_box_are_its_surface():
    """One fine box of 4x6x8 coarse cells inside the domain: 2(4*6 + 4*8 + 6*8) coarse faces,
    each on a distinct (coarse cell, direction, side)."""
    Nc = 16
    crse = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 8), [0, 0, 0], [Nc - 1] * 3, 1, 1)
    fine = oracle.Level([[4, 6, 8, 11, 17, 23]], [0, 0, 0], [2 * Nc - 1] * 3, 1, 1)
    cf = oracle.CFFaces(crse, fine, 2)
    assert cf.n == 2 * (4 * 6 + 4 * 8 + 6 * 8)
    assert len({tuple(f) for f in cf.faces}) == cf.n
    # every coarse cell named lies outside the box and next to it
    for x, y, z, d, sc in cf.faces:
        inside = 2 <= x <= 5 and 3 <= y <= 8 and 4 <= z <= 11
        assert not inside


def test_amr_keeps_constant_state():
    Nc = 8
    crse, fine = _fine_setup(Nc)
    cd = crse.from_dense(np.full((1, Nc, Nc, Nc), 2.0))
    fd = fine.from_dense(np.full((1, 2 * Nc, 2 * Nc, 2 * Nc), 2.0))
    c_out, f_out = oracle.amr_advance(crse, fine, 1, 0.075, cd, fd, 2)
    assert np.all(crse.to_dense(c_out) == 2.0)
    fo = fine.to_dense(f_out)
    assert np.all(fo[~np.isnan(fo)] == 2.0)


# --------------------------------------------------------------------------- workloads

def test_heat64_workload_runs_and_conserves():
    cfg = synth.WORKLOADS["c1"]
    N = cfg["N"]
    lo, hi = whole_domain((N, N, N))
    L = oracle.Level(oracle.chop(lo, hi, cfg["max_grid_size"]), lo, hi, cfg["ngrow"], 1)
    u = L.from_dense(synth.initial_field(cfg))
    lam = 1.0 * synth.dt_for(cfg) * float(N * N)
    assert abs(lam - 0.15) < 1e-15
    out = oracle.advance(L, u, 1, lam, cfg["nsteps"])
    mass = math.fsum(np.abs(L.to_dense(u)).ravel().tolist())
    assert abs(oracle.domain_sum(L, out) - oracle.domain_sum(L, u)) <= cfg["nsteps"] * 1e-15 * mass


def test_fill_with_offset_domain_equals_numpy_wrap():
    """A domain whose lower corner is not the origin: the wrap is relative to domain_lo."""
    lo, hi = [-3, 2, 5], [2, 6, 11]  # 6 x 5 x 7 cells
    boxes = oracle.chop(lo, hi, 3)
    L = oracle.Level(boxes, lo, hi, 2, 1)
    dense = _rand((1, 7, 5, 6), seed=21)
    u = L.from_dense(dense)
    oracle.fill_boundary(L, u)
    padded = np.pad(dense[0], 2, mode="wrap")
    for b, B in enumerate(boxes):
        s = [B[d] - lo[d] for d in range(3)]
        e = [B[3 + d] - lo[d] + 1 + 4 for d in range(3)]
        np.testing.assert_array_equal(L.fab(u, b)[0], padded[s[2]:e[2], s[1]:e[1], s[0]:e[0]])


@pytest.mark.parametrize("ratio", [2, 4])
def test_average_down_matches_block_mean(ratio):
    """Random fine data: the average-down equals numpy's mean over r x r x r blocks."""
    Nc = 8
    crse, fine = _fine_setup(Nc, ratio=ratio)
    dense_f = _rand((1, ratio * Nc, ratio * Nc, ratio * Nc), seed=4)
    fd = fine.from_dense(dense_f)
    cd = crse.from_dense(np.zeros((1, Nc, Nc, Nc)))
    oracle.average_down(fine, crse, ratio, fd, cd)
    block = dense_f[0].reshape(Nc, ratio, Nc, ratio, Nc, ratio).mean(axis=(1, 3, 5))
    dense = crse.to_dense(cd)[0]
    for B in fine.boxes:
        sl = (slice(B[2] // ratio, B[5] // ratio + 1), slice(B[1] // ratio, B[4] // ratio + 1),
              slice(B[0] // ratio, B[3] // ratio + 1))
        np.testing.assert_allclose(dense[sl], block[sl], rtol=0, atol=ratio * 4e-16 * np.max(np.abs(block)))


@pytest.mark.parametrize("R", [1, 2, 4])
def test_threaded_oracle_gives_the_same_bits(R):
    """The paper's threaded loop over boxes (Sec. 3.3; the CPU baseline) against the
    single-threaded oracle: identical bits, on an uneven layout."""
    lo, hi = [0, 0, 0], [23, 15, 19]
    boxes = np.array([[0, 0, 0, 9, 15, 7], [10, 0, 0, 23, 6, 7], [10, 7, 0, 23, 15, 7], [0, 0, 8, 5, 15, 19],
                      [6, 0, 8, 23, 8, 12], [6, 9, 8, 23, 15, 12], [6, 0, 13, 23, 15, 19]], dtype=np.int32)
    L = oracle.Level(boxes, lo, hi, R, 2)
    u = L.from_dense(_rand((2, 20, 16, 24), seed=40 + R))
    lam = {1: 0.15, 2: 0.1125, 4: 0.09}[R]
    np.testing.assert_array_equal(oracle.advance_omp(L, u, R, lam, 3), oracle.advance(L, u, R, lam, 3))
