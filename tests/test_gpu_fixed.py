"""GPU parity of the fixed-point-difference path (MF_FIXED_DIFF, FP64 storage) against the FP64
oracle, through the C ABI.

The path evaluates the same flux-form forward-Euler step as the FP64 kernel on a level held as
64-bit fixed point inside an advance: the Laplacian formed exactly in 64-bit integers, the update
rounded onto a per-step, per-component grid taken from the level maximum.  Bars: max-norm
relative error <= 1e-12 against the FP64 oracle, identical bits for every tile shape, box layout
and schedule, the grid following a decaying solution (a Nyquist mode shrinking by 0.8 per step),
zero and extreme-magnitude fields, and the rejection of what the path does not take.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.coeffs import symbol as coeffs_symbol

torch = pytest.importorskip("torch")
mf = pytest.importorskip("paper_1604_03570_gb300")

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FIX = mf.MF_FIXED_DIFF

UNEVEN = np.array([
    [0, 0, 0, 9, 15, 7], [10, 0, 0, 23, 6, 7], [10, 7, 0, 23, 15, 7],
    [0, 0, 8, 5, 15, 19], [6, 0, 8, 23, 8, 12], [6, 9, 8, 23, 15, 12], [6, 0, 13, 23, 15, 19]], dtype=np.int32)
UNEVEN_DOM = ([0, 0, 0], [23, 15, 19])
LAM = {1: 0.15, 2: 0.1125, 4: 0.09}


def rel_err(got, ref):
    e = 0.0
    for c in range(ref.shape[0]):
        e = max(e, float(np.max(np.abs(got[c] - ref[c])) / np.max(np.abs(ref[c]))))
    return e


def level(lo, hi, boxes=None, mgs=None, ncomp=1, ngrow=1):
    return mf.MultiFab(lo, hi, max_grid_size=mgs, boxes=boxes, ncomp=ncomp, ngrow=ngrow, dtype="f64")


def oracle_advance(boxes, lo, hi, g, C, R, lam, nsteps, dense):
    L = oracle.Level(boxes, lo, hi, g, C)
    return L.to_dense(oracle.advance(L, L.from_dense(dense), R, lam, nsteps))


@pytest.mark.parametrize("R", [1, 2, 4])
@pytest.mark.parametrize("layout", ["uniform", "uneven"])
def test_fixed_diff_matches_oracle(R, layout):
    """32^3 in 16^3 boxes, or the 24x16x20 domain in 7 uneven boxes; ragged (whole-row) 5x7
    tiles; 2 components of very different magnitude (each has its own grid)."""
    if layout == "uniform":
        lo, hi = [0, 0, 0], [31, 31, 31]
        boxes = oracle.chop(lo, hi, 16)
    else:
        lo, hi = UNEVEN_DOM
        boxes = UNEVEN
    shape = tuple(h - l + 1 for l, h in zip(lo[::-1], hi[::-1]))
    Nx = hi[0] - lo[0] + 1
    D = np.array([1.0, 0.625])
    dt = LAM[R] / float(Nx * Nx)
    rng = np.random.default_rng(100 + R)
    dense = rng.standard_normal((2,) + shape)
    dense[1] *= 3e-4
    g = level(lo, hi, boxes=boxes, ncomp=2, ngrow=R)
    g.set_tile((0, 5, 7))
    g.from_host(dense)
    g.advance(R, list(D), dt, 7, FIX)
    ref = oracle_advance(boxes, lo, hi, R, 2, R, D * LAM[R], 7, dense)
    err = rel_err(g.to_host(), ref)
    print("MEASURED fixed-diff R=%d %s rel_err %.3e" % (R, layout, err))
    assert err <= FP64_TOL


@pytest.mark.parametrize("R", [1, 2])
def test_fixed_diff_bits_independent_of_layout_tiles_and_schedule(R):
    """The result of each cell depends on its stencil values and on the level maximum only:
    identical bits for 1, 8 and 18 boxes, several tile shapes (the balanced whole-box schedule
    included), 1 or 2 rows per thread and 16- or 32-byte groups."""
    lo, hi = [0, 0, 0], [31, 31, 31]
    dense = np.random.default_rng(7).standard_normal((1, 32, 32, 32))
    dt = LAM[R] / 1024.0
    # 18 uneven boxes: x split at 10 and 21 (odd widths: box faces inside 16-byte groups),
    # y at 5 and 17, z at 12
    xs, ys, zs = [(0, 9), (10, 20), (21, 31)], [(0, 4), (5, 16), (17, 31)], [(0, 11), (12, 31)]
    odd = np.array([[x[0], y[0], z[0], x[1], y[1], z[1]] for z in zs for y in ys for x in xs], dtype=np.int32)
    runs = [(None, 32, (0, 8, 16), (1, 0, 16)), (None, 16, (0, 4, 8), (2, 0, 16)), (None, 16, (0, 0, 0), (1, 0, 32)),
            (odd, None, (0, 3, 5), (2, 8, 16)), (odd, None, (0, 16, 0), (1, 4, 32))]
    outs = []
    for boxes, mgs, tile, sched in runs:
        g = level(lo, hi, boxes=boxes, mgs=mgs, ngrow=R)
        g.set_tile(tile)
        mf.mf_set_schedule(g.h, *sched)
        g.from_host(dense)
        g.advance(R, [1.0], dt, 6, FIX)
        outs.append(g.to_host())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    ref = oracle_advance(oracle.chop(lo, hi, 16), lo, hi, R, 1, R, LAM[R], 6, dense)
    assert rel_err(outs[0], ref) <= FP64_TOL


@pytest.mark.parametrize("R,nsteps", [(1, 60), (2, 50)])
def test_fixed_diff_grid_follows_a_decaying_mode(R, nsteps):
    """The Nyquist mode, an exact checkerboard of +-0.75, decays by g = 1 + 3 lam sigma_R(pi) =
    -0.8 per step at R = 1 (lam 0.15) and R = 2 (lam 0.1125): after n steps every cell is
    0.75 g^n in magnitude.  All cells keep equal magnitudes, so truncation to the grid keeps the
    field a checkerboard, and the error relative to the current maximum stays <= 1e-12 only if
    each step takes its grid from the current level maximum: a grid kept from the first step
    gives about 1e-11 here.  (The input must be exact: the rounding noise of a sampled sine,
    about 1e-17, lives in slowly decaying modes and would outgrow the 0.8^n mode.)"""
    N = 32
    lam = LAM[R]
    sign = 1.0 - 2.0 * (np.indices((N, N, N)).sum(axis=0) % 2)
    dense = (0.75 * sign)[None]
    gk = 1.0 + lam * 3.0 * coeffs_symbol(R, math.pi)
    exact = (0.75 * gk ** nsteps * sign)[None]
    g = level([0, 0, 0], [N - 1] * 3, mgs=16, ngrow=R)
    g.from_host(dense)
    g.advance(R, [1.0], lam / (N * N), nsteps, FIX)
    err = rel_err(g.to_host(), exact)
    print("MEASURED fixed-diff decaying Nyquist mode R=%d |g|^n %.2e rel_err %.3e" % (R, abs(gk) ** nsteps, err))
    assert abs(gk) ** nsteps < 1e-4
    assert err <= FP64_TOL


@pytest.mark.parametrize("scale", [0.0, 1e-280, 1e250])
def test_fixed_diff_zero_and_extreme_magnitudes(scale):
    """A zero field stays zero; fields near the ends of the FP64 range the path covers (level
    maximum at least 2^(B - 1022), about 1e-290 at R = 1) match the oracle."""
    lo, hi = [0, 0, 0], [15, 15, 15]
    dense = scale * np.random.default_rng(11).standard_normal((1, 16, 16, 16))
    g = level(lo, hi, mgs=8, ngrow=1)
    g.from_host(dense)
    g.advance(1, [1.0], 0.15 / 256.0, 5, FIX)
    out = g.to_host()
    if scale == 0.0:
        assert np.all(out == 0.0)
        return
    ref = oracle_advance(oracle.chop(lo, hi, 8), lo, hi, 1, 1, 1, 0.15, 5, dense)
    assert rel_err(out, ref) <= FP64_TOL


def test_fixed_diff_reports_a_non_finite_value_and_recovers():
    lo, hi = [0, 0, 0], [15, 15, 15]
    dense = np.random.default_rng(12).standard_normal((1, 16, 16, 16))
    bad = dense.copy()
    bad[0, 3, 4, 5] = np.nan
    g = level(lo, hi, mgs=8, ngrow=1)
    g.from_host(bad)
    g.advance(1, [1.0], 0.15 / 256.0, 3, FIX)
    with pytest.raises(mf.MFError) as e:
        g.to_host()
    assert e.value.code == mf.MF_ECUDA and "non-finite" in str(e.value)
    g.from_host(dense)
    g.advance(1, [1.0], 0.15 / 256.0, 3, FIX)
    ref = oracle_advance(oracle.chop(lo, hi, 8), lo, hi, 1, 1, 1, 0.15, 3, dense)
    assert rel_err(g.to_host(), ref) <= FP64_TOL


def test_fixed_diff_rejects_what_it_does_not_take():
    lo, hi = [0, 0, 0], [15, 15, 15]
    g32 = mf.MultiFab(lo, hi, max_grid_size=8, ncomp=1, ngrow=1, dtype="f32")
    with pytest.raises(mf.MFError) as e:
        g32.advance(1, [1.0], 1e-4, 1, FIX)
    assert e.value.code == mf.MF_EINVAL
    g = level(lo, hi, mgs=8, ngrow=1)
    for flags in (FIX | mf.MF_PLAIN_PER_BOX,):
        with pytest.raises(mf.MFError) as e:
            g.advance(1, [1.0], 1e-4, 1, flags)
        assert e.value.code == mf.MF_EINVAL
    with pytest.raises(mf.MFError) as e:
        g.rk3_advance(1, [1.0], 1e-4, 1, FIX)
    assert e.value.code == mf.MF_EINVAL
    mf.mf_set_kernel(g.h, mf.MF_KERNEL_GLOBAL)
    with pytest.raises(mf.MFError) as e:
        g.advance(1, [1.0], 1e-4, 1, FIX)
    assert e.value.code == mf.MF_EINVAL
