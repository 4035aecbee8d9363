"""GPU tests of regional storage (mf_create_regional): a level whose boxes are logical tiles of
larger regions (Sec. 2, Fig. 2) computes exactly what the same boxes stored one FArrayBox each
compute, and matches the FP64 oracle run on those boxes.

Bars: identical bits against the per-box layout for the forward-Euler advance (R = 1, 2, 4;
FP64 and FP32; one region per 32^3 block or a single region that is its own periodic image),
the fixed-point FP64 steps, the RK3 stages, the two-level advance with a regional fine level,
and the box-addressed copies; <= 1e-12 max-norm relative error against the oracle in FP64."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
mf = pytest.importorskip("paper_1604_03570_gb300")

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
LAM = {1: 0.15, 2: 0.1125, 4: 0.09}
N = 64
LO, HI = [0, 0, 0], [N - 1] * 3
BOXES = synth.uneven_boxes(N, 96, base=32, quantum=8)  # 96 boxes of 8^3 - 32^3


def rel_err(got, ref):
    return max(float(np.max(np.abs(got[c] - ref[c])) / np.max(np.abs(ref[c]))) for c in range(ref.shape[0]))


def pair(boxes, max_region, **kw):
    """The same boxes stored per box and in regions."""
    a = mf.MultiFab(LO, HI, boxes=boxes, **kw)
    b = mf.MultiFab(LO, HI, boxes=boxes, max_region=max_region, **kw)
    return a, b


def field(C, seed, dtype):
    x = np.random.default_rng(seed).standard_normal((C, N, N, N))
    return x.astype(np.float32).astype(np.float64) if dtype == "f32" else x


@pytest.mark.parametrize("max_region", [32, 64])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("R", [1, 2, 4])
def test_regional_advance_equals_per_box_and_matches_oracle(R, dtype, max_region):
    a, b = pair(BOXES, max_region, ncomp=2, ngrow=R, dtype=dtype)
    nreg = mf.mf_nregions(b.h)
    assert nreg == (8 if max_region == 32 else 1) and mf.mf_nboxes(b.h) == len(BOXES)
    dense = field(2, 40 + R, dtype)
    D = [1.0, 0.625]
    dt = LAM[R] / float(N * N)
    for g in (a, b):
        g.from_host(dense)
        g.advance(R, D, dt, 5)
    got_a, got_b = a.to_host(), b.to_host()
    np.testing.assert_array_equal(got_b, got_a)
    if dtype == "f64":
        L = oracle.Level(BOXES, LO, HI, R, 2)
        ref = L.to_dense(oracle.advance(L, L.from_dense(dense), R, np.array(D) * LAM[R], 5))
        err = rel_err(got_b, ref)
        print("MEASURED regional R=%d %d regions rel_err %.3e" % (R, nreg, err))
        assert err <= FP64_TOL


def test_regional_box_copies_address_the_boxes():
    """fab_to_host of box i (the box grown by its ghost cells) after a fill gives what the
    per-box layout's FArrayBox i holds after its fill; fab_from_host writes the box's cells."""
    a, b = pair(BOXES, 32, ncomp=1, ngrow=2, dtype="f64")
    dense = field(1, 7, "f64")
    for g in (a, b):
        g.from_host(dense)
        g.fill_boundary()
    for i in range(0, len(BOXES), 7):
        np.testing.assert_array_equal(b.fab_to_host(i), a.fab_to_host(i))
    i = 5
    arr = a.fab_to_host(i) + 1.0
    b.fab_from_host(i, arr)
    out = b.to_host()
    B = BOXES[i]
    g = 2
    np.testing.assert_array_equal(out[:, B[2]:B[5] + 1, B[1]:B[4] + 1, B[0]:B[3] + 1], arr[:, g:-g, g:-g, g:-g])
    rest = out.copy()
    rest[:, B[2]:B[5] + 1, B[1]:B[4] + 1, B[0]:B[3] + 1] = dense[:, B[2]:B[5] + 1, B[1]:B[4] + 1, B[0]:B[3] + 1]
    np.testing.assert_array_equal(rest, dense)


def test_regional_fixed_point_steps_and_rk3_equal_per_box():
    a, b = pair(BOXES, 32, ncomp=1, ngrow=2, dtype="f64")
    dense = field(1, 9, "f64")
    for g in (a, b):
        g.from_host(dense)
        g.advance(2, [1.0], LAM[2] / (N * N), 6, mf.MF_FIXED_DIFF)
    np.testing.assert_array_equal(b.to_host(), a.to_host())
    a, b = pair(BOXES, 64, ncomp=1, ngrow=4, dtype="f32")
    dense = field(1, 10, "f32")
    for g in (a, b):
        g.from_host(dense)
        g.rk3_advance(4, [1.0], 0.5 * LAM[4] / (N * N), 3)
    np.testing.assert_array_equal(b.to_host(), a.to_host())


def test_regional_fine_level_in_the_two_level_advance():
    """Refluxed two-level advance at ratio 2: the fine level's three patches chopped into 4^3
    boxes, stored per box or as regions (the patches again); identical bits on both levels, and
    the oracle on the chopped boxes within 1e-12."""
    Nc = 16
    clo, chi = [0, 0, 0], [Nc - 1] * 3
    base = np.array([[4, 4, 4, 7, 11, 7], [8, 4, 4, 11, 7, 9], [0, 0, 12, 3, 3, 15]])
    patches = np.concatenate([base[:, :3] * 2, (base[:, 3:] + 1) * 2 - 1], axis=1)
    fboxes = np.concatenate([oracle.chop(p[:3], p[3:], 4) for p in patches]).astype(np.int32)
    flo, fhi = [0, 0, 0], [2 * Nc - 1] * 3
    cboxes = oracle.chop(clo, chi, 8)
    modes = synth.sine_modes(1604, 51, 4, 3)
    cden = synth.eval_modes((Nc, Nc, Nc), modes)[None]
    fden = synth.eval_modes((2 * Nc,) * 3, modes)[None]
    dt_c = 0.075 / (Nc * Nc)
    outs = []
    for max_region in (None, 64):
        gc = mf.MultiFab(clo, chi, boxes=cboxes, ngrow=1, dtype="f64")
        gf = mf.MultiFab(flo, fhi, boxes=fboxes, ngrow=1, dtype="f64", max_region=max_region)
        if max_region:
            assert mf.mf_nregions(gf.h) < len(fboxes)
        gc.from_host(cden)
        gf.from_host(fden)
        mf.mf_amr_advance(gc.h, gf.h, 1, [1.0], dt_c, 2, 2, 2, mf.MF_REFLUX)
        outs.append((gc.to_host(), gf.to_host()))
    np.testing.assert_array_equal(outs[1][0], outs[0][0])
    np.testing.assert_array_equal(outs[1][1], outs[0][1])
    CL = oracle.Level(cboxes, clo, chi, 1, 1)
    FL = oracle.Level(fboxes, flo, fhi, 1, 1)
    c_out, f_out = oracle.amr_advance(CL, FL, 1, dt_c * float(Nc * Nc), CL.from_dense(cden), FL.from_dense(fden), 2,
                                      reflux_faces=True)
    assert rel_err(outs[1][0], CL.to_dense(c_out)) <= FP64_TOL
    fr = FL.to_dense(f_out)
    mask = ~np.isnan(fr)
    np.testing.assert_array_equal(mask, ~np.isnan(outs[1][1]))
    assert float(np.max(np.abs(outs[1][1][mask] - fr[mask])) / np.max(np.abs(fr[mask]))) <= FP64_TOL
