"""Host-side tests of libmf (no GPU): the library loads and exports the C ABI, the box chop and
the FillBoundary intersection lists are right, argument errors come back as error codes.

The FillBoundary list is checked against the definition (Sec. 3.1): every ghost cell of
every box is written exactly once, from the valid cell owning its periodic point."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

mf = pytest.importorskip("paper_1604_03570_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(mf.lib, n), n
    assert sorted(mf.EXPORTS) == names


@pytest.mark.parametrize("N,mgs", [((64, 64, 64), 32), ((10, 4, 5), 4), ((256, 256, 256), 64)])
def test_chop_matches_oracle(N, mgs):
    lo, hi = [0, 0, 0], [N[0] - 1, N[1] - 1, N[2] - 1]
    h = mf.mf_create(lo, hi, mgs, 1, 1, "f64")
    try:
        np.testing.assert_array_equal(mf.mf_get_boxes(h), oracle.chop(lo, hi, mgs))
    finally:
        mf.mf_destroy(h)


def _check_fb_regions(h, boxes, dlo, dhi, g, expect_cover=True):
    """Brute-force set check of the FillBoundary list."""
    regs = mf.mf_get_fb_regions(h)
    L = [dhi[d] - dlo[d] + 1 for d in range(3)]
    written = {}
    for r in regs:
        db, sb = int(r[0]), int(r[1])
        dl, sl, n = r[2:5], r[5:8], r[8:11]
        assert np.all(n > 0)
        B, A = boxes[db], boxes[sb]
        for d in range(3):
            # source inside the source box's valid region
            assert A[d] <= sl[d] and sl[d] + n[d] - 1 <= A[3 + d]
            # destination inside the grown destination box, and a periodic image of the source
            assert B[d] - g <= dl[d] and dl[d] + n[d] - 1 <= B[3 + d] + g
            assert (dl[d] - sl[d]) % L[d] == 0
        for z in range(n[2]):
            for y in range(n[1]):
                for x in range(n[0]):
                    key = (db, dl[0] + x, dl[1] + y, dl[2] + z)
                    assert key not in written, "ghost cell written twice"
                    written[key] = sb
    # every written cell is a ghost cell, and (for covering levels) every ghost cell is written
    for (db, i, j, k) in written:
        B = boxes[db]
        assert not (B[0] <= i <= B[3] and B[1] <= j <= B[4] and B[2] <= k <= B[5])
    if expect_cover:
        total = sum(int(np.prod(B[3:] - B[:3] + 1 + 2 * g) - np.prod(B[3:] - B[:3] + 1)) for B in boxes)
        assert len(written) == total
    return len(written)


def test_fb_list_covers_every_ghost_once_uniform():
    lo, hi = [0, 0, 0], [15, 15, 15]
    h = mf.mf_create(lo, hi, 8, 1, 2, "f32")
    try:
        boxes = mf.mf_get_boxes(h)
        n = _check_fb_regions(h, boxes, lo, hi, 2)
        assert mf.mf_fb_regions(h)[1] == n
    finally:
        mf.mf_destroy(h)


def test_fb_list_covers_every_ghost_once_uneven():
    lo, hi = [0, 0, 0], [11, 7, 9]
    boxes = np.array([
        [0, 0, 0, 4, 7, 3], [5, 0, 0, 11, 2, 3], [5, 3, 0, 11, 7, 3],
        [0, 0, 4, 2, 7, 9], [3, 0, 4, 11, 4, 6], [3, 5, 4, 11, 7, 6], [3, 0, 7, 11, 7, 9]], dtype=np.int32)
    h = mf.mf_create_boxes(lo, hi, boxes, 2, 2, "f64")
    try:
        _check_fb_regions(h, boxes, lo, hi, 2)
    finally:
        mf.mf_destroy(h)


def test_fb_list_partial_level_matches_oracle_count():
    lo, hi = [0, 0, 0], [31, 31, 31]
    boxes = np.array([[8, 8, 8, 15, 23, 15], [16, 8, 8, 23, 15, 19], [0, 0, 24, 7, 7, 31]], dtype=np.int32)
    h = mf.mf_create_boxes(lo, hi, boxes, 1, 1, "f32")
    try:
        n = _check_fb_regions(h, boxes, lo, hi, 1, expect_cover=False)
        L = oracle.Level(boxes, lo, hi, 1, 1)
        u = L.from_dense(np.zeros((1, 32, 32, 32)))
        assert n == oracle.fill_boundary(L, u)
    finally:
        mf.mf_destroy(h)


def test_many_small_boxes_list_builds_quickly():
    """4096+ uneven boxes: the bin hash keeps the list build far from O(n^2)."""
    import time
    boxes = synth.uneven_boxes(256, 8192 // 8)
    t0 = time.time()
    h = mf.mf_create_boxes([0, 0, 0], [255, 255, 255], boxes, 2, 2, "f32")
    try:
        n, ghosts = mf.mf_fb_regions(h)
        assert n > 0 and ghosts > 0
        total = sum(int(np.prod(B[3:] - B[:3] + 1 + 4) - np.prod(B[3:] - B[:3] + 1)) for B in boxes)
        assert ghosts == total
    finally:
        mf.mf_destroy(h)
    assert time.time() - t0 < 20


def test_step_bytes_formula():
    h = mf.mf_create([0, 0, 0], [255, 255, 255], 64, 1, 1, "f32")
    try:
        V = 256 ** 3
        G = 64 * (66 ** 3 - 64 ** 3)
        Gf = 64 * 6 * 64 * 64
        assert mf.mf_fb_regions(h)[1] == G
        assert mf.mf_step_bytes(h, 1) == 4 * (2 * V + 2 * G + Gf)
    finally:
        mf.mf_destroy(h)


def test_layout_bytes_alignment():
    for dt, s in (("f64", 8), ("f32", 4), ("bf16", 2)):
        h = mf.mf_create([0, 0, 0], [63, 63, 63], 32, 3, 1, dt)
        try:
            b = mf.mf_bytes(h)
            assert b % 512 == 0
            assert b >= 2 * 3 * 8 * 34 ** 3 * s
        finally:
            mf.mf_destroy(h)


@pytest.mark.parametrize("bad", ["overlap", "outside", "ngrow", "ncomp", "dtype", "empty", "no_boxes", "too_large"])
def test_create_rejects_bad_arguments(bad):
    lo, hi = [0, 0, 0], [15, 15, 15]
    boxes = [[0, 0, 0, 7, 7, 7], [8, 0, 0, 15, 7, 7]]
    kw = dict(ncomp=1, ngrow=1, dtype="f64")
    if bad == "no_boxes":
        boxes = np.zeros((0, 6), dtype=np.int32)
    elif bad == "too_large":  # one FArrayBox of 1302^3 > 2^31 elements (offsets inside one are 32-bit)
        lo, hi = [0, 0, 0], [1299, 1299, 1299]
        boxes = [[0, 0, 0, 1299, 1299, 1299]]
    if bad == "overlap":
        boxes = [[0, 0, 0, 7, 7, 7], [7, 0, 0, 15, 7, 7]]
    elif bad == "outside":
        boxes = [[0, 0, 0, 7, 7, 16]]
    elif bad == "ngrow":
        kw["ngrow"] = 16
    elif bad == "ncomp":
        kw["ncomp"] = 0
    elif bad == "dtype":
        kw["dtype"] = 7
    elif bad == "empty":
        boxes = [[0, 0, 0, 7, -1, 7]]
    with pytest.raises(mf.MFError) as e:
        mf.mf_create_boxes(lo, hi, boxes, kw["ncomp"], kw["ngrow"], kw["dtype"])
    assert e.value.code == mf.MF_EINVAL


def test_calls_before_attach_fail_with_state_error():
    h = mf.mf_create([0, 0, 0], [15, 15, 15], 8, 1, 1, "f32")
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_fill_boundary(h)
        assert e.value.code == mf.MF_ESTATE
        with pytest.raises(mf.MFError) as e:
            mf.mf_advance(h, 1, [1.0], 1e-6, 1)
        assert e.value.code == mf.MF_ESTATE
        with pytest.raises(mf.MFError) as e:
            mf.mf_attach(h, 0x1001, 1 << 30, 0)
        assert e.value.code == mf.MF_EALIGN
    finally:
        mf.mf_destroy(h)


def test_set_tile_roundtrip():
    h = mf.mf_create([0, 0, 0], [63, 63, 63], 32, 1, 1, "f32")
    try:
        assert mf.mf_get_tile(h)[1] is True
        mf.mf_set_tile(h, (32, 8, 4))
        assert mf.mf_get_tile(h) == ((32, 8, 4), False)
        mf.mf_set_tile(h, None)
        assert mf.mf_get_tile(h)[1] is True
    finally:
        mf.mf_destroy(h)


@pytest.mark.parametrize("rows,stages,gb", [(3, 0, 16), (0, 3, 16), (0, 32, 16), (0, 0, 24)])
def test_set_schedule_rejects_out_of_range_values(rows, stages, gb):
    """Rows per thread 1-2, ring slots a power of two up to 16, row groups of 16 or 32 bytes."""
    h = mf.mf_create([0, 0, 0], [63, 63, 63], 32, 1, 1, "f32")
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_set_schedule(h, rows, stages, gb)
        assert e.value.code == mf.MF_EINVAL
        mf.mf_set_schedule(h, 2, 8, 32)  # in range: accepted before any device memory exists
    finally:
        mf.mf_destroy(h)


def test_eval_modes_box_equals_the_block_of_the_full_grid():
    """The sub-box evaluator of the seeded inputs gives the same bits as the full grid."""
    import synth
    m = synth.sine_modes(1604, 100, 4, 8)
    full = synth.eval_modes((32, 32, 32), m)
    blk = synth.eval_modes_box(32, (5, 7, 9), (10, 12, 14), m)
    np.testing.assert_array_equal(full[9:19, 7:19, 5:19], blk)


def test_two_level_step_bytes_by_hand():
    """The benchmark's algorithmic bytes of one coarse step: coarse 32^3 in 8 boxes of 16^3,
    one fine box of 16^3 at ratio 2, 2 substeps, FP32, its whole ghost shell interpolated."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    fb = np.array([[8, 8, 8, 23, 23, 23]])
    g_interp = 18 ** 3 - 16 ** 3
    coarse = 2 * 32 ** 3 + 8 * 6 * 16 * 16       # valid cells read + written, face halo read
    fine = 2 * (2 * 16 ** 3 + 6 * 16 * 16)      # per substep
    interp = 2 * (g_interp + 2 * g_interp / 8)  # ghost writes + coarse reads at two times
    avg = 16 ** 3 + 16 ** 3 / 8
    assert bench.amr_step_bytes(4, 32, 16, fb, 2, 2, g_interp) == 4 * (coarse + fine + interp + avg)


def test_level_step_bytes_by_hand():
    """The benchmark's compulsory bytes of one step of a level of uneven boxes: two boxes of
    8x16x32 and 32x32x32, 2 components, radius 2, FP32."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    boxes = np.array([[0, 0, 0, 7, 15, 31], [8, 0, 0, 39, 31, 31]])
    V = 8 * 16 * 32 + 32 ** 3
    face = 2 * (8 * 16 + 16 * 32 + 8 * 32) + 6 * 32 * 32
    assert bench.manybox_step_bytes(4, 2, boxes, 2) == 4 * 2 * (2 * V + 2 * face)


@pytest.mark.parametrize("N,mgs,g,C,dtype", [(256, 64, 1, 1, "f32"), (512, 128, 4, 5, "f32"), (64, 32, 1, 1, "f64"),
                                              (256, 64, 2, 2, "bf16")])
def test_bench_level_bytes_match_the_library_layout(N, mgs, g, C, dtype):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import paper_1604_03570_gb300 as mf
    h = mf.mf_create([0, 0, 0], [N - 1] * 3, mgs, C, g, dtype)
    try:
        S = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
        assert bench.level_bytes(N, mgs, g, C, S) == mf.mf_bytes(h) // 2
    finally:
        mf.mf_destroy(h)


@pytest.mark.parametrize("ratio,g", [(2, 1), (2, 2), (4, 1), (4, 2)])
def test_interp_work_list_holds_exactly_the_oracles_cells(ratio, g):
    """The interpolation work list (built on the host, no device memory) holds as many cells as
    the oracle interpolates: the fine ghost cells whose point lies in no fine box."""
    Nc = 16
    base = np.array([[4, 4, 4, 7, 11, 7], [8, 4, 4, 11, 7, 9], [0, 0, 12, 3, 3, 15]])
    fb = np.concatenate([base[:, :3] * ratio, (base[:, 3:] + 1) * ratio - 1], axis=1).astype(np.int32)
    hc = mf.mf_create([0, 0, 0], [Nc - 1] * 3, 8, 1, 1, "f64")
    hf = mf.mf_create_boxes([0, 0, 0], [ratio * Nc - 1] * 3, fb, 1, g, "f64")
    try:
        n, runs = mf.mf_interp_cells(hf, hc, ratio)
        CL = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, 8), [0, 0, 0], [Nc - 1] * 3, 1, 1)
        FL = oracle.Level(fb, [0, 0, 0], [ratio * Nc - 1] * 3, g, 1)
        assert n == oracle.interp_cf(FL, CL, ratio, 0.0, CL.alloc(), CL.alloc(), FL.alloc()) > 0
        assert 0 < runs < n  # runs of several cells
        with pytest.raises(mf.MFError) as e:
            mf.mf_interp_cells(hf, hc, 3)
        assert e.value.code == mf.MF_EINVAL
    finally:
        mf.mf_destroy(hf)
        mf.mf_destroy(hc)


def test_interp_work_list_of_the_sphere_workload():
    """The two-level workload: the work list, the oracle and the bench's shell count agree."""
    cfg = synth.WORKLOADS["c4"]
    Nc, r = cfg["N"], cfg["ratio"]
    fb = synth.sphere_fine_boxes(Nc, ratio=r)
    hc = mf.mf_create([0, 0, 0], [Nc - 1] * 3, cfg["max_grid_size"], 1, 1, "f32")
    hf = mf.mf_create_boxes([0, 0, 0], [r * Nc - 1] * 3, fb, 1, 1, "f32")
    try:
        n, runs = mf.mf_interp_cells(hf, hc, r)
        ext = fb[:, 3:] - fb[:, :3] + 1
        assert n == int(((ext + 2).prod(axis=1) - ext.prod(axis=1)).sum()) - mf.mf_fb_regions(hf)[1]
        CL = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, cfg["max_grid_size"]), [0, 0, 0], [Nc - 1] * 3, 1, 1)
        FL = oracle.Level(fb, [0, 0, 0], [r * Nc - 1] * 3, 1, 1)
        assert n == oracle.interp_cf(FL, CL, r, 0.0, CL.alloc(), CL.alloc(), FL.alloc())
        assert n / runs > 10  # runs follow the ghost slabs, not x alone
    finally:
        mf.mf_destroy(hf)
        mf.mf_destroy(hc)


def test_reflux_faces_match_the_oracle():
    """The refluxing plan (host lists only) has the oracle's coarse-fine faces and corrected
    coarse cells: a small layout with periodic images, and the 225-box sphere workload."""
    small = np.array([[8, 8, 4, 15, 23, 19], [16, 8, 4, 23, 15, 11], [0, 24, 26, 5, 31, 31],
                      [26, 24, 26, 31, 31, 31]], dtype=np.int32)
    for Nc, mgs, fb in ((16, 8, small), (256, 64, synth.sphere_fine_boxes(256, ratio=2))):
        hc = mf.mf_create([0, 0, 0], [Nc - 1] * 3, mgs, 1, 1, "f64")
        hf = mf.mf_create_boxes([0, 0, 0], [2 * Nc - 1] * 3, fb, 1, 1, "f64")
        try:
            n, cells = mf.mf_reflux_faces(hf, hc, 2)
            CL = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, mgs), [0, 0, 0], [Nc - 1] * 3, 1, 1)
            FL = oracle.Level(fb, [0, 0, 0], [2 * Nc - 1] * 3, 1, 1)
            cf = oracle.CFFaces(CL, FL, 2)
            assert n == cf.n > 0
            assert cells == len({tuple(f[:3]) for f in cf.faces})
        finally:
            mf.mf_destroy(hf)
            mf.mf_destroy(hc)
    # fine boxes that are not whole coarse cells are refused
    hc = mf.mf_create([0, 0, 0], [15, 15, 15], 8, 1, 1, "f64")
    hf = mf.mf_create_boxes([0, 0, 0], [31, 31, 31], np.array([[1, 0, 0, 8, 7, 7]], dtype=np.int32), 1, 1, "f64")
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_reflux_faces(hf, hc, 2)
        assert e.value.code == mf.MF_EINVAL
    finally:
        mf.mf_destroy(hf)
        mf.mf_destroy(hc)


def test_average_down_work_list_holds_exactly_the_oracles_cells():
    """The average-down work list (host lists only) covers the coarse cells the oracle writes:
    a small layout at ratio 2 and 4, and the 225-box sphere workload."""
    base = np.array([[4, 4, 4, 7, 11, 7], [8, 4, 4, 11, 7, 9], [0, 0, 12, 3, 3, 15]])
    cases = [(16, 8, r, np.concatenate([base[:, :3] * r, (base[:, 3:] + 1) * r - 1], axis=1).astype(np.int32))
             for r in (2, 4)]
    cases.append((256, 64, 2, synth.sphere_fine_boxes(256, ratio=2)))
    for Nc, mgs, r, fb in cases:
        hc = mf.mf_create([0, 0, 0], [Nc - 1] * 3, mgs, 1, 1, "f64")
        hf = mf.mf_create_boxes([0, 0, 0], [r * Nc - 1] * 3, fb, 1, 1, "f64")
        try:
            n, regions = mf.mf_avgdown_cells(hf, hc, r)
            CL = oracle.Level(oracle.chop([0, 0, 0], [Nc - 1] * 3, mgs), [0, 0, 0], [Nc - 1] * 3, 1, 1)
            FL = oracle.Level(fb, [0, 0, 0], [r * Nc - 1] * 3, 1, 1)
            assert n == oracle.average_down(FL, CL, r, FL.alloc(), CL.alloc()) > 0
            assert len(fb) <= regions
        finally:
            mf.mf_destroy(hf)
            mf.mf_destroy(hc)
