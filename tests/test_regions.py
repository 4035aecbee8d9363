"""Host-side tests of regional storage (no GPU): the regions mf_create_regional groups a box list
into, and the handle's box and region views.

Sec. 2 (Fig. 2): a grid's data may live in regions, each one contiguous block, while the tiles
of the iteration space are logical.  The regions here must be rectangles that their boxes cover
exactly (or single boxes), disjoint, with every side at most max_region cells; every box lies
in exactly one region.  The checks paint cells on small grids (brute force) and compare volumes
on the 512^3 many-box layout."""
import numpy as np
import pytest

import synth

mf = pytest.importorskip("paper_1604_03570_gb300")


def check_regions(boxes, regs, of, max_region):
    boxes = np.asarray(boxes)
    assert of.shape == (len(boxes),) and of.min() >= 0 and of.max() < len(regs)
    for r, R in enumerate(regs):
        members = boxes[of == r]
        assert len(members) >= 1
        for b in members:  # inside its region
            assert np.all(b[:3] >= R[:3]) and np.all(b[3:] <= R[3:])
        ext = R[3:] - R[:3] + 1
        vol = int(np.prod((members[:, 3:] - members[:, :3] + 1).astype(np.int64), axis=1).sum())
        assert vol == int(np.prod(ext.astype(np.int64)))  # covered exactly (boxes are disjoint)
        if len(members) > 1:
            assert np.all(ext <= max_region)
    # regions pairwise disjoint (sweep on x)
    order = np.argsort(regs[:, 0])
    for i in range(len(order)):
        a = regs[order[i]]
        for j in range(i + 1, len(order)):
            b = regs[order[j]]
            if b[0] > a[3]:
                break
            assert np.any(np.maximum(a[:3], b[:3]) > np.minimum(a[3:], b[3:]))


def paint(shape, boxes, lo=(0, 0, 0)):
    """owner[x, y, z] = index of the box holding the cell, -1 for none."""
    own = -np.ones(shape, dtype=np.int64)
    for i, b in enumerate(boxes):
        sl = tuple(slice(b[d] - lo[d], b[3 + d] - lo[d] + 1) for d in range(3))
        assert np.all(own[sl] == -1)
        own[sl] = i
    return own


def test_many_box_level_groups_into_128_cubed_regions():
    """The 512^3 layout of 32768 boxes (cut from 32^3 blocks) has a box-free plane at every
    multiple of 32, so it falls into the 64 blocks of 128^3."""
    boxes = synth.uneven_boxes(512, 32768)
    regs, of = mf.mf_box_regions(boxes, 128)
    assert len(regs) == 64
    assert np.all(regs[:, 3:] - regs[:, :3] + 1 == 128)
    assert np.all(regs[:, :3] % 128 == 0)
    check_regions(boxes, regs, of, 128)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("max_region", [6, 16, 40])
def test_regions_of_random_guillotine_layouts_by_painting(seed, max_region):
    """Random recursive cuts of a 40 x 24 x 16 block (odd positions too), some boxes dropped
    (holes): every cell of a region is a cell of one of its boxes."""
    rng = np.random.default_rng(seed)
    todo, boxes = [[0, 0, 0, 39, 23, 15]], []
    while todo:
        b = todo.pop()
        ext = [b[3 + d] - b[d] + 1 for d in range(3)]
        d = int(np.argmax(ext))
        if ext[d] < 4 or rng.random() < 0.15:
            boxes.append(b)
            continue
        p = b[d] + int(rng.integers(1, ext[d]))
        a, c = list(b), list(b)
        a[3 + d], c[d] = p - 1, p
        todo += [a, c]
    boxes = np.asarray([b for b in boxes if rng.random() > 0.1], dtype=np.int32)
    regs, of = mf.mf_box_regions(boxes, max_region)
    check_regions(boxes, regs, of, max_region)
    own = paint((40, 24, 16), boxes)
    for r, R in enumerate(regs):
        cells = own[R[0]:R[3] + 1, R[1]:R[4] + 1, R[2]:R[5] + 1]
        assert np.all(cells >= 0) and set(np.unique(cells)) == set(np.nonzero(of == r)[0])


def test_a_pinwheel_is_one_region_or_none():
    """Four 2x1 slabs around a 1x1 centre column (a pinwheel of a 3x3 square): every plane
    crosses a box.  The square is covered, so it is one region where it fits; with regions of
    at most 2 cells per side nothing can be cut, and each box is its own region."""
    boxes = np.array([[0, 0, 0, 1, 0, 3], [2, 0, 0, 2, 1, 3], [1, 2, 0, 2, 2, 3], [0, 1, 0, 0, 2, 3],
                      [1, 1, 0, 1, 1, 3]], dtype=np.int32)
    paint((3, 3, 4), boxes)
    regs, of = mf.mf_box_regions(boxes, 64)
    np.testing.assert_array_equal(regs, [[0, 0, 0, 2, 2, 3]])
    regs, of = mf.mf_box_regions(boxes, 2)
    assert len(regs) == 5
    np.testing.assert_array_equal(regs[of], boxes)


def test_regional_handle_keeps_its_boxes_and_reports_its_regions():
    lo, hi = [0, 0, 0], [63, 63, 31]
    boxes = mf._chop(lo, hi, 16)
    h = mf.mf_create_regional(lo, hi, boxes, 2, 2, "f32", 32)
    try:
        np.testing.assert_array_equal(mf.mf_get_boxes(h), boxes)
        regs, of = mf.mf_get_regions(h)
        assert len(regs) == 4 and np.all(regs[:, 3:] - regs[:, :3] + 1 == 32)
        check_regions(boxes, regs, of, 32)
        # the ghost exchange is between regions only: 4 regions of 32^3 in a periodic 64x64x32
        # domain, 2 ghost cells
        _, ghosts = mf.mf_fb_regions(h)
        assert ghosts == 4 * (36 ** 3 - 32 ** 3)
    finally:
        mf.mf_destroy(h)
    h = mf.mf_create_boxes(lo, hi, boxes, 2, 2, "f32")
    try:
        regs, of = mf.mf_get_regions(h)
        np.testing.assert_array_equal(regs, boxes)
        np.testing.assert_array_equal(of, np.arange(len(boxes)))
    finally:
        mf.mf_destroy(h)


@pytest.mark.parametrize("max_region", [0, -3, 241])
def test_regional_create_rejects_region_sizes_out_of_range(max_region):
    with pytest.raises(mf.MFError) as e:
        mf.mf_create_regional([0, 0, 0], [15, 15, 15], mf._chop([0, 0, 0], [15, 15, 15], 8), 1, 1, "f64",
                              max_region)
    assert e.value.code == mf.MF_EINVAL


def test_regional_create_rejects_overlapping_boxes():
    boxes = np.array([[0, 0, 0, 7, 7, 7], [4, 0, 0, 11, 7, 7]], dtype=np.int32)
    with pytest.raises(mf.MFError) as e:
        mf.mf_create_regional([0, 0, 0], [15, 15, 15], boxes, 1, 1, "f64", 32)
    assert e.value.code == mf.MF_EINVAL


def test_class_tiles_are_checked_and_reported():
    """Tile shapes per box-size class (the box's y extent: <= 8, 16, 32, 64, above): arguments
    checked, the classes present reported, mf_set_tile resets them (host only)."""
    boxes = synth.uneven_boxes(64, 96, base=32, quantum=8)
    h = mf.mf_create_boxes([0, 0, 0], [63, 63, 63], boxes, 1, 1, "f32")
    try:
        ny = boxes[:, 4] - boxes[:, 1] + 1
        present = {int(np.searchsorted([8, 16, 32, 64], v)) for v in ny}
        assert set(mf.mf_get_class_tiles(h)) == present
        assert all(v == (-1, -1) for v in mf.mf_get_class_tiles(h).values())
        mf.mf_set_class_tile(h, 0, 4, 0)
        assert mf.mf_get_class_tiles(h)[0] == (4, 0)
        for bad in [(5, 4, 8), (-1, 4, 8), (0, -2, 8), (0, 4, -3)]:
            with pytest.raises(mf.MFError) as e:
                mf.mf_set_class_tile(h, *bad)
            assert e.value.code == mf.MF_EINVAL
        mf.mf_set_tile(h, (0, 8, 8))
        assert all(v == (-1, -1) for v in mf.mf_get_class_tiles(h).values())
    finally:
        mf.mf_destroy(h)
    assert mf.mf_autotune_cache_reset() is None


def test_region_edge_cases():
    """Negative coordinates, a box larger than max_region (kept as its own region), and
    max_region 1 (only single-cell boxes could share; none do)."""
    boxes = np.array([[-8, -8, -8, -1, -1, -1], [0, -8, -8, 7, -1, -1],       # two 8^3 boxes side by side
                      [-8, 0, -8, 7, 39, -1]], dtype=np.int32)              # a 16 x 40 x 8 slab
    regs, of = mf.mf_box_regions(boxes, 16)
    check_regions(boxes, regs, of, 16)
    assert of[0] == of[1] and of[2] != of[0]                                   # the cubes merge, the slab stays
    np.testing.assert_array_equal(regs[of[2]], boxes[2])
    np.testing.assert_array_equal(regs[of[0]], [-8, -8, -8, 7, -1, -1])
    regs, of = mf.mf_box_regions(boxes, 1)
    assert len(regs) == 3
    np.testing.assert_array_equal(regs[of], boxes)
    one = mf.mf_box_regions(boxes[:1], 4)
    np.testing.assert_array_equal(one[0], boxes[:1])


def test_regional_step_bytes_count_the_regions_faces():
    """mf_step_bytes of a regional level is the per-box formula S*C*(2V + 2G + G_face) on its
    regions: the same valid cells, fewer ghost and face cells (host only)."""
    lo, hi = [0, 0, 0], [63, 63, 63]
    boxes = synth.uneven_boxes(64, 96, base=32, quantum=8)
    a = mf.mf_create_boxes(lo, hi, boxes, 2, 2, "f32")
    b = mf.mf_create_regional(lo, hi, boxes, 2, 2, "f32", 64)   # one region: the whole domain
    try:
        V = 64 ** 3
        _, Ga = mf.mf_fb_regions(a)
        _, Gb = mf.mf_fb_regions(b)
        assert Gb == 68 ** 3 - 64 ** 3 and Gb < Ga
        ext = boxes[:, 3:] - boxes[:, :3] + 1
        face_a = int((2 * (ext[:, 0] * ext[:, 1] + ext[:, 1] * ext[:, 2] + ext[:, 0] * ext[:, 2])).sum()) * 2
        face_b = 6 * 64 * 64 * 2
        assert mf.mf_step_bytes(a, 2) == 4 * 2 * (2 * V + 2 * Ga + face_a)
        assert mf.mf_step_bytes(b, 2) == 4 * 2 * (2 * V + 2 * Gb + face_b)
    finally:
        mf.mf_destroy(a)
        mf.mf_destroy(b)
