"""The seeded input generators (`synth/`): the counter-based generator against its published
definition, and the invariants of the box lists and fields that every workload relies on."""
import numpy as np
import pytest

import synth


def test_splitmix64_output_function_matches_the_published_sequence():
    """SplitMix64 seeded with 0 (state advanced by the golden-ratio increment, then the output
    function): the published first four outputs."""
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    state = [(k * 0x9E3779B97F4A7C15) % 2 ** 64 for k in (1, 2, 3, 4)]
    got = [int(v) for v in synth._mix(np.array(state, dtype=np.uint64))]
    assert got == expect


def test_draws_are_counter_based_and_in_range():
    a = synth.splitmix64(7, 3, np.arange(1000))
    b = synth.splitmix64(7, 3, np.arange(500, 1000))
    np.testing.assert_array_equal(a[500:], b)                  # value depends on the index only
    assert len(np.unique(a)) == 1000
    assert not np.array_equal(a, synth.splitmix64(7, 4, np.arange(1000)))  # streams differ
    u = synth.uniform(7, 3, np.arange(100000))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def _check_disjoint_cover(boxes, N):
    owner = np.zeros((N, N, N), dtype=np.int32)
    for b in boxes:
        owner[b[2]:b[5] + 1, b[1]:b[4] + 1, b[0]:b[3] + 1] += 1
    return owner


@pytest.mark.parametrize("target", [4096, 32768])
def test_uneven_boxes_tile_the_domain(target):
    N = 512
    boxes = synth.uneven_boxes(N, target)
    assert boxes.shape == (target, 6) and boxes.dtype == np.int32
    ext = boxes[:, 3:] - boxes[:, :3] + 1
    assert ext.min() >= 8 and ext.max() <= 32 and (ext % 8 == 0).all() and (boxes[:, :3] % 8 == 0).all()
    assert int(ext.prod(axis=1).sum()) == N ** 3
    assert (_check_disjoint_cover(boxes, N) == 1).all()
    np.testing.assert_array_equal(boxes, synth.uneven_boxes(N, target))  # seeded: reproducible


def test_sphere_fine_boxes_cover_the_tagged_sphere():
    Nc, r = 256, 2
    boxes = synth.sphere_fine_boxes(Nc, ratio=r)
    Nf = Nc * r
    ext = boxes[:, 3:] - boxes[:, :3] + 1
    assert boxes.min() >= 0 and boxes[:, 3:].max() < Nf
    assert ext.min() >= 16 and ext.max() <= 64
    assert (boxes[:, :3] % 8 == 0).all() and (ext % 8 == 0).all()      # blocking factor 8
    cover = _check_disjoint_cover(boxes, Nf)
    assert cover.max() == 1                                             # disjoint
    x = (np.arange(Nc) + 0.5) / Nc - 0.5
    tag = (x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2) <= 0.25 ** 2
    fine_of_tag = np.repeat(np.repeat(np.repeat(tag, r, 0), r, 1), r, 2)
    assert cover[fine_of_tag].min() == 1                                # every tagged cell refined
    assert cover.sum() < 0.1 * Nf ** 3                                  # and not the whole domain


def test_initial_field_is_layout_free_and_seeded():
    cfg = dict(synth.WORKLOADS["c2"])
    a = synth.initial_field(cfg, N=32)
    b = synth.initial_field(cfg, N=32)
    np.testing.assert_array_equal(a, b)
    assert a.shape == (1, 32, 32, 32) and np.isfinite(a).all()
    modes = synth.sine_modes(synth.FIELD_SEED, 3, 8, 16)
    full = synth.eval_modes((32, 32, 32), modes)
    assert full.shape == (32, 32, 32) and np.abs(full).max() <= 1.0


def test_device_field_generator_matches_host_generator():
    """initial_field_device (torch) gives the host generator's field: identical noise draws,
    modes to rounding."""
    torch = pytest.importorskip("torch")
    cfg = dict(synth.WORKLOADS["c3"])
    host = synth.initial_field(cfg, N=24)
    dev = synth.initial_field_device(cfg, "cpu", N=24).numpy()
    assert host.shape == dev.shape
    assert float(np.max(np.abs(host - dev))) <= 1e-14
    no_modes = dict(cfg, nmodes=0)
    np.testing.assert_array_equal(synth.initial_field(no_modes, N=12), synth.initial_field_device(no_modes, "cpu", N=12).numpy())
