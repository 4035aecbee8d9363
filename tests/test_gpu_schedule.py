"""GPU tests of the schedule choices: tile shapes per box-size class within one launch give the
same bits as one shape for all boxes (and the oracle within 1e-12 in FP64), and the autotuner's
schedule cache (MF_AUTOTUNE_CACHE) is written, reused within the process, and read back from its
file by a fresh lookup."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
mf = pytest.importorskip("paper_1604_03570_gb300")

pytestmark = pytest.mark.gpu

N = 64
LO, HI = [0, 0, 0], [N - 1] * 3
BOXES = synth.uneven_boxes(N, 96, base=32, quantum=8)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_class_tiles_give_identical_bits(dtype):
    dense = np.random.default_rng(5).standard_normal((1, N, N, N))
    if dtype == "f32":
        dense = dense.astype(np.float32).astype(np.float64)
    dt = 0.1125 / (N * N)
    outs = []
    for classes in ({}, {0: (4, 8), 1: (0, 0), 2: (8, 32)}, {0: (0, 16), 2: (32, 8)}):
        g = mf.MultiFab(LO, HI, boxes=BOXES, ngrow=2, dtype=dtype)
        g.set_tile((0, 16, 16))
        for k, (ty, tz) in classes.items():
            mf.mf_set_class_tile(g.h, k, ty, tz)
        assert mf.mf_get_schedule(g.h)["class_tiles"] == classes
        g.from_host(dense)
        g.advance(2, [1.0], dt, 4)
        outs.append(g.to_host())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    if dtype == "f64":
        L = oracle.Level(BOXES, LO, HI, 2, 1)
        ref = L.to_dense(oracle.advance(L, L.from_dense(dense), 2, 0.1125, 4))
        assert float(np.max(np.abs(outs[0] - ref)) / np.max(np.abs(ref))) <= 1e-12


def test_autotune_cache_is_reused_and_read_from_its_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("MF_AUTOTUNE_CACHE", str(path))
    mf.mf_autotune_cache_reset()
    dense = np.random.default_rng(6).standard_normal((1, N, N, N)).astype(np.float32).astype(np.float64)
    dt = 0.1125 / (N * N)
    try:
        def run():
            g = mf.MultiFab(LO, HI, boxes=BOXES, ngrow=2, dtype="f32")
            g.from_host(dense)
            g.advance(2, [1.0], dt, 3)
            return g.to_host(), mf.mf_get_schedule(g.h)

        out1, s1 = run()
        lines = path.read_text().splitlines()
        assert len(lines) == 1
        out2, s2 = run()  # the same geometry: the process's choice, no second line
        assert s2 == s1 and len(path.read_text().splitlines()) == 1
        np.testing.assert_array_equal(out2, out1)
        # another choice written into the file, read back after the process forgets its own
        f = lines[0].split()
        f[1:8] = ["0", "8", "8", "1", "8", "16", "1"]
        f[8:] = ["-1"] * 10
        path.write_text(" ".join(f) + "\n")
        mf.mf_autotune_cache_reset()
        out3, s3 = run()
        assert s3["tile"] == (0, 8, 8) and s3["rows"] == 1 and s3["stages"] == 8 and s3["class_tiles"] == {}
        np.testing.assert_array_equal(out3, out1)
    finally:
        monkeypatch.delenv("MF_AUTOTUNE_CACHE")
        mf.mf_autotune_cache_reset()
