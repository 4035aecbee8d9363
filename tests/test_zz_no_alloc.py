"""The allocation-free sum entry point (mf_sum_strided_noalloc) against mf_sum.

Some callers cannot allocate device memory (another component owns every allocation, or an
allocation inside a real-time loop is not allowed).  For them the library offers a sum that
uses a fixed scratch array compiled into the library.  This test calls it through the C ABI
three times in a row, on differently sized and typed inputs, and checks each result against the
handle-based mf_sum of the same cells (both compensated FP64 sums, each within 2 ulp of the
correctly rounded sum).  It runs last so that a failure here leaves every other test run.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mf = pytest.importorskip("paper_1604_03570_gb300")

pytestmark = pytest.mark.gpu


def _reference(dense, dtype, mgs):
    """mf_sum of a MultiFab holding the dense field (the existing entry point)."""
    nz, ny, nx = dense.shape
    lvl = mf.MultiFab([0, 0, 0], [nx - 1, ny - 1, nz - 1], max_grid_size=mgs, ncomp=1, ngrow=1, dtype=dtype)
    lvl.from_host(dense[None])
    return lvl.sum(0)


def _strided_device_copy(dense, torch_dtype, pad):
    """The field in a padded device array: rows of nx + pad elements, returned with its strides."""
    nz, ny, nx = dense.shape
    full = torch.zeros((nz, ny, nx + pad), dtype=torch_dtype, device="cuda")
    full[:, :, :nx] = torch.from_numpy(dense).to(torch_dtype)
    torch.cuda.synchronize()
    return full, nx + pad, ny * (nx + pad)


def test_noalloc_sum_matches_mf_sum_on_calls_in_a_row():
    """Three calls in a row on one shared scratch array: FP64 (8 blocks), FP32 (64 blocks),
    then BF16 (1 block, on the legacy stream).  The last call is smaller than the one before
    it, so stale partial sums of the 64-block call would show in its result."""
    rng = np.random.default_rng(2718)
    calls = [("f64", (40, 24, 33), torch.float64, None),
             ("f32", (64, 64, 64), torch.float32, None),
             ("bf16", (5, 7, 9), torch.bfloat16, 0)]
    for dtype, (nz, ny, nx), tdt, stream in calls:
        if dtype == "bf16":
            dense = rng.integers(-128, 128, size=(nz, ny, nx)) / 16.0  # 8 significant bits: exact in BF16
        else:
            dense = 1.0 + rng.standard_normal((nz, ny, nx))
        if dtype == "f32":
            dense = dense.astype(np.float32).astype(np.float64)
        ref = _reference(dense, dtype, 16)
        arr, sy, sz = _strided_device_copy(dense, tdt, pad=7)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        got = mf.mf_sum_strided_noalloc(arr.data_ptr(), dtype, nx, ny, nz, sy, sz, stream)
        exact = math.fsum(dense.ravel().tolist())
        assert abs(got - ref) <= 4 * math.ulp(abs(ref)), (dtype, got, ref)
        assert abs(got - exact) <= 2 * math.ulp(abs(exact)), (dtype, got, exact)


def test_noalloc_sum_refuses_a_capturing_stream():
    """The call waits for its result, so on a stream that is capturing a graph it returns
    MF_ESTATE without enqueueing anything, and the capture stays usable."""
    arr = torch.ones(64, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(mf.MFError) as e:
            mf.mf_sum_strided_noalloc(arr.data_ptr(), "f32", 64, 1, 1, 64, 64, s.cuda_stream)
        arr.add_(1.0)
    assert e.value.code == mf.MF_ESTATE
    g.replay()
    torch.cuda.synchronize()
    assert float(arr.sum()) == 128.0
    assert mf.mf_sum_strided_noalloc(arr.data_ptr(), "f32", 64, 1, 1, 64, 64) == 128.0


def test_noalloc_sum_rejects_inputs_beyond_its_scratch():
    arr = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(mf.MFError) as e:
        mf.mf_sum_strided_noalloc(arr.data_ptr(), "f32", 1024, 1024, 257, 1024, 1024 * 1024)
    assert e.value.code == mf.MF_EINVAL
    assert "limit" in str(e.value)
