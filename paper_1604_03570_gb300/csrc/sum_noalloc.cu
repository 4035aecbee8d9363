// sum_noalloc.cu -- compensated FP64 sum of a strided 3-D device array that allocates no
// memory at all: the per-block partial sums live in a file-scope device array instead of a
// buffer made by cudaMalloc or a library allocator.
//
// Who needs it: code that may not call cudaMalloc -- work running while another component
// owns every device allocation (a framework's caching allocator or a fixed memory pool),
// callers in real-time loops where an allocation could stall or fail, and plug-ins loaded
// into processes that forbid new device allocations.  They pass the data and receive the
// result; the library touches only this fixed scratch array.
//
// The array is allocated when the library is loaded on a device and stays there until the
// process exits (every GPU that loads the library holds kMaxBlocks * 16 bytes = 1 MiB).
// All calls share it: two calls whose kernels overlap on the GPU race on it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/mf.h"
#include "mf_internal.h"
#include "reduce_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr long long kCellsPerBlock = (long long)kThreads * kCellsPerThread;
constexpr int kMaxBlocks = 65536;  // input limit: kMaxBlocks * kCellsPerBlock = 268,435,456 cells
constexpr int kMaxDevices = 64;

// partials[0 .. nblocks) per block, partials[kMaxBlocks] the final (sum, 0)
static __device__ __align__(256) double2 g_scratch[kMaxBlocks + 1];

static void *g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device, set once

int fail_na(int code, const char *msg) { return mfk::set_error(code, msg); }

__device__ __forceinline__ double load_f64(const double *p) { return *p; }
__device__ __forceinline__ double load_f64(const float *p) { return (double)*p; }
__device__ __forceinline__ double load_f64(const __nv_bfloat16 *p) { return (double)__bfloat162float(*p); }

// One block per kCellsPerBlock consecutive cells of the (x, y, z) linear order.
template <typename S>
__global__ void __launch_bounds__(kThreads)
    k_sum_strided_partial(const S *__restrict__ data, int nx, int ny, long long sy, long long sz, long long ncell,
                          double2 *partials) {
    double s = 0.0, c = 0.0;
    const long long first = (long long)blockIdx.x * kCellsPerBlock;
    for (int i = threadIdx.x; i < kCellsPerBlock; i += kThreads) {
        const long long q = first + i;
        if (q >= ncell) break;
        const long long x = q % nx, r = q / nx, y = r % ny, z = r / ny;
        mfk::neu_add(s, c, load_f64(data + z * sz + y * sy + x));
    }
    mfk::block_reduce(s, c);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(s, c);
}

__global__ void __launch_bounds__(kThreads) k_sum_strided_final(double2 *partials, int n) {
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) mfk::neu_merge(s, c, partials[i].x, partials[i].y);
    mfk::block_reduce(s, c);
    if (threadIdx.x == 0) partials[kMaxBlocks] = make_double2(__dadd_rn(s, c), 0.0);
}

// Device address of the scratch array for the current device: looked up on the first call
// made on that device (with that device current), then reused.
int scratch_for_current_device(double2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_na(MF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_na(MF_EINVAL, "device ordinal above the supported 64");
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return fail_na(MF_ECUDA, "cudaGetSymbolAddress of the sum scratch failed");
        g_scratch_addr[dev] = p;
    }
    *out = (double2 *)g_scratch_addr[dev];
    return 0;
}

}  // namespace

extern "C" int mf_sum_strided_noalloc(const void *data, int dtype, int nx, int ny, int nz, long long sy, long long sz,
                                      double *out, void *stream) {
    if (!data || !out) return fail_na(MF_EINVAL, "null data or out");
    if (nx < 1 || ny < 1 || nz < 1) return fail_na(MF_EINVAL, "extents must be >= 1");
    if (sy < nx || sz < sy * (long long)ny) return fail_na(MF_EINVAL, "strides overlap the rows or planes");
    if (dtype != MF_F64 && dtype != MF_F32 && dtype != MF_BF16) return fail_na(MF_EINVAL, "unknown dtype");
    const long long ncell = (long long)nx * ny * nz;
    const long long nblocks = (ncell + kCellsPerBlock - 1) / kCellsPerBlock;
    if (nblocks > kMaxBlocks) {
        char buf[160];
        snprintf(buf, sizeof buf, "input of %lld cells exceeds the %lld-cell limit of the static scratch", ncell,
                 (long long)kMaxBlocks * kCellsPerBlock);
        return fail_na(MF_EINVAL, buf);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the call ends by waiting for its result, which a capturing stream cannot do: refuse
    // before enqueueing anything, so that the caller's capture stays intact
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess) return fail_na(MF_ECUDA, cudaGetErrorString(ce));
    if (cs != cudaStreamCaptureStatusNone)
        return fail_na(MF_ESTATE, "mf_sum_strided_noalloc waits for its result and cannot run on a capturing stream");
    double2 *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    switch (dtype) {
        case MF_F64:
            k_sum_strided_partial<<<(int)nblocks, kThreads, 0, s>>>((const double *)data, nx, ny, sy, sz, ncell,
                                                                   scratch);
            break;
        case MF_F32:
            k_sum_strided_partial<<<(int)nblocks, kThreads, 0, s>>>((const float *)data, nx, ny, sy, sz, ncell,
                                                                   scratch);
            break;
        default:
            k_sum_strided_partial<<<(int)nblocks, kThreads, 0, s>>>((const __nv_bfloat16 *)data, nx, ny, sy, sz,
                                                                   ncell, scratch);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_na(MF_ECUDA, cudaGetErrorString(e));
    k_sum_strided_final<<<1, kThreads, 0, s>>>(scratch, (int)nblocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_na(MF_ECUDA, cudaGetErrorString(e));
    double2 res;
    e = cudaMemcpyAsync(&res, scratch + kMaxBlocks, sizeof(double2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_na(MF_ECUDA, cudaGetErrorString(e));
    *out = res.x;
    return 0;
}
