// reduce_common.cuh -- FP64 compensated (Neumaier) accumulation and the fixed-shape block
// reduction used by the whole-level sum kernels.
#pragma once

#include <cuda_runtime.h>

namespace mfk {

// Neumaier: running sum s with compensation c.
__device__ __forceinline__ void neu_add(double &s, double &c, double x) {
    double t = __dadd_rn(s, x);
    if (::fabs(s) >= ::fabs(x)) c = __dadd_rn(c, __dadd_rn(__dsub_rn(s, t), x));
    else c = __dadd_rn(c, __dadd_rn(__dsub_rn(x, t), s));
    s = t;
}
// Combine (s2, c2) into (s, c): TwoSum of the heads, compensations added.
__device__ __forceinline__ void neu_merge(double &s, double &c, double s2, double c2) {
    neu_add(s, c, s2);
    c = __dadd_rn(c, c2);
}

__device__ __forceinline__ void block_reduce(double &s, double &c) {
    for (int off = 16; off > 0; off >>= 1) {
        double s2 = __shfl_down_sync(0xffffffffu, s, off);
        double c2 = __shfl_down_sync(0xffffffffu, c, off);
        neu_merge(s, c, s2, c2);
    }
    __shared__ double ss[32], sc[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { ss[wid] = s; sc[wid] = c; }
    __syncthreads();
    if (wid == 0) {
        s = lane < nw ? ss[lane] : 0.0;
        c = lane < nw ? sc[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            double s2 = __shfl_down_sync(0xffffffffu, s, off);
            double c2 = __shfl_down_sync(0xffffffffu, c, off);
            neu_merge(s, c, s2, c2);
        }
    }
}

}  // namespace mfk
