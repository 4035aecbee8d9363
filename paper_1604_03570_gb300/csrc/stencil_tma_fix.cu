// stencil_tma_fix.cu -- the TMA-staged stencil with exact fixed-point differences for FP64
// storage (fixed_diff.cuh), and the reduction that gives an advance its first fixed-point grid.
// A translation unit of its own so that it compiles in parallel with the other variants.
#include "stencil_tma_kernel.cuh"

namespace mfk {

cudaError_t launch_stencil_tma_fix(int R, int rows, int gb, int nt, const StencilTmaParams &p, int grid,
                                   cudaStream_t s) {
    if (p.ntiles == 0) return cudaSuccess;
    if (p.nstages > kMaxStages || p.nstages < 2 * R + 1 || (p.nstages & (p.nstages - 1))) return cudaErrorInvalidValue;
    if (!tma_has_group(F64, R, rows, gb) || !p.fix_in || !p.fix_out || !p.fix_clear) return cudaErrorInvalidValue;
    return tma_dispatch<double>(R, rows, gb, LaunchF<double, FixA, false>{nt, p, grid, s}, cudaErrorInvalidValue);
}

namespace {
struct OccFix {
    int nt, smem;
    template <int R, int ROWS, int GB> int run() {
        if (nt < 64 || nt > TmaBounds<R, FixA>::threads || nt % 32) return 0;
        if (tma_configure<double, FixA, R, ROWS, GB, false>(smem) != cudaSuccess) return 0;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stencil_tma<double, FixA, R, ROWS, GB, false>, nt,
                                                          smem) != cudaSuccess)
            return 0;
        return per_sm;
    }
};
}  // namespace

int tma_ctas_per_sm_fix(int R, int rows, int gb, int nt, int smem) {
    return tma_dispatch<double>(R, rows, gb, OccFix{nt, smem}, 0);
}

int tma_max_threads_fix(int R) { return R == 1 ? TmaBounds<1, FixA>::threads : R == 2 ? TmaBounds<2, FixA>::threads : TmaBounds<4, FixA>::threads; }

// The largest |u| of one FP64 level, per component, as fix_key (the high word of the encoding
// without its sign): block (box * ncomp + comp, z slice), warps over the slice's valid rows,
// lanes along x; one atomicMax per warp.
__global__ void __launch_bounds__(256) k_fix_emax(const double *base, const FabInfo *ftab, int ncomp, int zsplit,
                                                  unsigned int *out) {
    const int b = blockIdx.x / ncomp, c = blockIdx.x % ncomp;
    const FabInfo f = ftab[b];
    const int nz = f.n[2];
    const int z0 = (int)((long long)nz * blockIdx.y / zsplit), z1 = (int)((long long)nz * (blockIdx.y + 1) / zsplit);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned int m = 0u;
    const int nrows = (z1 - z0) * f.n[1];
    for (int r = warp; r < nrows; r += nw) {
        const int z = z0 + r / f.n[1], y = r % f.n[1];
        const double *row = base + f.org + c * f.cstride + (long long)z * f.plane + (long long)y * f.px;
        for (int x = lane; x < f.n[0]; x += 32) m = max(m, fix_key(row[x]));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0 && m) atomicMax(out + c, m);
}

cudaError_t launch_fix_emax(const void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, unsigned int *out,
                            cudaStream_t s) {
    if (nfab < 1 || ncomp < 1) return cudaSuccess;
    const long long blocks = (long long)nfab * ncomp;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    // enough z slices for four CTAs per SM when the level has few boxes
    long long zs = (4LL * sm_count() + blocks - 1) / blocks;
    if (zs > maxz) zs = maxz;
    if (zs < 1) zs = 1;
    k_fix_emax<<<dim3((unsigned)blocks, (unsigned)zs), 256, 0, s>>>((const double *)base, ftab, ncomp, (int)zs, out);
    return cudaGetLastError();
}

}  // namespace mfk
