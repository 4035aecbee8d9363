// stencil_tma_fix.cu -- fixed-point time stepping for FP64 levels (fixed_diff.cuh): the TMA-staged
// stencil over a level held as 64-bit fixed point, and the passes that enter and leave that
// representation.  A translation unit of its own so that it compiles in parallel with the other
// variants.
#include "stencil_tma_kernel.cuh"

namespace mfk {

cudaError_t launch_stencil_tma_fix(int R, int rows, int gb, int nt, const StencilTmaParams &p, int grid,
                                   cudaStream_t s) {
    if (p.ntiles == 0) return cudaSuccess;
    if (p.nstages > kMaxStages || p.nstages < 2 * R + 1 || (p.nstages & (p.nstages - 1))) return cudaErrorInvalidValue;
    if (!tma_has_group_fix(R, rows, gb) || !p.fix_in || !p.fix_out || !p.fix_clear) return cudaErrorInvalidValue;
    return tma_dispatch<long long>(R, rows, gb, LaunchF<long long, FixA, false>{nt, p, grid, s}, cudaErrorInvalidValue);
}

namespace {
struct OccFix {
    int nt, smem;
    template <int R, int ROWS, int GB> int run() {
        if (nt < 64 || nt > TmaThreads<long long, R, FixA, ROWS, GB>::value || nt % 32) return 0;
        if (tma_configure<long long, FixA, R, ROWS, GB, false>(smem) != cudaSuccess) return 0;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stencil_tma<long long, FixA, R, ROWS, GB, false>,
                                                          nt, smem) != cudaSuccess)
            return 0;
        return per_sm;
    }
};

// Rows of the valid cells of one (box, component) in a z slice: block (box * ncomp + comp, slice),
// warps over the rows, lanes along x.  f(row pointer, x) per cell.
template <typename F>
__device__ __forceinline__ void for_valid_rows(const FabInfo &f, int c, int zsplit, long long base_off, F &&fn) {
    const int nz = f.n[2];
    const int z0 = (int)((long long)nz * blockIdx.y / zsplit), z1 = (int)((long long)nz * (blockIdx.y + 1) / zsplit);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nrows = (z1 - z0) * f.n[1];
    for (int r = warp; r < nrows; r += nw) {
        const int z = z0 + r / f.n[1], y = r % f.n[1];
        const long long row = base_off + f.org + c * f.cstride + (long long)z * f.plane + (long long)y * f.px;
        for (int x = lane; x < f.n[0]; x += 32) fn(row + x);
    }
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
    return v;
}

int zslices(int nfab, int ncomp, int maxz) {
    const long long blocks = (long long)nfab * ncomp;
    long long zs = (4LL * sm_count() + blocks - 1) / blocks;  // four CTAs per SM for few boxes
    if (zs > maxz) zs = maxz;
    return zs < 1 ? 1 : (int)zs;
}
}  // namespace

int tma_ctas_per_sm_fix(int R, int rows, int gb, int nt, int smem) {
    return tma_dispatch<long long>(R, rows, gb, OccFix{nt, smem}, 0);
}

namespace {
struct MaxThreadsFix {
    template <int R, int ROWS, int GB> int run() { return TmaThreads<long long, R, FixA, ROWS, GB>::value; }
};
}  // namespace

int tma_max_threads_fix(int R, int rows, int gb) { return tma_dispatch<long long>(R, rows, gb, MaxThreadsFix{}, 0); }

bool tma_has_group_fix(int R, int rows, int gb) {
    if (gb == 16) return rows >= 1 && rows <= (R == 4 ? 1 : 2);
    return gb == 32 && ((R == 1 && rows <= 2) || (R == 2 && rows == 1));
}

// The largest |u| of one FP64 level, per component, as fix_key into set->key.
__global__ void __launch_bounds__(256) k_fix_emax(const double *base, const FabInfo *ftab, int ncomp, int zsplit,
                                                  FixSet *set) {
    const int b = blockIdx.x / ncomp, c = blockIdx.x % ncomp;
    unsigned int m = 0u;
    for_valid_rows(ftab[b], c, zsplit, 0, [&](long long e) { m = max(m, fix_key(base[e])); });
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&set->key[c], m);
}

// FP64 -> fixed point on the first grid of each component, in place; set->E and set->M recorded.
template <int R>
__global__ void __launch_bounds__(256) k_fix_in(void *base, const FabInfo *ftab, int ncomp, int zsplit, FixSet *set,
                                                int *err) {
    const int b = blockIdx.x / ncomp, c = blockIdx.x % ncomp;
    const unsigned int key = set->key[c];
    const int E = fix_first_grid(key, FixW<R>::B);
    if (threadIdx.x == 0) {
        set->E[c] = E;  // every block writes the same value
        if (key >= 0x7ff00000u) atomicOr(err, 2);
    }
    unsigned long long m = 0ull;
    for_valid_rows(ftab[b], c, zsplit, 0, [&](long long e) {
        const long long K = fix_from_f64(((const double *)base)[e], E);
        ((long long *)base)[e] = K;
        const unsigned long long sg = (unsigned long long)(K >> 63);
        m |= ((unsigned long long)K ^ sg) - sg;
    });
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, d);
    if ((threadIdx.x & 31) == 0 && m) atomicOr(&set->M[c], m);
}

// Fixed point on grid set->E -> FP64, in place.
__global__ void __launch_bounds__(256) k_fix_out(void *base, const FabInfo *ftab, int ncomp, int zsplit,
                                                 const FixSet *set) {
    const int b = blockIdx.x / ncomp, c = blockIdx.x % ncomp;
    const int E = set->E[c];
    for_valid_rows(ftab[b], c, zsplit, 0, [&](long long e) {
        ((double *)base)[e] = fix_to_f64(((const long long *)base)[e], E);
    });
}

cudaError_t launch_fix_emax(const void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, FixSet *set,
                            cudaStream_t s) {
    if (nfab < 1 || ncomp < 1) return cudaSuccess;
    if ((long long)nfab * ncomp > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int zs = zslices(nfab, ncomp, maxz);
    k_fix_emax<<<dim3((unsigned)(nfab * ncomp), (unsigned)zs), 256, 0, s>>>((const double *)base, ftab, ncomp, zs, set);
    return cudaGetLastError();
}

cudaError_t launch_fix_in(int R, void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, FixSet *set, int *err,
                          cudaStream_t s) {
    if (nfab < 1 || ncomp < 1) return cudaSuccess;
    if ((long long)nfab * ncomp > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int zs = zslices(nfab, ncomp, maxz);
    const dim3 grid((unsigned)(nfab * ncomp), (unsigned)zs);
    switch (R) {
        case 1: k_fix_in<1><<<grid, 256, 0, s>>>(base, ftab, ncomp, zs, set, err); break;
        case 2: k_fix_in<2><<<grid, 256, 0, s>>>(base, ftab, ncomp, zs, set, err); break;
        case 4: k_fix_in<4><<<grid, 256, 0, s>>>(base, ftab, ncomp, zs, set, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fix_out(void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, const FixSet *set,
                           cudaStream_t s) {
    if (nfab < 1 || ncomp < 1) return cudaSuccess;
    if ((long long)nfab * ncomp > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int zs = zslices(nfab, ncomp, maxz);
    k_fix_out<<<dim3((unsigned)(nfab * ncomp), (unsigned)zs), 256, 0, s>>>(base, ftab, ncomp, zs, set);
    return cudaGetLastError();
}

}  // namespace mfk
