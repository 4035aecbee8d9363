// stencil_tma.cu -- launches of the TMA-staged flux-form stencil for plain forward-Euler
// steps, and the residency queries of the balanced schedule; the kernel is in
// stencil_tma_kernel.cuh, its Runge-Kutta-stage instantiations in stencil_tma_rk.cu.
#include "stencil_tma_kernel.cuh"

namespace mfk {

template <typename S, typename A, int R, int ROWS, int GB>
static int tma_occ(int nt, int smem) {
    if (nt < 64 || nt > TmaThreads<S, R, A, ROWS, GB>::value || nt % 32) return 0;
    if (tma_configure<S, A, R, ROWS, GB, false>(smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stencil_tma<S, A, R, ROWS, GB, false>, nt, smem) !=
        cudaSuccess)
        return 0;
    return per_sm;
}

// Residency of the storage type's two instantiations (FP64 differences or not): the smaller,
// so that one schedule fits both in one wave.
template <typename S>
struct OccF {
    int nt, smem;
    template <int R, int ROWS, int GB> int run() {
        return std::min(tma_occ<S, typename NativeArith<S>::T, R, ROWS, GB>(nt, smem),
                        tma_occ<S, double, R, ROWS, GB>(nt, smem));
    }
};

int tma_ctas_per_sm(int dtype, int R, int rows, int gb, int nt, int smem) {
    switch (dtype) {
        case F64: return tma_dispatch<double>(R, rows, gb, OccF<double>{nt, smem}, 0);
        case F32: return tma_dispatch<float>(R, rows, gb, OccF<float>{nt, smem}, 0);
        case BF16: return tma_dispatch<__nv_bfloat16>(R, rows, gb, OccF<__nv_bfloat16>{nt, smem}, 0);
    }
    return 0;
}

int tma_max_threads(int dtype, int R) {
    if (dtype == BF16) return TmaThreads<__nv_bfloat16, 1, float, 1, 16>::value;
    return R == 1 ? TmaBounds<1>::threads : R == 2 ? TmaBounds<2>::threads : TmaBounds<4>::threads;
}
int tma_max_rows(int) { return 2; }
bool tma_has_group(int dtype, int R, int rows, int gb) {
    if (gb == 16) return rows >= 1 && rows <= tma_max_rows(R) && !(R == 4 && rows == 2 && dtype == BF16);
    return gb == 32 && dtype != BF16 && R <= 2 && rows == 1;
}

cudaError_t launch_stencil_tma(int dtype, int R, bool fp64diff, int rows, int gb, int nt, const StencilTmaParams &p,
                               int grid, cudaStream_t s) {
    if (p.ntiles == 0) return cudaSuccess;
    if (p.nstages > kMaxStages || p.nstages < 2 * R + 1 || (p.nstages & (p.nstages - 1))) return cudaErrorInvalidValue;
    if (!tma_has_group(dtype, R, rows, gb)) return cudaErrorInvalidValue;
    if (p.u0[0]) return launch_stencil_tma_rk(dtype, R, fp64diff, rows, gb, nt, p, grid, s);
    return launch_tma_variant<false>(dtype, R, fp64diff, rows, gb, nt, p, grid, s);
}

}  // namespace mfk
