// stencil_tma_rk.cu -- the TMA-staged stencil's Runge-Kutta-stage instantiations (Sec. 4.2):
// each launch writes rk_a * u0 + rk_b * (forward-Euler value), u0 the state at the start of
// the step.  A translation unit of its own so that the two sets compile in parallel.
#include "stencil_tma_kernel.cuh"

namespace mfk {

cudaError_t launch_stencil_tma_rk(int dtype, int R, bool fp64diff, int rows, int gb, int nt, const StencilTmaParams &p,
                                  int grid, cudaStream_t s) {
    return launch_tma_variant<true>(dtype, R, fp64diff, rows, gb, nt, p, grid, s);
}

}  // namespace mfk
