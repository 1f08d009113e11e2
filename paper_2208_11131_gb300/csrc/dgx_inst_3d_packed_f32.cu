// z-marching 3-D FP32-bulk stage kernels over packed total-degree storage (degrees 1 and 3).
#include "dgx_stage3z.cuh"

namespace dgx {

cudaError_t launch_stage3z_packed(int degree, const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid)
{
    if (degree == 1) return run_stage3z_variant<1, true>(a, t, s, grid);
    if (degree == 3) return run_stage3z_variant<3, true>(a, t, s, grid);
    return cudaErrorInvalidValue;
}

}  // namespace dgx
