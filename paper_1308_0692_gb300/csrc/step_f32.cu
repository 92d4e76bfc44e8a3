// FP32 instantiations of the fused step (perturbation h stored and marched in float;
// wall impermeability sums and residual reductions across threads in double).
#include "step_kernel.cuh"

using namespace lbmk;

#define LBM_CASE32(M_, G_)                                                                    \
    if (m == M_ && g == G_)                                                                   \
        return resid ? launch_one<float, float, M_, G_, true, false, false>(a, grid, s)       \
                     : launch_one<float, float, M_, G_, false, false, false>(a, grid, s);

cudaError_t launch_step_f32(int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
    LBM_CASE32(3, 1)
    LBM_CASE32(4, 1)
    LBM_CASE32(6, 1)
    LBM_CASE32(6, 2)
    LBM_CASE32(8, 1)
    LBM_CASE32(8, 2)
    LBM_CASE32(12, 1)
    LBM_CASE32(12, 2)
    LBM_CASE32(12, 4)
    return cudaErrorInvalidValue;
}
