// FP64 instantiations of the fused step (storage and arithmetic in double).
#include "step_kernel.cuh"

using namespace lbmk;

#define LBM_CASE64(M_, G_)                                                                    \
    if (m == M_ && g == G_)                                                                   \
        return resid ? launch_one<double, double, M_, G_, true, false, false>(a, grid, s)     \
                     : launch_one<double, double, M_, G_, false, false, false>(a, grid, s);

cudaError_t launch_step_f64(int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
    LBM_CASE64(3, 1)
    LBM_CASE64(4, 1)
    LBM_CASE64(6, 1)
    LBM_CASE64(6, 2)
    LBM_CASE64(8, 2)
    LBM_CASE64(8, 4)
    LBM_CASE64(12, 2)
    LBM_CASE64(12, 4)
    return cudaErrorInvalidValue;
}
