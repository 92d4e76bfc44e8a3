// FP32 fused step, 3/4/6/8 nodes per axis (perturbation stored and marched in float;
// wall sums across velocity rows and residual reductions across threads in double).
// (instantiation list; the kernel is in step_kernel.cuh)
#include "step_kernel.cuh"

using namespace lbmk;

cudaError_t launch_step_f32_small(int m, int g, int pf, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
    if (m == 3 && g == 1 && pf == 0)
        return resid ? launch_one<float, float, 3, 1, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 3, 1, false, false, false, false>(a, grid, s);
    if (m == 4 && g == 1 && pf == 0)
        return resid ? launch_one<float, float, 4, 1, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 4, 1, false, false, false, false>(a, grid, s);
    if (m == 6 && g == 1 && pf == 0)
        return resid ? launch_one<float, float, 6, 1, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 6, 1, false, false, false, false>(a, grid, s);
    if (m == 6 && g == 2 && pf == 0)
        return resid ? launch_one<float, float, 6, 2, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 6, 2, false, false, false, false>(a, grid, s);
    if (m == 8 && g == 1 && pf == 0)
        return resid ? launch_one<float, float, 8, 1, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 8, 1, false, false, false, false>(a, grid, s);
    if (m == 8 && g == 2 && pf == 0)
        return resid ? launch_one<float, float, 8, 2, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 8, 2, false, false, false, false>(a, grid, s);
    if (m == 8 && g == 4 && pf == 0)
        return resid ? launch_one<float, float, 8, 4, true, false, false, false>(a, grid, s)
                     : launch_one<float, float, 8, 4, false, false, false, false>(a, grid, s);
    if (m == 8 && g == 2 && pf == 1)
        return resid ? launch_one<float, float, 8, 2, true, false, false, true>(a, grid, s)
                     : launch_one<float, float, 8, 2, false, false, false, true>(a, grid, s);
    if (m == 8 && g == 4 && pf == 1)
        return resid ? launch_one<float, float, 8, 4, true, false, false, true>(a, grid, s)
                     : launch_one<float, float, 8, 4, false, false, false, true>(a, grid, s);
    return cudaErrorInvalidValue;
}
