// FP64 fused step, 8/12 nodes per axis (storage and arithmetic in double).
// (instantiation list; the kernel is in step_kernel.cuh)
#include "step_kernel.cuh"

using namespace lbmk;

cudaError_t launch_step_f64_large(int m, int g, int pf, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
    if (m == 8 && g == 2 && pf == 0)
        return resid ? launch_one<double, double, 8, 2, true, false, false, false>(a, grid, s)
                     : launch_one<double, double, 8, 2, false, false, false, false>(a, grid, s);
    if (m == 8 && g == 4 && pf == 0)
        return resid ? launch_one<double, double, 8, 4, true, false, false, false>(a, grid, s)
                     : launch_one<double, double, 8, 4, false, false, false, false>(a, grid, s);
    if (m == 12 && g == 3 && pf == 0)
        return resid ? launch_one<double, double, 12, 3, true, false, false, false>(a, grid, s)
                     : launch_one<double, double, 12, 3, false, false, false, false>(a, grid, s);
    if (m == 12 && g == 4 && pf == 0)
        return resid ? launch_one<double, double, 12, 4, true, false, false, false>(a, grid, s)
                     : launch_one<double, double, 12, 4, false, false, false, false>(a, grid, s);
    if (m == 12 && g == 6 && pf == 0)
        return resid ? launch_one<double, double, 12, 6, true, false, false, false>(a, grid, s)
                     : launch_one<double, double, 12, 6, false, false, false, false>(a, grid, s);
    if (m == 8 && g == 4 && pf == 1)
        return resid ? launch_one<double, double, 8, 4, true, false, false, true>(a, grid, s)
                     : launch_one<double, double, 8, 4, false, false, false, true>(a, grid, s);
    if (m == 12 && g == 6 && pf == 1)
        return resid ? launch_one<double, double, 12, 6, true, false, false, true>(a, grid, s)
                     : launch_one<double, double, 12, 6, false, false, false, true>(a, grid, s);
    return cudaErrorInvalidValue;
}
