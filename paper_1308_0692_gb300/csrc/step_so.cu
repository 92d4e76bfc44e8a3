// Second-order variant of the step (instantiation list; the kernel is in step_so.cuh):
// FP64 and FP32 storage, the default warps per segment of each velocity-set size.
#include "step_so.cuh"

using namespace lbmk;

cudaError_t launch_step_so(int prec, int m, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
#define LBM_SO(TS_, TC_, M_, G_)                                                                     \
    if (m == M_) return resid ? launch_so<TS_, TC_, M_, G_, true>(a, grid, s) : launch_so<TS_, TC_, M_, G_, false>(a, grid, s);
    if (prec == 0) {
        LBM_SO(double, double, 3, 1)
        LBM_SO(double, double, 4, 1)
        LBM_SO(double, double, 6, 2)
        LBM_SO(double, double, 8, 4)
        LBM_SO(double, double, 12, 4)
    } else {
        LBM_SO(float, float, 3, 1)
        LBM_SO(float, float, 4, 1)
        LBM_SO(float, float, 6, 1)
        LBM_SO(float, float, 8, 2)
        LBM_SO(float, float, 12, 4)
    }
#undef LBM_SO
    return cudaErrorInvalidValue;
}
