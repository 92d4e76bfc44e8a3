// Second-order variant of the step (instantiation list; the kernel is in step_so.cuh):
// FP64 and FP32 storage, per velocity-set size the warps per segment offered.
#include "step_so.cuh"

using namespace lbmk;

#define LBM_SO_LIST(X)                                                                        \
    X(double, double, 3, 1) X(double, double, 4, 1) X(double, double, 6, 2) X(double, double, 8, 4) \
    X(double, double, 12, 4) X(double, double, 12, 6) X(double, double, 12, 12)                     \
    X(float, float, 3, 1) X(float, float, 4, 1) X(float, float, 6, 1) X(float, float, 8, 2)         \
    X(float, float, 12, 4) X(float, float, 12, 6)

bool so_supported(int prec, int m, int g)
{
#define LBM_SO_HAVE(TS_, TC_, M_, G_) \
    if ((prec == 0) == (sizeof(TS_) == 8) && m == M_ && g == G_) return true;
    LBM_SO_LIST(LBM_SO_HAVE)
#undef LBM_SO_HAVE
    return false;
}

cudaError_t launch_step_so(int prec, int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
#define LBM_SO(TS_, TC_, M_, G_)                                        \
    if ((prec == 0) == (sizeof(TS_) == 8) && m == M_ && g == G_)        \
        return resid ? launch_so<TS_, TC_, M_, G_, true>(a, grid, s) : launch_so<TS_, TC_, M_, G_, false>(a, grid, s);
    LBM_SO_LIST(LBM_SO)
#undef LBM_SO
    return cudaErrorInvalidValue;
}
