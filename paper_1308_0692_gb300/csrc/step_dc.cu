// Kernels of the mixed-precision refinement of the FP32 march:
//   defect  : one step evaluated in FP64 arithmetic on the FP32 state, storing the
//             change M(h) - h (the defect) as float, with its norms;
//   correct : the FP32 step of the homogeneous problem (wall driving removed) plus a
//             source array -- the correction equation delta = L(delta) + defect.
#include "step_kernel.cuh"

using namespace lbmk;

#define LBM_CASE_DEF(M_, G_)                                                                 \
    if (m == M_) return launch_one<float, double, M_, G_, false, false, true>(a, grid, s);

cudaError_t launch_defect_f32(int m, const StepArgs &a, int grid, cudaStream_t s)
{
    LBM_CASE_DEF(3, 1)
    LBM_CASE_DEF(4, 1)
    LBM_CASE_DEF(6, 1)
    LBM_CASE_DEF(8, 2)
    LBM_CASE_DEF(12, 4)
    return cudaErrorInvalidValue;
}

#define LBM_CASE_COR(M_, G_)                                                                  \
    if (m == M_ && g == G_)                                                                   \
        return resid ? launch_one<float, float, M_, G_, true, true, false>(a, grid, s)        \
                     : launch_one<float, float, M_, G_, false, true, false>(a, grid, s);

cudaError_t launch_correct_f32(int m, int g, bool resid, const StepArgs &a, int grid,
                               cudaStream_t s)
{
    LBM_CASE_COR(3, 1)
    LBM_CASE_COR(4, 1)
    LBM_CASE_COR(6, 1)
    LBM_CASE_COR(8, 1)
    LBM_CASE_COR(12, 2)
    return cudaErrorInvalidValue;
}
