// FP32 fused step with TMA (bulk asynchronous copy) staging of the upwind halo for the
// wall-free segments (instantiation list; the kernel is in step_tma.cuh).
#include "step_tma.cuh"

using namespace lbmk;

cudaError_t launch_step_f32_tma(int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s,
                               bool merged)
{
#define LBM_TMA(M_, G_) \
    if (m == M_ && g == G_) return resid ? launch_tma<M_, G_, true>(a, grid, s, merged) : launch_tma<M_, G_, false>(a, grid, s, merged);
    LBM_TMA(8, 2)
    LBM_TMA(8, 4)
    LBM_TMA(12, 3)
    LBM_TMA(12, 4)
    LBM_TMA(12, 6)
#undef LBM_TMA
    return cudaErrorInvalidValue;
}

cudaError_t prepare_step_f32_tma(int m, int g)
{
    if (m == 8 && g == 2) return prepare_tma<8, 2>();
    if (m == 8 && g == 4) return prepare_tma<8, 4>();
    if (m == 12 && g == 3) return prepare_tma<12, 3>();
    if (m == 12 && g == 4) return prepare_tma<12, 4>();
    if (m == 12 && g == 6) return prepare_tma<12, 6>();
    return cudaErrorInvalidValue;
}
