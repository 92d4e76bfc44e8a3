// Kernels of the mixed-precision refinement of the FP32 march:
//   defect  : one step evaluated in FP64 arithmetic on the FP32 state, storing the
//             change M(h) - h (the defect) as float, with its norms;
//   correct : the FP32 step of the homogeneous problem (wall driving removed) plus a
//             source array -- the correction equation delta = L(delta) + defect.
// (generated instantiation list; the kernel is in step_kernel.cuh)
#include "step_kernel.cuh"

using namespace lbmk;

cudaError_t launch_defect_f32(int m, const StepArgs &a, int grid, cudaStream_t s)
{
    if (m == 3) return launch_one<float, double, 3, 1, false, false, true>(a, grid, s);
    if (m == 4) return launch_one<float, double, 4, 1, false, false, true>(a, grid, s);
    if (m == 6) return launch_one<float, double, 6, 2, false, false, true>(a, grid, s);
    if (m == 8) return launch_one<float, double, 8, 4, false, false, true>(a, grid, s);
    if (m == 12) return launch_one<float, double, 12, 6, false, false, true>(a, grid, s);
    return cudaErrorInvalidValue;
}

int defect_lanes(int m) { return m == 12 ? 6 : m == 8 ? 4 : m == 6 ? 2 : 1; }
int correct_lanes(int m) { return m == 12 ? 4 : m == 8 ? 2 : 1; }

cudaError_t launch_correct_f32(int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s)
{
    if (m == 3 && g == 1)
        return resid ? launch_one<float, float, 3, 1, true, true, false>(a, grid, s)
                     : launch_one<float, float, 3, 1, false, true, false>(a, grid, s);
    if (m == 4 && g == 1)
        return resid ? launch_one<float, float, 4, 1, true, true, false>(a, grid, s)
                     : launch_one<float, float, 4, 1, false, true, false>(a, grid, s);
    if (m == 6 && g == 1)
        return resid ? launch_one<float, float, 6, 1, true, true, false>(a, grid, s)
                     : launch_one<float, float, 6, 1, false, true, false>(a, grid, s);
    if (m == 8 && g == 2)
        return resid ? launch_one<float, float, 8, 2, true, true, false>(a, grid, s)
                     : launch_one<float, float, 8, 2, false, true, false>(a, grid, s);
    if (m == 12 && g == 4)
        return resid ? launch_one<float, float, 12, 4, true, true, false>(a, grid, s)
                     : launch_one<float, float, 12, 4, false, true, false>(a, grid, s);
    return cudaErrorInvalidValue;
}
