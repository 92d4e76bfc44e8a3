// FP32 step with the interior as a TMA-staged column march (instantiation list; the kernel
// is in step_march.cuh).  Load path 4 keeps two rows of copies in flight per warp (ring of
// four row slots), load path 5 three (ring of five), load path 6 none (ring of two, two
// blocks per SM), load path 7 is path 4 with the relaxation of each row deferred until
// after the next row's transport (steps without the residual), load path 8 is path 4 on the
// strip-tiled state (one contiguous copy per warp and row), load path 9 path 8 with the stores
// as bulk asynchronous copies from shared memory too.  M = 4 (the 16-velocity sets D2Q^h_16
// and D2Q_16) has the tiled forms only.
#include "step_march.cuh"

using namespace lbmk;

#define LBM_MARCH_LIST(X)     \
    X(12, 6, 4, false, 0)     \
    X(12, 6, 5, false, 0)     \
    X(12, 6, 2, false, 0)     \
    X(12, 6, 4, true, 0)      \
    X(12, 12, 4, false, 0)    \
    X(12, 12, 5, false, 0)    \
    X(8, 4, 5, false, 0)      \
    X(8, 2, 5, false, 0)      \
    X(12, 6, 4, false, 1)     \
    X(12, 6, 4, false, 2)     \
    X(8, 4, 4, false, 1)      \
    X(8, 4, 4, false, 2)      \
    X(4, 2, 4, false, 1)      \
    X(4, 2, 4, false, 2)

bool march_supported(int m, int g, int slots, bool defer, int tiled)
{
#define LBM_MARCH_HAVE(M_, G_, S_, D_, T_) \
    if (m == M_ && g == G_ && slots == S_ && defer == D_ && tiled == T_) return true;
    LBM_MARCH_LIST(LBM_MARCH_HAVE)
#undef LBM_MARCH_HAVE
    return false;
}

cudaError_t launch_step_f32_march(int m, int g, int slots, bool defer, int tiled, bool resid, const StepArgs &a,
                                  int grid, cudaStream_t s)
{
#define LBM_MARCH_LAUNCH(M_, G_, S_, D_, T_)                                                       \
    if (m == M_ && g == G_ && slots == S_ && defer == D_ && tiled == T_)                          \
        return resid ? launch_march<M_, G_, S_, D_, true, T_>(a, grid, s)                          \
                     : launch_march<M_, G_, S_, D_, false, T_>(a, grid, s);
    LBM_MARCH_LIST(LBM_MARCH_LAUNCH)
#undef LBM_MARCH_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t prepare_step_f32_march(int m, int g, int slots, bool defer, int tiled, int *grid)
{
#define LBM_MARCH_PREP(M_, G_, S_, D_, T_) \
    if (m == M_ && g == G_ && slots == S_ && defer == D_ && tiled == T_) return prepare_march<M_, G_, S_, D_, T_>(grid);
    LBM_MARCH_LIST(LBM_MARCH_PREP)
#undef LBM_MARCH_PREP
    return cudaErrorInvalidValue;
}
