// Second-order step on the strip-tiled FP32 state (instantiation list): the cells with no
// face flux reaching a wall (x in [32, nx - 32), y in [2, ny - 3]) as the column march of
// step_march.cuh with ORDER = 2, and beside it, as its programmatic dependent launch, the
// second-order segment kernel of step_so.cuh over the rest (rows 0, 1, ny - 2, ny - 1 and
// the 32-cell side segments of the other rows), indexing the same tiles.
//
// Load path 8: ring of five row slots (two rows of copies in flight), direct stores; load
// path 9: ring of four (one row in flight) with the stores as bulk asynchronous copies from
// shared memory (the staging buffer leaves no room for a fifth slot at D2Q^h_144).
#include "step_march.cuh"
#include "step_so.cuh"

using namespace lbmk;

namespace {

// At most 64 registers a thread: two of its blocks then fit on an SM beside a march block
// (up to 200 registers x 192 threads), as the first-order wall kernel's do; with one the
// wall segments were still running when the march had finished.
template <int M, int G, bool RESID>
__global__ void __maxnreg__(64) step_so_wall_beside_march_kernel(const StepArgs a)
{
    step_so_body<float, float, M, G, RESID, true, true>(a, blockIdx.x);
    // see step_wall_beside_march_kernel: the grid completes after the march grid
    if (blockIdx.x == 0) asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

template <int M, int G, int S, int TILED, bool RESID>
cudaError_t launch_so_march(const StepArgs &a, int grid, cudaStream_t s)
{
    using Sh = MarchShape<M, G, S, TILED>;
    step_march_kernel<M, G, S, RESID, false, TILED, 2><<<grid, Sh::THREADS, Sh::SMEM, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_wall_segs == 0) return e;
    return launch_wall_beside<G>(step_so_wall_beside_march_kernel<M, G, RESID>, a, grid, s);
}

}  // namespace

#define LBM_SO_MARCH_LIST(X) \
    X(12, 6, 4, 2)           \
    X(12, 6, 5, 1)           \
    X(8, 4, 4, 2)            \
    X(8, 4, 5, 1)

bool so_march_supported(int m, int g, int slots, int tiled)
{
#define LBM_SOM_HAVE(M_, G_, S_, T_) \
    if (m == M_ && g == G_ && slots == S_ && tiled == T_) return true;
    LBM_SO_MARCH_LIST(LBM_SOM_HAVE)
#undef LBM_SOM_HAVE
    return false;
}

cudaError_t launch_step_f32_so_march(int m, int g, int slots, int tiled, bool resid, const StepArgs &a, int grid,
                                     cudaStream_t s)
{
#define LBM_SOM_LAUNCH(M_, G_, S_, T_)                                    \
    if (m == M_ && g == G_ && slots == S_ && tiled == T_)                 \
        return resid ? launch_so_march<M_, G_, S_, T_, true>(a, grid, s) \
                     : launch_so_march<M_, G_, S_, T_, false>(a, grid, s);
    LBM_SO_MARCH_LIST(LBM_SOM_LAUNCH)
#undef LBM_SOM_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t prepare_step_f32_so_march(int m, int g, int slots, int tiled, int *grid)
{
#define LBM_SOM_PREP(M_, G_, S_, T_) \
    if (m == M_ && g == G_ && slots == S_ && tiled == T_) return prepare_march<M_, G_, S_, false, T_, 2>(grid);
    LBM_SO_MARCH_LIST(LBM_SOM_PREP)
#undef LBM_SOM_PREP
    return cudaErrorInvalidValue;
}
