// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#define LBM_MAX_M 12
#define LBM_MAX_V (LBM_MAX_M * LBM_MAX_M)
#define LBM_BLOCK 256
#define LBM_TILE_W 64        // cells per tile row of the strip-tiled state
#define LBM_TILE_SHIFT 32    // tile boundaries at x = 32 (mod 64): the march's strips are whole tiles

// offset of cell (x, y), velocity 0, in the strip-tiled state of n velocities
__host__ __device__ inline long tile_off(long x, long y, int n, long tile_pitch)
{
    const long xs = x + LBM_TILE_SHIFT;
    return (xs / LBM_TILE_W) * tile_pitch + y * (long)n * LBM_TILE_W + (xs % LBM_TILE_W);
}
// tiles of a row of nx cells, and floats of a tiled state
inline long tiles_for(int nx) { return (nx + LBM_TILE_SHIFT + LBM_TILE_W - 1) / LBM_TILE_W; }
inline size_t tiled_values(int n, int nx, int ny) { return (size_t)tiles_for(nx) * ny * n * LBM_TILE_W; }

// Per-velocity coefficient table of one simulation, structure of arrays, in device memory.
// Rows (each LBM_MAX_V long), velocity a = iy*M + ix:
enum {
    TAB_A0 = 0,    // 1 - nu_x - nu_y           (upwind transport, own cell)
    TAB_NUX,       // |xi_x| dt / dx            (upwind neighbour in x)
    TAB_NUY,       // |xi_y| dt / dy            (upwind neighbour in y)
    TAB_CW,        // omega * w_a               (relaxation towards w_a (rho + xi.j))
    TAB_GB_LIN,    // w_a (1 + xi_x U_bottom)   (bottom-wall ghost, coefficient of rho'_w)
    TAB_GB_C,      // w_a xi_x U_bottom / u_ref (bottom-wall ghost, driving term)
    TAB_GT_LIN,    // same, top wall
    TAB_GT_C,
    TAB_W,         // w_a                       (side-wall ghost, walls at rest)
    TAB_ROWS
};

struct TableHeader {
    double xi1[LBM_MAX_M];   // 1-D nodes (ascending)
    double w1[LBM_MAX_M];    // 1-D weights
    double b;                // 1 - omega
    double inv_dx_wall;      // 1 / sum_{xi_x>0} xi_x w  (side walls)
    double inv_dy_wall;      // 1 / sum_{xi_y>0} xi_y w  (bottom / top walls)
};

// Arguments of one fused step launch (passed by value: the 1-D coefficient tables
// live in the kernel-parameter constant bank).
struct StepArgs {
    const void *h;        // state at time n   [n][ncells]
    void *hn;             // state at time n+1 [n][ncells]
    const void *src;      // optional source added after relaxation (correction sweeps)
    double *partials;     // per-block residual partial sums [2 * gridDim.x]
    int nx, ny;
    long ncells;
    // state layout: value (velocity a, cell x, y) at a * pa + y * py + x.  A planar state
    // [a][y][x] (pa = ncells, py = nx): the step kernels index it as a * ncells + c, the
    // diagnostics and the host-transfer relayout take the pitches
    long pa, py;
    // strip-tiled FP32 state of the tiled column march (load path 8), 0 when planar: tiles of
    // LBM_TILE_W cells in x, tile t holding x in [64 t - 32, 64 t + 32), laid out
    // [t][y][a][x - 64 t + 32], so that one row of a 64-cell strip is one contiguous stretch
    // of n * 256 bytes; value (a, x, y) at tile_off(x, y, n, tile_pitch) + a * LBM_TILE_W
    long tile_pitch;      // floats per tile: ny * n * LBM_TILE_W
    int cavity;
    int homogeneous;      // drop the wall driving terms (correction sweeps)
    const int *wall_segs; // segments (32 consecutive cells) that contain a wall cell
    int n_wall_segs;
    long partials_offset; // first partials slot of the wall kernel
    int *status;          // set to 1 by a device-side wait that gave up
    int merged;           // bulk and wall segments in one launch
    int bulk_blocks;      // merged launch: blocks taking the wall-free segments
    int wall_blocks;      // merged TMA launch: leading blocks taking the wall segments
    int *counters;        // column march: [0] next item, [1] finished blocks (zero between launches)
    int march_strips;     // column march: 64-cell strips of the interior
    int march_chunks;     // column march: chunks of the interior rows
    // 1-D tables over the M nodes of one axis (velocity a = iy*M + ix)
    double xi[LBM_MAX_M];   // nodes
    double nux[LBM_MAX_M];  // |xi| dt / dx (0 for a single periodic Couette column)
    double nuy[LBM_MAX_M];  // |xi| dt / dy
    double w1[LBM_MAX_M];   // 1-D weights (w_a = w1[ix] w1[iy])
    float xi_f[LBM_MAX_M], nux_f[LBM_MAX_M], nuy_f[LBM_MAX_M], w1_f[LBM_MAX_M];
    // second-order transport, per axis (0: x, 1: y) and node with Courant number nu:
    // P = nu (3 - nu) / 2, B = nu (2 - nu), and the second upwind cell's coefficient
    // -C = -nu (1 - nu) / 2 held negated (step_so.cuh, step_march.cuh)
    double so_p[2][LBM_MAX_M], so_b[2][LBM_MAX_M], so_c[2][LBM_MAX_M];
    float so_p_f[2][LBM_MAX_M], so_b_f[2][LBM_MAX_M], so_c_f[2][LBM_MAX_M];
    double omega, b;        // dt / Kn, 1 - omega
    float omega_f, b_f;
    double inv_dx_wall;     // 1 / sum_{xi_x>0} xi_x w  (side walls)
    double inv_dy_wall;     // 1 / sum_{xi_y>0} xi_y w  (bottom / top walls)
    double u_bottom, u_top; // wall speeds
    double inv_u_ref;       // 1 / u_ref
};

// Launchers (step_*.cu).  `g` selects the warps per 32-cell segment; a launch is the
// bulk kernel over `grid` blocks followed by the wall kernel over the wall segments; the
// residual partials of one step occupy grid + wall_grid(g, n_wall_segs) slots.
cudaError_t launch_step(int prec, int m, int g, int pf, bool resid, const StepArgs &a, int grid,
                        cudaStream_t s);
cudaError_t launch_defect(int m, const StepArgs &a, int grid, cudaStream_t s);
int default_lanes_per_cell(int prec, int m);
inline int segs_per_block(int g) { return g >= 8 ? 1 : 8 / g; }
inline int wall_grid(int g, int n_wall_segs) { return (n_wall_segs + segs_per_block(g) - 1) / segs_per_block(g); }
bool step_supported(int prec, int m, int g, int pf);

// Reductions and diagnostics (reduce.cu)
cudaError_t launch_finalize_residual(const double *partials, int nparts, double *result,
                                     cudaStream_t s);
// Sum `nparts` (d, n) pairs in a fixed order into out[0..1] (and r, flag when nres >= 4).
cudaError_t launch_finalize_pairs(const double *partials, int nparts, double *out, int nres,
                                  cudaStream_t s);
cudaError_t launch_norms(const void *a, const void *b, long count, int prec, double *partials,
                         int nparts, double *out, cudaStream_t s);
int norms_blocks(long count);
// moments of a planar state (tile_pitch 0) or of the strip-tiled FP32 state (its tile pitch);
// need_p false: rho, u_x, u_y only (outputs 3-5 are not written)
cudaError_t launch_moments(int prec, const void *h, long pa, long py, const double *tab64, const TableHeader *hdr,
                           int m, int nx, int ny, double u_ref, double *out6, cudaStream_t s, long tile_pitch = 0,
                           bool need_p = true);
cudaError_t launch_face_flux(int prec, const void *h, long pa, long py, const double *tab64, const TableHeader *hdr,
                             int m, int nx, int ny, int cavity, double u_ref, double *flux_y,
                             double *flux_x, double *wall_sums, cudaStream_t s);
// face fluxes with the second-order transport's face values (step_so.cuh)
cudaError_t launch_face_flux2(int prec, const void *h, long pa, long py, const double *tab64, const TableHeader *hdr,
                              int m, int nx, int ny, int cavity, double u_ref, double *flux_y, double *flux_x,
                              cudaStream_t s);
// copy between the host-order planar FP64 state [a][y][x] and a device state of the given
// layout and precision (to_layout: planar FP64 -> layout; else layout -> planar FP64)
cudaError_t launch_relayout(int prec, bool to_layout, double *planar, void *state, int n, int nx, int ny,
                            long pa, long py, cudaStream_t s);

cudaError_t launch_convert(const double *src, float *dst, long count, cudaStream_t s);
// FP32 state planar [a][y][x] <-> strip-tiled (to_tiled: planar -> tiled)
cudaError_t launch_tile_convert(bool to_tiled, const float *src, float *dst, int n, int nx, int ny, long tile_pitch,
                                cudaStream_t s);
// the same for velocities a0 .. a0 + na - 1 of the n
cudaError_t launch_tile_convert_range(bool to_tiled, const float *src, float *dst, int n, int a0, int na, int nx,
                                      int ny, long tile_pitch, cudaStream_t s);
// state h from device FP64 moments [6][ncells] (rho, u_x, u_y, P_xx, P_xy, P_yy)
cudaError_t launch_moments_state(int prec, const double *mom, int nx, int ny, long pa, long py, int m,
                                 const TableHeader *hdr, double u_ref, void *h, cudaStream_t s);
cudaError_t launch_add_f32(float *y, const float *x, long count, cudaStream_t s);
cudaError_t launch_widen(const float *src, double *dst, long count, cudaStream_t s);

// warm start (mlp.cu): h from normalised predicted moments [ncells][6]
cudaError_t launch_warm_state(const float *pred, int nx, int ny, long pa, long py, int m, const double *xi1,
                              const double *w1, double uw_over_uref, void *h, int prec, cudaStream_t s,
                              bool tiled32 = false);

// Host quadrature (quadrature.cpp)
bool lbm_rule_1d(int kind, int n, std::vector<double> &nodes, std::vector<double> &weights);
