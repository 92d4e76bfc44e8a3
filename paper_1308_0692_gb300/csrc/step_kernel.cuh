// Fused time-step kernel of the finite-difference LB march (sm_103a).
//
// One launch = one time step of the paper's fully discrete scheme (Ghiroldi & Gibelli,
// arXiv:1308.0692, Eqs. 1, 5-9 and the discretisation paragraph): first-order upwind
// transport with Maxwell diffuse-wall ghosts, then explicit-Euler relaxation towards
// the linearised equilibrium w_a (rho + xi_a . j), all in one pass over memory.
//
// Work decomposition.  The state is SoA h[a][c], c = y*nx + x, a = iy*M + ix.  The
// cells are cut into segments of 32 consecutive cells; a segment is handled by G warps
// of one block, lane = cell within the segment, warp g of the segment owning the M/G
// velocity rows iy in [g*M/G, (g+1)*M/G).  Every load and store of one velocity plane is
// therefore one full 128-byte line per warp.  Per velocity a lane reads the own-cell
// value and the two upwind neighbours (the x neighbour lies in the same line or the next,
// the y neighbour one grid row away and is read by the neighbouring blocks at about the
// same time: both are served from L1/L2, DRAM sees each value about once), keeps the
// transported value in registers and accumulates the row sums sum_ix h*, sum_ix xi_x h*.
// The moments rho', j' of a cell are completed across its G warps through shared memory
// (fixed summation order: every warp of the segment gets the same bits); the second pass
// relaxes the registers and stores them.
//
// Coefficients.  The velocity set is a tensor product, so every per-velocity coefficient
// factors into 1-D tables indexed by ix (a compile-time index: a constant-bank operand of
// the kernel parameters) and by iy (one register per velocity row):
//   transport   h* = h + nu_x[ix] (h_x - h) + nu_y[iy] (h_y - h),
//   relaxation  h' = (1 - omega) h* + w[ix] (Q_iy + xi[ix] J_iy),
//               Q_iy = omega w[iy] (rho' + xi[iy] j'_y),  J_iy = omega w[iy] j'_x,
// which is h* - omega (h* - w_a (rho' + xi_a . j')) with w_a = w[ix] w[iy].
//
// Walls.  Segments that contain a wall-adjacent cell are handled by a second kernel
// (PART = true) over the list of such segments, so that the bulk kernel carries no wall
// code and keeps a small register footprint.  It first forms rho'_w of each wall face from
// the incoming populations (Eq. 9 as a discrete flux balance): products and sums within a
// velocity row in the arithmetic type, the sums over rows and over the G warps in FP64 --
// per-velocity FP64 work on every lane of a wall segment made this kernel a third of
// the step on GB300, whose FP64 rate is 1/64 of FP32.  The ghost
// w_a [rho'_w (1 + xi_t U) + xi_t U / u_ref] (Eq. 8) is the upwind value across the wall.
//
// Template parameters: TS storage type, TC arithmetic type, M nodes per axis, G warps
// per segment; RESID: accumulate ||h^{n+1} - h^n||^2 and ||h^{n+1}||^2 (FP64 across
// threads); SOURCE: add a source array after relaxation (correction sweeps of the
// mixed-precision refinement); DEFECT: write h^{n+1} - h^n instead of h^{n+1} (FP64
// defect of an FP32 state); PART: wall kernel; PF: bulk variant that issues all own-cell
// and y-neighbour loads of the warp's velocity rows before the arithmetic (more loads in
// flight per warp, more registers); TILED: the state is strip-tiled (lbm_internal.h,
// tile_off) instead of planar -- used by the wall kernel beside the tiled column march.
#pragma once

#include "lbm_internal.h"

namespace lbmk {

template <typename TC>
__device__ __forceinline__ TC pick(const double *d, const float *f, int i);
template <>
__device__ __forceinline__ double pick<double>(const double *d, const float *, int i) { return d[i]; }
template <>
__device__ __forceinline__ float pick<float>(const double *, const float *f, int i) { return f[i]; }

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

template <int G>
struct Shape {
    static constexpr int SPB = G >= 8 ? 1 : 8 / G;   // segments per block
    static constexpr int WARPS = G * SPB;
    static constexpr int THREADS = 32 * WARPS;
};

template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT, bool PART,
          bool PF = false, bool TILED = false>
__device__ __forceinline__ void step_body(const StepArgs &a, const int bid)
{
    constexpr int SPB = Shape<G>::SPB;
    constexpr int WARPS = Shape<G>::WARPS;
    constexpr int RPL = M / G;            // velocity rows per warp
    constexpr int HALF = M / 2;           // ix < HALF: xi < 0; ix >= M - HALF: xi > 0
    constexpr bool ACC = RESID || DEFECT;
    constexpr bool WALLS = PART;
    static_assert(M % G == 0, "warps per segment must divide M");

    __shared__ TC s_mom[3][G][SPB][32];
    __shared__ double s_wall[WALLS ? 4 : 1][G][SPB][32];
    __shared__ double s_red[2][WARPS];

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = warp / G, g = warp - sl * G;
    const long ncells = a.ncells;
    const int nx = a.nx, ny = a.ny;
    long seg;
    bool active;
    if (PART) {
        const long k = (long)bid * SPB + sl;
        active = k < a.n_wall_segs;
        seg = active ? a.wall_segs[k] : 0;
    } else {
        seg = (long)bid * SPB + sl;
        active = seg * 32 < ncells;
    }
    const long cell0 = seg * 32 + lane;
    const bool in_grid = cell0 < ncells;
    const long c = in_grid ? cell0 : ncells - 1;   // lanes past the end mirror the last cell
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const bool cav = a.cavity != 0;
    const bool is_wall = in_grid && (y == 0 || y == ny - 1 || (cav && (x == 0 || x == nx - 1)));
    // bulk kernel: wall-free segments only (the same answer for all G warps of a segment)
    const bool work = PART ? active : (active && !__any_sync(FULL, is_wall));
    const bool valid = work && in_grid;

    const bool wl = WALLS && cav && x == 0, wr = WALLS && cav && x == nx - 1;
    const bool wb = WALLS && y == 0, wt = WALLS && y == ny - 1;
    static_assert(!TILED || (!PF && !SOURCE && !DEFECT), "the tiled state is marched by plain steps only");
    // offsets of the cell and its four neighbours in the state, and the stride between
    // velocities: planar (cell index, stride ncells) or strip-tiled (cavity only)
    long c_at, c_left, c_right, c_below, c_above, vstride;
    if constexpr (TILED) {
        const long tp = a.tile_pitch;
        vstride = LBM_TILE_W;
        c_at = tile_off(x, y, M * M, tp);
        c_left = x > 0 ? tile_off(x - 1, y, M * M, tp) : c_at;
        c_right = x < nx - 1 ? tile_off(x + 1, y, M * M, tp) : c_at;
        c_below = y > 0 ? c_at - (long)M * M * LBM_TILE_W : c_at;
        c_above = y < ny - 1 ? c_at + (long)M * M * LBM_TILE_W : c_at;
    } else {
        vstride = ncells;
        c_at = c;
        c_left = (x > 0) ? c - 1 : (cav ? c : c + nx - 1);        // periodic in Couette
        c_right = (x < nx - 1) ? c + 1 : (cav ? c : c - (nx - 1));
        c_below = (y > 0) ? c - nx : c;
        c_above = (y < ny - 1) ? c + nx : c;
    }
    const TS *__restrict__ h = reinterpret_cast<const TS *>(a.h);

    // ---- wall densities rho'_w of the faces this cell touches (Eq. 9) ----
    // Partial sums over the M velocities of one row are formed in the arithmetic type
    // (exact products of the stored values for FP64; single precision for FP32), the sums
    // across rows and across the G warps in FP64.
    double rb = 0.0, rt = 0.0, rl = 0.0, rr = 0.0;
    if (WALLS) {
        double sb = 0.0, st = 0.0, sls = 0.0, srs = 0.0;
        // Segments in the bottom or top row need the y-wall sums of every lane.  The other
        // wall segments (a cavity's side walls) hold one or two wall cells: their sums are
        // formed cooperatively for those cells only, the velocities dealt to the lanes (products in the
        // arithmetic type, the sum in FP64).
        const bool rows_wall = __any_sync(FULL, in_grid && (y == 0 || y == ny - 1));
        if (work && !rows_wall && cav) {
            constexpr int NSIDE = RPL * HALF;          // velocities of this warp towards one side wall
            for (int side = 0; side < 2; ++side) {
                unsigned m = __ballot_sync(FULL, in_grid && (side == 0 ? x == 0 : x == nx - 1));
                while (m) {
                    const int L = __ffs(m) - 1;
                    m &= m - 1;
                    const long cL = __shfl_sync(FULL, c_at, L);
                    double part = 0.0;
                    for (int k = lane; k < NSIDE; k += 32) {
                        const int r = k / HALF, q = k - r * HALF;
                        const int iy = g * RPL + r, ix = side == 0 ? q : M - HALF + q;
                        const TC v = (TC)ldg(h + (long)(iy * M + ix) * vstride + cL);
                        const TC xv = pick<TC>(a.xi, a.xi_f, ix) * v;
                        part += side == 0 ? -(double)xv : (double)xv;
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(FULL, part, off);
                    if (lane == L) {
                        if (side == 0) sls = part;
                        else srs = part;
                    }
                }
            }
        } else if (work) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int iy = g * RPL + r;
                const double xiy = a.xi[iy];
                TC rowsum = 0, left = 0, right = 0;
#pragma unroll
                for (int ix = 0; ix < M; ++ix) {
                    const TC v = (TC)ldg(h + (long)(iy * M + ix) * vstride + c_at);
                    rowsum += v;
                    if (ix < HALF) left -= pick<TC>(a.xi, a.xi_f, ix) * v;       // towards the left wall
                    if (ix >= M - HALF) right += pick<TC>(a.xi, a.xi_f, ix) * v; // towards the right wall
                }
                if (xiy < 0.0) sb -= xiy * (double)rowsum;             // towards the bottom wall
                if (xiy > 0.0) st += xiy * (double)rowsum;             // towards the top wall
                sls += (double)left;
                srs += (double)right;
            }
        }
        s_wall[0][g][sl][lane] = sb;
        s_wall[WALLS ? 1 : 0][g][sl][lane] = st;
        s_wall[WALLS ? 2 : 0][g][sl][lane] = sls;
        s_wall[WALLS ? 3 : 0][g][sl][lane] = srs;
        __syncthreads();
        sb = st = sls = srs = 0.0;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            sb += s_wall[0][q][sl][lane];
            st += s_wall[WALLS ? 1 : 0][q][sl][lane];
            sls += s_wall[WALLS ? 2 : 0][q][sl][lane];
            srs += s_wall[WALLS ? 3 : 0][q][sl][lane];
        }
        rb = sb * a.inv_dy_wall;
        rt = st * a.inv_dy_wall;
        rl = sls * a.inv_dx_wall;
        rr = srs * a.inv_dx_wall;
    }

    // ---- transport (upwind) + moment row sums, h* kept in registers ----
    // Ghost values (Eq. 8) are evaluated in the arithmetic type from the FP64 densities.
    TC hs[RPL * M];
    TC rho = 0, jx = 0, jy = 0;
    if (work && !WALLS && PF) {
        // bulk path, loads issued ahead of use: all own-cell and y-neighbour values of the
        // warp's rows first, then the x neighbours and the arithmetic
        TC hyv[RPL * M];
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC xiy = pick<TC>(a.xi, a.xi_f, iy);
            const long cy = xiy > TC(0) ? c_below : (xiy < TC(0) ? c_above : c_at);
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const TS *hp = h + (long)(iy * M + ix) * vstride;
                hs[r * M + ix] = (TC)ldg(hp + c_at);
                hyv[r * M + ix] = (TC)ldg(hp + cy);
            }
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC xiy = pick<TC>(a.xi, a.xi_f, iy);
            const TC nuy = pick<TC>(a.nuy, a.nuy_f, iy);
            TC R = 0, X = 0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const TS *hp = h + (long)(iy * M + ix) * vstride;
                const TC hc = hs[r * M + ix];
                TC v = hc;
                if (ix >= M - HALF || ix < HALF) {
                    const TC hx = (TC)ldg(hp + (ix >= M - HALF ? c_left : c_right));
                    v += pick<TC>(a.nux, a.nux_f, ix) * (hx - hc);
                }
                v += nuy * (hyv[r * M + ix] - hc);
                hs[r * M + ix] = v;
                R += v;
                X += pick<TC>(a.xi, a.xi_f, ix) * v;
            }
            rho += R;
            jx += X;
            jy += xiy * R;
        }
    } else if (work) {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC xiy = pick<TC>(a.xi, a.xi_f, iy);
            const TC nuy = pick<TC>(a.nuy, a.nuy_f, iy);
            const bool ypos = xiy > TC(0), yneg = xiy < TC(0);
            const long cy = ypos ? c_below : (yneg ? c_above : c_at);
            const bool ywall = WALLS && ((ypos && wb) || (yneg && wt));
            const TC rho_y = (TC)(ypos ? rb : rt);
            const TC u_y = (TC)(ypos ? a.u_bottom : a.u_top);
            const TC drive_y = a.homogeneous ? TC(0) : (TC)((ypos ? a.u_bottom : a.u_top) * a.inv_u_ref);
            const TC wy = pick<TC>(a.w1, a.w1_f, iy);
            const TC rl_t = (TC)rl, rr_t = (TC)rr;
            TC R = 0, X = 0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const TS *hp = h + (long)(iy * M + ix) * vstride;
                const TC hc = (TC)ldg(hp + c_at);
                const TC xix = pick<TC>(a.xi, a.xi_f, ix);
                const TC wxy = pick<TC>(a.w1, a.w1_f, ix) * wy;
                TC v = hc;
                if (ix >= M - HALF || ix < HALF) {
                    TC hx;
                    if (WALLS && (ix >= M - HALF ? wl : wr))
                        hx = wxy * (ix >= M - HALF ? rl_t : rr_t);
                    else
                        hx = (TC)ldg(hp + (ix >= M - HALF ? c_left : c_right));
                    v += pick<TC>(a.nux, a.nux_f, ix) * (hx - hc);
                }
                TC hy;
                if (WALLS && ywall)
                    hy = wxy * (rho_y * (TC(1) + xix * u_y) + xix * drive_y);
                else
                    hy = (TC)ldg(hp + cy);
                v += nuy * (hy - hc);
                hs[r * M + ix] = v;
                R += v;
                X += xix * v;
            }
            rho += R;
            jx += X;
            jy += xiy * R;
        }
    }
    if (G > 1) {
        s_mom[0][g][sl][lane] = rho;
        s_mom[1][g][sl][lane] = jx;
        s_mom[2][g][sl][lane] = jy;
        __syncthreads();
        rho = jx = jy = 0;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            rho += s_mom[0][q][sl][lane];
            jx += s_mom[1][q][sl][lane];
            jy += s_mom[2][q][sl][lane];
        }
    }

    // ---- relaxation, store, residual ----
    TC psd = 0, psn = 0;
    if (work) {
        const TC b = pick<TC>(&a.b, &a.b_f, 0);
        const TC om = pick<TC>(&a.omega, &a.omega_f, 0);
        TS *__restrict__ hn = reinterpret_cast<TS *>(a.hn);
        const TS *__restrict__ src = reinterpret_cast<const TS *>(a.src);
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC wom = om * pick<TC>(a.w1, a.w1_f, iy);
            const TC q = wom * (rho + pick<TC>(a.xi, a.xi_f, iy) * jy);
            const TC jj = wom * jx;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const long off = (long)(iy * M + ix) * vstride + c_at;
                const TC t = q + pick<TC>(a.xi, a.xi_f, ix) * jj;
                TC v = b * hs[r * M + ix] + pick<TC>(a.w1, a.w1_f, ix) * t;
                if (SOURCE) v += (TC)ldg(src + off);
                if (ACC) {
                    const TC hc = (TC)ldg(h + off);
                    const TC d = v - hc;
                    psd += d * d;
                    psn += v * v;
                    if (DEFECT) v = d;
                }
                if (valid) hn[off] = (TS)v;
            }
        }
    }

    if (ACC) {
        double sd = valid ? (double)psd : 0.0, sn = valid ? (double)psn : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sd += __shfl_xor_sync(FULL, sd, off);
            sn += __shfl_xor_sync(FULL, sn, off);
        }
        if (lane == 0) {
            s_red[0][warp] = sd;
            s_red[1][warp] = sn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double td = 0.0, tn = 0.0;
            for (int wi = 0; wi < WARPS; ++wi) {
                td += s_red[0][wi];
                tn += s_red[1][wi];
            }
            const long slot = (PART ? a.partials_offset : 0) + bid;
            a.partials[2 * slot] = td;
            a.partials[2 * slot + 1] = tn;
        }
    }
}

template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT, bool PART,
          bool PF = false>
__global__ void __launch_bounds__(Shape<G>::THREADS) step_kernel(const StepArgs a)
{
    step_body<TS, TC, M, G, RESID, SOURCE, DEFECT, PART, PF>(a, blockIdx.x);
}

// Bulk and wall segments in one launch: blocks [0, bulk_blocks) take the wall-free
// segments, the rest the wall segments (block-uniform branch).  Used when wall segments
// are a large share of the grid (small grids), where two serialised launches would leave
// the GPU half idle.
template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT>
__global__ void __launch_bounds__(Shape<G>::THREADS) step_kernel_merged(const StepArgs a)
{
    if ((int)blockIdx.x < a.bulk_blocks)
        step_body<TS, TC, M, G, RESID, SOURCE, DEFECT, false, false>(a, blockIdx.x);
    else
        step_body<TS, TC, M, G, RESID, SOURCE, DEFECT, true, false>(a, blockIdx.x - a.bulk_blocks);
}

// Bulk kernel over `grid` blocks, then the wall kernel over the listed wall segments.
// PF selects the bulk variant that issues a warp's loads ahead of their use.
template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT, bool PF = false>
cudaError_t launch_one(const StepArgs &a, int grid, cudaStream_t s)
{
    constexpr int T = Shape<G>::THREADS;
    if (a.merged && !PF) {
        StepArgs b = a;
        b.partials_offset = grid;
        b.bulk_blocks = grid;
        const int wgrid = (a.n_wall_segs + Shape<G>::SPB - 1) / Shape<G>::SPB;
        step_kernel_merged<TS, TC, M, G, RESID, SOURCE, DEFECT><<<grid + wgrid, T, 0, s>>>(b);
        return cudaGetLastError();
    }
    step_kernel<TS, TC, M, G, RESID, SOURCE, DEFECT, false, PF><<<grid, T, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_wall_segs == 0) return e;
    StepArgs b = a;
    b.partials_offset = grid;
    const int wgrid = (a.n_wall_segs + Shape<G>::SPB - 1) / Shape<G>::SPB;
    step_kernel<TS, TC, M, G, RESID, SOURCE, DEFECT, true, false><<<wgrid, T, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace lbmk
