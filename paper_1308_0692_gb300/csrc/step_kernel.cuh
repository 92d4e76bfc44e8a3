// Fused time-step kernel of the finite-difference LB march (sm_103a).
//
// One launch = one time step of the paper's fully discrete scheme (Ghiroldi & Gibelli,
// arXiv:1308.0692, Eqs. 1, 5-9 and the discretisation paragraph): first-order upwind
// transport with Maxwell diffuse-wall ghosts, then explicit-Euler relaxation towards
// the linearised equilibrium w_a (rho + xi_a . j), all in one pass over memory.
//
// Work decomposition.  The state is SoA h[a][c], c = y*nx + x, a = iy*M + ix.  A cell
// is handled by G lanes of one warp; lane group g owns the M/G velocity rows iy in
// [g*M/G, (g+1)*M/G).  Lanes of the same g hold consecutive cells, so every load/store
// of one velocity plane is a contiguous, coalesced 32/G-element segment.  Per velocity
// the lane reads the own-cell value and the two upwind neighbours (the x neighbour lies
// in the same segment, the y neighbour one grid row away: both are served from L1/L2,
// DRAM sees each value about once), keeps the transported value in registers and
// accumulates the row sums sum_ix h*, sum_ix xi_x h*.  The moments rho', j' of the
// cell are completed with warp shuffles across the G lanes; the second pass relaxes
// the registers and stores them.
//
// Coefficients.  The velocity set is a tensor product, so every per-velocity
// coefficient factors into 1-D tables indexed by ix (a compile-time index: a constant
// bank operand of the kernel parameters) and by iy (one register per velocity row):
//   transport   h* = h + nu_x[ix] (h_x - h) + nu_y[iy] (h_y - h),
//   relaxation  h' = (1 - omega) h* + w[ix] (Q_iy + xi[ix] J_iy),
//               Q_iy = omega w[iy] (rho' + xi[iy] j'_y),  J_iy = omega w[iy] j'_x,
// which is h* - omega (h* - w_a (rho' + xi_a . j')) with w_a = w[ix] w[iy].
//
// Walls.  Warps that contain a wall-adjacent cell take a separate code path: they first
// form rho'_w of each wall face in FP64 from the incoming populations (Eq. 9 as a
// discrete flux balance), reduced over the G lanes, and use the ghost
// w_a [rho'_w (1 + xi_t U) + xi_t U / u_ref] (Eq. 8) as the upwind value across the
// wall.  Interior warps run the wall-free path.
//
// Template parameters: TS storage type, TC arithmetic type, M nodes per axis, G lanes per
// cell; RESID: accumulate ||h^{n+1} - h^n||^2 and ||h^{n+1}||^2 (FP64 across threads);
// SOURCE: add a source array after relaxation (correction sweeps of the mixed-precision
// refinement); DEFECT: write h^{n+1} - h^n instead of h^{n+1} (FP64 defect of an FP32
// state).
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

template <typename TS, typename TC, int M, int G, bool SOURCE, bool DEFECT, bool ACC, bool WALLS>
__device__ __forceinline__ void cell_update(const StepArgs &a, const long c, const int x, const int y,
                                            const bool valid, const int g, TC &psd, TC &psn)
{
    constexpr int RPL = M / G;
    constexpr int CPW = 32 / G;
    constexpr int HALF = M / 2;           // ix < HALF: xi < 0; ix >= M - HALF: xi > 0
    const unsigned FULL = 0xffffffffu;
    const long ncells = a.ncells;
    const int nx = a.nx, ny = a.ny;
    const bool cav = a.cavity != 0;
    const bool wl = WALLS && cav && x == 0, wr = WALLS && cav && x == nx - 1;
    const bool wb = WALLS && y == 0, wt = WALLS && y == ny - 1;
    const long c_left = (x > 0) ? c - 1 : (cav ? c : c + nx - 1);        // periodic in Couette
    const long c_right = (x < nx - 1) ? c + 1 : (cav ? c : c - (nx - 1));
    const long c_below = (y > 0) ? c - nx : c;
    const long c_above = (y < ny - 1) ? c + nx : c;
    const TS *__restrict__ h = reinterpret_cast<const TS *>(a.h);

    // ---- wall densities rho'_w of the faces this cell touches (FP64, Eq. 9) ----
    double rb = 0.0, rt = 0.0, rl = 0.0, rr = 0.0;
    if (WALLS) {
        double sb = 0.0, st = 0.0, sl = 0.0, sr = 0.0;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const double xiy = a.xi[iy];
            double rowsum = 0.0, left = 0.0, right = 0.0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const double v = (double)ldg(h + (long)(iy * M + ix) * ncells + c);
                rowsum += v;
                if (ix < HALF) left -= a.xi[ix] * v;       // moving towards the left wall
                if (ix >= M - HALF) right += a.xi[ix] * v; // moving towards the right wall
            }
            if (xiy < 0.0) sb -= xiy * rowsum;             // moving towards the bottom wall
            if (xiy > 0.0) st += xiy * rowsum;             // moving towards the top wall
            sl += left;
            sr += right;
        }
#pragma unroll
        for (int off = CPW; off < 32; off <<= 1) {
            sb += __shfl_xor_sync(FULL, sb, off);
            st += __shfl_xor_sync(FULL, st, off);
            sl += __shfl_xor_sync(FULL, sl, off);
            sr += __shfl_xor_sync(FULL, sr, off);
        }
        rb = sb * a.inv_dy_wall;
        rt = st * a.inv_dy_wall;
        rl = sl * a.inv_dx_wall;
        rr = sr * a.inv_dx_wall;
    }

    // Per-row context of the upwind y neighbour and of the y-wall ghost.
    struct Row {
        TC xiy, nuy;
        long cy;
        bool ywall;
        double rho_y, u_y, drive_y, wy;
    };
    auto row_ctx = [&](int iy) {
        Row rw;
        rw.xiy = pick<TC>(a.xi, a.xi_f, iy);
        rw.nuy = pick<TC>(a.nuy, a.nuy_f, iy);
        const bool ypos = rw.xiy > TC(0), yneg = rw.xiy < TC(0);
        rw.cy = ypos ? c_below : (yneg ? c_above : c);
        rw.ywall = WALLS && ((ypos && wb) || (yneg && wt));
        rw.rho_y = ypos ? rb : rt;
        rw.u_y = ypos ? a.u_bottom : a.u_top;
        rw.drive_y = a.homogeneous ? 0.0 : rw.u_y * a.inv_u_ref;
        rw.wy = a.w1[iy];
        return rw;
    };
    // transported value h*_a of velocity (iy, ix) at this cell
    auto transport = [&](const Row &rw, const int iy, const int ix) -> TC {
        const TS *hp = h + (long)(iy * M + ix) * ncells;
        const TC hc = (TC)ldg(hp + c);
        TC v = hc;
        if (ix >= M - HALF || ix < HALF) {
            TC hx;
            if (WALLS && (ix >= M - HALF ? wl : wr))
                hx = (TC)(a.w1[ix] * rw.wy * (ix >= M - HALF ? rl : rr));
            else
                hx = (TC)ldg(hp + (ix >= M - HALF ? c_left : c_right));
            v += pick<TC>(a.nux, a.nux_f, ix) * (hx - hc);
        }
        TC hy;
        if (WALLS && rw.ywall)
            hy = (TC)(a.w1[ix] * rw.wy * (rw.rho_y * (1.0 + a.xi[ix] * rw.u_y) + a.xi[ix] * rw.drive_y));
        else
            hy = (TC)ldg(hp + rw.cy);
        return v + rw.nuy * (hy - hc);
    };

    // ---- transport + moment row sums (h* kept in registers) ----
    TC hs[RPL * M];
    TC rho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int iy = g * RPL + r;
        const Row rw = row_ctx(iy);
        TC R = 0, X = 0;
#pragma unroll
        for (int ix = 0; ix < M; ++ix) {
            const TC v = transport(rw, iy, ix);
            hs[r * M + ix] = v;
            R += v;
            X += pick<TC>(a.xi, a.xi_f, ix) * v;
        }
        rho += R;
        jx += X;
        jy += rw.xiy * R;
    }
#pragma unroll
    for (int off = CPW; off < 32; off <<= 1) {
        rho += __shfl_xor_sync(FULL, rho, off);
        jx += __shfl_xor_sync(FULL, jx, off);
        jy += __shfl_xor_sync(FULL, jy, off);
    }

    // ---- relaxation, store, residual ----
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
            const long off = (long)(iy * M + ix) * ncells + c;
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

// PART = false: every segment of CPW consecutive cells that contains no wall cell
//               (segments with a wall cell are skipped: a warp-uniform test);
// PART = true:  the segments listed in a.wall_segs (those with a wall cell), one per warp.
// Separate kernels keep the register footprint of the bulk kernel free of the wall code.
template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT, bool PART>
__global__ void __launch_bounds__(LBM_BLOCK) step_kernel(const StepArgs a)
{
    constexpr int CPW = 32 / G;           // cells per warp (one segment)
    constexpr int WPB = LBM_BLOCK / 32;   // warps per block
    constexpr bool ACC = RESID || DEFECT;
    static_assert(M % G == 0 && 32 % G == 0, "lanes per cell must divide M and 32");
    __shared__ double s_red[2][WPB];

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / CPW, cl = lane - g * CPW;
    const long ncells = a.ncells;
    const int nx = a.nx, ny = a.ny;
    long seg;
    bool active;
    if (PART) {
        const long k = (long)blockIdx.x * WPB + warp;
        active = k < a.n_wall_segs;
        seg = active ? a.wall_segs[k] : 0;
    } else {
        seg = (long)blockIdx.x * WPB + warp;
        active = seg * CPW < ncells;
    }
    const long cell0 = seg * CPW + cl;
    const bool valid = active && cell0 < ncells;
    const long c = cell0 < ncells ? cell0 : ncells - 1;   // inactive lanes mirror the last cell
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const bool wall = valid && (y == 0 || y == ny - 1 || (a.cavity && (x == 0 || x == nx - 1)));

    TC psd = 0, psn = 0;
    bool work;
    if (PART) work = active;                      // listed wall segment
    else work = active && !__any_sync(FULL, wall);  // bulk: wall-free segments only
    if (work) {
        if (PART)
            cell_update<TS, TC, M, G, SOURCE, DEFECT, ACC, true>(a, c, x, y, valid, g, psd, psn);
        else
            cell_update<TS, TC, M, G, SOURCE, DEFECT, ACC, false>(a, c, x, y, valid, g, psd, psn);
    }

    if (ACC) {
        double sd = (valid && work) ? (double)psd : 0.0, sn = (valid && work) ? (double)psn : 0.0;
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
            for (int wi = 0; wi < WPB; ++wi) {
                td += s_red[0][wi];
                tn += s_red[1][wi];
            }
            const long slot = (PART ? a.partials_offset : 0) + blockIdx.x;
            a.partials[2 * slot] = td;
            a.partials[2 * slot + 1] = tn;
        }
    }
}

// Bulk kernel over `grid` blocks, then the wall kernel over the listed wall segments.
template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT>
cudaError_t launch_one(const StepArgs &a, int grid, cudaStream_t s)
{
    step_kernel<TS, TC, M, G, RESID, SOURCE, DEFECT, false><<<grid, LBM_BLOCK, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_wall_segs == 0) return e;
    StepArgs b = a;
    b.partials_offset = grid;
    const int wgrid = (a.n_wall_segs + LBM_BLOCK / 32 - 1) / (LBM_BLOCK / 32);
    step_kernel<TS, TC, M, G, RESID, SOURCE, DEFECT, true><<<wgrid, LBM_BLOCK, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace lbmk
