// Fused time-step kernel of the finite-difference LB march (sm_103a).
//
// One launch = one time step of the paper's fully discrete scheme (Ghiroldi & Gibelli,
// arXiv:1308.0692, Eqs. 1, 5-9 and the discretisation paragraph): first-order upwind
// transport with Maxwell diffuse-wall ghosts, then explicit-Euler relaxation towards
// the linearised equilibrium w_a (rho + xi_a . j), all in one pass over memory.
//
// Work decomposition.  The state is SoA h[a][c], c = y*nx + x.  A cell is handled by G
// lanes of one warp; lane group g owns the M/G velocity rows iy in [g*M/G, (g+1)*M/G)
// (a = iy*M + ix).  Lanes of the same g hold consecutive cells, so each load/store of
// one velocity plane is a contiguous, coalesced 32/G-element segment.  Per velocity the
// lane reads the own-cell value and the two upwind neighbours (the x neighbour is in
// the same or an adjacent warp, the y neighbour one row away: both served from L1/L2;
// DRAM sees each value once), keeps the transported value in registers, and
// accumulates the row sums sum_ix h*, sum_ix xi_x h*.  The moments rho', j' of the
// cell are then completed with warp shuffles across the G lanes, and the second pass
// relaxes the registers and stores them.  Wall cells first form rho'_w of each wall face
// in FP64 from the incoming populations (Eq. 9 as a discrete flux balance), again
// reduced over the G lanes, and use the ghost w_a [rho'_w (1 + xi_t U) + xi_t U/u_ref]
// (Eq. 8) as upwind value.
//
// Template parameters: TS storage type, TC arithmetic type, M nodes per axis, G lanes per
// cell, RESID: accumulate ||h^{n+1} - h^n||^2 and ||h^{n+1}||^2 (FP64 across threads);
// SOURCE: add a source array after relaxation (correction sweeps of the mixed-precision
// refinement); DEFECT: write h^{n+1} - h^n instead of h^{n+1} (FP64 defect of an FP32
// state).
#pragma once

#include "lbm_internal.h"

namespace lbmk {

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p)
{
    return __ldg(p);
}

template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT>
__global__ void __launch_bounds__(LBM_BLOCK) step_kernel(const StepArgs a)
{
    constexpr int NV = M * M;
    constexpr int RPL = M / G;            // velocity rows per lane
    constexpr int CPW = 32 / G;           // cells per warp
    constexpr int CPB = LBM_BLOCK / G;    // cells per block
    constexpr int HALF = M / 2;           // ix < HALF: xi < 0; ix >= M - HALF: xi > 0
    static_assert(M % G == 0 && 32 % G == 0, "lanes per cell must divide M and 32");

    __shared__ TC s_a0[NV], s_nux[NV], s_nuy[NV], s_cw[NV];
    __shared__ TC s_xi[M];
    __shared__ double s_xi64[M];
    __shared__ double s_red[2][LBM_BLOCK / 32];

    const TC *tab = (sizeof(TC) == 8) ? reinterpret_cast<const TC *>(a.tab64)
                                      : reinterpret_cast<const TC *>(a.tab32);
    for (int i = threadIdx.x; i < NV; i += LBM_BLOCK) {
        s_a0[i] = tab[TAB_A0 * LBM_MAX_V + i];
        s_nux[i] = tab[TAB_NUX * LBM_MAX_V + i];
        s_nuy[i] = tab[TAB_NUY * LBM_MAX_V + i];
        s_cw[i] = tab[TAB_CW * LBM_MAX_V + i];
    }
    if (threadIdx.x < M) {
        s_xi64[threadIdx.x] = a.hdr->xi1[threadIdx.x];
        s_xi[threadIdx.x] = (TC)a.hdr->xi1[threadIdx.x];
    }
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / CPW, cl = lane - g * CPW;
    const long ncells = a.ncells;
    const long cell0 = (long)blockIdx.x * CPB + warp * CPW + cl;
    const bool valid = cell0 < ncells;
    const long c = valid ? cell0 : ncells - 1;   // inactive lanes mirror the last cell
    const int nx = a.nx, ny = a.ny;
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const bool cav = a.cavity != 0;
    const bool wl = cav && x == 0, wr = cav && x == nx - 1;
    const bool wb = y == 0, wt = y == ny - 1;
    const long c_left = (x > 0) ? c - 1 : (cav ? c : c + nx - 1);        // periodic in Couette
    const long c_right = (x < nx - 1) ? c + 1 : (cav ? c : c - (nx - 1));
    const long c_below = wb ? c : c - nx;
    const long c_above = wt ? c : c + nx;
    const TS *__restrict__ h = reinterpret_cast<const TS *>(a.h);
    const double *__restrict__ t64 = a.tab64;
    const bool homog = a.homogeneous != 0;

    // ---- wall densities rho'_w of the faces this cell touches (FP64, Eq. 9) ----
    double rb = 0.0, rt = 0.0, rl = 0.0, rr = 0.0;
    if (__any_sync(FULL, wl || wr || wb || wt)) {
        double sb = 0.0, st = 0.0, sl = 0.0, sr = 0.0;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const double xiy = s_xi64[iy];
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const double v = (double)ld_stream(h + (long)(iy * M + ix) * ncells + c);
                const double xix = s_xi64[ix];
                if (xiy < 0.0) sb -= xiy * v;      // leaving the gas through the bottom wall
                if (xiy > 0.0) st += xiy * v;      // ... through the top wall
                if (ix < HALF) sl -= xix * v;      // ... through the left wall
                if (ix >= M - HALF) sr += xix * v; // ... through the right wall
            }
        }
#pragma unroll
        for (int off = CPW; off < 32; off <<= 1) {
            sb += __shfl_xor_sync(FULL, sb, off);
            st += __shfl_xor_sync(FULL, st, off);
            sl += __shfl_xor_sync(FULL, sl, off);
            sr += __shfl_xor_sync(FULL, sr, off);
        }
        rb = sb * a.hdr->inv_dy_wall;
        rt = st * a.hdr->inv_dy_wall;
        rl = sl * a.hdr->inv_dx_wall;
        rr = sr * a.hdr->inv_dx_wall;
    }

    // ---- transport (upwind) + moment row sums ----
    TC hs[RPL * M];
    TC rho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int iy = g * RPL + r;
        const TC xiy = s_xi[iy];
        const bool ypos = xiy > TC(0), yneg = xiy < TC(0);
        const long cy = ypos ? c_below : (yneg ? c_above : c);
        const bool ywall = (ypos && wb) || (yneg && wt);
        const double rho_y = ypos ? rb : rt;
        const int row_lin = ypos ? TAB_GB_LIN : TAB_GT_LIN;
        const int row_c = ypos ? TAB_GB_C : TAB_GT_C;
        TC R = 0, X = 0;
#pragma unroll
        for (int ix = 0; ix < M; ++ix) {
            const int al = iy * M + ix;
            const TS *hp = h + (long)al * ncells;
            const TC hc = (TC)ld_stream(hp + c);
            TC hx = hc;
            if (ix >= M - HALF) {                        // xi_x > 0: upwind is the left cell
                hx = wl ? (TC)(rl * __ldg(t64 + TAB_W * LBM_MAX_V + al)) : (TC)ld_stream(hp + c_left);
            } else if (ix < HALF) {                      // xi_x < 0: upwind is the right cell
                hx = wr ? (TC)(rr * __ldg(t64 + TAB_W * LBM_MAX_V + al)) : (TC)ld_stream(hp + c_right);
            }
            TC hy;
            if (ywall) {
                double gv = rho_y * __ldg(t64 + row_lin * LBM_MAX_V + al);
                if (!homog) gv += __ldg(t64 + row_c * LBM_MAX_V + al);
                hy = (TC)gv;
            } else {
                hy = (TC)ld_stream(hp + cy);
            }
            const TC v = s_a0[al] * hc + s_nux[al] * hx + s_nuy[al] * hy;
            hs[r * M + ix] = v;
            R += v;
            X += s_xi[ix] * v;
        }
        rho += R;
        jx += X;
        jy += xiy * R;
    }
#pragma unroll
    for (int off = CPW; off < 32; off <<= 1) {
        rho += __shfl_xor_sync(FULL, rho, off);
        jx += __shfl_xor_sync(FULL, jx, off);
        jy += __shfl_xor_sync(FULL, jy, off);
    }

    // ---- relaxation, store, residual ----
    const TC b = (TC)a.hdr->b;
    TS *__restrict__ hn = reinterpret_cast<TS *>(a.hn);
    const TS *__restrict__ src = reinterpret_cast<const TS *>(a.src);
    TC psd = 0, psn = 0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int iy = g * RPL + r;
        const TC q = rho + s_xi[iy] * jy;
#pragma unroll
        for (int ix = 0; ix < M; ++ix) {
            const int al = iy * M + ix;
            const TC e = q + s_xi[ix] * jx;
            TC v = b * hs[r * M + ix] + s_cw[al] * e;
            if (SOURCE) v += (TC)ld_stream(src + (long)al * ncells + c);
            if (RESID || DEFECT) {
                const TC hc = (TC)ld_stream(h + (long)al * ncells + c);
                const TC d = v - hc;
                psd += d * d;
                psn += v * v;
                if (DEFECT) v = d;
            }
            if (valid) hn[(long)al * ncells + c] = (TS)v;
        }
    }

    if (RESID || DEFECT) {
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
            for (int wi = 0; wi < LBM_BLOCK / 32; ++wi) {
                td += s_red[0][wi];
                tn += s_red[1][wi];
            }
            a.partials[2 * blockIdx.x] = td;
            a.partials[2 * blockIdx.x + 1] = tn;
        }
    }
}

template <typename TS, typename TC, int M, int G, bool RESID, bool SOURCE, bool DEFECT>
cudaError_t launch_one(const StepArgs &a, int grid, cudaStream_t s)
{
    step_kernel<TS, TC, M, G, RESID, SOURCE, DEFECT><<<grid, LBM_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
