// Second-order variant of the fused step (an extension of the paper's scheme): the
// transport is the finite-volume update h*_i = h_i - (F_out - F_in) per direction with the
// upwind-biased second-order (Beam-Warming) face flux
//     F = nu [h_u + (1 - nu)/2 (h_u - h_uu)]      (h_u upwind cell, h_uu the next one),
// first order (F = nu h_u) where h_uu would lie beyond a wall, nu times the wall-emitted
// population (Eq. 8) across a wall face.  The wall density of Eq. (9) balances the outflow
// through the wall face as this flux computes it: it is formed from the face values
// h + (1 - nu)/2 (h - h_inner) of the wall-adjacent cell.  Paired with symmetric splitting
// and exact relaxation (relaxation factor exp(-omega) on the stored half-relaxed state,
// set by the host), the steady state converges at second order in the grid spacing.
//
// Same decomposition as step_kernel.cuh (32-cell segments, G warps per segment owning M/G
// velocity rows, moments through shared memory, wall segments in a second kernel), with
// register loads of the two upwind neighbours per direction.  TILED: the state is the
// strip-tiled FP32 layout of the column march (lbm_internal.h); the kernel then serves as
// the wall kernel beside the second-order march (step_so_march.cu).
#pragma once

#include "step_kernel.cuh"

namespace lbmk {

// a * b + c rounded once, in the arithmetic type
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename TS, typename TC, int M, int G, bool RESID, bool PART, bool TILED = false>
__device__ __forceinline__ void step_so_body(const StepArgs &a, const int bid)
{
    constexpr int SPB = Shape<G>::SPB;
    constexpr int WARPS = Shape<G>::WARPS;
    constexpr int RPL = M / G;
    constexpr int HALF = M / 2;   // ix < HALF: xi < 0; ix >= M - HALF: xi > 0
    static_assert(M % G == 0, "warps per segment must divide M");

    __shared__ TC s_mom[3][G][SPB][32];
    __shared__ double s_wall[PART ? 4 : 1][G][SPB][32];
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
    const long c = in_grid ? cell0 : ncells - 1;
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const bool cav = a.cavity != 0;
    const bool xmove = cav || nx > 1;
    const bool is_wall = in_grid && (y == 0 || y == ny - 1 || (cav && (x == 0 || x == nx - 1)));
    const bool work = PART ? active : (active && !__any_sync(FULL, is_wall));
    const bool valid = work && in_grid;
    const TS *__restrict__ h = reinterpret_cast<const TS *>(a.h);

    // offset of velocity 0 of cell (xx, yy) and the stride between velocities: planar, or
    // strip-tiled (cavity only)
    auto at = [&](int xx, int yy) -> long {
        if constexpr (TILED) return tile_off(xx, yy, M * M, a.tile_pitch);
        else return (long)yy * nx + xx;
    };
    const long vstride = TILED ? (long)LBM_TILE_W : ncells;
    // neighbour cells along x (periodic in Couette, clamped in the cavity) and y (clamped);
    // a clamped index is only ever read where its value is not used
    auto xcell = [&](int k) -> long {
        int xx = x + k;
        if (!cav) xx = ((xx % nx) + nx) % nx;
        else xx = xx < 0 ? 0 : (xx > nx - 1 ? nx - 1 : xx);
        return at(xx, y);
    };
    auto ycell = [&](int k) -> long {
        int yy = y + k;
        yy = yy < 0 ? 0 : (yy > ny - 1 ? ny - 1 : yy);
        return at(x, yy);
    };
    const long cat = at(x, y);
    const long cxm1 = xcell(-1), cxm2 = xcell(-2), cxp1 = xcell(1), cxp2 = xcell(2);
    const long cym1 = ycell(-1), cym2 = ycell(-2), cyp1 = ycell(1), cyp2 = ycell(2);

    // ---- wall densities (Eq. 9) balancing the second-order outflow through each wall face ----
    // Segments in the bottom or top row form the y-wall sums on every lane (partial sums of
    // a velocity row in the arithmetic type, across rows and warps in FP64).  A side wall
    // touches one or two cells of a segment: their sums are formed cooperatively, the
    // velocities towards that wall dealt to the lanes (products in the arithmetic type, the
    // sum in FP64), instead of by every lane of the segment.
    // the densities and the wall terms of Eq. (8) in the arithmetic type, formed once per
    // lane and only in warps with a lane at that wall (FP64 work runs on this GPU's slowest
    // pipe: forming all four on every lane of a wall segment kept it two thirds busy)
    TC rb = 0, rt = 0, rl = 0, rr = 0;
    TC ub = 0, ut = 0, db = 0, dt = 0;
    const bool rows_wall = PART && __any_sync(FULL, in_grid && (y == 0 || y == ny - 1));
    if (PART) {
        double sb = 0.0, st = 0.0, sls = 0.0, srs = 0.0;
        if (work && rows_wall) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int iy = g * RPL + r;
                const int ys = iy >= M - HALF ? 1 : (iy < HALF ? -1 : 0);
                if (ys == 0) continue;
                const TC nuy = pick<TC>(a.nuy, a.nuy_f, iy);
                const TC kap = TC(0.5) * (TC(1) - nuy);
                // towards the bottom wall (xi_y < 0): inner cell y + 1; top: y - 1
                const long cin = ys < 0 ? cyp1 : cym1;
                TC sy = 0;
#pragma unroll
                for (int ix = 0; ix < M; ++ix) {
                    const TS *hp = h + (long)(iy * M + ix) * vstride;
                    const TC v = (TC)ldg(hp + cat);
                    sy += v + kap * (v - (TC)ldg(hp + cin));
                }
                const double xiy = a.xi[iy];
                if (ys < 0) sb -= xiy * (double)sy;
                else st += xiy * (double)sy;
            }
        }
        if (work && cav) {
            constexpr int NSIDE = RPL * HALF;   // velocities of this warp towards one side wall
            for (int side = 0; side < 2; ++side) {
                unsigned mask = __ballot_sync(FULL, in_grid && (side == 0 ? x == 0 : x == nx - 1));
                while (mask) {
                    const int L = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const long cL = __shfl_sync(FULL, cat, L);
                    const long cI = __shfl_sync(FULL, side == 0 ? cxp1 : cxm1, L);   // inner neighbour
                    double part = 0.0;
                    for (int k = lane; k < NSIDE; k += 32) {
                        const int r = k / HALF, q = k - r * HALF;
                        const int iy = g * RPL + r, ix = side == 0 ? q : M - HALF + q;
                        const TS *hp = h + (long)(iy * M + ix) * vstride;
                        const TC v = (TC)ldg(hp + cL);
                        const TC nux = pick<TC>(a.nux, a.nux_f, ix);
                        const TC fv = v + TC(0.5) * (TC(1) - nux) * (v - (TC)ldg(hp + cI));
                        const TC xf = pick<TC>(a.xi, a.xi_f, ix) * fv;
                        part += side == 0 ? -(double)xf : (double)xf;
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(FULL, part, off);
                    if (lane == L) {
                        if (side == 0) sls = part;
                        else srs = part;
                    }
                }
            }
        }
        s_wall[0][g][sl][lane] = sb;
        s_wall[PART ? 1 : 0][g][sl][lane] = st;
        s_wall[PART ? 2 : 0][g][sl][lane] = sls;
        s_wall[PART ? 3 : 0][g][sl][lane] = srs;
        __syncthreads();
        // totals over the warps of the segment
        auto total = [&](int k) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < G; ++q) t += s_wall[k][q][sl][lane];
            return t;
        };
        if (__any_sync(FULL, in_grid && y == 0)) rb = (TC)(total(0) * a.inv_dy_wall);
        if (__any_sync(FULL, in_grid && y == ny - 1)) rt = (TC)(total(1) * a.inv_dy_wall);
        if (cav && __any_sync(FULL, in_grid && x == 0)) rl = (TC)(total(2) * a.inv_dx_wall);
        if (cav && __any_sync(FULL, in_grid && x == nx - 1)) rr = (TC)(total(3) * a.inv_dx_wall);
        if (rows_wall) {
            ub = (TC)a.u_bottom;
            ut = (TC)a.u_top;
            db = a.homogeneous ? TC(0) : (TC)(a.u_bottom * a.inv_u_ref);
            dt = a.homogeneous ? TC(0) : (TC)(a.u_top * a.inv_u_ref);
        }
    }

    // ---- second-order transport + moment row sums ----
    // h* = h - D_x - D_y, per direction the face-flux difference with Courant number nu,
    // P = nu (3 - nu) / 2, B = nu (2 - nu), C = nu (1 - nu) / 2 (host tables) and h_1, h_2
    // the first and second upwind cells:
    //     D = P h - B h_1 + C h_2     two or more cells from the upwind wall (or periodic)
    //     D = P h - P h_1             the second cell (first-order inflow face)
    //     D = nu h - nu g             the wall-adjacent cell (g: the wall-emitted population)
    // Every neighbour is loaded (clamped index, unused where its coefficient is 0) and the
    // case only selects coefficients, so that the loads of all velocities can be in flight
    // together.  Position along a direction counted from its upwind end: 0 is the
    // wall-adjacent cell.
    const int ixp = x, ixn = nx - 1 - x, iyp = y, iyn = ny - 1 - y;
    TC hs[RPL * M];
    TC rho = 0, jx = 0, jy = 0;
    if (work) {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC xiy = pick<TC>(a.xi, a.xi_f, iy);
            // sign of xi_y from the node index (nodes ascend; odd full-range sets have a 0)
            const int ys = iy >= M - HALF ? 1 : (iy < HALF ? -1 : 0);
            const int jpos = ys > 0 ? iyp : iyn;
            const TC nuy = pick<TC>(a.nuy, a.nuy_f, iy);
            const TC Py = pick<TC>(a.so_p[1], a.so_p_f[1], iy), By = pick<TC>(a.so_b[1], a.so_b_f[1], iy),
                     Cy = pick<TC>(a.so_c[1], a.so_c_f[1], iy);
            const bool y0 = jpos == 0, y1 = jpos == 1;
            const TC ay = ys == 0 ? TC(0) : (y0 ? nuy : Py);
            const TC by = (ys == 0 || y0) ? TC(0) : (y1 ? Py : By);
            const TC cy = (ys == 0 || y0 || y1) ? TC(0) : Cy;     // the table holds -C
            const long c1y = ys > 0 ? cym1 : cyp1, c2y = ys > 0 ? cym2 : cyp2;
            // wall-emitted population across a bottom or top wall face (Eq. 8), PART only
            const TC gy = (PART && ys != 0 && y0) ? nuy : TC(0);
            const TC rho_y = ys > 0 ? rb : rt;
            const TC u_y = ys > 0 ? ub : ut;
            const TC drive_y = ys > 0 ? db : dt;
            const TC wy = pick<TC>(a.w1, a.w1_f, iy);
            TC R = 0, X = 0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const TS *hp = h + (long)(iy * M + ix) * vstride;
                const TC hc = (TC)ldg(hp + cat);
                const TC h1y = (TC)ldg(hp + c1y), h2y = (TC)ldg(hp + c2y);
                const TC xix = pick<TC>(a.xi, a.xi_f, ix);
                TC v = fma_(-ay, hc, hc);
                v = fma_(by, h1y, v);
                v = fma_(cy, h2y, v);
                const int xs = ix >= M - HALF ? 1 : (ix < HALF ? -1 : 0);
                if (xmove && xs != 0) {
                    const TC nu = pick<TC>(a.nux, a.nux_f, ix);
                    const TC Px = pick<TC>(a.so_p[0], a.so_p_f[0], ix), Bx = pick<TC>(a.so_b[0], a.so_b_f[0], ix),
                             Cx = pick<TC>(a.so_c[0], a.so_c_f[0], ix);
                    const TC h1x = (TC)ldg(hp + (xs > 0 ? cxm1 : cxp1)), h2x = (TC)ldg(hp + (xs > 0 ? cxm2 : cxp2));
                    const int i = xs > 0 ? ixp : ixn;
                    const bool x0 = cav && i == 0, x1 = cav && i == 1;
                    const TC ax = x0 ? nu : Px;
                    const TC bx = x0 ? TC(0) : (x1 ? Px : Bx);
                    const TC cx = (x0 || x1) ? TC(0) : Cx;      // the table holds -C
                    v = fma_(-ax, hc, v);
                    v = fma_(bx, h1x, v);
                    v = fma_(cx, h2x, v);
                    if (PART && x0) v += nu * (pick<TC>(a.w1, a.w1_f, ix) * wy * (xs > 0 ? rl : rr));
                }
                if (PART && gy != TC(0)) {
                    const TC wxy = pick<TC>(a.w1, a.w1_f, ix) * wy;
                    v += gy * (wxy * (rho_y * (TC(1) + xix * u_y) + xix * drive_y));
                }
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

    // ---- relaxation (factor from the host: exp(-omega) for exact symmetric splitting) ----
    TC psd = 0, psn = 0;
    if (work) {
        const TC b = pick<TC>(&a.b, &a.b_f, 0);
        const TC om = pick<TC>(&a.omega, &a.omega_f, 0);
        TS *__restrict__ hn = reinterpret_cast<TS *>(a.hn);
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC wom = om * pick<TC>(a.w1, a.w1_f, iy);
            const TC q = wom * (rho + pick<TC>(a.xi, a.xi_f, iy) * jy);
            const TC jj = wom * jx;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const long off = (long)(iy * M + ix) * vstride + cat;
                const TC t = q + pick<TC>(a.xi, a.xi_f, ix) * jj;
                const TC v = b * hs[r * M + ix] + pick<TC>(a.w1, a.w1_f, ix) * t;
                if (RESID) {
                    const TC d = v - (TC)ldg(h + off);
                    psd += d * d;
                    psn += v * v;
                }
                if (valid) hn[off] = (TS)v;
            }
        }
    }
    if (RESID) {
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

template <typename TS, typename TC, int M, int G, bool RESID, bool PART>
__global__ void __launch_bounds__(Shape<G>::THREADS) step_so_kernel(const StepArgs a)
{
    step_so_body<TS, TC, M, G, RESID, PART>(a, blockIdx.x);
}

// bulk kernel over `grid` blocks, then the wall kernel over the wall segments
template <typename TS, typename TC, int M, int G, bool RESID>
cudaError_t launch_so(const StepArgs &a, int grid, cudaStream_t s)
{
    constexpr int T = Shape<G>::THREADS;
    step_so_kernel<TS, TC, M, G, RESID, false><<<grid, T, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_wall_segs == 0) return e;
    StepArgs b = a;
    b.partials_offset = grid;
    const int wgrid = (a.n_wall_segs + Shape<G>::SPB - 1) / Shape<G>::SPB;
    step_so_kernel<TS, TC, M, G, RESID, true><<<wgrid, T, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace lbmk
