// Hybrid half-range / full-range Couette channel (the coupling the paper's conclusion
// proposes; this project's reading, not the paper's algorithm): cells within `layer` cells
// of either plate carry the half-range set D2Q^h_{(2N)^2}, the cells between them the
// full-range Gauss-Hermite set of N nodes per axis.  Per step and cell (FP64):
//   * first-order upwind transport in y on the cell's own set (Eq. 1), Maxwell diffuse
//     plates (Eqs. 8-9, the wall density as a discrete flux balance over the cell's set);
//   * across an interface the upwind values come from the tensor Hermite projection of
//     order N - 1 of the neighbour's distribution,
//         c_mn = sum_a h_a He_m(xi_x,a) He_n(xi_y,a) / (m! n!),
//         h~_b = w_b sum_{m,n} c_mn He_m(xi_x,b) He_n(xi_y,b);
//   * the flux through an interface face is the half-range one (both half-spaces summed in
//     the half-range set, the full-range side by its projection onto it): the full-range
//     cell's transported state gets (lam + mu xi_x) w so that its mass and x-momentum
//     exchange through that face equals it (sum w = sum xi_x^2 w = 1 for the full-range
//     rule);
//   * relaxation towards w (rho + xi . j) in the cell's own set (Eqs. 1, 5-7).
// Cells with an interface face: one warp per cell (projections in shared memory); all other
// cells: a lane group per cell, several cells per warp, the upwind values read directly.  The
// state is packed cell after cell, each cell's values in its own set's velocity order
// (a = iy * M + ix).  dt = cfl dy / max |xi_y| over the sets present,
// dt <= Kn.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

lbm_status lbm_norms_fail(lbm_status s, const char *msg);
bool lbm_rule_1d(int kind, int n, std::vector<double> &nodes, std::vector<double> &weights);

namespace {

constexpr int HMAXV = 144;     // half-range N <= 6
constexpr int HMAXQ = 5;       // Hermite order N - 1
constexpr int HWARPS = 4;      // cells per block

struct HybSet {
    int n;
    int lanes;                 // lanes per cell in the plain-cell kernel: n rounded up to a power of two, <= 32
    double xi_x[HMAXV], xi_y[HMAXV], w[HMAXV];
    double he_x[HMAXQ + 1][HMAXV], he_y[HMAXQ + 1][HMAXV];
    double d_x, d_y;           // sums over xi > 0 of xi w per axis (wall-flux normalisers, Eq. 9)
    double nux[HMAXV], nuy[HMAXV];  // |xi_x| dt / dx, |xi_y| dt / dy (set on the host once dt is known)
    // signs of xi_x, xi_y (-1, 0, 1): the upwind and half-space tests as integer compares (an
    // FP64 compare takes the FP64 pipe, the bound of these kernels)
    signed char sx[HMAXV], sy[HMAXV];
};

constexpr int HMAXF = 36;      // full-range N <= 6

struct HybTables {
    HybSet set[2];             // 0: half-range, 1: full-range
    double inv_fact[HMAXQ + 1];
    // projection matrices, transposed: pt[t][a * n_s + b] = w_b sum_{m,n} He_m(xi_x,a) He_n(xi_y,a)
    // He_m(xi_x,b) He_n(xi_y,b) / (m! n!), a a velocity of set t, b of the other set s = 1 - t
    double pt[2][HMAXV * HMAXF];
};

struct HybArgs {
    const HybTables *tab;
    const int *off;            // [ny + 1] first value of each cell in the packed state
    const unsigned char *half; // [ncells] 1: half-range cell
    const double *h;
    double *hn;
    double *part;              // [2 ncells] residual sums per cell (||h^{n+1} - h^n||^2, ||h^{n+1}||^2)
    int nx, ny, order;
    int cavity;                // 0: Couette column (no x transport), 1: cavity (walls on all faces)
    double omega;
    double u_bottom, u_top, u_ref;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Tensor Hermite projection of order N - 1 of distribution h (set ti) onto the other set,
// into out[]: out_b = w_b sum_{m,n} c_mn He_m(xi_x,b) He_n(xi_y,b) with
// c_mn = sum_a h_a He_m(xi_x,a) He_n(xi_y,a) / (m! n!), applied as the precomputed matrix.
// Target sets of more than 16 velocities: each lane whole sums for outputs lane, lane + 32,
// ...; smaller ones: the source velocities split over 32 / lanes lane groups, the partial sums
// combined by shuffles (every lane of the warp calls this).
__device__ void project_warp(const HybTables &tb, int ti, const double *h, double *out)
{
    const int lane = threadIdx.x & 31;
    const HybSet &T = tb.set[ti], &S = tb.set[ti ^ 1];
    const double *pt = tb.pt[ti];
    const int nt = T.n, ns = S.n;
    if (ns > 16) {
        for (int b = lane; b < ns; b += 32) {
            double s4[4] = {0.0, 0.0, 0.0, 0.0};
            int a = 0;
            for (; a + 4 <= nt; a += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s4[q] += pt[(a + q) * ns + b] * h[a + q];
            }
            for (; a < nt; ++a) s4[0] += pt[a * ns + b] * h[a];
            out[b] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
    } else {
        const int ls = S.lanes, parts = 32 / ls, part = lane / ls, b = lane - part * ls;
        double acc = 0.0;
        if (b < ns)
            for (int a = part; a < nt; a += parts) acc += pt[a * ns + b] * h[a];
        for (int o = ls; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (part == 0 && b < ns) out[b] = acc;
    }
    __syncwarp();
}

// Values of neighbour cell k as seen by a cell of set sj, into buf[0..S.n): its own values
// for the same set, else their projection.
__device__ void neighbour_values(const HybArgs &a, int k, int sj, double *buf)
{
    const HybTables &tb = *a.tab;
    const HybSet &S = tb.set[sj];
    const int sk = a.half[k] ? 0 : 1;
    const double *hk = a.h + a.off[k];
    if (sk == sj) {
        for (int b = threadIdx.x & 31; b < S.n; b += 32) buf[b] = hk[b];
        __syncwarp();
    } else {
        project_warp(tb, sk, hk, buf);
    }
}

// Ghost of Eq. 8 (perturbation form) for the velocities leaving wall `face` (0 bottom, 1 top,
// 2 left, 3 right; the side walls at rest), into buf; rho_w by Eq. 9 over the cell's own set.
__device__ void wall_ghost(const HybArgs &a, const HybSet &S, const double *hc, int face, double *buf)
{
    const int lane = threadIdx.x & 31;
    double part = 0.0;
    for (int b = lane; b < S.n; b += 32) {
        const int sn = face == 0 ? S.sy[b] : face == 1 ? -S.sy[b] : face == 2 ? S.sx[b] : -S.sx[b];
        if (sn < 0) {
            const double xn = face == 0 ? S.xi_y[b] : face == 1 ? -S.xi_y[b] : face == 2 ? S.xi_x[b] : -S.xi_x[b];
            part += -xn * hc[b];
        }
    }
    const double rho_w = warp_sum(part) / (face < 2 ? S.d_y : S.d_x);
    const double u = face == 0 ? a.u_bottom : face == 1 ? a.u_top : 0.0;
    for (int b = lane; b < S.n; b += 32) {
        const double xt = face < 2 ? S.xi_x[b] : S.xi_y[b];
        buf[b] = S.w[b] * (rho_w * (1.0 + xt * u) + xt * u / a.u_ref);
    }
    __syncwarp();
}

// (mass, x-momentum, y-momentum) flux sum |xi_d| (1, xi_x, xi_y) v over the velocities of S
// moving along +axis (positive) or -axis; axis 0 = x, 1 = y.
__device__ void face_moments(const HybSet &S, const double *v, int axis, bool positive, double (&m)[3])
{
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int b = threadIdx.x & 31; b < S.n; b += 32) {
        const int sd = axis == 0 ? S.sx[b] : S.sy[b];
        if (positive ? sd > 0 : sd < 0) {
            const double xd = axis == 0 ? S.xi_x[b] : S.xi_y[b];
            const double t = fabs(xd) * v[b];
            p0 += t;
            p1 += t * S.xi_x[b];
            p2 += t * S.xi_y[b];
        }
    }
    m[0] = warp_sum(p0);
    m[1] = warp_sum(p1);
    m[2] = warp_sum(p2);
}

struct HybShared {
    double nbv[HWARPS][4][HMAXV];   // left, right, below, above: upwind values in the cell's set
    double ph[HWARPS][HMAXV], nb[HWARPS][HMAXV];
};

// A cell with an interface face (a neighbour in the other set): one warp, warp `wi` of the
// block's shared buffers.
__device__ void interface_cell(const HybArgs &a, HybShared &sh, int wi, int c, double dt, double dx, double dy,
                               int resid)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    const HybTables &tb = *a.tab;
    const int sj = a.half[c] ? 0 : 1;
    const HybSet &S = tb.set[sj];
    const HybSet &H = tb.set[0];
    const double *hc = a.h + a.off[c];
    const int x = c % nx, y = c / nx;
    double(*nbv)[HMAXV] = sh.nbv[wi];
    // upwind values: x (cavity only) and y neighbours in this cell's set, or the walls' ghosts;
    // the four faces as (axis, side, neighbour or -1)
    int nbc[4] = {-1, -1, -1, -1};
    if (a.cavity) {
        if (x > 0) neighbour_values(a, nbc[0] = c - 1, sj, nbv[0]);
        else wall_ghost(a, S, hc, 2, nbv[0]);
        if (x < nx - 1) neighbour_values(a, nbc[1] = c + 1, sj, nbv[1]);
        else wall_ghost(a, S, hc, 3, nbv[1]);
    }
    if (y > 0) neighbour_values(a, nbc[2] = c - nx, sj, nbv[2]);
    else wall_ghost(a, S, hc, 0, nbv[2]);
    if (y < ny - 1) neighbour_values(a, nbc[3] = c + nx, sj, nbv[3]);
    else wall_ghost(a, S, hc, 1, nbv[3]);
    // interface faces of a full-range cell: mass and momentum exchange made equal to the
    // half-range evaluation of the face
    double cr[3] = {0.0, 0.0, 0.0};
    bool any_if = false;
    if (sj == 1)
        for (int f = 0; f < 4; ++f) any_if |= nbc[f] >= 0 && a.half[nbc[f]];
    if (any_if) {
        double *ph = sh.ph[wi], *nb = sh.nb[wi];
        project_warp(tb, 1, hc, ph);                            // this cell seen in H
        for (int f = 0; f < 4; ++f) {
            if (nbc[f] < 0 || !a.half[nbc[f]]) continue;
            const int axis = f >> 1;
            const bool lower = (f & 1) == 0;                  // the neighbour is on the lower side
            neighbour_values(a, nbc[f], 0, nb);               // its own half-range values
            double up[3], dn[3], got[3], sent[3];
            face_moments(H, lower ? nb : ph, axis, true, up);
            face_moments(H, lower ? ph : nb, axis, false, dn);
            face_moments(S, nbv[f], axis, lower, got);
            face_moments(S, hc, axis, !lower, sent);
            const double fac = dt / (axis == 0 ? dx : dy);
            for (int q = 0; q < 3; ++q) {
                const double want = lower ? up[q] - dn[q] : dn[q] - up[q];
                cr[q] += fac * (want - (got[q] - sent[q]));
            }
        }
    }
    // transport, moments, relaxation
    double hs[(HMAXV + 31) / 32];
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < (HMAXV + 31) / 32; ++i) {
        const int b = lane + 32 * i;
        double v = 0.0;
        if (b < S.n) {
            const double ex = S.xi_x[b], ey = S.xi_y[b];
            const double h0 = hc[b];
            double hx = h0, nux = 0.0;
            const int sgx = S.sx[b], sgy = S.sy[b];
            if (a.cavity) {
                hx = sgx > 0 ? nbv[0][b] : (sgx < 0 ? nbv[1][b] : h0);
                nux = S.nux[b];
            }
            const double hy = sgy > 0 ? nbv[2][b] : (sgy < 0 ? nbv[3][b] : h0);
            const double nuy = S.nuy[b];
            v = h0 - nux * (h0 - hx) - nuy * (h0 - hy);
            if (any_if) v += (cr[0] + cr[1] * ex + cr[2] * ey) * S.w[b];
            rho += v;
            jx += ex * v;
            jy += ey * v;
        }
        hs[i] = v;
    }
    rho = warp_sum(rho);
    jx = warp_sum(jx);
    jy = warp_sum(jy);
    double *out = a.hn + a.off[c];
    double pd = 0.0, pn = 0.0;
#pragma unroll
    for (int i = 0; i < (HMAXV + 31) / 32; ++i) {
        const int b = lane + 32 * i;
        if (b < S.n) {
            const double heq = S.w[b] * (rho + S.xi_x[b] * jx + S.xi_y[b] * jy);
            const double o = hs[i] - a.omega * (hs[i] - heq);
            out[b] = o;
            if (resid) {
                const double d = o - hc[b];
                pd += d * d;
                pn += o * o;
            }
        }
    }
    if (resid) {
        pd = warp_sum(pd);
        pn = warp_sum(pn);
        if (lane == 0) {
            a.part[2 * c] = pd;
            a.part[2 * c + 1] = pn;
        }
    }
}

// sum over the `width` lanes of an aligned lane group (width a power of two <= 32)
__device__ __forceinline__ double group_sum(double v, int width)
{
    for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int HMAXPL = (HMAXV + 31) / 32;     // velocities per lane in the plain-cell kernel

// Cells whose existing neighbours all carry the cell's own set (no interface face): the
// same update as hybrid_step_kernel without projections.  A warp takes a task, a run of
// consecutive cells of one set (contiguous in the packed state); a group of S.lanes lanes
// takes a cell, lane g its velocities g, g + lanes, ...; the upwind values are read straight
// from the neighbour cells, the wall densities and moments are sums over the group.
__device__ void plain_task(const HybArgs &a, const int2 tk, int resid)
{
    const int lane = threadIdx.x & 31;
    const HybTables &tb = *a.tab;
    const HybSet &S = tb.set[a.half[tk.x] ? 0 : 1];
    const int n = S.n, L = S.lanes;
    const int sub = lane / L, g = lane - sub * L;
    const bool on = sub < tk.y;
    const int c = tk.x + (on ? sub : 0);         // idle groups repeat the first cell and store nothing
    const int nx = a.nx, ny = a.ny, x = c % nx, y = c / nx;
    const double *hc = a.h + a.off[c];
    const bool cav = a.cavity != 0;
    const bool wl = cav && x == 0, wr = cav && x == nx - 1, wb = y == 0, wt = y == ny - 1;
    const double *hl = (cav && !wl) ? a.h + a.off[c - 1] : hc;
    const double *hr = (cav && !wr) ? a.h + a.off[c + 1] : hc;
    const double *hd = !wb ? a.h + a.off[c - nx] : hc;
    const double *hu = !wt ? a.h + a.off[c + nx] : hc;
    double hv[HMAXPL];
    double pw[4] = {0.0, 0.0, 0.0, 0.0};         // outflow through the bottom, top, left, right walls
    const bool walls = __any_sync(0xffffffffu, wl || wr || wb || wt);
#pragma unroll
    for (int i = 0; i < HMAXPL; ++i) {
        const int b = g + L * i;
        hv[i] = 0.0;
        if (b < n) {
            const double v = hc[b];
            hv[i] = v;
            if (walls) {
                const double ex = S.xi_x[b], ey = S.xi_y[b];
                const int sgx = S.sx[b], sgy = S.sy[b];
                if (sgy < 0) pw[0] -= ey * v;
                if (sgy > 0) pw[1] += ey * v;
                if (sgx < 0) pw[2] -= ex * v;
                if (sgx > 0) pw[3] += ex * v;
            }
        }
    }
    // wall densities (Eq. 9 as a flux balance over the cell's set)
    double rw[4] = {0.0, 0.0, 0.0, 0.0};
    if (walls) {
#pragma unroll
        for (int f = 0; f < 4; ++f) rw[f] = group_sum(pw[f], L) / (f < 2 ? S.d_y : S.d_x);
    }
    const double ub = a.u_bottom, ut = a.u_top;
    double hs[HMAXPL];
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < HMAXPL; ++i) {
        const int b = g + L * i;
        double v = 0.0;
        if (b < n) {
            const double ex = S.xi_x[b], ey = S.xi_y[b], wb_ = S.w[b];
            const double h0 = hv[i];
            const int sgx = S.sx[b], sgy = S.sy[b];
            double hx = h0, nux = 0.0;
            if (cav) {
                if (sgx > 0) hx = wl ? wb_ * rw[2] : hl[b];          // side walls at rest
                else if (sgx < 0) hx = wr ? wb_ * rw[3] : hr[b];
                nux = S.nux[b];
            }
            double hy = h0;
            if (sgy > 0) hy = wb ? wb_ * (rw[0] * (1.0 + ex * ub) + ex * ub / a.u_ref) : hd[b];
            else if (sgy < 0) hy = wt ? wb_ * (rw[1] * (1.0 + ex * ut) + ex * ut / a.u_ref) : hu[b];
            const double nuy = S.nuy[b];
            v = h0 - nux * (h0 - hx) - nuy * (h0 - hy);
            rho += v;
            jx += ex * v;
            jy += ey * v;
        }
        hs[i] = v;
    }
    rho = group_sum(rho, L);
    jx = group_sum(jx, L);
    jy = group_sum(jy, L);
    double *out = a.hn + a.off[c];
    double pd = 0.0, pn = 0.0;
#pragma unroll
    for (int i = 0; i < HMAXPL; ++i) {
        const int b = g + L * i;
        if (b < n) {
            const double heq = S.w[b] * (rho + S.xi_x[b] * jx + S.xi_y[b] * jy);
            const double o = hs[i] - a.omega * (hs[i] - heq);
            if (on) out[b] = o;
            if (resid) {
                const double d = o - hv[i];
                pd += d * d;
                pn += o * o;
            }
        }
    }
    if (resid) {
        pd = group_sum(pd, L);
        pn = group_sum(pn, L);
        if (on && g == 0) {
            a.part[2 * c] = pd;
            a.part[2 * c + 1] = pn;
        }
    }
}

// One step: the blocks for the interface cells first (their projections are the long
// latency chains), then the plain-cell tasks, so that both run side by side in one launch.
__global__ void __launch_bounds__(32 * HWARPS, 5) hybrid_step_kernel(const HybArgs a, const int *cells, int ncells,
                                                                   const int2 *tasks, int ntasks, double dt, double dx,
                                                                   double dy, int resid)
{
    __shared__ HybShared sh;
    const int wi = threadIdx.x >> 5;
    const int if_blocks = (ncells + HWARPS - 1) / HWARPS;
    if ((int)blockIdx.x < if_blocks) {
        const int ci = (int)blockIdx.x * HWARPS + wi;
        if (ci < ncells) interface_cell(a, sh, wi, cells[ci], dt, dx, dy, resid);     // whole warps
    } else {
        const int t = ((int)blockIdx.x - if_blocks) * HWARPS + wi;
        if (t < ntasks) plain_task(a, tasks[t], resid);
    }
}

// residual sums over the cells: one block, each thread a fixed stride of cells, then a fixed
// tree (the same order every call)
constexpr int HFIN = 1024;
__global__ void __launch_bounds__(HFIN) hybrid_finalize_kernel(const double *part, int ncells, double *out)
{
    __shared__ double sd[HFIN], sn[HFIN];
    double d = 0.0, n = 0.0;
    for (int j = threadIdx.x; j < ncells; j += HFIN) {
        d += part[2 * j];
        n += part[2 * j + 1];
    }
    sd[threadIdx.x] = d;
    sn[threadIdx.x] = n;
    __syncthreads();
    for (int w = HFIN / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sd[threadIdx.x] += sd[threadIdx.x + w];
            sn[threadIdx.x] += sn[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sd[0];
        out[1] = sn[0];
    }
}

// Couette column: the x-momentum flux through the ny + 1 faces (interface faces evaluated in
// the half-range set); one warp per face k
__global__ void __launch_bounds__(32 * HWARPS) hybrid_face_flux_kernel(const HybArgs a, double u_ref, double *pxy)
{
    __shared__ HybShared sh;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int k = blockIdx.x * HWARPS + wi;
    if (k > a.ny) return;
    const HybTables &tb = *a.tab;
    double *lo = sh.nbv[wi][0], *hi = sh.nbv[wi][1];
    double up = 0.0, dn = 0.0;
    if (k > 0 && k < a.ny && a.half[k - 1] != a.half[k]) {
        const HybSet &H = tb.set[0];
        neighbour_values(a, k - 1, 0, lo);
        neighbour_values(a, k, 0, hi);
        double mu[3], md[3];
        face_moments(H, lo, 1, true, mu);
        face_moments(H, hi, 1, false, md);
        up = mu[1];
        dn = -md[1];                                            // sum over xi_y < 0 of xi_y xi_x h
    } else {
        const int cb = k == 0 ? 0 : k - 1, ca = k == a.ny ? a.ny - 1 : k;
        const HybSet &Sb = tb.set[a.half[cb] ? 0 : 1], &Sa = tb.set[a.half[ca] ? 0 : 1];
        const double *vb = a.h + a.off[cb], *va = a.h + a.off[ca];
        if (k == 0) {
            wall_ghost(a, Sb, vb, 0, lo);
            vb = lo;
        }
        if (k == a.ny) {
            wall_ghost(a, Sa, va, 1, hi);
            va = hi;
        }
        double pu = 0.0, pd = 0.0;
        for (int b = lane; b < Sb.n; b += 32)
            if (Sb.xi_y[b] > 0) pu += Sb.xi_x[b] * Sb.xi_y[b] * vb[b];
        for (int b = lane; b < Sa.n; b += 32)
            if (Sa.xi_y[b] < 0) pd += Sa.xi_x[b] * Sa.xi_y[b] * va[b];
        up = warp_sum(pu);
        dn = warp_sum(pd);
    }
    if (lane == 0) pxy[k] = u_ref * (up + dn);
}

// (u_x, u_y) of every cell from its own set: u = u_ref sum xi h / (1 + u_ref sum h)
__global__ void __launch_bounds__(32 * HWARPS) hybrid_velocity_kernel(const HybArgs a, double u_ref, double *ux,
                                                                       double *uy)
{
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * HWARPS + (threadIdx.x >> 5);
    if (c >= a.nx * a.ny) return;
    const HybSet &S = a.tab->set[a.half[c] ? 0 : 1];
    const double *hc = a.h + a.off[c];
    double s0 = 0.0, sx = 0.0, sy = 0.0;
    for (int b = lane; b < S.n; b += 32) {
        s0 += hc[b];
        sx += S.xi_x[b] * hc[b];
        sy += S.xi_y[b] * hc[b];
    }
    s0 = warp_sum(s0);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
        const double rho = 1.0 + u_ref * s0;
        ux[c] = u_ref * sx / rho;
        uy[c] = u_ref * sy / rho;
    }
}

}  // namespace

struct lbm_hybrid {
    int geom, n_half, nx, ny, layer, order;
    double kn, u_bottom, u_top, cfl, dt, dx, dy, omega, u_ref;
    std::vector<int> off;
    std::vector<unsigned char> half;
    long unknowns;
    cudaStream_t stream;
    HybTables *d_tab;
    int *d_off;
    unsigned char *d_half;
    double *d_h[2], *d_part, *d_res;
    double *h_res;           // pinned
    int cur;
    bool have_resid;
    int n_if, n_tasks;       // interface cells, plain-cell tasks
    int *d_if;               // [n_if] cells with an interface face
    int2 *d_tasks;           // [n_tasks] runs of plain cells (first cell, count)
};

namespace {

lbm_status hfail(lbm_status s, const std::string &m) { return lbm_norms_fail(s, m.c_str()); }

bool fill_set(HybSet &S, int kind, int n, int order, double &max_y)
{
    std::vector<double> x, w;
    if (!lbm_rule_1d(kind, n, x, w)) return false;
    const int m = (int)x.size();
    S.n = m * m;
    if (S.n > HMAXV) return false;
    S.lanes = 1;
    while (S.lanes < S.n && S.lanes < 32) S.lanes *= 2;
    S.d_x = S.d_y = 0.0;
    max_y = 0.0;
    for (int iy = 0; iy < m; ++iy)
        for (int ix = 0; ix < m; ++ix) {
            const int a = iy * m + ix;
            S.xi_x[a] = x[ix];
            S.xi_y[a] = x[iy];
            S.w[a] = w[ix] * w[iy];
            S.sx[a] = (signed char)((x[ix] > 0) - (x[ix] < 0));
            S.sy[a] = (signed char)((x[iy] > 0) - (x[iy] < 0));
            if (x[iy] > 0) S.d_y += x[iy] * S.w[a];
            if (x[ix] > 0) S.d_x += x[ix] * S.w[a];
            max_y = std::max(max_y, std::fabs(x[iy]));
            // probabilists' Hermite polynomials by the three-term recurrence
            for (int axis = 0; axis < 2; ++axis) {
                const double v = axis == 0 ? x[ix] : x[iy];
                double (*he)[HMAXV] = axis == 0 ? S.he_x : S.he_y;
                he[0][a] = 1.0;
                if (order >= 1) he[1][a] = v;
                for (int k = 1; k < order; ++k) he[k + 1][a] = v * he[k][a] - k * he[k - 1][a];
            }
        }
    return true;
}

HybArgs hargs(const lbm_hybrid *hb)
{
    HybArgs a;
    std::memset(&a, 0, sizeof a);
    a.tab = hb->d_tab;
    a.off = hb->d_off;
    a.half = hb->d_half;
    a.h = hb->d_h[hb->cur];
    a.hn = hb->d_h[hb->cur ^ 1];
    a.part = hb->d_part;
    a.nx = hb->nx;
    a.ny = hb->ny;
    a.cavity = hb->geom == LBM_CAVITY;
    a.order = hb->order;
    a.omega = hb->omega;
    a.u_bottom = hb->u_bottom;
    a.u_top = hb->u_top;
    a.u_ref = hb->u_ref;
    return a;
}

}  // namespace

extern "C" {

lbm_status lbm_hybrid_init(int geom, int n_half, int nx, int ny, double kn, double u_bottom, double u_top, int layer,
                           double cfl, void *stream, lbm_hybrid **out)
{
    if (!out) return hfail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_half < 2 || n_half > 6) return hfail(LBM_EINVAL, "the hybrid needs 2 <= N <= 6 nodes per half-axis");
    if (geom != LBM_COUETTE && geom != LBM_CAVITY) return hfail(LBM_EINVAL, "unknown geometry");
    if (geom == LBM_COUETTE && nx != 1) return hfail(LBM_EINVAL, "the hybrid Couette channel is one column (nx = 1)");
    if (geom == LBM_CAVITY && nx < 2) return hfail(LBM_EINVAL, "cavity needs nx >= 2");
    if (ny < 2 || layer < 0 || !(kn > 0) || !(cfl > 0) || !std::isfinite(u_bottom) || !std::isfinite(u_top))
        return hfail(LBM_EINVAL, "invalid hybrid problem (ny >= 2, layer >= 0, Kn > 0, cfl > 0)");
    if ((long)nx * ny > 16L * 1024 * 1024) return hfail(LBM_EINVAL, "grid too large for the hybrid kernels");
    lbm_hybrid *hb = new (std::nothrow) lbm_hybrid;
    if (!hb) return hfail(LBM_ENOMEM, "host allocation failed");
    hb->geom = geom;
    hb->n_half = n_half;
    hb->nx = nx;
    hb->ny = ny;
    hb->layer = layer;
    hb->order = n_half - 1;
    hb->kn = kn;
    hb->u_bottom = u_bottom;
    hb->u_top = u_top;
    hb->cfl = cfl;
    hb->stream = (cudaStream_t)stream;
    hb->cur = 0;
    hb->have_resid = false;
    hb->d_tab = nullptr;
    hb->d_off = nullptr;
    hb->d_half = nullptr;
    hb->d_h[0] = hb->d_h[1] = nullptr;
    hb->d_part = hb->d_res = nullptr;
    hb->h_res = nullptr;
    hb->d_if = nullptr;
    hb->d_tasks = nullptr;
    hb->n_if = hb->n_tasks = 0;
    std::vector<HybTables> tabv(1);     // ~130 KB: on the heap, zero-initialised
    HybTables &tab = tabv[0];
    double my_h = 0, my_f = 0;
    if (!fill_set(tab.set[0], LBM_HALF_RANGE_GH, n_half, hb->order, my_h) ||
        !fill_set(tab.set[1], LBM_FULL_RANGE_GH, n_half, hb->order, my_f)) {
        delete hb;
        return hfail(LBM_EINVAL, "quadrature construction failed");
    }
    double f = 1.0;
    for (int k = 0; k <= HMAXQ; ++k) {
        if (k > 0) f *= k;
        tab.inv_fact[k] = 1.0 / f;
    }
    if (tab.set[1].n > HMAXF) {
        delete hb;
        return hfail(LBM_EINVAL, "full-range set too large for the hybrid projection");
    }
    // the projections as matrices (transposed, source velocity major)
    for (int t = 0; t < 2; ++t) {
        const HybSet &T = tab.set[t], &S = tab.set[1 - t];
        for (int a = 0; a < T.n; ++a)
            for (int b = 0; b < S.n; ++b) {
                double v = 0.0;
                for (int m = 0; m <= hb->order; ++m)
                    for (int n = 0; n <= hb->order; ++n)
                        v += tab.inv_fact[m] * tab.inv_fact[n] * T.he_x[m][a] * T.he_y[n][a] * S.he_x[m][b] *
                             S.he_y[n][b];
                tab.pt[t][a * S.n + b] = S.w[b] * v;
            }
    }
    const long nc = (long)nx * ny;
    hb->half.resize(nc);
    hb->off.resize(nc + 1);
    bool any_h = false, any_f = false;
    long o = 0;
    for (long c = 0; c < nc; ++c) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const int dwall = geom == LBM_CAVITY ? std::min(std::min(x, nx - 1 - x), std::min(y, ny - 1 - y))
                                             : std::min(y, ny - 1 - y);
        hb->half[c] = dwall < layer ? 1 : 0;
        (hb->half[c] ? any_h : any_f) = true;
        hb->off[c] = (int)std::min(o, (long)INT_MAX);      // checked below
        o += hb->half[c] ? tab.set[0].n : tab.set[1].n;
    }
    if (o > (long)INT_MAX) {
        delete hb;
        return hfail(LBM_EINVAL, "too many unknowns for the hybrid's 32-bit cell offsets");
    }
    hb->off[nc] = (int)o;
    hb->unknowns = o;
    // cells with a neighbour in the other set go to the projecting kernel; runs of the others
    // (consecutive cells of one set, as many as fill a warp) to the plain-cell kernel
    std::vector<int> if_cells;
    std::vector<int2> tasks;
    for (long c = 0; c < nc; ++c) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const unsigned char hc_ = hb->half[c];
        bool iface = (y > 0 && hb->half[c - nx] != hc_) || (y < ny - 1 && hb->half[c + nx] != hc_);
        if (geom == LBM_CAVITY) iface = iface || (x > 0 && hb->half[c - 1] != hc_) || (x < nx - 1 && hb->half[c + 1] != hc_);
        if (iface) {
            if_cells.push_back((int)c);
            continue;
        }
        const int cap = 32 / tab.set[hc_ ? 0 : 1].lanes;
        if (!tasks.empty()) {
            int2 &tk = tasks.back();
            if (tk.x + tk.y == c && hb->half[tk.x] == hc_ && tk.y < cap) {
                ++tk.y;
                continue;
            }
        }
        tasks.push_back(make_int2((int)c, 1));
    }
    hb->n_if = (int)if_cells.size();
    hb->n_tasks = (int)tasks.size();
    // dt = cfl / (max|xi_x|/dx + max|xi_y|/dy) over the sets present (the x term dropped for
    // the Couette column), dt <= Kn; the sets are symmetric, so max |xi_x| = max |xi_y|
    hb->dy = 1.0 / ny;
    hb->dx = geom == LBM_CAVITY ? 1.0 / nx : hb->dy;
    const double my = std::max(any_h ? my_h : 0.0, any_f ? my_f : 0.0);
    hb->dt = cfl / (my / hb->dy + (geom == LBM_CAVITY ? my / hb->dx : 0.0));
    if (std::isfinite(kn) && hb->dt > kn) hb->dt = kn;
    hb->omega = std::isfinite(kn) ? hb->dt / kn : 0.0;
    for (int k = 0; k < 2; ++k) {
        HybSet &S = tab.set[k];
        for (int b = 0; b < S.n; ++b) {
            S.nux[b] = std::fabs(S.xi_x[b]) * hb->dt / hb->dx;
            S.nuy[b] = std::fabs(S.xi_y[b]) * hb->dt / hb->dy;
        }
    }
    const double ur = std::max(std::fabs(u_bottom), std::fabs(u_top));
    hb->u_ref = ur > 0 ? ur : 1.0;
    cudaError_t e = cudaMalloc(&hb->d_tab, sizeof(HybTables));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_off, sizeof(int) * (nc + 1));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_half, nc);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_h[0], sizeof(double) * o);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_h[1], sizeof(double) * o);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_part, sizeof(double) * 2 * nc);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_res, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMallocHost(&hb->h_res, sizeof(double) * 2);
    if (e == cudaSuccess && hb->n_if > 0) e = cudaMalloc(&hb->d_if, sizeof(int) * hb->n_if);
    if (e == cudaSuccess && hb->n_tasks > 0) e = cudaMalloc(&hb->d_tasks, sizeof(int2) * hb->n_tasks);
    if (e == cudaSuccess && hb->n_if > 0)
        e = cudaMemcpyAsync(hb->d_if, if_cells.data(), sizeof(int) * hb->n_if, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess && hb->n_tasks > 0)
        e = cudaMemcpyAsync(hb->d_tasks, tasks.data(), sizeof(int2) * hb->n_tasks, cudaMemcpyHostToDevice,
                            hb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb->d_tab, &tab, sizeof tab, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb->d_off, hb->off.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb->d_half, hb->half.data(), nc, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hb->d_h[0], 0, sizeof(double) * o, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (e != cudaSuccess) {
        lbm_hybrid_destroy(hb);
        return hfail(LBM_ECUDA, std::string("allocating the hybrid channel: ") + cudaGetErrorString(e));
    }
    *out = hb;
    return LBM_OK;
}

void lbm_hybrid_destroy(lbm_hybrid *hb)
{
    if (!hb) return;
    if (hb->stream) cudaStreamSynchronize(hb->stream);
    else cudaDeviceSynchronize();
    cudaFree(hb->d_tab);
    cudaFree(hb->d_off);
    cudaFree(hb->d_half);
    cudaFree(hb->d_h[0]);
    cudaFree(hb->d_h[1]);
    cudaFree(hb->d_part);
    cudaFree(hb->d_res);
    cudaFree(hb->d_if);
    cudaFree(hb->d_tasks);
    if (hb->h_res) cudaFreeHost(hb->h_res);
    delete hb;
}

lbm_status lbm_hybrid_query(const lbm_hybrid *hb, long *unknowns, int *half_range_cells, double *dt)
{
    if (!hb) return hfail(LBM_EINVAL, "hybrid is NULL");
    if (unknowns) *unknowns = hb->unknowns;
    if (half_range_cells) {
        int c = 0;
        for (unsigned char v : hb->half) c += v;
        *half_range_cells = c;
    }
    if (dt) *dt = hb->dt;
    return LBM_OK;
}

lbm_status lbm_hybrid_set_state(lbm_hybrid *hb, const double *h)
{
    if (!hb || !h) return hfail(LBM_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(hb->d_h[hb->cur], h, sizeof(double) * hb->unknowns, cudaMemcpyHostToDevice,
                                    hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    hb->have_resid = false;
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("setting the state: ") + cudaGetErrorString(e));
}

lbm_status lbm_hybrid_get_state(lbm_hybrid *hb, double *h)
{
    if (!hb || !h) return hfail(LBM_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(h, hb->d_h[hb->cur], sizeof(double) * hb->unknowns, cudaMemcpyDeviceToHost,
                                    hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("reading the state: ") + cudaGetErrorString(e));
}

lbm_status lbm_hybrid_step(lbm_hybrid *hb, long nsteps)
{
    if (!hb || nsteps < 0) return hfail(LBM_EINVAL, "invalid step arguments");
    const int nc = hb->nx * hb->ny;
    for (long s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        const int blocks = (hb->n_if + HWARPS - 1) / HWARPS + (hb->n_tasks + HWARPS - 1) / HWARPS;
        hybrid_step_kernel<<<blocks, 32 * HWARPS, 0, hb->stream>>>(hargs(hb), hb->d_if, hb->n_if, hb->d_tasks,
                                                                   hb->n_tasks, hb->dt, hb->dx, hb->dy, last ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && last) {
            hybrid_finalize_kernel<<<1, HFIN, 0, hb->stream>>>(hb->d_part, nc, hb->d_res);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return hfail(LBM_ECUDA, std::string("launching the hybrid step: ") + cudaGetErrorString(e));
        hb->cur ^= 1;
    }
    if (nsteps > 0) hb->have_resid = true;
    return LBM_OK;
}

lbm_status lbm_hybrid_residual(lbm_hybrid *hb, double *r)
{
    if (!hb || !r) return hfail(LBM_EINVAL, "NULL argument");
    if (!hb->have_resid) return hfail(LBM_EINVAL, "no step taken since the state was set");
    cudaError_t e = cudaMemcpyAsync(hb->h_res, hb->d_res, sizeof(double) * 2, cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (e != cudaSuccess) return hfail(LBM_ECUDA, std::string("reading the residual: ") + cudaGetErrorString(e));
    const double d = hb->h_res[0], n = hb->h_res[1];
    if (!std::isfinite(d) || !std::isfinite(n)) return hfail(LBM_ENONFINITE, "non-finite residual");
    *r = n > 0 ? std::sqrt(d / n) : (d == 0 ? 0.0 : INFINITY);
    return LBM_OK;
}

lbm_status lbm_hybrid_solve(lbm_hybrid *hb, double tol, long max_steps, int every, long *steps, double *r)
{
    if (!hb || every < 1 || max_steps < 0 || !(tol >= 0)) return hfail(LBM_EINVAL, "invalid solve arguments");
    long taken = 0;
    double res = INFINITY;
    while (taken < max_steps) {
        lbm_status st = lbm_hybrid_step(hb, every);
        if (st != LBM_OK) return st;
        taken += every;
        st = lbm_hybrid_residual(hb, &res);
        if (st != LBM_OK) return st;
        if (res < tol) break;
    }
    if (steps) *steps = taken;
    if (r) *r = res;
    return LBM_OK;
}

lbm_status lbm_hybrid_velocity(lbm_hybrid *hb, double *ux, double *uy)
{
    if (!hb || !ux || !uy) return hfail(LBM_EINVAL, "NULL argument");
    const int nc = hb->nx * hb->ny;
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * 2 * nc);
    if (e == cudaSuccess) {
        hybrid_velocity_kernel<<<(nc + HWARPS - 1) / HWARPS, 32 * HWARPS, 0, hb->stream>>>(hargs(hb), hb->u_ref, d,
                                                                                            d + nc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ux, d, sizeof(double) * nc, cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(uy, d + nc, sizeof(double) * nc, cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (d) cudaFree(d);
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("hybrid velocity: ") + cudaGetErrorString(e));
}

lbm_status lbm_hybrid_face_flux(lbm_hybrid *hb, double *pxy)
{
    if (!hb || !pxy) return hfail(LBM_EINVAL, "NULL argument");
    if (hb->geom != LBM_COUETTE) return hfail(LBM_EUNSUPPORTED, "face fluxes are reported for the Couette column");
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * (hb->ny + 1));
    if (e == cudaSuccess) {
        hybrid_face_flux_kernel<<<(hb->ny + 1 + HWARPS - 1) / HWARPS, 32 * HWARPS, 0, hb->stream>>>(hargs(hb),
                                                                                                    hb->u_ref, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(pxy, d, sizeof(double) * (hb->ny + 1), cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (d) cudaFree(d);
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("hybrid face flux: ") + cudaGetErrorString(e));
}

}  // extern "C"
