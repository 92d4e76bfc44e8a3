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
// cells: the plain-cell kernel, one lane per cell with the 1-D node tables of its set in the
// kernel parameters.  State layout: tiles of up to 32 consecutive cells (in the cell order
// c = y nx + x) of one set; velocity a of the cell in position p of a tile lies at
// tile base + p + 32 a, so that a warp reads one velocity of a tile's cells as one
// contiguous stretch (toff[c] = tile base + p).  Host transfers keep the packed order,
// cell after cell, each cell's values in its own set's velocity order (a = iy * M + ix).
// dt = cfl dy / max |xi_y| over the sets present, dt <= Kn.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
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

// Device copy of the tables in the arithmetic type T of the interface cells (double for the
// FP64 march, float for the FP32 one: GB300 retires FP64 at 2 lanes per cycle per SM)
template <typename T>
struct HybSetT {
    int n, lanes;
    T xi_x[HMAXV], xi_y[HMAXV], w[HMAXV];
    T d_x, d_y;
    T nux[HMAXV], nuy[HMAXV];
    signed char sx[HMAXV], sy[HMAXV];
};

template <typename T>
struct HybTabT {
    HybSetT<T> set[2];
    T pt[2][HMAXV * HMAXF];
};

constexpr int HST = 32;        // stride between the velocities of a cell in the tiled state

struct HybArgs {
    const void *tab;           // HybTabT<double> or HybTabT<float>, the type the interface cells compute in
    const int *toff;           // [ncells] velocity 0 of each cell in the tiled state
    const unsigned char *half; // [ncells] 1: half-range cell
    const void *h;             // state (FP64, or FP32 in the mixed-precision march), tiled
    void *hn;
    const float *src;          // correction march: the FP64 defect added after relaxation (else NULL)
    double *part;              // [2 ncells] residual sums per cell (||h^{n+1} - h^n||^2, ||h^{n+1}||^2)
    int nx, ny, order;
    int cavity;                // 0: Couette column (no x transport), 1: cavity (walls on all faces)
    int homogeneous;           // correction march: the walls' driving terms dropped
    double omega;
    double u_bottom, u_top, u_ref;
};

// a * b + c rounded once, in the arithmetic type
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
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
template <typename T>
__device__ void project_warp(const HybTabT<T> &tb, int ti, const T *h, T *out)
{
    const int lane = threadIdx.x & 31;
    const HybSetT<T> &Tg = tb.set[ti], &S = tb.set[ti ^ 1];
    const T *pt = tb.pt[ti];
    const int nt = Tg.n, ns = S.n;
    if (ns > 16) {
        for (int b = lane; b < ns; b += 32) {
            T s4[4] = {0, 0, 0, 0};
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
        T acc = 0;
        if (b < ns)
            for (int a = part; a < nt; a += parts) acc += pt[a * ns + b] * h[a];
        for (int o = ls; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (part == 0 && b < ns) out[b] = acc;
    }
    __syncwarp();
}

// The n values of cell k into buf[0..n) (a warp; velocity b at toff[k] + HST b).
template <typename TS, typename T>
__device__ void gather_cell(const TS *h, const int *toff, int k, int n, T *buf)
{
    const TS *hk = h + toff[k];
    for (int b = threadIdx.x & 31; b < n; b += 32) buf[b] = (T)hk[(long)HST * b];
    __syncwarp();
}

// Values of neighbour cell k as seen by a cell of set sj, into buf[0..S.n): its own values
// for the same set, else their projection (tmp: the neighbour's values, gathered first).
template <typename TS, typename T>
__device__ void neighbour_values(const HybArgs &a, int k, int sj, T *buf, T *tmp)
{
    const HybTabT<T> &tb = *static_cast<const HybTabT<T> *>(a.tab);
    const int sk = a.half[k] ? 0 : 1;
    const TS *h = static_cast<const TS *>(a.h);
    if (sk == sj) {
        gather_cell(h, a.toff, k, tb.set[sj].n, buf);
    } else {
        gather_cell(h, a.toff, k, tb.set[sk].n, tmp);
        project_warp(tb, sk, tmp, buf);
    }
}

// Ghost of Eq. 8 (perturbation form) for the velocities leaving wall `face` (0 bottom, 1 top,
// 2 left, 3 right; the side walls at rest), into buf; rho_w by Eq. 9 over the cell's own set.
template <typename T>
__device__ void wall_ghost(const HybArgs &a, const HybSetT<T> &S, const T *hc, int face, T *buf)
{
    const int lane = threadIdx.x & 31;
    T part = 0;
    for (int b = lane; b < S.n; b += 32) {
        const int sn = face == 0 ? S.sy[b] : face == 1 ? -S.sy[b] : face == 2 ? S.sx[b] : -S.sx[b];
        if (sn < 0) {
            const T xn = face == 0 ? S.xi_y[b] : face == 1 ? -S.xi_y[b] : face == 2 ? S.xi_x[b] : -S.xi_x[b];
            part += -xn * hc[b];
        }
    }
    const T rho_w = warp_sum(part) / (face < 2 ? S.d_y : S.d_x);
    const T u = (T)(face == 0 ? a.u_bottom : face == 1 ? a.u_top : 0.0);
    for (int b = lane; b < S.n; b += 32) {
        const T xt = face < 2 ? S.xi_x[b] : S.xi_y[b];
        buf[b] = S.w[b] * (rho_w * (T(1) + xt * u) + (a.homogeneous ? T(0) : xt * u / (T)a.u_ref));
    }
    __syncwarp();
}

// (mass, x-momentum, y-momentum) flux sum |xi_d| (1, xi_x, xi_y) v over the velocities of S
// moving along +axis (positive) or -axis; axis 0 = x, 1 = y.
template <typename T>
__device__ void face_moments(const HybSetT<T> &S, const T *v, int axis, bool positive, T (&m)[3])
{
    T p0 = 0, p1 = 0, p2 = 0;
    for (int b = threadIdx.x & 31; b < S.n; b += 32) {
        const int sd = axis == 0 ? S.sx[b] : S.sy[b];
        if (positive ? sd > 0 : sd < 0) {
            const T xd = axis == 0 ? S.xi_x[b] : S.xi_y[b];
            const T t = (xd < 0 ? -xd : xd) * v[b];
            p0 += t;
            p1 += t * S.xi_x[b];
            p2 += t * S.xi_y[b];
        }
    }
    m[0] = warp_sum(p0);
    m[1] = warp_sum(p1);
    m[2] = warp_sum(p2);
}

template <typename T>
struct HybShared {
    T nbv[HWARPS][4][HMAXV];   // left, right, below, above: upwind values in the cell's set
    T ph[HWARPS][HMAXV], nb[HWARPS][HMAXV];
    T own[HWARPS][HMAXV], tmp[HWARPS][HMAXV];   // the cell's values; a neighbour's before projection
};

// A cell with an interface face (a neighbour in the other set): one warp, warp `wi` of the
// block's shared buffers; arithmetic in the storage type TS.
template <typename TS>
__device__ void interface_cell(const HybArgs &a, HybShared<TS> &sh, int wi, int c, double dt_dx, double dt_dy,
                               int resid)
{
    using T = TS;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    const HybTabT<T> &tb = *static_cast<const HybTabT<T> *>(a.tab);
    const int sj = a.half[c] ? 0 : 1;
    const HybSetT<T> &S = tb.set[sj];
    const HybSetT<T> &H = tb.set[0];
    T *hc = sh.own[wi];
    gather_cell(static_cast<const TS *>(a.h), a.toff, c, S.n, hc);
    T *tmp = sh.tmp[wi];
    const int x = c % nx, y = c / nx;
    T(*nbv)[HMAXV] = sh.nbv[wi];
    // upwind values: x (cavity only) and y neighbours in this cell's set, or the walls' ghosts;
    // the four faces as (axis, side, neighbour or -1)
    int nbc[4] = {-1, -1, -1, -1};
    if (a.cavity) {
        if (x > 0) neighbour_values<TS>(a, nbc[0] = c - 1, sj, nbv[0], tmp);
        else wall_ghost(a, S, hc, 2, nbv[0]);
        if (x < nx - 1) neighbour_values<TS>(a, nbc[1] = c + 1, sj, nbv[1], tmp);
        else wall_ghost(a, S, hc, 3, nbv[1]);
    }
    if (y > 0) neighbour_values<TS>(a, nbc[2] = c - nx, sj, nbv[2], tmp);
    else wall_ghost(a, S, hc, 0, nbv[2]);
    if (y < ny - 1) neighbour_values<TS>(a, nbc[3] = c + nx, sj, nbv[3], tmp);
    else wall_ghost(a, S, hc, 1, nbv[3]);
    // interface faces of a full-range cell: mass and momentum exchange made equal to the
    // half-range evaluation of the face
    T cr[3] = {0, 0, 0};
    bool any_if = false;
    if (sj == 1)
        for (int f = 0; f < 4; ++f) any_if |= nbc[f] >= 0 && a.half[nbc[f]];
    if (any_if) {
        T *ph = sh.ph[wi], *nb = sh.nb[wi];
        project_warp(tb, 1, hc, ph);                            // this cell seen in H
        for (int f = 0; f < 4; ++f) {
            if (nbc[f] < 0 || !a.half[nbc[f]]) continue;
            const int axis = f >> 1;
            const bool lower = (f & 1) == 0;                  // the neighbour is on the lower side
            neighbour_values<TS>(a, nbc[f], 0, nb, tmp);      // its own half-range values
            T up[3], dn[3], got[3], sent[3];
            face_moments(H, lower ? nb : ph, axis, true, up);
            face_moments(H, lower ? ph : nb, axis, false, dn);
            face_moments(S, nbv[f], axis, lower, got);
            face_moments(S, hc, axis, !lower, sent);
            const T fac = (T)(axis == 0 ? dt_dx : dt_dy);
            for (int q = 0; q < 3; ++q) {
                const T want = lower ? up[q] - dn[q] : dn[q] - up[q];
                cr[q] += fac * (want - (got[q] - sent[q]));
            }
        }
    }
    // transport, moments, relaxation
    T hs[(HMAXV + 31) / 32];
    T rho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < (HMAXV + 31) / 32; ++i) {
        const int b = lane + 32 * i;
        T v = 0;
        if (b < S.n) {
            const T ex = S.xi_x[b], ey = S.xi_y[b];
            const T h0 = hc[b];
            T hx = h0, nux = 0;
            const int sgx = S.sx[b], sgy = S.sy[b];
            if (a.cavity) {
                hx = sgx > 0 ? nbv[0][b] : (sgx < 0 ? nbv[1][b] : h0);
                nux = S.nux[b];
            }
            const T hy = sgy > 0 ? nbv[2][b] : (sgy < 0 ? nbv[3][b] : h0);
            const T nuy = S.nuy[b];
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
    TS *out = static_cast<TS *>(a.hn) + a.toff[c];
    constexpr bool MIXED = std::is_same<TS, float>::value;      // the FP32 march's correction sweeps
    const float *src = (MIXED && a.src) ? a.src + a.toff[c] : nullptr;
    const T om = (T)a.omega;
    T pd = 0, pn = 0;
#pragma unroll
    for (int i = 0; i < (HMAXV + 31) / 32; ++i) {
        const int b = lane + 32 * i;
        if (b < S.n) {
            const T heq = S.w[b] * (rho + S.xi_x[b] * jx + S.xi_y[b] * jy);
            T o = hs[i] - om * (hs[i] - heq);
            if (MIXED && src) o += (T)src[(long)HST * b];
            out[(long)HST * b] = o;
            if (resid) {
                const T d = o - hc[b];
                pd += d * d;
                pn += o * o;
            }
        }
    }
    if (resid) {
        pd = warp_sum(pd);
        pn = warp_sum(pn);
        if (lane == 0) {
            a.part[2 * c] = (double)pd;
            a.part[2 * c + 1] = (double)pn;
        }
    }
}

// Plain cells of one set: all their existing neighbours carry the same set.  Per tile (up to
// 32 consecutive cells of the set) G warps, lane p the tile's cell p, warp g the velocity rows
// iy in [g M / G, (g + 1) M / G); the set's 1-D nodes, weights and Courant numbers are kernel
// parameters (velocity a = iy M + ix: xi = (xi[ix], xi[iy]), w = w1[ix] w1[iy]).  The same
// update as interface_cell without projections: first-order upwind transport with the wall
// ghosts of Eqs. 8-9 (the wall density a flux balance over the cell's set), relaxation
// towards w (rho + xi . j) (Eqs. 1, 5-7).  Interface cells of a tile are left to their own
// kernel; idle lanes mirror the tile's first cell and store nothing.
// TC: the arithmetic and storage type (double for the FP64 march, float for the FP32 one)
template <typename TC>
struct PlainArgs {
    const int *toff;
    const unsigned char *iface;   // [ncells] 1: a neighbour carries the other set
    const TC *h;
    TC *hn;
    double *part;
    const float *src;             // correction march: the defect added after relaxation (else NULL)
    int nx, ny, cavity, homogeneous;
    TC omega, b, u_bottom, u_top, inv_u_ref;   // b = 1 - omega
    double inv_dx_wall, inv_dy_wall;   // 1 / sum_{xi > 0} xi w over the set, per axis
    TC xi[12], w1[12], nux[12], nuy[12];
    TC a0[144];                        // 1 - nu_x - nu_y per velocity a = iy M + ix
};

// blocks of four warps: G warps per tile, 4 / G tiles per block
template <int M, int G>
struct PlainShape {
    static constexpr int TPB = HWARPS / G;             // tiles per block
    static_assert(M % G == 0 && HWARPS % G == 0 && M <= 12, "warps split the velocity rows evenly");
};

template <int M, int G, typename TC>
__device__ __forceinline__ void plain_tiles(const PlainArgs<TC> &p, const int2 *tiles, int ntiles, int bid, int resid,
                                            double (*s_x)[G][4][32])
{
    constexpr int TPB = PlainShape<M, G>::TPB, RPL = M / G, HALF = M / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tl = warp / G, g = warp - tl * G;
    const int t = bid * TPB + tl;
    int c0 = 0, k = 0;
    if (t < ntiles) {
        const int2 T = tiles[t];
        c0 = T.x;
        k = T.y;
    }
    const int cl = lane < k ? c0 + lane : c0;
    const bool on = lane < k && !p.iface[cl];
    const int nx = p.nx, ny = p.ny, x = cl % nx, y = cl / nx;
    const bool cav = p.cavity != 0;
    const bool wl = cav && x == 0, wr = cav && x == nx - 1, wb = y == 0, wt = y == ny - 1;
    const TC *h = p.h;
    const long oc = p.toff[cl];
    // same-set neighbours of a plain cell; an idle or interface lane reads only its own cell
    const long ol = (on && cav && !wl) ? p.toff[cl - 1] : oc;
    const long orr = (on && cav && !wr) ? p.toff[cl + 1] : oc;
    const long od = (on && !wb) ? p.toff[cl - nx] : oc;
    const long ou = (on && !wt) ? p.toff[cl + nx] : oc;

    // ---- wall densities, where a lane of the block touches a wall ----
    TC rw[4] = {0, 0, 0, 0};
    if (__syncthreads_or((int)(on && (wl || wr || wb || wt)))) {
        double pw[4] = {0.0, 0.0, 0.0, 0.0};     // outflow through the bottom, top, left, right walls
        // products and the sums over one velocity row in the arithmetic type, the sums over
        // rows and warps in FP64 (as the single-domain kernels do; per-velocity FP64 sums kept
        // the FP64 pipe of the FP32 hybrid step 38 % busy)
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            TC ys = 0, ls = 0, rs = 0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const TC v = h[oc + (long)HST * (iy * M + ix)];
                ys += v;
                if (ix < HALF) ls -= p.xi[ix] * v;
                if (ix >= M - HALF) rs += p.xi[ix] * v;
            }
            if (iy < HALF) pw[0] -= (double)(p.xi[iy] * ys);
            if (iy >= M - HALF) pw[1] += (double)(p.xi[iy] * ys);
            pw[2] += (double)ls;
            pw[3] += (double)rs;
        }
        if (G > 1) {
#pragma unroll
            for (int f = 0; f < 4; ++f) s_x[tl][g][f][lane] = pw[f];
            __syncthreads();
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                pw[f] = 0.0;
#pragma unroll
                for (int q = 0; q < G; ++q) pw[f] += s_x[tl][q][f][lane];
            }
            __syncthreads();
        }
        rw[0] = (TC)(pw[0] * p.inv_dy_wall);
        rw[1] = (TC)(pw[1] * p.inv_dy_wall);
        rw[2] = (TC)(pw[2] * p.inv_dx_wall);
        rw[3] = (TC)(pw[3] * p.inv_dx_wall);
    }

    // ---- transport and moment sums ----
    // h* = (1 - nu_x - nu_y) h + nu_x h_x + nu_y h_y; rho, j_x per velocity, j_y per row.
    // The wall ghosts are formed only in tiles that touch a wall (WALLS): as a select in every
    // tile they doubled the FP64 operations of the step.
    // the FP32 march's correction sweeps drop the walls' driving terms and add the defect; the
    // FP64 march never does (its kernels carry no code for it)
    constexpr bool MIXED = std::is_same<TC, float>::value;
    const TC ub = p.u_bottom, ut = p.u_top;
    const TC drive = (MIXED && p.homogeneous) ? TC(0) : p.inv_u_ref;     // the walls' driving term
    TC hs[RPL * M];
    TC R = 0, X = 0, Y = 0;
    auto transport = [&](auto walls_tag) {
        constexpr bool WALLS = decltype(walls_tag)::value;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC nuy = p.nuy[iy], wy = p.w1[iy];
            TC Rr = 0, Xr = 0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const long a = (long)HST * (iy * M + ix);
                const TC h0 = h[oc + a];
                TC v = p.a0[iy * M + ix] * h0;
                if (cav) {
                    TC hx = h0;
                    if (ix >= M - HALF) {
                        hx = h[ol + a];
                        if (WALLS && wl) hx = p.w1[ix] * wy * rw[2];          // side walls at rest
                    } else if (ix < HALF) {
                        hx = h[orr + a];
                        if (WALLS && wr) hx = p.w1[ix] * wy * rw[3];
                    }
                    v = fma_(p.nux[ix], hx, v);
                }
                TC hy = h0;
                if (iy >= M - HALF) {
                    hy = h[od + a];
                    if (WALLS && wb) hy = p.w1[ix] * wy * (rw[0] * (TC(1) + p.xi[ix] * ub) + p.xi[ix] * ub * drive);
                } else if (iy < HALF) {
                    hy = h[ou + a];
                    if (WALLS && wt) hy = p.w1[ix] * wy * (rw[1] * (TC(1) + p.xi[ix] * ut) + p.xi[ix] * ut * drive);
                }
                v = fma_(nuy, hy, v);
                hs[r * M + ix] = v;
                Rr += v;
                Xr = fma_(p.xi[ix], v, Xr);
            }
            R += Rr;
            X += Xr;
            Y = fma_(p.xi[iy], Rr, Y);
        }
    };
    if (__any_sync(0xffffffffu, wl || wr || wb || wt)) transport(std::true_type{});
    else transport(std::false_type{});
    if (G > 1) {
        s_x[tl][g][0][lane] = R;
        s_x[tl][g][1][lane] = X;
        s_x[tl][g][2][lane] = Y;
        __syncthreads();
        R = X = Y = 0;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            R += (TC)s_x[tl][q][0][lane];
            X += (TC)s_x[tl][q][1][lane];
            Y += (TC)s_x[tl][q][2][lane];
        }
        __syncthreads();
    }

    // ---- relaxation h' = (1 - omega) h* + omega w (rho + xi . j), store, residual sums ----
    TC pd = 0, pn = 0;
    const float *src = (MIXED && p.src) ? p.src + oc : nullptr;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int iy = g * RPL + r;
        const TC ow = p.omega * p.w1[iy];
        const TC A = ow * fma_(p.xi[iy], Y, R), B = ow * X;
#pragma unroll
        for (int ix = 0; ix < M; ++ix) {
            const long a = (long)HST * (iy * M + ix);
            TC o = fma_(p.b, hs[r * M + ix], p.w1[ix] * fma_(p.xi[ix], B, A));
            if (MIXED && src) o += (TC)src[a];
            if (on) p.hn[oc + a] = o;
            if (resid) {
                const TC d = o - h[oc + a];
                pd += d * d;
                pn += o * o;
            }
        }
    }
    if (resid) {
        if (G > 1) {
            s_x[tl][g][0][lane] = (double)pd;
            s_x[tl][g][1][lane] = (double)pn;
            __syncthreads();
            double sd = 0.0, sn = 0.0;
#pragma unroll
            for (int q = 0; q < G; ++q) {
                sd += s_x[tl][q][0][lane];
                sn += s_x[tl][q][1][lane];
            }
            pd = (TC)sd;
            pn = (TC)sn;
        }
        if (on && g == 0) {
            p.part[2 * cl] = (double)pd;
            p.part[2 * cl + 1] = (double)pn;
        }
    }
}

// Warps per half-range tile (2N nodes per axis): four where they split the velocity rows
// evenly, else two; a full-range tile (N nodes) takes one warp
__host__ __device__ constexpr int half_warps(int n) { return (2 * n) % 4 == 0 ? 4 : 2; }

// One step, one launch: the blocks for the interface cells first (one warp per cell: their
// projections are long latency chains), then those for the half-range and the full-range
// tiles, so that all three run side by side.
struct StepLists {
    const int *cells;          // interface cells
    int ncells;
    const int2 *tiles[2];      // half-range, full-range tiles with a plain cell
    int ntiles[2];
};

// blocks a SM the FP32 build asks for: eight (64 registers a thread) where that does not
// spill, six for the 100-velocity half-range set; FP64 as the compiler chooses
template <int N, typename TS>
constexpr int hybrid_min_blocks() { return sizeof(TS) == 8 ? 1 : (N == 5 ? 6 : 8); }

template <int N, typename TS>
__global__ void __launch_bounds__(32 * HWARPS, hybrid_min_blocks<N, TS>()) hybrid_step_kernel(const HybArgs a, const PlainArgs<TS> ph,
                                                                   const PlainArgs<TS> pf, const StepLists L,
                                                                   double dt_dx, double dt_dy, int resid)
{
    constexpr int GH = half_warps(N);
    __shared__ union {
        HybShared<TS> sh;
        double hx[HWARPS / GH][GH][4][32];
        double fx[HWARPS][1][4][32];
    } u;
    const int bid = (int)blockIdx.x;
    const int ifb = (L.ncells + HWARPS - 1) / HWARPS;
    const int hbk = (L.ntiles[0] + HWARPS / GH - 1) / (HWARPS / GH);
    if (bid < ifb) {
        const int wi = threadIdx.x >> 5, ci = bid * HWARPS + wi;
        if (ci < L.ncells) interface_cell<TS>(a, u.sh, wi, L.cells[ci], dt_dx, dt_dy, resid);    // whole warps
    } else if (bid < ifb + hbk) {
        plain_tiles<2 * N, GH>(ph, L.tiles[0], L.ntiles[0], bid - ifb, resid, u.hx);
    } else {
        plain_tiles<N, 1>(pf, L.tiles[1], L.ntiles[1], bid - ifb - hbk, resid, u.fx);
    }
}

template <int N, typename TS>
cudaError_t launch_step_n(const HybArgs &a, const PlainArgs<TS> &ph, const PlainArgs<TS> &pf, const StepLists &L,
                          double dt_dx, double dt_dy, int resid, cudaStream_t st)
{
    constexpr int GH = half_warps(N);
    const int blocks = (L.ncells + HWARPS - 1) / HWARPS + (L.ntiles[0] + HWARPS / GH - 1) / (HWARPS / GH) +
                       (L.ntiles[1] + HWARPS - 1) / HWARPS;
    if (blocks == 0) return cudaSuccess;
    hybrid_step_kernel<N, TS><<<blocks, 32 * HWARPS, 0, st>>>(a, ph, pf, L, dt_dx, dt_dy, resid);
    return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_hybrid_step(int n, const HybArgs &a, const PlainArgs<TS> &ph, const PlainArgs<TS> &pf,
                               const StepLists &L, double dt_dx, double dt_dy, int resid, cudaStream_t st)
{
    switch (n) {
    case 2: return launch_step_n<2, TS>(a, ph, pf, L, dt_dx, dt_dy, resid, st);
    case 3: return launch_step_n<3, TS>(a, ph, pf, L, dt_dx, dt_dy, resid, st);
    case 4: return launch_step_n<4, TS>(a, ph, pf, L, dt_dx, dt_dy, resid, st);
    case 5: return launch_step_n<5, TS>(a, ph, pf, L, dt_dx, dt_dy, resid, st);
    case 6: return launch_step_n<6, TS>(a, ph, pf, L, dt_dx, dt_dy, resid, st);
    default: return cudaErrorInvalidValue;
    }
}

// elementwise over the tiled state (padding included): float <-> double, y += x, and the FP64
// defect d = m - h as float with its sums over the cells' values (packed index i -> cell by
// binary search over poff, as the relayout)
__global__ void hybrid_f32_to_f64_kernel(const float *x, double *y, long n)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] = x[i];
}

__global__ void hybrid_f64_to_f32_kernel(const double *x, float *y, long n)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] = (float)x[i];
}

__global__ void hybrid_add_f32_kernel(float *y, const float *x, long n)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] += x[i];
}

__global__ void __launch_bounds__(256) hybrid_defect_kernel(const double *m, const float *h, float *d, const int *poff,
                                                            const int *toff, int ncells, double *sums)
{
    __shared__ double sd[256], sn[256];
    const long total = poff[ncells];
    double a = 0.0, b = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        int lo = 0, hi = ncells - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (poff[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const long ti = toff[lo] + (long)HST * (i - poff[lo]);
        const double mv = m[ti], dv = mv - (double)h[ti];
        d[ti] = (float)dv;
        a += dv * dv;
        b += mv * mv;
    }
    sd[threadIdx.x] = a;
    sn[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sd[threadIdx.x] += sd[threadIdx.x + w];
            sn[threadIdx.x] += sn[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[2 * blockIdx.x] = sd[0];
        sums[2 * blockIdx.x + 1] = sn[0];
    }
}

// packed FP64 (cell after cell) <-> tiled state of type TS: one thread per value
template <typename TS>
__global__ void hybrid_relayout_kernel(const void *src, void *dst, const int *poff, const int *toff, int ncells,
                                       int to_tiled)
{
    const long total = poff[ncells];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        // the cell of packed value i: poff is ascending
        int lo = 0, hi = ncells - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (poff[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const long b = i - poff[lo], ti = toff[lo] + (long)HST * b;
        if (to_tiled) static_cast<TS *>(dst)[ti] = (TS)static_cast<const double *>(src)[i];
        else static_cast<double *>(dst)[i] = (double)static_cast<const TS *>(src)[ti];
    }
}

// residual sums over the cells: one block, each thread a fixed stride of cells, then a fixed
// tree (the same order every call)
constexpr int HFIN = 1024;
// stage 1: block b sums the pairs of cells [b HCHUNK, (b + 1) HCHUNK) into out[2 b..2 b + 1];
// stage 2 (one block) sums those partials: the same fixed order at every call
constexpr int HCHUNK = 8192;
__global__ void __launch_bounds__(HFIN) hybrid_finalize_kernel(const double *part, int ncells, double *out)
{
    __shared__ double sd[HFIN], sn[HFIN];
    double d = 0.0, n = 0.0;
    const int first = (int)blockIdx.x * HCHUNK, last = min(ncells, first + HCHUNK);
    for (int j = first + (int)threadIdx.x; j < last; j += HFIN) {
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
        out[2 * blockIdx.x] = sd[0];
        out[2 * blockIdx.x + 1] = sn[0];
    }
}

// Couette column: the x-momentum flux through the ny + 1 faces (interface faces evaluated in
// the half-range set); one warp per face k
__global__ void __launch_bounds__(32 * HWARPS) hybrid_face_flux_kernel(const HybArgs a, double u_ref, double *pxy)
{
    __shared__ HybShared<double> sh;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int k = blockIdx.x * HWARPS + wi;
    if (k > a.ny) return;
    const HybTabT<double> &tb = *static_cast<const HybTabT<double> *>(a.tab);
    double *lo = sh.nbv[wi][0], *hi = sh.nbv[wi][1];
    double up = 0.0, dn = 0.0;
    if (k > 0 && k < a.ny && a.half[k - 1] != a.half[k]) {
        const HybSetT<double> &H = tb.set[0];
        neighbour_values<double>(a, k - 1, 0, lo, sh.tmp[wi]);
        neighbour_values<double>(a, k, 0, hi, sh.tmp[wi]);
        double mu[3], md[3];
        face_moments(H, lo, 1, true, mu);
        face_moments(H, hi, 1, false, md);
        up = mu[1];
        dn = -md[1];                                            // sum over xi_y < 0 of xi_y xi_x h
    } else {
        const int cb = k == 0 ? 0 : k - 1, ca = k == a.ny ? a.ny - 1 : k;
        const HybSetT<double> &Sb = tb.set[a.half[cb] ? 0 : 1], &Sa = tb.set[a.half[ca] ? 0 : 1];
        double *vb = sh.own[wi], *va = sh.tmp[wi];
        gather_cell(static_cast<const double *>(a.h), a.toff, cb, Sb.n, vb);
        gather_cell(static_cast<const double *>(a.h), a.toff, ca, Sa.n, va);
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
    const HybSetT<double> &S = static_cast<const HybTabT<double> *>(a.tab)->set[a.half[c] ? 0 : 1];
    const double *hc = static_cast<const double *>(a.h) + a.toff[c];
    double s0 = 0.0, sx = 0.0, sy = 0.0;
    for (int b = lane; b < S.n; b += 32) {
        const double v = hc[(long)HST * b];
        s0 += v;
        sx += S.xi_x[b] * v;
        sy += S.xi_y[b] * v;
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
    std::vector<int> off;    // [ncells + 1] packed (host-transfer) offsets, cell after cell
    std::vector<unsigned char> half;
    long unknowns;           // values of the packed state
    long tiled;              // doubles of the tiled device state (tiles padded to 32 cells)
    cudaStream_t stream;
    HybTabT<double> *d_tab;  // the tables for the FP64 kernels
    HybTabT<float> *d_tab32; // and for the FP32 march
    int *d_poff, *d_toff;    // packed offsets; tiled offsets of velocity 0 of each cell
    unsigned char *d_half, *d_iface;
    double *d_h[2], *d_part, *d_res;
    double *h_res;           // pinned
    int cur;
    bool have_resid;
    int n_if;                // cells with an interface face
    int *d_if;               // [n_if]
    int n_tiles[2];          // tiles of the half-range (0) and full-range (1) set holding a plain cell
    int2 *d_tiles[2];        // (first cell, count)
    int m1[2];               // nodes per axis of each set
    double x1[2][12], w1[2][12], inv_dx_wall[2], inv_dy_wall[2];
    // FP32 march (lbm_hybrid_set_precision): tiled float buffers, the state ping-pong (0, 1),
    // the FP64 defect (2) and the correction ping-pong (3, 4); the FP64 buffers d_h then serve
    // as scratch (the defect's FP64 step, host transfers)
    int prec;
    float *d_f[5];
    double *d_sums;          // [2 * HDEF] partial sums of the defect pass
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

constexpr int HDEF = 152 * 4;   // blocks of the defect pass

// Step arguments from state h to hn (the current ones by default), with an optional source
// (correction march, homogeneous walls)
HybArgs hargs(const lbm_hybrid *hb, const void *h = nullptr, void *hn = nullptr, const float *src = nullptr,
              int homogeneous = 0)
{
    HybArgs a;
    std::memset(&a, 0, sizeof a);
    a.tab = hb->d_tab;
    a.toff = hb->d_toff;
    a.half = hb->d_half;
    const bool f32 = hb->prec == LBM_FP32_PERTURB;
    a.h = h ? h : (f32 ? (const void *)hb->d_f[hb->cur] : (const void *)hb->d_h[hb->cur]);
    a.hn = hn ? hn : (f32 ? (void *)hb->d_f[hb->cur ^ 1] : (void *)hb->d_h[hb->cur ^ 1]);
    a.src = src;
    a.homogeneous = homogeneous;
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

// the plain-cell kernel's arguments for set `set` in arithmetic type TC (coefficients formed
// in FP64 and rounded once)
template <typename TC>
PlainArgs<TC> plain_args(const lbm_hybrid *hb, int set, const HybArgs &a)
{
    PlainArgs<TC> p;
    std::memset(&p, 0, sizeof p);
    p.toff = hb->d_toff;
    p.iface = hb->d_iface;
    p.h = static_cast<const TC *>(a.h);
    p.hn = static_cast<TC *>(a.hn);
    p.part = hb->d_part;
    p.src = a.src;
    p.nx = hb->nx;
    p.ny = hb->ny;
    p.cavity = hb->geom == LBM_CAVITY;
    p.homogeneous = a.homogeneous;
    p.omega = (TC)hb->omega;
    p.b = (TC)(1.0 - hb->omega);
    p.u_bottom = (TC)hb->u_bottom;
    p.u_top = (TC)hb->u_top;
    p.inv_u_ref = (TC)(1.0 / hb->u_ref);
    p.inv_dx_wall = hb->inv_dx_wall[set];
    p.inv_dy_wall = hb->inv_dy_wall[set];
    const int m = hb->m1[set];
    double nux[12], nuy[12];
    for (int i = 0; i < m; ++i) {
        nux[i] = p.cavity ? std::fabs(hb->x1[set][i]) * hb->dt / hb->dx : 0.0;
        nuy[i] = std::fabs(hb->x1[set][i]) * hb->dt / hb->dy;
        p.xi[i] = (TC)hb->x1[set][i];
        p.w1[i] = (TC)hb->w1[set][i];
        p.nux[i] = (TC)nux[i];
        p.nuy[i] = (TC)nuy[i];
    }
    for (int iy = 0; iy < m; ++iy)
        for (int ix = 0; ix < m; ++ix) p.a0[iy * m + ix] = (TC)(1.0 - nux[ix] - nuy[iy]);
    return p;
}

// One step from a.h into a.hn in precision TS (the residual partials when resid)
template <typename TS>
cudaError_t hybrid_launch(const lbm_hybrid *hb, const HybArgs &a0, int resid)
{
    HybArgs a = a0;
    a.tab = std::is_same<TS, float>::value ? (const void *)hb->d_tab32 : (const void *)hb->d_tab;
    StepLists L;
    L.cells = hb->d_if;
    L.ncells = hb->n_if;
    for (int t = 0; t < 2; ++t) {
        L.tiles[t] = hb->d_tiles[t];
        L.ntiles[t] = hb->n_tiles[t];
    }
    // the interface faces' dt / dx and dt / dy, divided once here (the device's FP64 divide
    // would run on every lane of every interface warp)
    return launch_hybrid_step<TS>(hb->n_half, a, plain_args<TS>(hb, 0, a), plain_args<TS>(hb, 1, a), L,
                                  hb->dt / hb->dx, hb->dt / hb->dy, resid, hb->stream);
}

// the two-stage reduction of the residual partials into d_res[0..1]
cudaError_t hybrid_finalize(const lbm_hybrid *hb)
{
    const int nc = hb->nx * hb->ny, nb1 = (nc + HCHUNK - 1) / HCHUNK;
    hybrid_finalize_kernel<<<nb1, HFIN, 0, hb->stream>>>(hb->d_part, nc, hb->d_res + 2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        hybrid_finalize_kernel<<<1, HFIN, 0, hb->stream>>>(hb->d_res + 2, nb1, hb->d_res);
        e = cudaGetLastError();
    }
    return e;
}

int elem_blocks(long n) { return (int)std::max(1L, std::min<long>((n + 255) / 256, 152L * 16)); }

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
    hb->d_tab32 = nullptr;
    hb->d_poff = hb->d_toff = nullptr;
    hb->d_half = hb->d_iface = nullptr;
    hb->d_h[0] = hb->d_h[1] = nullptr;
    hb->d_part = hb->d_res = nullptr;
    hb->h_res = nullptr;
    hb->d_if = nullptr;
    hb->d_tiles[0] = hb->d_tiles[1] = nullptr;
    hb->n_if = hb->n_tiles[0] = hb->n_tiles[1] = 0;
    hb->prec = LBM_FP64;
    for (auto &f : hb->d_f) f = nullptr;
    hb->d_sums = nullptr;
    std::vector<HybTables> tabv(1);     // ~130 KB: on the heap, zero-initialised
    HybTables &tab = tabv[0];
    double my_h = 0, my_f = 0;
    if (!fill_set(tab.set[0], LBM_HALF_RANGE_GH, n_half, hb->order, my_h) ||
        !fill_set(tab.set[1], LBM_FULL_RANGE_GH, n_half, hb->order, my_f)) {
        delete hb;
        return hfail(LBM_EINVAL, "quadrature construction failed");
    }
    for (int t = 0; t < 2; ++t) {       // the sets' 1-D rules for the plain-cell kernel
        std::vector<double> x, w;
        lbm_rule_1d(t == 0 ? LBM_HALF_RANGE_GH : LBM_FULL_RANGE_GH, n_half, x, w);
        hb->m1[t] = (int)x.size();
        for (int i = 0; i < hb->m1[t]; ++i) {
            hb->x1[t][i] = x[i];
            hb->w1[t][i] = w[i];
        }
        hb->inv_dx_wall[t] = 1.0 / tab.set[t].d_x;
        hb->inv_dy_wall[t] = 1.0 / tab.set[t].d_y;
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
    // cells with a neighbour in the other set go to the projecting kernel, the others to the
    // plain-cell kernel; the tiled layout: runs of consecutive cells of one set cut into tiles
    // of up to 32 cells, each tile n_set x 32 doubles
    std::vector<int> if_cells;
    std::vector<unsigned char> iface(nc, 0);
    for (long c = 0; c < nc; ++c) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const unsigned char hc_ = hb->half[c];
        bool ifc = (y > 0 && hb->half[c - nx] != hc_) || (y < ny - 1 && hb->half[c + nx] != hc_);
        if (geom == LBM_CAVITY) ifc = ifc || (x > 0 && hb->half[c - 1] != hc_) || (x < nx - 1 && hb->half[c + 1] != hc_);
        iface[c] = ifc ? 1 : 0;
        if (ifc) if_cells.push_back((int)c);
    }
    std::vector<int> toff(nc);
    std::vector<int2> tiles[2];
    long tb = 0;
    for (long c = 0; c < nc;) {
        const int set = hb->half[c] ? 0 : 1;
        long e = c + 1;
        while (e < nc && e - c < 32 && hb->half[e] == hb->half[c]) ++e;
        bool plain = false;
        for (long q = c; q < e; ++q) {
            toff[q] = (int)std::min(tb + (q - c), (long)INT_MAX);     // checked below
            plain |= !iface[q];
        }
        if (plain) tiles[set].push_back(make_int2((int)c, (int)(e - c)));
        tb += 32L * tab.set[set].n;
        c = e;
    }
    if (tb > (long)INT_MAX) {
        delete hb;
        return hfail(LBM_EINVAL, "too many unknowns for the hybrid's 32-bit cell offsets");
    }
    hb->tiled = tb;
    hb->n_if = (int)if_cells.size();
    hb->n_tiles[0] = (int)tiles[0].size();
    hb->n_tiles[1] = (int)tiles[1].size();
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
    // device tables in both arithmetic types
    std::vector<HybTabT<double>> t64(1);
    std::vector<HybTabT<float>> t32(1);
    for (int t = 0; t < 2; ++t) {
        const HybSet &S = tab.set[t];
        HybSetT<double> &D = t64[0].set[t];
        HybSetT<float> &F = t32[0].set[t];
        D.n = F.n = S.n;
        D.lanes = F.lanes = S.lanes;
        D.d_x = S.d_x;
        D.d_y = S.d_y;
        F.d_x = (float)S.d_x;
        F.d_y = (float)S.d_y;
        for (int b = 0; b < S.n; ++b) {
            D.xi_x[b] = S.xi_x[b];
            D.xi_y[b] = S.xi_y[b];
            D.w[b] = S.w[b];
            D.nux[b] = S.nux[b];
            D.nuy[b] = S.nuy[b];
            F.xi_x[b] = (float)S.xi_x[b];
            F.xi_y[b] = (float)S.xi_y[b];
            F.w[b] = (float)S.w[b];
            F.nux[b] = (float)S.nux[b];
            F.nuy[b] = (float)S.nuy[b];
            D.sx[b] = F.sx[b] = S.sx[b];
            D.sy[b] = F.sy[b] = S.sy[b];
        }
        for (int i = 0; i < HMAXV * HMAXF; ++i) {
            t64[0].pt[t][i] = tab.pt[t][i];
            t32[0].pt[t][i] = (float)tab.pt[t][i];
        }
    }
    cudaError_t e = cudaMalloc(&hb->d_tab, sizeof(HybTabT<double>));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_tab32, sizeof(HybTabT<float>));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_poff, sizeof(int) * (nc + 1));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_toff, sizeof(int) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_half, nc);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_iface, nc);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_h[0], sizeof(double) * tb);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_h[1], sizeof(double) * tb);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_part, sizeof(double) * 2 * nc);
    // the residual sums and the first-stage partials of their reduction
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_res, sizeof(double) * 2 * (1 + (nc + HCHUNK - 1) / HCHUNK));
    if (e == cudaSuccess) e = cudaMallocHost(&hb->h_res, sizeof(double) * 2);
    if (e == cudaSuccess && hb->n_if > 0) e = cudaMalloc(&hb->d_if, sizeof(int) * hb->n_if);
    for (int t = 0; t < 2 && e == cudaSuccess; ++t)
        if (hb->n_tiles[t] > 0) e = cudaMalloc(&hb->d_tiles[t], sizeof(int2) * hb->n_tiles[t]);
    if (e == cudaSuccess && hb->n_if > 0)
        e = cudaMemcpyAsync(hb->d_if, if_cells.data(), sizeof(int) * hb->n_if, cudaMemcpyHostToDevice, hb->stream);
    for (int t = 0; t < 2 && e == cudaSuccess; ++t)
        if (hb->n_tiles[t] > 0)
            e = cudaMemcpyAsync(hb->d_tiles[t], tiles[t].data(), sizeof(int2) * hb->n_tiles[t], cudaMemcpyHostToDevice,
                                hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb->d_tab, t64.data(), sizeof(HybTabT<double>), cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb->d_tab32, t32.data(), sizeof(HybTabT<float>), cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb->d_poff, hb->off.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb->d_toff, toff.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb->d_half, hb->half.data(), nc, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb->d_iface, iface.data(), nc, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hb->d_h[0], 0, sizeof(double) * tb, hb->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hb->d_h[1], 0, sizeof(double) * tb, hb->stream);
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
    cudaFree(hb->d_tab32);
    cudaFree(hb->d_poff);
    cudaFree(hb->d_toff);
    cudaFree(hb->d_half);
    cudaFree(hb->d_iface);
    cudaFree(hb->d_h[0]);
    cudaFree(hb->d_h[1]);
    cudaFree(hb->d_part);
    cudaFree(hb->d_res);
    cudaFree(hb->d_if);
    cudaFree(hb->d_tiles[0]);
    cudaFree(hb->d_tiles[1]);
    for (auto f : hb->d_f) cudaFree(f);
    cudaFree(hb->d_sums);
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

// packed <-> tiled through the other state buffer (it is rewritten by the next step)
static cudaError_t hybrid_relayout(lbm_hybrid *hb, const void *src, void *dst, bool to_tiled)
{
    const int nc = hb->nx * hb->ny, blocks = elem_blocks(hb->unknowns);
    if (hb->prec == LBM_FP32_PERTURB)
        hybrid_relayout_kernel<float><<<blocks, 256, 0, hb->stream>>>(src, dst, hb->d_poff, hb->d_toff, nc, to_tiled ? 1 : 0);
    else
        hybrid_relayout_kernel<double><<<blocks, 256, 0, hb->stream>>>(src, dst, hb->d_poff, hb->d_toff, nc, to_tiled ? 1 : 0);
    return cudaGetLastError();
}

// the current state's buffer (FP64 or FP32, tiled)
static void *hybrid_state(lbm_hybrid *hb)
{
    return hb->prec == LBM_FP32_PERTURB ? (void *)hb->d_f[hb->cur] : (void *)hb->d_h[hb->cur];
}

// the current state as FP64 in a tiled buffer (itself, or its FP64 copy in scratch d_h[0])
static cudaError_t hybrid_state_f64(lbm_hybrid *hb, const double **out)
{
    if (hb->prec != LBM_FP32_PERTURB) {
        *out = hb->d_h[hb->cur];
        return cudaSuccess;
    }
    hybrid_f32_to_f64_kernel<<<elem_blocks(hb->tiled), 256, 0, hb->stream>>>(hb->d_f[hb->cur], hb->d_h[0], hb->tiled);
    *out = hb->d_h[0];
    return cudaGetLastError();
}

lbm_status lbm_hybrid_set_state(lbm_hybrid *hb, const double *h)
{
    if (!hb || !h) return hfail(LBM_EINVAL, "NULL argument");
    // scratch: the FP64 buffer the state is not in
    double *scratch = hb->prec == LBM_FP32_PERTURB ? hb->d_h[0] : hb->d_h[hb->cur ^ 1];
    cudaError_t e = cudaMemcpyAsync(scratch, h, sizeof(double) * hb->unknowns, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = hybrid_relayout(hb, scratch, hybrid_state(hb), true);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    hb->have_resid = false;
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("setting the state: ") + cudaGetErrorString(e));
}

lbm_status lbm_hybrid_get_state(lbm_hybrid *hb, double *h)
{
    if (!hb || !h) return hfail(LBM_EINVAL, "NULL argument");
    double *scratch = hb->prec == LBM_FP32_PERTURB ? hb->d_h[0] : hb->d_h[hb->cur ^ 1];
    cudaError_t e = hybrid_relayout(hb, hybrid_state(hb), scratch, false);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, scratch, sizeof(double) * hb->unknowns, cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("reading the state: ") + cudaGetErrorString(e));
}

lbm_status lbm_hybrid_step(lbm_hybrid *hb, long nsteps)
{
    if (!hb || nsteps < 0) return hfail(LBM_EINVAL, "invalid step arguments");
    const int nc = hb->nx * hb->ny;
    (void)nc;
    for (long s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        const HybArgs a = hargs(hb);
        cudaError_t e = hb->prec == LBM_FP32_PERTURB ? hybrid_launch<float>(hb, a, last ? 1 : 0)
                                                     : hybrid_launch<double>(hb, a, last ? 1 : 0);
        if (e == cudaSuccess && last) e = hybrid_finalize(hb);
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
    double res = INFINITY, best = INFINITY;
    int flat = 0;
    while (taken < max_steps) {
        lbm_status st = lbm_hybrid_step(hb, every);
        if (st != LBM_OK) return st;
        taken += every;
        st = lbm_hybrid_residual(hb, &res);
        if (st != LBM_OK) return st;
        if (res < tol) break;
        // the FP32 march stops at its rounding floor: no 1 % improvement over 20 checks
        if (hb->prec == LBM_FP32_PERTURB) {
            if (res < 0.99 * best) {
                best = res;
                flat = 0;
            } else if (++flat >= 20) {
                break;
            }
        }
    }
    if (steps) *steps = taken;
    if (r) *r = res;
    return LBM_OK;
}

lbm_status lbm_hybrid_set_precision(lbm_hybrid *hb, int prec)
{
    if (!hb) return hfail(LBM_EINVAL, "hybrid is NULL");
    if (prec != LBM_FP64 && prec != LBM_FP32_PERTURB) return hfail(LBM_EINVAL, "unknown precision");
    if (prec == hb->prec) return LBM_OK;
    cudaError_t e = cudaSuccess;
    if (prec == LBM_FP32_PERTURB) {
        for (int i = 0; i < 5 && e == cudaSuccess; ++i)
            if (!hb->d_f[i]) {
                e = cudaMalloc(&hb->d_f[i], sizeof(float) * hb->tiled);
                if (e == cudaSuccess) e = cudaMemsetAsync(hb->d_f[i], 0, sizeof(float) * hb->tiled, hb->stream);
            }
        if (e == cudaSuccess && !hb->d_sums) e = cudaMalloc(&hb->d_sums, sizeof(double) * 2 * HDEF);
        if (e == cudaSuccess) {
            hybrid_f64_to_f32_kernel<<<elem_blocks(hb->tiled), 256, 0, hb->stream>>>(hb->d_h[hb->cur], hb->d_f[hb->cur],
                                                                                   hb->tiled);
            e = cudaGetLastError();
        }
    } else {
        hybrid_f32_to_f64_kernel<<<elem_blocks(hb->tiled), 256, 0, hb->stream>>>(hb->d_f[hb->cur], hb->d_h[hb->cur],
                                                                               hb->tiled);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (e != cudaSuccess) return hfail(LBM_ECUDA, std::string("changing the hybrid's precision: ") + cudaGetErrorString(e));
    hb->prec = prec;
    hb->have_resid = false;
    return LBM_OK;
}

// FP64 defect of the FP32 state: D = M64(H) - H into d_f[2]; *dsum = ||D||^2, *nsum = ||M64(H)||^2
static lbm_status hybrid_defect(lbm_hybrid *hb, double *dsum, double *nsum)
{
    const float *H = hb->d_f[hb->cur];
    hybrid_f32_to_f64_kernel<<<elem_blocks(hb->tiled), 256, 0, hb->stream>>>(H, hb->d_h[0], hb->tiled);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = hybrid_launch<double>(hb, hargs(hb, hb->d_h[0], hb->d_h[1]), 0);
    if (e == cudaSuccess) {
        hybrid_defect_kernel<<<HDEF, 256, 0, hb->stream>>>(hb->d_h[1], H, hb->d_f[2], hb->d_poff, hb->d_toff,
                                                          hb->nx * hb->ny, hb->d_sums);
        e = cudaGetLastError();
    }
    std::vector<double> sums(2 * HDEF);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums.data(), hb->d_sums, sizeof(double) * 2 * HDEF, cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (e != cudaSuccess) return hfail(LBM_ECUDA, std::string("hybrid defect pass: ") + cudaGetErrorString(e));
    double d = 0.0, n = 0.0;
    for (int b = 0; b < HDEF; ++b) {
        d += sums[2 * b];
        n += sums[2 * b + 1];
    }
    if (!std::isfinite(d) || !std::isfinite(n)) return hfail(LBM_ENONFINITE, "non-finite hybrid defect");
    *dsum = d;
    *nsum = n;
    return LBM_OK;
}

lbm_status lbm_hybrid_refine(lbm_hybrid *hb, double tol, int max_sweeps, double refine_tol, long max_steps, int every,
                             long *correction_steps, double *defect)
{
    if (!hb) return hfail(LBM_EINVAL, "hybrid is NULL");
    if (hb->prec != LBM_FP32_PERTURB) return hfail(LBM_EINVAL, "refinement applies to the FP32 march");
    if (!(tol > 0) || max_sweeps < 0 || refine_tol < 0 || max_steps < 1 || every < 1)
        return hfail(LBM_EINVAL, "invalid refinement arguments");
    double dsum, nsum;
    lbm_status st = hybrid_defect(hb, &dsum, &nsum);
    if (st != LBM_OK) return st;
    double r64 = nsum > 0 ? std::sqrt(dsum / nsum) : 0.0;
    const double hnorm = std::sqrt(nsum), ctol = refine_tol > 0 ? refine_tol : 0.1 * tol;
    long ksum = 0;
    for (int sw = 0; sw < max_sweeps && r64 >= tol && hnorm > 0; ++sw) {
        // correction march delta <- L(delta) + D from delta = 0 (walls without driving)
        float *C[2] = {hb->d_f[3], hb->d_f[4]};
        int cc = 0;
        cudaError_t e = cudaMemsetAsync(C[0], 0, sizeof(float) * hb->tiled, hb->stream);
        long k = 0;
        double cbest = INFINITY;
        int cflat = 0;
        while (e == cudaSuccess && k < max_steps) {
            for (int j = 1; j <= every && e == cudaSuccess; ++j) {
                e = hybrid_launch<float>(hb, hargs(hb, C[cc], C[cc ^ 1], hb->d_f[2], 1), j == every ? 1 : 0);
                cc ^= 1;
            }
            if (e == cudaSuccess) e = hybrid_finalize(hb);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hb->h_res, hb->d_res, sizeof(double) * 2, cudaMemcpyDeviceToHost, hb->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
            if (e != cudaSuccess) break;
            k += every;
            // change per step relative to ||M64(H)||, below ctol: the correction's own error is
            // its per-step change times the conditioning of the slow modes
            const double change = std::sqrt(hb->h_res[0]) / hnorm;
            if (!std::isfinite(change)) return hfail(LBM_ENONFINITE, "non-finite hybrid correction");
            if (change < ctol) break;
            if (change < 0.99 * cbest) {
                cbest = change;
                cflat = 0;
            } else if (++cflat >= 20) {
                break;
            }
        }
        if (e == cudaSuccess) {
            hybrid_add_f32_kernel<<<elem_blocks(hb->tiled), 256, 0, hb->stream>>>(hb->d_f[hb->cur], C[cc], hb->tiled);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return hfail(LBM_ECUDA, std::string("hybrid correction march: ") + cudaGetErrorString(e));
        ksum += k;
        const double prev = r64;
        st = hybrid_defect(hb, &dsum, &nsum);
        if (st != LBM_OK) return st;
        r64 = nsum > 0 ? std::sqrt(dsum / nsum) : 0.0;
        if (r64 > 0.5 * prev) break;          // at the FP32 rounding floor
    }
    hb->have_resid = false;
    if (correction_steps) *correction_steps = ksum;
    if (defect) *defect = r64;
    return LBM_OK;
}

lbm_status lbm_hybrid_velocity(lbm_hybrid *hb, double *ux, double *uy)
{
    if (!hb || !ux || !uy) return hfail(LBM_EINVAL, "NULL argument");
    const int nc = hb->nx * hb->ny;
    double *d = nullptr;
    const double *h64 = nullptr;
    cudaError_t e = hybrid_state_f64(hb, &h64);
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(double) * 2 * nc);
    if (e == cudaSuccess) {
        hybrid_velocity_kernel<<<(nc + HWARPS - 1) / HWARPS, 32 * HWARPS, 0, hb->stream>>>(hargs(hb, h64), hb->u_ref, d,
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
    const double *h64 = nullptr;
    cudaError_t e = hybrid_state_f64(hb, &h64);
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(double) * (hb->ny + 1));
    if (e == cudaSuccess) {
        hybrid_face_flux_kernel<<<(hb->ny + 1 + HWARPS - 1) / HWARPS, 32 * HWARPS, 0, hb->stream>>>(hargs(hb, h64),
                                                                                                    hb->u_ref, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(pxy, d, sizeof(double) * (hb->ny + 1), cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (d) cudaFree(d);
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("hybrid face flux: ") + cudaGetErrorString(e));
}

}  // extern "C"
