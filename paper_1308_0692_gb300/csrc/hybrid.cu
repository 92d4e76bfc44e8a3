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
// One warp per cell; the state is packed cell after cell, each cell's values in its own
// set's velocity order (a = iy * M + ix).  dt = cfl dy / max |xi_y| over the sets present,
// dt <= Kn.
#include <algorithm>
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
    double xi_x[HMAXV], xi_y[HMAXV], w[HMAXV];
    double he_x[HMAXQ + 1][HMAXV], he_y[HMAXQ + 1][HMAXV];
    double d_x, d_y;           // sums over xi > 0 of xi w per axis (wall-flux normalisers, Eq. 9)
};

struct HybTables {
    HybSet set[2];             // 0: half-range, 1: full-range
    double inv_fact[HMAXQ + 1];
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

// Hermite coefficients of distribution h (set T) into coef[(order+1)^2] (lane-parallel: one
// coefficient per lane, summed over the velocities in order), then the projection onto the
// velocities of S into out[]: out_b = w_b sum c_mn He_m(xi_x,b) He_n(xi_y,b).
__device__ void project_warp(const HybTables &tb, const HybSet &T, const double *h, const HybSet &S, int order,
                             double *coef, double *out)
{
    const int lane = threadIdx.x & 31, nq = order + 1;
    for (int l = lane; l < nq * nq; l += 32) {
        const int m = l / nq, n = l - m * nq;
        double c = 0.0;
        for (int a = 0; a < T.n; ++a) c += h[a] * T.he_x[m][a] * T.he_y[n][a];
        coef[l] = c * tb.inv_fact[m] * tb.inv_fact[n];
    }
    __syncwarp();
    for (int b = lane; b < S.n; b += 32) {
        double v = 0.0;
        for (int m = 0; m < nq; ++m)
            for (int n = 0; n < nq; ++n) v += coef[m * nq + n] * S.he_x[m][b] * S.he_y[n][b];
        out[b] = S.w[b] * v;
    }
    __syncwarp();
}

// Values of neighbour cell k as seen by a cell of set sj, into buf[0..S.n): its own values
// for the same set, else their projection.
__device__ void neighbour_values(const HybArgs &a, int k, int sj, double *coef, double *buf)
{
    const HybTables &tb = *a.tab;
    const HybSet &S = tb.set[sj];
    const int sk = a.half[k] ? 0 : 1;
    const double *hk = a.h + a.off[k];
    if (sk == sj) {
        for (int b = threadIdx.x & 31; b < S.n; b += 32) buf[b] = hk[b];
        __syncwarp();
    } else {
        project_warp(tb, tb.set[sk], hk, S, a.order, coef, buf);
    }
}

// Ghost of Eq. 8 (perturbation form) for the velocities leaving wall `face` (0 bottom, 1 top,
// 2 left, 3 right; the side walls at rest), into buf; rho_w by Eq. 9 over the cell's own set.
__device__ void wall_ghost(const HybArgs &a, const HybSet &S, const double *hc, int face, double *buf)
{
    const int lane = threadIdx.x & 31;
    double part = 0.0;
    for (int b = lane; b < S.n; b += 32) {
        const double xn = face == 0 ? S.xi_y[b] : face == 1 ? -S.xi_y[b] : face == 2 ? S.xi_x[b] : -S.xi_x[b];
        if (xn < 0) part += -xn * hc[b];
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
        const double xd = axis == 0 ? S.xi_x[b] : S.xi_y[b];
        if (positive ? xd > 0 : xd < 0) {
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
    double coef[HWARPS][(HMAXQ + 1) * (HMAXQ + 1)];
    double nbv[HWARPS][4][HMAXV];   // left, right, below, above: upwind values in the cell's set
    double ph[HWARPS][HMAXV], nb[HWARPS][HMAXV];
};

__global__ void __launch_bounds__(32 * HWARPS) hybrid_step_kernel(const HybArgs a, double dt, double dx, double dy,
                                                                   int resid)
{
    __shared__ HybShared sh;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int c = blockIdx.x * HWARPS + wi;
    const int nx = a.nx, ny = a.ny;
    if (c >= nx * ny) return;                    // whole warps; only warp-level sync below
    const HybTables &tb = *a.tab;
    const int sj = a.half[c] ? 0 : 1;
    const HybSet &S = tb.set[sj];
    const HybSet &H = tb.set[0];
    const double *hc = a.h + a.off[c];
    const int x = c % nx, y = c / nx;
    double *coef = sh.coef[wi];
    double(*nbv)[HMAXV] = sh.nbv[wi];
    // upwind values: x (cavity only) and y neighbours in this cell's set, or the walls' ghosts;
    // the four faces as (axis, side, neighbour or -1)
    int nbc[4] = {-1, -1, -1, -1};
    if (a.cavity) {
        if (x > 0) neighbour_values(a, nbc[0] = c - 1, sj, coef, nbv[0]);
        else wall_ghost(a, S, hc, 2, nbv[0]);
        if (x < nx - 1) neighbour_values(a, nbc[1] = c + 1, sj, coef, nbv[1]);
        else wall_ghost(a, S, hc, 3, nbv[1]);
    }
    if (y > 0) neighbour_values(a, nbc[2] = c - nx, sj, coef, nbv[2]);
    else wall_ghost(a, S, hc, 0, nbv[2]);
    if (y < ny - 1) neighbour_values(a, nbc[3] = c + nx, sj, coef, nbv[3]);
    else wall_ghost(a, S, hc, 1, nbv[3]);
    // interface faces of a full-range cell: mass and momentum exchange made equal to the
    // half-range evaluation of the face
    double cr[3] = {0.0, 0.0, 0.0};
    bool any_if = false;
    if (sj == 1)
        for (int f = 0; f < 4; ++f) any_if |= nbc[f] >= 0 && a.half[nbc[f]];
    if (any_if) {
        double *ph = sh.ph[wi], *nb = sh.nb[wi];
        project_warp(tb, S, hc, H, a.order, coef, ph);          // this cell seen in H
        for (int f = 0; f < 4; ++f) {
            if (nbc[f] < 0 || !a.half[nbc[f]]) continue;
            const int axis = f >> 1;
            const bool lower = (f & 1) == 0;                  // the neighbour is on the lower side
            neighbour_values(a, nbc[f], 0, coef, nb);         // its own half-range values
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
            if (a.cavity) {
                hx = ex > 0 ? nbv[0][b] : (ex < 0 ? nbv[1][b] : h0);
                nux = fabs(ex) * dt / dx;
            }
            const double hy = ey > 0 ? nbv[2][b] : (ey < 0 ? nbv[3][b] : h0);
            const double nuy = fabs(ey) * dt / dy;
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
            const double d = o - hc[b];
            pd += d * d;
            pn += o * o;
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

// residual sums in cell order
__global__ void hybrid_finalize_kernel(const double *part, int ny, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double d = 0.0, n = 0.0;
        for (int j = 0; j < ny; ++j) {
            d += part[2 * j];
            n += part[2 * j + 1];
        }
        out[0] = d;
        out[1] = n;
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
    double *coef = sh.coef[wi], *lo = sh.nbv[wi][0], *hi = sh.nbv[wi][1];
    double up = 0.0, dn = 0.0;
    if (k > 0 && k < a.ny && a.half[k - 1] != a.half[k]) {
        const HybSet &H = tb.set[0];
        neighbour_values(a, k - 1, 0, coef, lo);
        neighbour_values(a, k, 0, coef, hi);
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
    S.d_x = S.d_y = 0.0;
    max_y = 0.0;
    for (int iy = 0; iy < m; ++iy)
        for (int ix = 0; ix < m; ++ix) {
            const int a = iy * m + ix;
            S.xi_x[a] = x[ix];
            S.xi_y[a] = x[iy];
            S.w[a] = w[ix] * w[iy];
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
    HybTables tab;
    std::memset(&tab, 0, sizeof tab);
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
        hb->off[c] = (int)o;
        o += hb->half[c] ? tab.set[0].n : tab.set[1].n;
    }
    hb->off[nc] = (int)o;
    hb->unknowns = o;
    // dt = cfl / (max|xi_x|/dx + max|xi_y|/dy) over the sets present (the x term dropped for
    // the Couette column), dt <= Kn; the sets are symmetric, so max |xi_x| = max |xi_y|
    hb->dy = 1.0 / ny;
    hb->dx = geom == LBM_CAVITY ? 1.0 / nx : hb->dy;
    const double my = std::max(any_h ? my_h : 0.0, any_f ? my_f : 0.0);
    hb->dt = cfl / (my / hb->dy + (geom == LBM_CAVITY ? my / hb->dx : 0.0));
    if (std::isfinite(kn) && hb->dt > kn) hb->dt = kn;
    hb->omega = std::isfinite(kn) ? hb->dt / kn : 0.0;
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
    const int grid = (nc + HWARPS - 1) / HWARPS;
    for (long s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        hybrid_step_kernel<<<grid, 32 * HWARPS, 0, hb->stream>>>(hargs(hb), hb->dt, hb->dx, hb->dy, last ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && last) {
            hybrid_finalize_kernel<<<1, 32, 0, hb->stream>>>(hb->d_part, nc, hb->d_res);
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
