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
    double d_y;                // sum over xi_y > 0 of xi_y w (wall-flux normaliser, Eq. 9)
};

struct HybTables {
    HybSet set[2];             // 0: half-range, 1: full-range
    double inv_fact[HMAXQ + 1];
};

struct HybArgs {
    const HybTables *tab;
    const int *off;            // [ny + 1] first value of each cell in the packed state
    const unsigned char *half; // [ny] 1: half-range cell
    const double *h;
    double *hn;
    double *part;              // [2 ny] residual sums per cell (||h^{n+1} - h^n||^2, ||h^{n+1}||^2)
    int ny, order;
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

// Ghost of Eq. 8 (perturbation form) for the velocities leaving a plate, into buf.
__device__ void wall_ghost(const HybArgs &a, const HybSet &S, const double *hc, bool bottom, double *buf)
{
    const int lane = threadIdx.x & 31;
    double part = 0.0;
    for (int b = lane; b < S.n; b += 32) {
        const double xn = bottom ? S.xi_y[b] : -S.xi_y[b];   // normal into the gas
        if (xn < 0) part += -xn * hc[b];
    }
    const double rho_w = warp_sum(part) / S.d_y;                // Eq. 9, discrete flux balance
    const double u = bottom ? a.u_bottom : a.u_top;
    for (int b = lane; b < S.n; b += 32)
        buf[b] = S.w[b] * (rho_w * (1.0 + S.xi_x[b] * u) + S.xi_x[b] * u / a.u_ref);
    __syncwarp();
}

// (mass, x-momentum) half-space flux sum |xi_y| (1, xi_x) v over the velocities of S moving up
// (up = true) or down.
__device__ void half_flux(const HybSet &S, const double *v, bool up, double &m, double &p)
{
    double pm = 0.0, pp = 0.0;
    for (int b = threadIdx.x & 31; b < S.n; b += 32) {
        const double y = S.xi_y[b];
        if (up ? y > 0 : y < 0) {
            const double t = fabs(y) * v[b];
            pm += t;
            pp += t * S.xi_x[b];
        }
    }
    m = warp_sum(pm);
    p = warp_sum(pp);
}

struct HybShared {
    double coef[HWARPS][(HMAXQ + 1) * (HMAXQ + 1)];
    double lo[HWARPS][HMAXV], hi[HWARPS][HMAXV], ph[HWARPS][HMAXV], nb[HWARPS][HMAXV];
};

__global__ void __launch_bounds__(32 * HWARPS) hybrid_step_kernel(const HybArgs a, double dt, double dy, int resid)
{
    __shared__ HybShared sh;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int j = blockIdx.x * HWARPS + wi;
    if (j >= a.ny) return;                       // whole warps; only warp-level sync below
    const HybTables &tb = *a.tab;
    const int sj = a.half[j] ? 0 : 1;
    const HybSet &S = tb.set[sj];
    const HybSet &H = tb.set[0];
    const double *hc = a.h + a.off[j];
    double *lo = sh.lo[wi], *hi = sh.hi[wi], *coef = sh.coef[wi];
    // upwind values: from below for xi_y > 0, from above for xi_y < 0 (or the plates' ghosts)
    if (j > 0) neighbour_values(a, j - 1, sj, coef, lo);
    else wall_ghost(a, S, hc, true, lo);
    if (j < a.ny - 1) neighbour_values(a, j + 1, sj, coef, hi);
    else wall_ghost(a, S, hc, false, hi);
    // interface faces of a full-range cell: (mass, x-momentum) exchange made equal to the
    // half-range evaluation of the face
    double cm = 0.0, cp = 0.0;
    const bool lo_if = j > 0 && sj == 1 && a.half[j - 1];
    const bool hi_if = j < a.ny - 1 && sj == 1 && a.half[j + 1];
    if (lo_if || hi_if) {
        double *ph = sh.ph[wi], *nb = sh.nb[wi];
        project_warp(tb, S, hc, H, a.order, coef, ph);          // this cell seen in H
        if (lo_if) {
            neighbour_values(a, j - 1, 0, coef, nb);            // the half-range cell below, own values
            double um, up, dm, dp, gm, gp, sm, sp;
            half_flux(H, nb, true, um, up);
            half_flux(H, ph, false, dm, dp);
            half_flux(S, lo, true, gm, gp);
            half_flux(S, hc, false, sm, sp);
            cm += (um - dm) - (gm - sm);
            cp += (up - dp) - (gp - sp);
        }
        if (hi_if) {
            neighbour_values(a, j + 1, 0, coef, nb);            // the half-range cell above
            double um, up, dm, dp, gm, gp, sm, sp;
            half_flux(H, ph, true, um, up);
            half_flux(H, nb, false, dm, dp);
            half_flux(S, hi, false, gm, gp);
            half_flux(S, hc, true, sm, sp);
            cm += (dm - um) - (gm - sm);
            cp += (dp - up) - (gp - sp);
        }
    }
    const double fac = dt / dy;
    // transport, moments, relaxation
    double hs[(HMAXV + 31) / 32];
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < (HMAXV + 31) / 32; ++i) {
        const int b = lane + 32 * i;
        double v = 0.0;
        if (b < S.n) {
            const double y = S.xi_y[b];
            const double hy = y > 0 ? lo[b] : hi[b];
            const double nuy = fabs(y) * dt / dy;
            v = hc[b] - nuy * (hc[b] - hy);
            if (lo_if || hi_if) v += fac * (cm + cp * S.xi_x[b]) * S.w[b];
            rho += v;
            jx += S.xi_x[b] * v;
            jy += y * v;
        }
        hs[i] = v;
    }
    rho = warp_sum(rho);
    jx = warp_sum(jx);
    jy = warp_sum(jy);
    double *out = a.hn + a.off[j];
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
            a.part[2 * j] = pd;
            a.part[2 * j + 1] = pn;
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

// u_x per cell and the x-momentum flux through the ny + 1 faces (interface faces evaluated in
// the half-range set); one warp per face k (cell k as well when k < ny)
__global__ void __launch_bounds__(32 * HWARPS) hybrid_profile_kernel(const HybArgs a, double u_ref, double *ux,
                                                                      double *pxy)
{
    __shared__ HybShared sh;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int k = blockIdx.x * HWARPS + wi;
    if (k > a.ny) return;
    const HybTables &tb = *a.tab;
    const HybSet &H = tb.set[0];
    double *coef = sh.coef[wi], *lo = sh.lo[wi], *hi = sh.hi[wi];
    if (k < a.ny) {
        const HybSet &S = tb.set[a.half[k] ? 0 : 1];
        const double *hc = a.h + a.off[k];
        double s0 = 0.0, s1 = 0.0;
        for (int b = lane; b < S.n; b += 32) {
            s0 += hc[b];
            s1 += S.xi_x[b] * hc[b];
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (lane == 0) ux[k] = u_ref * s1 / (1.0 + u_ref * s0);
    }
    double up = 0.0, dn = 0.0;
    if (k > 0 && k < a.ny && a.half[k - 1] != a.half[k]) {
        neighbour_values(a, k - 1, 0, coef, lo);
        neighbour_values(a, k, 0, coef, hi);
        double um, dm;
        half_flux(H, lo, true, um, up);
        half_flux(H, hi, false, dm, dn);
        dn = -dn;                                               // sum over xi_y < 0 of xi_y xi_x h
    } else {
        const int cb = k == 0 ? 0 : k - 1, ca = k == a.ny ? a.ny - 1 : k;
        const HybSet &Sb = tb.set[a.half[cb] ? 0 : 1], &Sa = tb.set[a.half[ca] ? 0 : 1];
        const double *vb = a.h + a.off[cb], *va = a.h + a.off[ca];
        if (k == 0) {
            wall_ghost(a, Sb, vb, true, lo);
            vb = lo;
        }
        if (k == a.ny) {
            wall_ghost(a, Sa, va, false, hi);
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

}  // namespace

struct lbm_hybrid {
    int n_half, ny, layer, order;
    double kn, u_bottom, u_top, cfl, dt, dy, omega, u_ref;
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
    S.d_y = 0.0;
    max_y = 0.0;
    for (int iy = 0; iy < m; ++iy)
        for (int ix = 0; ix < m; ++ix) {
            const int a = iy * m + ix;
            S.xi_x[a] = x[ix];
            S.xi_y[a] = x[iy];
            S.w[a] = w[ix] * w[iy];
            if (x[iy] > 0) S.d_y += x[iy] * S.w[a];
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
    a.ny = hb->ny;
    a.order = hb->order;
    a.omega = hb->omega;
    a.u_bottom = hb->u_bottom;
    a.u_top = hb->u_top;
    a.u_ref = hb->u_ref;
    return a;
}

}  // namespace

extern "C" {

lbm_status lbm_hybrid_init(int n_half, int ny, double kn, double u_bottom, double u_top, int layer, double cfl,
                           void *stream, lbm_hybrid **out)
{
    if (!out) return hfail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_half < 2 || n_half > 6) return hfail(LBM_EINVAL, "the hybrid needs 2 <= N <= 6 nodes per half-axis");
    if (ny < 2 || layer < 0 || !(kn > 0) || !(cfl > 0) || !std::isfinite(u_bottom) || !std::isfinite(u_top))
        return hfail(LBM_EINVAL, "invalid hybrid problem (ny >= 2, layer >= 0, Kn > 0, cfl > 0)");
    lbm_hybrid *hb = new (std::nothrow) lbm_hybrid;
    if (!hb) return hfail(LBM_ENOMEM, "host allocation failed");
    hb->n_half = n_half;
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
    hb->half.resize(ny);
    hb->off.resize(ny + 1);
    bool any_h = false, any_f = false;
    long o = 0;
    for (int j = 0; j < ny; ++j) {
        hb->half[j] = (j < layer || j >= ny - layer) ? 1 : 0;
        (hb->half[j] ? any_h : any_f) = true;
        hb->off[j] = (int)o;
        o += hb->half[j] ? tab.set[0].n : tab.set[1].n;
    }
    hb->off[ny] = (int)o;
    hb->unknowns = o;
    // dt from the largest |xi_y| of the sets present (Couette column: y only), dt <= Kn
    hb->dy = 1.0 / ny;
    const double my = std::max(any_h ? my_h : 0.0, any_f ? my_f : 0.0);
    hb->dt = cfl / (my / hb->dy);
    if (std::isfinite(kn) && hb->dt > kn) hb->dt = kn;
    hb->omega = std::isfinite(kn) ? hb->dt / kn : 0.0;
    const double ur = std::max(std::fabs(u_bottom), std::fabs(u_top));
    hb->u_ref = ur > 0 ? ur : 1.0;
    cudaError_t e = cudaMalloc(&hb->d_tab, sizeof(HybTables));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_off, sizeof(int) * (ny + 1));
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_half, ny);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_h[0], sizeof(double) * o);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_h[1], sizeof(double) * o);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_part, sizeof(double) * 2 * ny);
    if (e == cudaSuccess) e = cudaMalloc(&hb->d_res, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMallocHost(&hb->h_res, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb->d_tab, &tab, sizeof tab, cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb->d_off, hb->off.data(), sizeof(int) * (ny + 1), cudaMemcpyHostToDevice, hb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb->d_half, hb->half.data(), ny, cudaMemcpyHostToDevice, hb->stream);
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
    const int grid = (hb->ny + HWARPS - 1) / HWARPS;
    for (long s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        hybrid_step_kernel<<<grid, 32 * HWARPS, 0, hb->stream>>>(hargs(hb), hb->dt, hb->dy, last ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && last) {
            hybrid_finalize_kernel<<<1, 32, 0, hb->stream>>>(hb->d_part, hb->ny, hb->d_res);
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

lbm_status lbm_hybrid_profile(lbm_hybrid *hb, double *ux, double *pxy)
{
    if (!hb || !ux || !pxy) return hfail(LBM_EINVAL, "NULL argument");
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * (2 * hb->ny + 1));
    if (e == cudaSuccess) {
        const int grid = (hb->ny + 1 + HWARPS - 1) / HWARPS;
        hybrid_profile_kernel<<<grid, 32 * HWARPS, 0, hb->stream>>>(hargs(hb), hb->u_ref, d, d + hb->ny);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ux, d, sizeof(double) * hb->ny, cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pxy, d + hb->ny, sizeof(double) * (hb->ny + 1), cudaMemcpyDeviceToHost, hb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
    if (d) cudaFree(d);
    return e == cudaSuccess ? LBM_OK : hfail(LBM_ECUDA, std::string("hybrid profile: ") + cudaGetErrorString(e));
}

}  // extern "C"
