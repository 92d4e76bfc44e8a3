// Reductions and diagnostics of the march (sm_103a): residual finalisation, squared
// norms, macroscopic moments (Eqs. 6-7 and the second moments behind p_xy) and the
// momentum flux through cell faces (the shear stress the scheme transmits; on a wall
// face the upwind value is the Maxwell ghost of Eqs. 8-9).  All accumulation in FP64.
#include <cmath>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int RED_BLOCK = 1024;

// Sum per-block partial pairs in a fixed order; result[0..1] = sums, and when
// nres >= 4: result[2] = sqrt(sd/sn) (0 if both are 0), result[3] = 1 if non-finite.
__global__ void __launch_bounds__(RED_BLOCK) finalize_kernel(const double *partials, int nparts,
                                                             double *result, int nres)
{
    __shared__ double s_d[RED_BLOCK / 32], s_n[RED_BLOCK / 32];
    double sd = 0.0, sn = 0.0;
    for (int i = threadIdx.x; i < nparts; i += RED_BLOCK) {
        sd += partials[2 * i];
        sn += partials[2 * i + 1];
    }
    for (int off = 16; off > 0; off >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, off);
        sn += __shfl_xor_sync(0xffffffffu, sn, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_d[warp] = sd;
        s_n[warp] = sn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double td = 0.0, tn = 0.0;
        for (int w = 0; w < RED_BLOCK / 32; ++w) {
            td += s_d[w];
            tn += s_n[w];
        }
        result[0] = td;
        result[1] = tn;
        if (nres >= 4) {
            const bool bad = !isfinite(td) || !isfinite(tn);
            result[2] = (tn > 0.0) ? sqrt(td / tn) : (td == 0.0 ? 0.0 : INFINITY);
            result[3] = bad ? 1.0 : 0.0;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) norms_kernel(const T *a, const T *b, long count,
                                                   double *partials)
{
    __shared__ double s_d[8], s_n[8];
    double sd = 0.0, sn = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const double va = (double)a[i];
        const double d = b ? va - (double)b[i] : va;
        sd += d * d;
        sn += va * va;
    }
    for (int off = 16; off > 0; off >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, off);
        sn += __shfl_xor_sync(0xffffffffu, sn, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_d[warp] = sd;
        s_n[warp] = sn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double td = 0.0, tn = 0.0;
        for (int w = 0; w < 8; ++w) {
            td += s_d[w];
            tn += s_n[w];
        }
        partials[2 * blockIdx.x] = td;
        partials[2 * blockIdx.x + 1] = tn;
    }
}

// Per cell: rho, ux, uy, pxx, pxy, pyy (linearised, Eq. (1) units).
template <typename T>
__global__ void moments_kernel(const T *h, long pa, long py, int nx, const TableHeader *hdr, int m, long ncells,
                               double u_ref, double *out)
{
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const long y = c / nx, co = y * py + (c - y * nx);
    double s0 = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
    for (int iy = 0; iy < m; ++iy) {
        const double ey = hdr->xi1[iy];
        for (int ix = 0; ix < m; ++ix) {
            const double ex = hdr->xi1[ix];
            const double v = (double)h[(long)(iy * m + ix) * pa + co];
            s0 += v;
            sx += ex * v;
            sy += ey * v;
            sxx += ex * ex * v;
            sxy += ex * ey * v;
            syy += ey * ey * v;
        }
    }
    const double rho = 1.0 + u_ref * s0;
    out[c] = rho;
    out[ncells + c] = u_ref * sx / rho;
    out[2 * ncells + c] = u_ref * sy / rho;
    out[3 * ncells + c] = 1.0 + u_ref * sxx;
    out[4 * ncells + c] = u_ref * sxy;
    out[5 * ncells + c] = 1.0 + u_ref * syy;
}

// The same moments of an FP32 state with the inner (x) sums in double-float arithmetic:
// each product xi_x v keeps its FMA rounding residual (xi_x itself carried as hi + lo) and
// each sum its TwoSum error, so the row sums are FP64-accurate; the outer (y) sums are FP64.
// FP64 accumulation of all 6 x M^2 products per cell is bound by this GPU's slow FP64 pipe
// (about 10 ms for 2048^2 x 144); this form does a ninth of the FP64 work.
struct DFAcc {
    float hi, lo;
};

__device__ __forceinline__ void df_add(DFAcc &a, float x)
{
    const float t = a.hi + x;
    const float z = t - a.hi;
    a.lo += (a.hi - (t - z)) + (x - z);
    a.hi = t;
}

// a += (xh + xl) v
__device__ __forceinline__ void df_add_prod(DFAcc &a, float xh, float xl, float v)
{
    const float p = xh * v;
    const float e = fmaf(xh, v, -p) + xl * v;
    df_add(a, p);
    a.lo += e;
}

// The state is planar (tile_pitch 0: velocity planes pa apart) or strip-tiled (velocity
// lines LBM_TILE_W apart from the cell's tile row).  P: also the P_ij sums (outputs 3-5).
template <bool P>
__global__ void moments_f32_kernel(const float *h, long pa, long py, int nx, const TableHeader *hdr, int m, long ncells,
                                   double u_ref, double *out, long tile_pitch)
{
    __shared__ float s_x[LBM_MAX_M][4];   // xi hi, lo; xi^2 hi, lo
    if (threadIdx.x < m) {
        const double x = hdr->xi1[threadIdx.x], x2 = x * x;
        const float xh = (float)x, x2h = (float)x2;
        s_x[threadIdx.x][0] = xh;
        s_x[threadIdx.x][1] = (float)(x - (double)xh);
        s_x[threadIdx.x][2] = x2h;
        s_x[threadIdx.x][3] = (float)(x2 - (double)x2h);
    }
    __syncthreads();
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const long y = c / nx, x = c - y * nx;
    const long base = tile_pitch > 0 ? tile_off(x, y, m * m, tile_pitch) : y * py + x;
    const long vstride = tile_pitch > 0 ? (long)LBM_TILE_W : pa;
    double s0 = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
    for (int iy = 0; iy < m; ++iy) {
        DFAcc r0 = {0.f, 0.f}, r1 = {0.f, 0.f}, r2 = {0.f, 0.f};
        for (int ix = 0; ix < m; ++ix) {
            const float v = h[base + (long)(iy * m + ix) * vstride];
            df_add(r0, v);
            df_add_prod(r1, s_x[ix][0], s_x[ix][1], v);
            if (P) df_add_prod(r2, s_x[ix][2], s_x[ix][3], v);
        }
        const double ey = hdr->xi1[iy];
        const double a0 = (double)r0.hi + (double)r0.lo, a1 = (double)r1.hi + (double)r1.lo;
        s0 += a0;
        sx += a1;
        sy += ey * a0;
        if (P) {
            sxx += (double)r2.hi + (double)r2.lo;
            sxy += ey * a1;
            syy += ey * ey * a0;
        }
    }
    const double rho = 1.0 + u_ref * s0;
    out[c] = rho;
    out[ncells + c] = u_ref * sx / rho;
    out[2 * ncells + c] = u_ref * sy / rho;
    if (P) {
        out[3 * ncells + c] = 1.0 + u_ref * sxx;
        out[4 * ncells + c] = u_ref * sxy;
        out[5 * ncells + c] = 1.0 + u_ref * syy;
    }
}

// rho'_w of a wall face of the cell at plane offset co; dir: 0 bottom, 1 top, 2 left, 3 right
template <typename T>
__device__ double wall_rho(const T *h, const TableHeader *hdr, int m, long pa, long co, int dir)
{
    double s = 0.0;
    for (int iy = 0; iy < m; ++iy) {
        for (int ix = 0; ix < m; ++ix) {
            const double xn = (dir == 0) ? hdr->xi1[iy] : (dir == 1) ? -hdr->xi1[iy]
                            : (dir == 2) ? hdr->xi1[ix] : -hdr->xi1[ix];
            if (xn < 0.0) s -= xn * (double)h[(long)(iy * m + ix) * pa + co];
        }
    }
    return s * ((dir < 2) ? hdr->inv_dy_wall : hdr->inv_dx_wall);
}

template <typename T>
__global__ void face_flux_y_kernel(const T *h, long pa, long py, const double *tab, const TableHeader *hdr, int m,
                                   int nx, int ny, double u_ref, double *out)
{
    const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nfaces = (long)(ny + 1) * nx;
    if (f >= nfaces) return;
    const int j = (int)(f / nx), x = (int)(f - (long)j * nx);
    const long below = (long)(j - 1) * py + x, above = (long)j * py + x;
    const double rb = (j == 0) ? wall_rho(h, hdr, m, pa, above, 0) : 0.0;
    const double rt = (j == ny) ? wall_rho(h, hdr, m, pa, below, 1) : 0.0;
    double s = 0.0;
    for (int iy = 0; iy < m; ++iy) {
        const double ey = hdr->xi1[iy];
        if (ey == 0.0) continue;
        for (int ix = 0; ix < m; ++ix) {
            const int al = iy * m + ix;
            double v;
            if (ey > 0.0)
                v = (j == 0) ? rb * tab[TAB_GB_LIN * LBM_MAX_V + al] + tab[TAB_GB_C * LBM_MAX_V + al]
                             : (double)h[(long)al * pa + below];
            else
                v = (j == ny) ? rt * tab[TAB_GT_LIN * LBM_MAX_V + al] + tab[TAB_GT_C * LBM_MAX_V + al]
                              : (double)h[(long)al * pa + above];
            s += hdr->xi1[ix] * ey * v;
        }
    }
    out[f] = u_ref * s;
}

template <typename T>
__global__ void face_flux_x_kernel(const T *h, long pa, long py, const double *tab, const TableHeader *hdr, int m,
                                   int nx, int ny, double u_ref, double *out)
{
    const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nfaces = (long)ny * (nx + 1);
    if (f >= nfaces) return;
    const int y = (int)(f / (nx + 1)), i = (int)(f - (long)y * (nx + 1));
    const long left = (long)y * py + i - 1, right = (long)y * py + i;
    const double rl = (i == 0) ? wall_rho(h, hdr, m, pa, right, 2) : 0.0;
    const double rr = (i == nx) ? wall_rho(h, hdr, m, pa, left, 3) : 0.0;
    double s = 0.0;
    for (int iy = 0; iy < m; ++iy) {
        const double ey = hdr->xi1[iy];
        for (int ix = 0; ix < m; ++ix) {
            const double ex = hdr->xi1[ix];
            if (ex == 0.0) continue;
            const int al = iy * m + ix;
            double v;
            if (ex > 0.0)
                v = (i == 0) ? rl * tab[TAB_W * LBM_MAX_V + al] : (double)h[(long)al * pa + left];
            else
                v = (i == nx) ? rr * tab[TAB_W * LBM_MAX_V + al] : (double)h[(long)al * pa + right];
            s += ex * ey * v;
        }
    }
    out[f] = u_ref * s;
}

// Face values of the second-order transport (step_so.cuh): the upwind reconstruction
// h_u + (1 - nu)/2 (h_u - h_uu), first order where h_uu lies beyond a wall, the wall ghost
// on a wall face with the wall density balancing the second-order outflow.
template <typename T>
__device__ double wall_rho2(const T *h, long pa, long py, const double *tab, const TableHeader *hdr, int m, int nx,
                            int ny, int x, int y, int dir)
{
    // dir: 0 bottom (inner y + 1), 1 top (y - 1), 2 left (x + 1), 3 right (x - 1)
    double s = 0.0;
    const long co = (long)y * py + x;
    const long ci = dir == 0 ? co + (ny > 1 ? py : 0) : dir == 1 ? co - (ny > 1 ? py : 0)
                  : dir == 2 ? co + (nx > 1 ? 1 : 0) : co - (nx > 1 ? 1 : 0);
    for (int iy = 0; iy < m; ++iy) {
        for (int ix = 0; ix < m; ++ix) {
            const int al = iy * m + ix;
            const double xn = (dir == 0) ? hdr->xi1[iy] : (dir == 1) ? -hdr->xi1[iy]
                            : (dir == 2) ? hdr->xi1[ix] : -hdr->xi1[ix];
            if (xn < 0.0) {
                const double nu = tab[(dir < 2 ? TAB_NUY : TAB_NUX) * LBM_MAX_V + al];
                const double hu = (double)h[(long)al * pa + co], huu = (double)h[(long)al * pa + ci];
                s -= xn * (hu + 0.5 * (1.0 - nu) * (hu - huu));
            }
        }
    }
    return s * ((dir < 2) ? hdr->inv_dy_wall : hdr->inv_dx_wall);
}

template <typename T>
__global__ void face_flux2_y_kernel(const T *h, long pa, long py, const double *tab, const TableHeader *hdr, int m,
                                    int nx, int ny, double u_ref, double *out)
{
    const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nfaces = (long)(ny + 1) * nx;
    if (f >= nfaces) return;
    const int j = (int)(f / nx), x = (int)(f - (long)j * nx);
    const double rb = (j == 0) ? wall_rho2(h, pa, py, tab, hdr, m, nx, ny, x, 0, 0) : 0.0;
    const double rt = (j == ny) ? wall_rho2(h, pa, py, tab, hdr, m, nx, ny, x, ny - 1, 1) : 0.0;
    double s = 0.0;
    for (int iy = 0; iy < m; ++iy) {
        const double ey = hdr->xi1[iy];
        if (ey == 0.0) continue;
        for (int ix = 0; ix < m; ++ix) {
            const int al = iy * m + ix;
            const double nu = tab[TAB_NUY * LBM_MAX_V + al];
            const T *ha = h + (long)al * pa;
            double v;
            if (ey > 0.0) {
                if (j == 0) v = rb * tab[TAB_GB_LIN * LBM_MAX_V + al] + tab[TAB_GB_C * LBM_MAX_V + al];
                else {
                    const double hu = (double)ha[(long)(j - 1) * py + x];
                    v = (j == 1) ? hu : hu + 0.5 * (1.0 - nu) * (hu - (double)ha[(long)(j - 2) * py + x]);
                }
            } else {
                if (j == ny) v = rt * tab[TAB_GT_LIN * LBM_MAX_V + al] + tab[TAB_GT_C * LBM_MAX_V + al];
                else {
                    const double hu = (double)ha[(long)j * py + x];
                    v = (j == ny - 1) ? hu : hu + 0.5 * (1.0 - nu) * (hu - (double)ha[(long)(j + 1) * py + x]);
                }
            }
            s += hdr->xi1[ix] * ey * v;
        }
    }
    out[f] = u_ref * s;
}

template <typename T>
__global__ void face_flux2_x_kernel(const T *h, long pa, long py, const double *tab, const TableHeader *hdr, int m,
                                    int nx, int ny, double u_ref, double *out)
{
    const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nfaces = (long)ny * (nx + 1);
    if (f >= nfaces) return;
    const int y = (int)(f / (nx + 1)), i = (int)(f - (long)y * (nx + 1));
    const double rl = (i == 0) ? wall_rho2(h, pa, py, tab, hdr, m, nx, ny, 0, y, 2) : 0.0;
    const double rr = (i == nx) ? wall_rho2(h, pa, py, tab, hdr, m, nx, ny, nx - 1, y, 3) : 0.0;
    double s = 0.0;
    for (int iy = 0; iy < m; ++iy) {
        const double ey = hdr->xi1[iy];
        for (int ix = 0; ix < m; ++ix) {
            const double ex = hdr->xi1[ix];
            if (ex == 0.0) continue;
            const int al = iy * m + ix;
            const double nu = tab[TAB_NUX * LBM_MAX_V + al];
            const T *ha = h + (long)al * pa + (long)y * py;
            double v;
            if (ex > 0.0) {
                if (i == 0) v = rl * tab[TAB_W * LBM_MAX_V + al];
                else {
                    const double hu = (double)ha[i - 1];
                    v = (i == 1) ? hu : hu + 0.5 * (1.0 - nu) * (hu - (double)ha[i - 2]);
                }
            } else {
                if (i == nx) v = rr * tab[TAB_W * LBM_MAX_V + al];
                else {
                    const double hu = (double)ha[i];
                    v = (i == nx - 1) ? hu : hu + 0.5 * (1.0 - nu) * (hu - (double)ha[i + 1]);
                }
            }
            s += ex * ey * v;
        }
    }
    out[f] = u_ref * s;
}

__global__ void convert_kernel(const double *src, float *dst, long count)
{
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        dst[i] = (float)src[i];
}

__global__ void widen_kernel(const float *src, double *dst, long count)
{
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        dst[i] = (double)src[i];
}

// h from the six moments of each cell, mom [6][ncells] = rho, u_x, u_y, P_xx, P_xy, P_yy:
// the second-order Hermite expansion h_a = w_a [rho' + xi_a . j' + 1/2 sum_ij (P'_ij -
// rho' delta_ij)(xi_i xi_j - delta_ij)] with rho' = (rho - 1)/u_ref, j' = rho u / u_ref,
// P' = (P - I)/u_ref (the inverse of the moment map of lbm_moments on sets exact to degree 4).
template <typename T>
__global__ void moments_state_kernel(const double *mom, int nx, long ncells, long pa, long py, int m,
                                     const TableHeader *hdr, double inv_u_ref, T *h)
{
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += stride) {
        const long y = c / nx, co = y * py + (c - y * nx);
        const double rho = mom[c];
        const double rp = (rho - 1.0) * inv_u_ref;
        const double jx = rho * mom[ncells + c] * inv_u_ref, jy = rho * mom[2 * ncells + c] * inv_u_ref;
        const double pxx = (mom[3 * ncells + c] - 1.0) * inv_u_ref, pxy = mom[4 * ncells + c] * inv_u_ref;
        const double pyy = (mom[5 * ncells + c] - 1.0) * inv_u_ref;
        for (int iy = 0; iy < m; ++iy) {
            const double ey = hdr->xi1[iy];
            for (int ix = 0; ix < m; ++ix) {
                const double ex = hdr->xi1[ix];
                const double v = hdr->w1[ix] * hdr->w1[iy] *
                                 (rp + ex * jx + ey * jy +
                                  0.5 * ((pxx - rp) * (ex * ex - 1.0) + 2.0 * pxy * ex * ey + (pyy - rp) * (ey * ey - 1.0)));
                h[(long)(iy * m + ix) * pa + co] = (T)v;
            }
        }
    }
}

// planar FP64 [a][c] <-> state of layout (pa, py) and type T
template <typename T>
__global__ void relayout_kernel(bool to_layout, double *planar, T *state, int n, int nx, long ncells, long pa,
                                long py)
{
    const long total = (long)n * ncells, stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const long al = i / ncells, c = i - al * ncells;
        const long y = c / nx;
        const long o = al * pa + y * py + (c - y * nx);
        if (to_layout)
            state[o] = (T)planar[i];
        else
            planar[i] = (double)state[o];
    }
}

__global__ void axpy_kernel(float *y, const float *x, long count)
{
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) y[i] += x[i];
}

}  // namespace

cudaError_t launch_moments_state(int prec, const double *mom, int nx, int ny, long pa, long py, int m,
                                 const TableHeader *hdr, double u_ref, void *h, cudaStream_t s)
{
    const long ncells = (long)nx * ny;
    if (prec == LBM_FP64)
        moments_state_kernel<double><<<152 * 8, 256, 0, s>>>(mom, nx, ncells, pa, py, m, hdr, 1.0 / u_ref, (double *)h);
    else
        moments_state_kernel<float><<<152 * 8, 256, 0, s>>>(mom, nx, ncells, pa, py, m, hdr, 1.0 / u_ref, (float *)h);
    return cudaGetLastError();
}

cudaError_t launch_relayout(int prec, bool to_layout, double *planar, void *state, int n, int nx, int ny,
                            long pa, long py, cudaStream_t s)
{
    const long ncells = (long)nx * ny;
    if (prec == LBM_FP64)
        relayout_kernel<double><<<152 * 8, 256, 0, s>>>(to_layout, planar, (double *)state, n, nx, ncells, pa, py);
    else
        relayout_kernel<float><<<152 * 8, 256, 0, s>>>(to_layout, planar, (float *)state, n, nx, ncells, pa, py);
    return cudaGetLastError();
}

cudaError_t launch_add_f32(float *y, const float *x, long count, cudaStream_t s)
{
    axpy_kernel<<<152 * 8, 256, 0, s>>>(y, x, count);
    return cudaGetLastError();
}

cudaError_t launch_convert(const double *src, float *dst, long count, cudaStream_t s)
{
    convert_kernel<<<152 * 8, 256, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

cudaError_t launch_widen(const float *src, double *dst, long count, cudaStream_t s)
{
    widen_kernel<<<152 * 8, 256, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

// Planar [a][y][x] <-> strip-tiled FP32 state: one block per row y of tile t, threads over
// the tile row's n * 64 values (contiguous in both layouts for each velocity); the padding
// positions of the tiled layout (x outside [0, nx)) are written as zero.
// Velocities a0 .. a0 + na - 1 only (the whole state: 0, n).
__global__ void __launch_bounds__(256) tile_convert_kernel(int to_tiled, const float *__restrict__ src,
                                                          float *__restrict__ dst, int n, int nx, int ny,
                                                          long tile_pitch, int a0, int na)
{
    const int t = blockIdx.x, y = blockIdx.y;
    const long ncells = (long)nx * ny;
    const long trow = (long)t * tile_pitch + (long)y * n * LBM_TILE_W;
    const int x0 = t * LBM_TILE_W - LBM_TILE_SHIFT;
    for (int i = a0 * LBM_TILE_W + threadIdx.x; i < (a0 + na) * LBM_TILE_W; i += blockDim.x) {
        const int a = i / LBM_TILE_W, p = i - a * LBM_TILE_W;
        const int x = x0 + p;
        const bool in = x >= 0 && x < nx;
        const long pl = (long)a * ncells + (long)y * nx + x;
        if (to_tiled) dst[trow + i] = in ? src[pl] : 0.f;
        else if (in) dst[pl] = src[trow + i];
    }
}

cudaError_t launch_tile_convert(bool to_tiled, const float *src, float *dst, int n, int nx, int ny, long tile_pitch,
                                cudaStream_t s)
{
    const dim3 grid((unsigned)tiles_for(nx), (unsigned)ny);
    tile_convert_kernel<<<grid, 256, 0, s>>>(to_tiled ? 1 : 0, src, dst, n, nx, ny, tile_pitch, 0, n);
    return cudaGetLastError();
}

cudaError_t launch_tile_convert_range(bool to_tiled, const float *src, float *dst, int n, int a0, int na, int nx,
                                      int ny, long tile_pitch, cudaStream_t s)
{
    if (a0 < 0 || na < 0 || a0 + na > n) return cudaErrorInvalidValue;
    if (na == 0) return cudaSuccess;
    const dim3 grid((unsigned)tiles_for(nx), (unsigned)ny);
    tile_convert_kernel<<<grid, 256, 0, s>>>(to_tiled ? 1 : 0, src, dst, n, nx, ny, tile_pitch, a0, na);
    return cudaGetLastError();
}

cudaError_t launch_finalize_pairs(const double *partials, int nparts, double *out, int nres,
                                  cudaStream_t s)
{
    finalize_kernel<<<1, RED_BLOCK, 0, s>>>(partials, nparts, out, nres);
    return cudaGetLastError();
}

cudaError_t launch_finalize_residual(const double *partials, int nparts, double *result,
                                     cudaStream_t s)
{
    finalize_kernel<<<1, RED_BLOCK, 0, s>>>(partials, nparts, result, 4);
    return cudaGetLastError();
}

int norms_blocks(long count)
{
    long b = (count + 256L * 8 - 1) / (256L * 8);
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

cudaError_t launch_norms(const void *a, const void *b, long count, int prec, double *partials,
                         int nparts, double *out, cudaStream_t s)
{
    if (prec == 0)
        norms_kernel<double><<<nparts, 256, 0, s>>>((const double *)a, (const double *)b, count,
                                                    partials);
    else
        norms_kernel<float><<<nparts, 256, 0, s>>>((const float *)a, (const float *)b, count,
                                                   partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_kernel<<<1, RED_BLOCK, 0, s>>>(partials, nparts, out, 2);
    return cudaGetLastError();
}

cudaError_t launch_moments(int prec, const void *h, long pa, long py, const double *tab64, const TableHeader *hdr,
                           int m, int nx, int ny, double u_ref, double *out6, cudaStream_t s, long tile_pitch,
                           bool need_p)
{
    (void)tab64;
    const long ncells = (long)nx * ny;
    const int grid = (int)((ncells + 255) / 256);
    if (prec == 0) {
        if (tile_pitch > 0) return cudaErrorInvalidValue;    // FP64 states are never tiled
        moments_kernel<double><<<grid, 256, 0, s>>>((const double *)h, pa, py, nx, hdr, m, ncells, u_ref, out6);
    } else if (need_p) {
        moments_f32_kernel<true><<<grid, 256, 0, s>>>((const float *)h, pa, py, nx, hdr, m, ncells, u_ref, out6,
                                                      tile_pitch);
    } else {
        moments_f32_kernel<false><<<grid, 256, 0, s>>>((const float *)h, pa, py, nx, hdr, m, ncells, u_ref, out6,
                                                       tile_pitch);
    }
    return cudaGetLastError();
}

cudaError_t launch_face_flux2(int prec, const void *h, long pa, long py, const double *tab64, const TableHeader *hdr,
                              int m, int nx, int ny, int cavity, double u_ref, double *flux_y, double *flux_x,
                              cudaStream_t s)
{
    const long ny_faces = (long)(ny + 1) * nx, nx_faces = (long)ny * (nx + 1);
    if (prec == LBM_FP64)
        face_flux2_y_kernel<double><<<(int)((ny_faces + 255) / 256), 256, 0, s>>>(
            (const double *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_y);
    else
        face_flux2_y_kernel<float><<<(int)((ny_faces + 255) / 256), 256, 0, s>>>(
            (const float *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !cavity || !flux_x) return e;
    if (prec == LBM_FP64)
        face_flux2_x_kernel<double><<<(int)((nx_faces + 255) / 256), 256, 0, s>>>(
            (const double *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_x);
    else
        face_flux2_x_kernel<float><<<(int)((nx_faces + 255) / 256), 256, 0, s>>>(
            (const float *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_x);
    return cudaGetLastError();
}

cudaError_t launch_face_flux(int prec, const void *h, long pa, long py, const double *tab64, const TableHeader *hdr,
                             int m, int nx, int ny, int cavity, double u_ref, double *flux_y,
                             double *flux_x, double *wall_sums, cudaStream_t s)
{
    (void)wall_sums;
    const long ny_faces = (long)(ny + 1) * nx;
    const long nx_faces = (long)ny * (nx + 1);
    if (prec == 0)
        face_flux_y_kernel<double><<<(int)((ny_faces + 255) / 256), 256, 0, s>>>(
            (const double *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_y);
    else
        face_flux_y_kernel<float><<<(int)((ny_faces + 255) / 256), 256, 0, s>>>(
            (const float *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !cavity || !flux_x) return e;
    if (prec == 0)
        face_flux_x_kernel<double><<<(int)((nx_faces + 255) / 256), 256, 0, s>>>(
            (const double *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_x);
    else
        face_flux_x_kernel<float><<<(int)((nx_faces + 255) / 256), 256, 0, s>>>(
            (const float *)h, pa, py, tab64, hdr, m, nx, ny, u_ref, flux_x);
    return cudaGetLastError();
}

lbm_status lbm_norms_fail(lbm_status s, const char *msg);   // error message (lbm_api.cu)

// ---------------------------------------------------------------------------------------
// FP64 throughput probe: eight independent FMA chains per thread on enough warps to keep
// every SM's FP64 pipe busy; the result is stored only if it equals a value it never takes,
// so the chains cannot be removed.  Measures the ceiling of the FP64 march on this GPU.
__device__ double g_fp64_probe_sink;

__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(long iters, double mul, double add)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1e-3 * threadIdx.x + k;
    for (long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], mul, add);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1.2345e300) g_fp64_probe_sink = s;
}

extern "C" lbm_status lbm_probe_fp64_rate(long iters, double *fma_per_s, void *stream)
{
    if (!fma_per_s || iters < 1) return lbm_norms_fail(LBM_EINVAL, "lbm_probe_fp64_rate: invalid argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int grid = 8 * sms, block = 256;
    float ms = 0.f;
    if (e == cudaSuccess) {
        fp64_fma_probe_kernel<<<grid, block, 0, s>>>(iters / 8 + 1, 0.9999999999999, 1e-13);   // warm-up
        e = cudaEventRecord(t0, s);
    }
    if (e == cudaSuccess) {
        fp64_fma_probe_kernel<<<grid, block, 0, s>>>(iters, 0.9999999999999, 1e-13);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return lbm_norms_fail(LBM_ECUDA, cudaGetErrorString(e));
    *fma_per_s = 8.0 * (double)iters * grid * block / (ms * 1e-3);
    return LBM_OK;
}
