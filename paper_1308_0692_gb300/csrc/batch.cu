// Batched march of many independent boundary-value problems (Couette channels and
// lid-driven cavities of different sizes, Knudsen numbers and wall speeds) in one
// persistent, cooperative kernel launch that advances every unconverged instance by a
// block of time steps, captured once into a CUDA graph and replayed.
//
// Each time step is the paper's fully discrete scheme (Eqs. 1, 5-9; the same arithmetic
// as step_kernel.cuh) applied to every active instance.  Work items are (instance,
// 32-cell segment) pairs in a schedule order chosen by the autotuner; the blocks of the
// persistent grid take items round-robin, a grid-wide barrier separates time steps, and
// every `resid_every` steps the per-instance residuals are reduced (FP64 atomics) and
// instances below the tolerance are frozen: from then on their items are skipped and
// their state stays in the buffer of the step at which they converged.
//
// The same kernel, in two more modes, refines converged FP32 instances all at once
// (lbm_batch_refine): BATCH_DEFECT evaluates one step in FP64 arithmetic on the FP32 state
// and stores the change M(h) - h; BATCH_CORRECT marches the correction delta <- L(delta) +
// D of the homogeneous problem (wall driving removed, the defect added after relaxation),
// freezing each instance once its per-step change is below the tolerance relative to the
// norm of its state.
//
// Every wait in the grid barrier is bounded (clock64 against a limit); a barrier that
// gives up sets an error word that all blocks check after each barrier, so the kernel
// returns and the host reports LBM_ETIMEOUT.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "step_kernel.cuh"

lbm_status lbm_norms_fail(lbm_status s, const char *msg);

namespace {

enum { BATCH_MARCH = 0, BATCH_CORRECT = 1, BATCH_DEFECT = 2 };

// Instance state layouts.  Couette channels: planar [n][ny][nx].  Cavities: strip-tiled, tiles
// of 32 columns (tile t holds x in [32 t, 32 t + 32)), each tile [y][pair][32 cells][2] with the
// two velocities (2p, 2p + 1) of a pair side by side in every cell: value (a, x, y) at
//   (x / 32) * tile_pitch + y * 32 n + (a / 2) * 64 + (x mod 32) * 2 + (a mod 2),
// tile_pitch = 32 n ny.  A row of a 32-column strip is then one contiguous stretch of 128 n
// bytes, and a warp's velocity pairs of that row one contiguous piece of it (the column march
// copies it with one bulk copy); the last tile of a width that is not a multiple of 32 is
// padded.
__host__ __device__ inline long tile32_off(int x, int y, int n, int ny)
{
    return (long)(x >> 5) * (32L * n * ny) + (long)y * (32L * n) + (long)(x & 31) * 2;
}
__host__ __device__ inline long tile32_vel(int a) { return (long)(a >> 1) * 64 + (a & 1); }

struct BatchInst {
    long off;           // element offset of the instance's state in each array
    long ncells;
    int nx, ny, cavity;
    int tiled;          // cavity: strip-tiled layout (tile32_off); else planar [n][ny][nx]
    double cx, cy;      // dt/dx (0 for a single periodic Couette column), dt/dy
    double omega, b;
    double u_bottom, u_top, inv_u_ref;
};

// values of an instance's state (with the padding of its last tile when tiled)
__host__ __device__ inline long inst_vals(const BatchInst &I, int nv)
{
    return I.tiled ? (long)((I.nx + 31) / 32) * I.ny * nv * 32 : (long)nv * I.ncells;
}
__host__ __device__ inline long inst_index(const BatchInst &I, int n, int a, int x, int y)
{
    return I.tiled ? tile32_off(x, y, n, I.ny) + tile32_vel(a) : (long)a * I.ncells + (long)y * I.nx + x;
}

// One work item: a 32-cell segment of one instance, with the instance's addressing (first
// 32 bytes: fetched one item group ahead, so that the state loads of a group do not wait
// for a chain of dependent metadata loads) and its step coefficients (second 32 bytes).
struct __align__(16) BatchItem {
    long off;            // element offset of the instance's state [n][ncells] in each array
    int ncells, inst, seg, nx, ny, cavity;
    float cx, cy, omega, b;                              // dt/dx (0: one periodic column), dt/dy, omega, 1 - omega
    float u_bottom, u_top, drive_bottom, drive_top;      // wall speeds, wall speed / u_ref
};
static_assert(sizeof(BatchItem) == 64, "two 32-byte halves");

// One work item of the column march (cavity instances): a strip of 32 columns [x0, x0 + 32)
// of rows [y0, y1) of one instance, and the instance's step coefficients.
struct __align__(16) MarchItem {
    long off;            // element offset of the instance's state [n][ncells] in each array
    int inst, nx, ny, x0, y0, y1;
    float cx, cy, omega, b;
    float u_bottom, u_top, drive_bottom, drive_top;
};
static_assert(sizeof(MarchItem) == 64, "four 16-byte loads");

struct BatchArgs {
    void *buf[2];
    const BatchInst *inst;
    int ninst;
    const BatchItem *items;       // the wall-free segments of the unconverged instances
    int nitems;
    const BatchItem *wall_items;  // the segments with a wall cell
    int nwall;
    double *acc;           // [ninst][2] residual sums of the current interval
    double *last_r;        // [ninst]
    double *best_r;        // [ninst] lowest residual so far (march mode; nullptr: no stagnation rule)
    int *flat;             // [ninst] residual checks since it last improved by 1 %
    long *frozen;          // [ninst] step count at convergence (LONG_MAX while active)
    unsigned *bar_count;
    unsigned *bar_gen;
    unsigned *mcount;      // column march: next item of the launch (all steps, step-major)
    unsigned *ifin;        // column march: [ninst] items of the instance finished in this launch
    unsigned *idone;       // column march: [ninst] steps of the instance completed in this launch
    const int *iitems;     // column march: [ninst] items of the instance per step
    int *err;
    long step0;
    int nsteps;
    int resid_every;
    double tol;
    const float *src;      // BATCH_CORRECT: the defect, added after relaxation
    const double *ref_n2;  // BATCH_CORRECT: squared norm of each instance's state (residual scale)
    const MarchItem *mitems;        // column-march items (cavity instances)
    int nmitems;
    const unsigned char *kind;      // [ninst] 1: marched by the column-march kernel, 0: by segments
    int kind_sel;                   // the kind whose residuals this launch reduces
    long long timeout_cycles;
    double xi[LBM_MAX_M], w1[LBM_MAX_M];
    float xi_f[LBM_MAX_M], w1_f[LBM_MAX_M];
    double inv_dx_wall, inv_dy_wall;
    float inv_dx_wall_f, inv_dy_wall_f;
};

// Grid-wide barrier with a bounded wait; returns false once any block has given up.  The
// verdict is read once per block (thread 0) and shared, so that every thread of a block
// takes the same branch (the column march's named barriers need all of a block's warps).
__device__ bool grid_barrier(const BatchArgs &a)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = a.bar_gen;
        const unsigned my_gen = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(a.bar_count, 0u);
            __threadfence();
            atomicAdd(a.bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == my_gen) {
                if (*(volatile int *)a.err != 0) break;
                if (clock64() - t0 > a.timeout_cycles) {
                    atomicExch(a.err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = *(volatile int *)a.err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename TC>
__device__ __forceinline__ TC pk(const double *d, const float *f, int i) { return lbmk::pick<TC>(d, f, i); }

// Addressing half of an item (zeros past the end of the list).
struct ItemAddr {
    long off;
    int ncells, inst, seg, nx, ny, cavity;
    bool valid;
};

__device__ __forceinline__ ItemAddr load_addr(const BatchItem *items, long nitems, long item)
{
    ItemAddr r;
    r.valid = item < nitems;
    int4 q0 = make_int4(0, 0, 0, 0), q1 = make_int4(0, 1, 1, 1);
    if (r.valid) {
        const int4 *p = reinterpret_cast<const int4 *>(items + item);
        q0 = __ldg(p);
        q1 = __ldg(p + 1);
    }
    r.off = (long)(((unsigned long long)(unsigned)q0.y << 32) | (unsigned)q0.x);
    r.ncells = q0.z;
    r.inst = q0.w;
    r.seg = q1.x;
    r.nx = q1.y;
    r.ny = q1.z;
    r.cavity = q1.w;
    return r;
}

// One group of SPB segments (one per warp group of the block): transport, moments and
// relaxation of the listed segments; WALLS selects the code path of segments that contain
// wall cells (FP64 wall densities across rows and warps, ghosts in the arithmetic type) --
// separate from the lean wall-free path so that the latter keeps a small register
// footprint.  The item's addressing `A` was fetched one group earlier; its coefficients and
// the instance's convergence flag are fetched here together with the state.  A segment of
// an instance that converged since the item list was built is read but not written.  All
// threads of the block call it together (shared-memory exchanges inside).
template <typename TS, typename TC, int M, int G, bool WALLS, int MODE>
__device__ __forceinline__ void batch_group(const BatchArgs &a, const BatchItem *items, long grp,
                                            const ItemAddr &A, long s, const TS *__restrict__ h,
                                            TS *__restrict__ hn, bool resid,
                                            TC (&s_mom)[3][G][lbmk::Shape<G>::SPB][32],
                                            double (&s_wall)[4][G][lbmk::Shape<G>::SPB][32])
{
    constexpr int SPB = lbmk::Shape<G>::SPB;
    constexpr int RPL = M / G;
    constexpr int HALF = M / 2;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = warp / G, g = warp - sl * G;
    const long item = grp * SPB + sl;
    const bool active = A.valid;
    // step coefficients: dt/dx, dt/dy, omega, 1 - omega, wall speeds, wall speeds / u_ref --
    // FP32 from the item, except in the FP64 defect pass, which takes the instance's FP64 values
    TC k_cx = 0, k_cy = 0, k_om = 1, k_b = 0, k_ub = 0, k_ut = 0, k_db = 0, k_dt = 0;
    bool live = false;
    if (active) {
        if (MODE == BATCH_DEFECT) {
            const BatchInst &I = a.inst[A.inst];
            k_cx = (TC)I.cx;
            k_cy = (TC)I.cy;
            k_om = (TC)I.omega;
            k_b = (TC)I.b;
            k_ub = (TC)I.u_bottom;
            k_ut = (TC)I.u_top;
            k_db = (TC)(I.u_bottom * I.inv_u_ref);
            k_dt = (TC)(I.u_top * I.inv_u_ref);
        } else {
            const float4 *p = reinterpret_cast<const float4 *>(items + item) + 2;
            const float4 k0 = __ldg(p), k1 = __ldg(p + 1);
            k_cx = (TC)k0.x;
            k_cy = (TC)k0.y;
            k_om = (TC)k0.z;
            k_b = (TC)k0.w;
            k_ub = (TC)k1.x;
            k_ut = (TC)k1.y;
            // homogeneous walls in the correction march: no driving term
            k_db = MODE == BATCH_CORRECT ? TC(0) : (TC)k1.z;
            k_dt = MODE == BATCH_CORRECT ? TC(0) : (TC)k1.w;
        }
        live = a.frozen[A.inst] > s;
    }
    const long ncells = A.ncells;
    const int nx = A.nx, ny = A.ny;
    const bool cav = A.cavity != 0;
    const long cell0 = (long)A.seg * 32 + lane;
    const bool in_grid = cell0 < ncells;
    const long c = in_grid ? cell0 : ncells - 1;
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const TS *hi = h + A.off;
    TS *hno = hn + A.off;
    // cell offsets (velocity 0) and the offset of velocity a, (a / 2) * ps + (a mod 2) * os:
    // cavities are strip-tiled, channels planar
    const bool tl = cav;
    auto cell_off = [&](int xx, int yy) -> long {
        return tl ? tile32_off(xx, yy, M * M, ny) : (long)yy * nx + xx;
    };
    const long ps = tl ? 64 : 2 * ncells, os = tl ? 1 : ncells;
    auto vo = [&](int aa) -> long { return (long)(aa >> 1) * ps + (aa & 1) * os; };
    const long c_at = cell_off(x, y);
    const long c_left = (x > 0) ? cell_off(x - 1, y) : (cav ? c_at : cell_off(nx - 1, y));
    const long c_right = (x < nx - 1) ? cell_off(x + 1, y) : (cav ? c_at : cell_off(0, y));
    const long c_below = (y > 0) ? cell_off(x, y - 1) : c_at;
    const long c_above = (y < ny - 1) ? cell_off(x, y + 1) : c_at;
    const bool wl = WALLS && cav && x == 0, wr = WALLS && cav && x == nx - 1;
    const bool wb = WALLS && y == 0, wt = WALLS && y == ny - 1;

    double rb = 0.0, rt = 0.0, rl = 0.0, rr = 0.0;
    if (WALLS) {
        // wall densities (Eq. 9).  Segments in the bottom or top row need the y-wall sums of
        // every lane: row sums in the arithmetic type, FP64 across rows and warps.  The other
        // wall segments (a cavity's side walls) hold one or two wall cells: their sums are
        // formed cooperatively for those cells only, the velocities dealt to the lanes (products in the
        // arithmetic type, the sum in FP64), instead of every lane reading all its
        // velocities -- in cavities of 128 cells per row half of all segments are of this kind.
        double sb = 0.0, st = 0.0, sls = 0.0, srs = 0.0;
        const bool rows_wall = __any_sync(FULL, in_grid && (y == 0 || y == ny - 1));
        if (active && !rows_wall && cav) {
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
                        const TC v = (TC)__ldg(hi + vo(iy * M + ix) + cL);
                        const TC xv = pk<TC>(a.xi, a.xi_f, ix) * v;
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
        } else if (active) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int iy = g * RPL + r;
                const double xiy = a.xi[iy];
                TC rowsum = 0, left = 0, right = 0;
#pragma unroll
                for (int ix = 0; ix < M; ++ix) {
                    const TC v = (TC)__ldg(hi + vo(iy * M + ix) + c_at);
                    rowsum += v;
                    if (ix < HALF) left -= pk<TC>(a.xi, a.xi_f, ix) * v;
                    if (ix >= M - HALF) right += pk<TC>(a.xi, a.xi_f, ix) * v;
                }
                if (xiy < 0.0) sb -= xiy * (double)rowsum;
                if (xiy > 0.0) st += xiy * (double)rowsum;
                sls += (double)left;
                srs += (double)right;
            }
        }
        s_wall[0][g][sl][lane] = sb;
        s_wall[1][g][sl][lane] = st;
        s_wall[2][g][sl][lane] = sls;
        s_wall[3][g][sl][lane] = srs;
        __syncthreads();
        sb = st = sls = srs = 0.0;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            sb += s_wall[0][q][sl][lane];
            st += s_wall[1][q][sl][lane];
            sls += s_wall[2][q][sl][lane];
            srs += s_wall[3][q][sl][lane];
        }
        rb = sb * a.inv_dy_wall;
        rt = st * a.inv_dy_wall;
        rl = sls * a.inv_dx_wall;
        rr = srs * a.inv_dx_wall;
    }

    TC hs[RPL * M];
    TC rho = 0, jx = 0, jy = 0;
    if (active) {
        const TC cx = k_cx, cy = k_cy;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC xiy = pk<TC>(a.xi, a.xi_f, iy);
            const TC nuy = (xiy < TC(0) ? -xiy : xiy) * cy;
            const bool ypos = xiy > TC(0), yneg = xiy < TC(0);
            const long cy_idx = ypos ? c_below : (yneg ? c_above : c_at);
            const bool ywall = WALLS && ((ypos && wb) || (yneg && wt));
            const TC rho_y = (TC)(ypos ? rb : rt);
            const TC u_y = ypos ? k_ub : k_ut;
            const TC drive_y = ypos ? k_db : k_dt;
            const TC wy = pk<TC>(a.w1, a.w1_f, iy);
            const TC rl_t = (TC)rl, rr_t = (TC)rr;
            TC R = 0, X = 0;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const TS *hp = hi + vo(iy * M + ix);
                const TC hc = (TC)__ldg(hp + c_at);
                const TC xix = pk<TC>(a.xi, a.xi_f, ix);
                TC v = hc;
                if (ix >= M - HALF || ix < HALF) {
                    TC hx;
                    if (WALLS && (ix >= M - HALF ? wl : wr))
                        hx = pk<TC>(a.w1, a.w1_f, ix) * wy * (ix >= M - HALF ? rl_t : rr_t);
                    else
                        hx = (TC)__ldg(hp + (ix >= M - HALF ? c_left : c_right));
                    v += (xix < TC(0) ? -xix : xix) * cx * (hx - hc);
                }
                TC hy;
                if (WALLS && ywall)
                    hy = pk<TC>(a.w1, a.w1_f, ix) * wy * (rho_y * (TC(1) + xix * u_y) + xix * drive_y);
                else
                    hy = (TC)__ldg(hp + cy_idx);
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

    TC psd = 0, psn = 0;
    const bool valid = live && in_grid;
    if (active) {
        const TC om = k_om, b = k_b;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC wom = om * pk<TC>(a.w1, a.w1_f, iy);
            const TC q = wom * (rho + pk<TC>(a.xi, a.xi_f, iy) * jy);
            const TC jj = wom * jx;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const long off = vo(iy * M + ix) + c_at;
                const TC t = q + pk<TC>(a.xi, a.xi_f, ix) * jj;
                TC v = b * hs[r * M + ix] + pk<TC>(a.w1, a.w1_f, ix) * t;
                if (MODE == BATCH_CORRECT) v += (TC)__ldg(a.src + A.off + off);
                TC d = 0;
                if (resid) {
                    d = v - (TC)__ldg(hi + off);
                    psd += d * d;
                    psn += v * v;
                }
                if (valid) hno[off] = (TS)(MODE == BATCH_DEFECT ? d : v);
            }
        }
    }
    if (resid && live) {
        double dsd = valid ? (double)psd : 0.0, dsn = valid ? (double)psn : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dsd += __shfl_xor_sync(FULL, dsd, off);
            dsn += __shfl_xor_sync(FULL, dsn, off);
        }
        if (lane == 0) {
            atomicAdd(a.acc + 2 * A.inst, dsd);
            atomicAdd(a.acc + 2 * A.inst + 1, dsn);
        }
    }
    __syncthreads();   // shared arrays are reused by the next group
}

template <typename TS, typename TC, int M, int G, int MODE>
__global__ void __launch_bounds__(lbmk::Shape<G>::THREADS, 2) batch_kernel(const BatchArgs a)
{
    constexpr int SPB = lbmk::Shape<G>::SPB;
    __shared__ TC s_mom[3][G][SPB][32];
    __shared__ double s_wall[4][G][SPB][32];

    for (int si = 0; si < a.nsteps; ++si) {
        const long s = a.step0 + si;
        const TS *__restrict__ h = reinterpret_cast<const TS *>(a.buf[s & 1]);
        TS *__restrict__ hn = reinterpret_cast<TS *>(a.buf[(s + 1) & 1]);
        const bool resid = MODE == BATCH_DEFECT || ((s + 1) % a.resid_every) == 0;
        // wall-free segments, then segments with wall cells, both round-robin over the blocks;
        // the addressing of the next group is fetched before the current group runs
        const int sl = (int)(threadIdx.x >> 5) / G;
        const long nb = ((long)a.nitems + SPB - 1) / SPB;
        ItemAddr cur = load_addr(a.items, a.nitems, (long)blockIdx.x * SPB + sl);
        for (long grp = blockIdx.x; grp < nb; grp += gridDim.x) {
            const ItemAddr nxt = load_addr(a.items, a.nitems, (grp + gridDim.x) * SPB + sl);
            batch_group<TS, TC, M, G, false, MODE>(a, a.items, grp, cur, s, h, hn, resid, s_mom, s_wall);
            cur = nxt;
        }
        const long nw = ((long)a.nwall + SPB - 1) / SPB;
        cur = load_addr(a.wall_items, a.nwall, (long)blockIdx.x * SPB + sl);
        for (long grp = blockIdx.x; grp < nw; grp += gridDim.x) {
            const ItemAddr nxt = load_addr(a.wall_items, a.nwall, (grp + gridDim.x) * SPB + sl);
            batch_group<TS, TC, M, G, true, MODE>(a, a.wall_items, grp, cur, s, h, hn, resid, s_mom, s_wall);
            cur = nxt;
        }
        if (MODE == BATCH_DEFECT) continue;    // one pass; the host reads the sums
        if (!grid_barrier(a)) return;
        if (resid) {
            if (blockIdx.x == 0) {
                for (int i = threadIdx.x; i < a.ninst; i += blockDim.x) {
                    if (a.frozen[i] <= s || a.kind[i] != a.kind_sel) continue;
                    const double sd = a.acc[2 * i];
                    // the correction's change is measured against the state it corrects
                    const double sn = MODE == BATCH_CORRECT ? a.ref_n2[i] : a.acc[2 * i + 1];
                    const double r = sn > 0.0 ? sqrt(sd / sn) : (sd == 0.0 ? 0.0 : INFINITY);
                    a.last_r[i] = r;
                    if (!(r == r) || isinf(r)) atomicExch(a.err, 2);
                    if (r < a.tol) {
                        a.frozen[i] = s + 1;
                    } else if (a.best_r && a.tol > 0) {
                        // the FP32 rounding floor: no 1 % improvement over 20 checks freezes too
                        if (r < 0.99 * a.best_r[i]) {
                            a.best_r[i] = r;
                            a.flat[i] = 0;
                        } else if (++a.flat[i] >= 20) {
                            a.frozen[i] = s + 1;
                        }
                    }
                    a.acc[2 * i] = 0.0;
                    a.acc[2 * i + 1] = 0.0;
                }
            }
            if (!grid_barrier(a)) return;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Compensated FP32 summation (Knuth's TwoSum error-free transformation): the pair (s, c)
// carries the sum and its rounding error, so that short sums come out as accurate as FP64
// ones -- FP64 arithmetic itself runs at a small fraction of the FP32 rate on this GPU.
// Plain IEEE additions (no reassociation; the library is built without fast-math).
__device__ __forceinline__ void comp_add(float &s, float &c, float x)
{
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// Column march over cavity instances.  A sub-block of G warps takes one item (a 32-column
// strip of a chunk of rows); warp g owns RPL velocity rows (one sign of xi_y, so its upwind y
// neighbour is the row below when xi_y > 0, the row above otherwise), lane l owns column
// x0 + l.  The strip marches up its rows through a ring of four row slots per warp in
// shared memory, two rows ahead.  The instance is strip-tiled (tile32_off: a tile is one
// 32-column strip), so a warp's velocity pairs of a row are one contiguous piece of
// 8 * RPL * M bytes: one bulk asynchronous copy (cp.async.bulk) fills the slot, and the x
// halo of each velocity pair (the left tile's last cell for pairs moving right, the right
// tile's first cell for pairs moving left) comes with one 8-byte cp.async per pair on the
// load/store unit; the slot's mbarrier counts the bulk copy's bytes and the halo copies'
// arrivals (cp.async.mbarrier.arrive.noinc).  Every value is read from memory once per step,
// plus one extra row per chunk and the halos (served by L2), and the x and y neighbours are
// read from the ring.  Per row the warps exchange their moment partials through shared
// memory (one named barrier per row, double-buffered), and with them the wall-density
// partials of the next row (Eq. 9: side walls from the wall cells' outgoing velocities, the
// top wall at the last row), so that the ghosts of the next row are known before its
// transport; the bottom wall's are formed before the first row of a chunk that starts at
// y = 0.  Arithmetic in FP32 with the same operations in the same order as batch_group; the
// wall sums and the residual sums are compensated FP32 (comp_add), which keeps FP64-grade
// sums off the slow FP64 pipe.  Stores: each lane writes its cell's velocity pairs as 8-byte
// stores, a warp instruction covering 256 contiguous bytes.  Every wait on a slot is bounded;
// after the limit the batch's error word is set and the waits of the launch are skipped
// (the grid barrier then ends the launch and the host reports LBM_ETIMEOUT).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void named_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int M, int G>
struct MarchShared {
    static constexpr int RPL = M / G;    // velocity rows per warp
    static constexpr int SUB = 8 / G;    // items per block of 8 warps
    static constexpr int NS = 4;         // row slots per warp
    static constexpr int PW = RPL * M / 2;   // velocity pairs per warp
    static constexpr int SLOT = PW * 32 + PW;   // float2: PW pair lines of 32 cells, then one halo per line
    float4 mom[SUB][2][G][32];           // [item][row parity][warp][lane]: (rho, jx, jy, -) partials
    float2 side[SUB][2][2][G];           // [item][parity][left, right][warp]: (sum, error)
    float2 tb[SUB][2][G][32];            // [item][parity][warp][lane]: bottom or top wall row
    float2 ring[8][NS][SLOT];            // [warp][slot]: velocity pairs (2q, 2q + 1) of a row
    uint64_t bar[8][NS];                 // [warp][slot]: fill of the slot complete
};

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
// nodes and 1-D weights of the velocity pair (2j, 2j + 1)
__device__ __forceinline__ float2 xi2(const BatchArgs &a, int j) { return make_float2(a.xi_f[2 * j], a.xi_f[2 * j + 1]); }
__device__ __forceinline__ float2 w2(const BatchArgs &a, int j) { return make_float2(a.w1_f[2 * j], a.w1_f[2 * j + 1]); }

__device__ __forceinline__ bool slot_try(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_addr(bar)), "r"(parity), "r"(1000000u)
                 : "memory");
    return done != 0;
}

// State of a warp's ring across items and steps: the parity each slot's next fill completes
// with (bit s) and which slots have a fill not yet waited for.
struct RingState {
    unsigned ph = 0, pend = 0;
};

template <int M, int G, int MODE>
__device__ __forceinline__ void march_item(const BatchArgs &a, const MarchItem *mi, long s, const float *h,
                                           float *hn, bool resid, MarchShared<M, G> &sh, RingState &rs)
{
    using Sh = MarchShared<M, G>;
    constexpr int P = M / 2, PH = P / 2;                  // pairs per velocity row; j >= PH move right
    constexpr int RPL = Sh::RPL, SUB = Sh::SUB, NS = Sh::NS, PW = Sh::PW;
    static_assert(SUB * G == 8 && PW <= 32 && (M / 2) % 2 == 0, "eight warps per block; halo lanes; pairs on one side");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = warp / G, g = warp - sub * G;
    const int bar_id = 1 + sub, bar_n = 32 * G;

    const int4 *q = reinterpret_cast<const int4 *>(mi);
    const int4 q0 = __ldg(q), q1 = __ldg(q + 1);
    const float4 k0 = __ldg(reinterpret_cast<const float4 *>(q + 2)),
                 k1 = __ldg(reinterpret_cast<const float4 *>(q + 3));
    const long off = (long)(((unsigned long long)(unsigned)q0.y << 32) | (unsigned)q0.x);
    const int inst = q0.z, nx = q0.w, ny = q1.x, x0 = q1.y, y0 = q1.z, y1 = q1.w;
    if (a.frozen[inst] <= s) return;          // converged: its state stays put
    const float cx = k0.x, cy = k0.y, om = k0.z, bb = k0.w;

    // this warp's velocity rows iy0 .. iy0 + RPL - 1 share the sign of xi_y
    const int iy0 = g * RPL;
    float xiyr[RPL], wyr[RPL], nuyr[RPL];
#pragma unroll
    for (int rr = 0; rr < RPL; ++rr) {
        xiyr[rr] = a.xi_f[iy0 + rr];
        wyr[rr] = a.w1_f[iy0 + rr];
        nuyr[rr] = (xiyr[rr] < 0.f ? -xiyr[rr] : xiyr[rr]) * cy;
    }
    const bool up = xiyr[0] > 0.f;            // upwind neighbour below; ghost at the bottom wall
    float2 nux2[P];                           // |xi_x| dt / dx per velocity pair
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const float u0 = a.xi_f[2 * j], u1 = a.xi_f[2 * j + 1];
        nux2[j] = make_float2((u0 < 0.f ? -u0 : u0) * cx, (u1 < 0.f ? -u1 : u1) * cx);
    }
    const int x = x0 + lane;
    const bool valid = x < nx;
    const bool wl = x == 0, wr = x == nx - 1;
    const bool side_l = x0 == 0, side_r = x0 + 32 >= nx, side = side_l || side_r;
    const int lr = nx - 1 - x0;               // lane of the right-wall cell when side_r
    // strip-tiled addressing: the strip is tile x0 / 32; a row is 32 n floats; this warp's
    // pairs start at pair iy0 * M / 2 of the row
    constexpr int NVEL = M * M;
    const long tp = 32L * NVEL * ny, trow = 32L * NVEL;
    const int tile = x0 >> 5, ntiles = (nx + 31) >> 5;
    const long wbase = off + (long)tile * tp + (long)(iy0 * M / 2) * 64;
    float2(*ring)[Sh::SLOT] = sh.ring[warp];
    uint64_t *bars = sh.bar[warp];
    // halo source of pair lane (lanes < PW): left tile's cell 31 for pairs moving right, right
    // tile's cell 0 for pairs moving left; a strip at a side wall takes its own tile there
    // (the wall lane uses the ghost instead)
    const int hq = lane < PW ? lane : 0, hj = hq % P;
    const long halo_off = hj >= PH ? (tile > 0 ? -tp + 62 : 0) : (tile + 1 < ntiles ? tp : 0);
    const float *hsrc = h + wbase + (long)hq * 64 + halo_off;

    auto wait_slot = [&](int sl) {
        if (!((rs.pend >> sl) & 1)) return;
        if (*(volatile int *)a.err == 0) {
            const long long t0 = clock64();
            bool ok = true;
            while (!slot_try(&bars[sl], (rs.ph >> sl) & 1u)) {
                if (clock64() - t0 > a.timeout_cycles) {
                    ok = false;
                    break;
                }
            }
            ok = __all_sync(FULL, ok);
            if (!ok && lane == 0) atomicExch(a.err, 1);
        }
        rs.ph ^= 1u << sl;
        rs.pend &= ~(1u << sl);
    };
    auto wait_row = [&](int r) { wait_slot(r & (NS - 1)); };
    // fill the slot of row r with this warp's pairs of the row and their halos
    auto copy_row = [&](int r, bool issue) {
        if (!issue) return;
        const int sl = r & (NS - 1);
        wait_slot(sl);                          // (never pending here: its row was consumed)
        float2 *slot = ring[sl];
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(&bars[sl])),
                         "r"((unsigned)(PW * 256))
                         : "memory");
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier reads of the slot first
        if (lane == 0)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                         ::"r"(smem_addr(slot)), "l"(h + wbase + (long)r * trow), "r"((unsigned)(PW * 256)),
                         "r"(smem_addr(&bars[sl]))
                         : "memory");
        if (lane < PW)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n"
                         "cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%2];\n" ::"r"(smem_addr(slot + PW * 32 + lane)),
                         "l"(hsrc + (long)r * trow), "r"(smem_addr(&bars[sl]))
                         : "memory");
        rs.pend |= 1u << sl;
    };
    // x-upwind neighbour of a lane's cell in pair line qq: the neighbouring cell of the line, or
    // for the strip's edge lane the halo (index base + qq * step of the slot)
    const int bl = lane > 0 ? lane - 1 : PW * 32, stl = lane > 0 ? 32 : 1;
    const int br = lane < 31 ? lane + 1 : PW * 32, str = lane < 31 ? 32 : 1;
    // moving up: rows r - 1, r in hand and r + 1, r + 2 in flight at row r; moving down:
    // r, r + 1 in hand and r + 2, r + 3 in flight.  The last row a warp reads:
    const int lim = up ? y1 - 1 : min(y1, ny - 1);
    if (up) {
        if (y0 > 0) copy_row(y0 - 1, true);
        copy_row(y0, true);
        copy_row(y0 + 1, y0 + 1 <= lim);
    } else {
        copy_row(y0, true);
        copy_row(y0 + 1, y0 + 1 <= lim);
        copy_row(y0 + 2, y0 + 2 <= lim);
    }

    // Eq. 9 sums: the outgoing velocities' normal fluxes at the wall cells of row r
    auto wall_partials = [&](int r, int p) {
        const float2 *row = ring[r & (NS - 1)];
        if (side_l && lane == 0) {
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr)
#pragma unroll
                for (int j = 0; j < PH; ++j) {
                    const float2 u = row[(rr * P + j) * 32];
                    comp_add(hi, lo, -(a.xi_f[2 * j] * u.x));
                    comp_add(hi, lo, -(a.xi_f[2 * j + 1] * u.y));
                }
            sh.side[sub][p][0][g] = make_float2(hi, lo);
        }
        if (side_r && lane == lr) {
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr)
#pragma unroll
                for (int j = PH; j < P; ++j) {
                    const float2 u = row[(rr * P + j) * 32 + lr];
                    comp_add(hi, lo, a.xi_f[2 * j] * u.x);
                    comp_add(hi, lo, a.xi_f[2 * j + 1] * u.y);
                }
            sh.side[sub][p][1][g] = make_float2(hi, lo);
        }
        if (r == 0 || r == ny - 1) {
            // sum over the warp's rows of |xi_y| times the row sum, each product with its
            // rounding error (FMA) kept; bottom wall: velocities moving down, top: moving up
            float th = 0.f, tl = 0.f;
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr) {
                float hi = 0.f, lo = 0.f;
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const float2 u = row[(rr * P + j) * 32 + lane];
                    comp_add(hi, lo, u.x);
                    comp_add(hi, lo, u.y);
                }
                const float ax = xiyr[rr] < 0.f ? -xiyr[rr] : xiyr[rr];
                const float ph = ax * hi, pl = fmaf(ax, hi, -ph) + ax * lo;
                comp_add(th, tl, ph);
                tl += pl;
            }
            const bool in = r == 0 ? !up : up;
            sh.tb[sub][p][g][lane] = in ? make_float2(th, tl) : make_float2(0.f, 0.f);
        }
    };
    float rho_l = 0.f, rho_r = 0.f, rho_w = 0.f;    // side walls; bottom or top wall of a wall row
    auto total = [&](const float2 *t, int stride, float inv) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int w = 0; w < G; ++w) {
            const float2 u = t[w * stride];
            comp_add(hi, lo, u.x);
            lo += u.y;
        }
        return fmaf(hi, inv, lo * inv);
    };
    auto read_walls = [&](int r, int p) {
        if (side_l) rho_l = total(&sh.side[sub][p][0][0], 1, a.inv_dx_wall_f);
        if (side_r) rho_r = total(&sh.side[sub][p][1][0], 1, a.inv_dx_wall_f);
        if (r == 0 || r == ny - 1) rho_w = total(&sh.tb[sub][p][0][lane], 32, a.inv_dy_wall_f);
    };
    wait_row(y0);
    {
        const int p0 = (y0 + 1) & 1;
        wall_partials(y0, p0);
        named_barrier(bar_id, bar_n);
        read_walls(y0, p0);
    }
    // wall speed and driving term of the wall this warp's velocities come from (Eq. 8)
    const float uw = up ? k1.x : k1.y;
    const float dw = MODE == BATCH_CORRECT ? 0.f : (up ? k1.z : k1.w);
    const float *sb = MODE == BATCH_CORRECT ? a.src + wbase : nullptr;

    float2 v[PW];
    // transport (Eqs. 1, 8-9) of row r into v[] (FP32x2 over velocity pairs, per velocity the
    // same operations as batch_group); SIDE: a side-wall cell in the strip, WROW: the y ghost
    // of a wall row.  Returns the partial moments (rho, jx, jy) of the warp's velocities.
    // (called with literal flags: each call site is inlined and specialised)
    auto transport = [&](bool SIDE, bool WROW, const float2 *cur, const float2 *yrow) {
        float R = 0.f, X = 0.f, Y = 0.f;
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            float2 R2 = make_float2(0.f, 0.f), X2 = make_float2(0.f, 0.f);
            const float2 wyy = splat(wyr[rr]);
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int qq = rr * P + j;
                const float2 hc = cur[qq * 32 + lane];
                float2 xn = cur[j >= PH ? bl + qq * stl : br + qq * str];
                if (SIDE) {
                    const float2 wa = __fmul2_rn(w2(a, j), wyy);
                    if (j >= PH && wl) xn = __fmul2_rn(wa, splat(rho_l));
                    if (j < PH && wr) xn = __fmul2_rn(wa, splat(rho_r));
                }
                float2 yn;
                if (WROW) {
                    const float2 wa = __fmul2_rn(w2(a, j), wyy);
                    const float2 gg = __ffma2_rn(xi2(a, j), splat(uw), splat(1.f));
                    yn = __fmul2_rn(wa, __ffma2_rn(xi2(a, j), splat(dw), __fmul2_rn(splat(rho_w), gg)));
                } else {
                    yn = yrow[qq * 32 + lane];
                }
                float2 t = __ffma2_rn(nux2[j], __fadd2_rn(xn, neg2(hc)), hc);
                t = __ffma2_rn(splat(nuyr[rr]), __fadd2_rn(yn, neg2(hc)), t);
                v[qq] = t;
                R2 = __fadd2_rn(R2, t);
                X2 = __ffma2_rn(xi2(a, j), t, X2);
            }
            const float Rr = R2.x + R2.y;
            R += Rr;
            X += X2.x + X2.y;
            Y += xiyr[rr] * Rr;
        }
        return make_float3(R, X, Y);
    };
    float psd = 0.f, psd_c = 0.f, psn = 0.f, psn_c = 0.f;
    // relaxation (Eqs. 5-7) towards w_a (rho + xi.j) and the store; RESID: residual sums
    float2 src[MODE == BATCH_CORRECT ? PW : 1];   // the correction's source of the current row
    auto relax = [&](bool RESID, const float2 *cur, float rho, float jx, float jy, int r) {
        float2 sd = make_float2(0.f, 0.f), sn = make_float2(0.f, 0.f);
        float2 *orow = reinterpret_cast<float2 *>(hn + wbase + (long)r * trow) + lane;
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            const float wom = om * wyr[rr];
            const float qv = wom * (rho + xiyr[rr] * jy);
            const float jj = wom * jx;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int qq = rr * P + j;
                const float2 t = __ffma2_rn(xi2(a, j), splat(jj), splat(qv));
                float2 nv = __ffma2_rn(w2(a, j), t, __fmul2_rn(splat(bb), v[qq]));
                if (MODE == BATCH_CORRECT) nv = __fadd2_rn(nv, src[qq]);
                if (RESID) {
                    const float2 d = __fadd2_rn(nv, neg2(cur[qq * 32 + lane]));
                    sd = __ffma2_rn(d, d, sd);
                    sn = __ffma2_rn(nv, nv, sn);
                }
                if (valid) orow[qq * 32] = nv;
            }
        }
        if (RESID && valid) {
            comp_add(psd, psd_c, sd.x + sd.y);
            comp_add(psn, psn_c, sn.x + sn.y);
        }
    };

    for (int r = y0; r < y1; ++r) {
        const int p = r & 1;
        // the rows of this step in hand: own row r and the upwind row (a wall row's ghost
        // needs none)
        wait_row(r);
        if (up ? r > 0 : r < ny - 1) wait_row(up ? r - 1 : r + 1);
        // refill: the slot of row r - 2 (moving up) or r - 1 (moving down), read by now
        if (up) copy_row(r + 2, r + 2 <= lim);
        else copy_row(r + 3, r + 3 <= lim);
        const float2 *cur = ring[r & (NS - 1)];
        const float2 *yrow = ring[(up ? r - 1 : r + 1) & (NS - 1)];
        if (MODE == BATCH_CORRECT) {          // issued now, used after the moment exchange
            const float2 *srow = reinterpret_cast<const float2 *>(sb + (long)r * trow) + lane;
#pragma unroll
            for (int k = 0; k < PW; ++k) src[k] = valid ? __ldg(srow + k * 32) : make_float2(0.f, 0.f);
        }
        // the y ghost of a wall row: bottom for warps moving up, top for warps moving down
        const bool wrow = up ? r == 0 : r == ny - 1;
        float3 rx;
        if (wrow) rx = side ? transport(true, true, cur, yrow) : transport(false, true, cur, yrow);
        else rx = side ? transport(true, false, cur, yrow) : transport(false, false, cur, yrow);
        sh.mom[sub][p][g][lane] = make_float4(rx.x, rx.y, rx.z, 0.f);
        // the next row's wall sums travel with this row's moments
        if (r + 1 < y1 && (side || r + 1 == ny - 1)) {
            wait_row(r + 1);
            wall_partials(r + 1, p);
        }
        named_barrier(bar_id, bar_n);
        float rho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
        for (int w = 0; w < G; ++w) {
            const float4 u = sh.mom[sub][p][w][lane];
            rho += u.x;
            jx += u.y;
            jy += u.z;
        }
        if (resid) relax(true, cur, rho, jx, jy, r);
        else relax(false, cur, rho, jx, jy, r);
        if (r + 1 < y1) read_walls(r + 1, p);
    }
    // every fill of the item has been waited for; none is left pending
    for (int sl = 0; sl < NS; ++sl) wait_slot(sl);
    __syncwarp();
    if (resid) {
        double dd = (double)psd + (double)psd_c, dn = (double)psn + (double)psn_c;
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            dd += __shfl_xor_sync(FULL, dd, o2);
            dn += __shfl_xor_sync(FULL, dn, o2);
        }
        if (lane == 0) {
            atomicAdd(a.acc + 2 * inst, dd);
            atomicAdd(a.acc + 2 * inst + 1, dn);
        }
    }
}

// The residual of instance i after step s (its sums complete): store it, check it is finite,
// and freeze the instance once below tol -- or, with tol > 0 in the march, once it has not
// improved by 1 % over 20 checks (the FP32 rounding floor); clear the sums for the next check.
template <int MODE>
__device__ void residual_decision(const BatchArgs &a, int i, long s)
{
    if (a.frozen[i] <= s) return;
    const double sd = a.acc[2 * i];
    // the correction's change is measured against the state it corrects
    const double sn = MODE == BATCH_CORRECT ? a.ref_n2[i] : a.acc[2 * i + 1];
    const double r = sn > 0.0 ? sqrt(sd / sn) : (sd == 0.0 ? 0.0 : INFINITY);
    a.last_r[i] = r;
    if (!(r == r) || isinf(r)) atomicExch(a.err, 2);
    if (r < a.tol) {
        a.frozen[i] = s + 1;
    } else if (a.best_r && a.tol > 0) {
        if (r < 0.99 * a.best_r[i]) {
            a.best_r[i] = r;
            a.flat[i] = 0;
        } else if (++a.flat[i] >= 20) {
            a.frozen[i] = s + 1;
        }
    }
    a.acc[2 * i] = 0.0;
    a.acc[2 * i + 1] = 0.0;
}

// Items of all the launch's steps form one sequence, step-major (item k of step si is number
// si * nmitems + k), handed out one at a time to the warp groups by a counter.  An item of
// step si > 0 first waits (bounded) until its instance has completed step si - 1 -- its reads
// of the old state and its writes of the new one then cannot overlap another step of the same
// instance -- so instances move through the steps independently and no grid-wide barrier is
// needed: a group that finishes early starts on the next step of the instances that are done.
// Every item waits only for items numbered before it, which groups resident in this
// cooperative launch are running, so the launch always progresses.  The group that finishes
// the last item of an instance's step evaluates its residual on residual steps (freezing it
// when converged) and then publishes the completed step.
template <int M, int G, int MODE>
__global__ void __launch_bounds__(256, G == M ? 3 : (2 * G == M ? 2 : 1)) batch_march_kernel(const BatchArgs a)
{
    using Sh = MarchShared<M, G>;
    constexpr int SUB = Sh::SUB;
    extern __shared__ __align__(16) unsigned char march_smem[];   // Sh, sized at launch
    Sh &sh = *reinterpret_cast<Sh *>(march_smem);
    __shared__ int s_item[SUB][2];            // fetched item of each warp group, double-buffered
    const int warp = (int)(threadIdx.x >> 5), sub = warp / G;
    const int bar_id = 1 + sub, bar_n = 32 * G;
    const bool fetcher = warp == sub * G && (threadIdx.x & 31) == 0;
    // each warp's ring slots: a fill completes with the bulk copy's bytes (armed by lane 0)
    // and one arrival per halo copy (Sh::PW lanes)
    if ((threadIdx.x & 31) == 0) {
        for (int sl = 0; sl < Sh::NS; ++sl)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(&sh.bar[warp][sl])),
                         "r"((unsigned)(1 + Sh::PW)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    RingState rs;
    const long total = (long)a.nsteps * a.nmitems;
    for (int k = 0;; ++k) {
        if (fetcher) s_item[sub][k & 1] = (int)atomicAdd(a.mcount, 1u);
        named_barrier(bar_id, bar_n);
        const long gi = (long)(unsigned)s_item[sub][k & 1];
        if (gi >= total) break;
        const int si = (int)(gi / a.nmitems), item = (int)(gi - (long)si * a.nmitems);
        const long s = a.step0 + si;
        const MarchItem *mi = a.mitems + item;
        const int inst = __ldg(&mi->inst);
        if (si > 0) {
            if (fetcher) {
                const long long t0 = clock64();
                while (*(volatile unsigned *)(a.idone + inst) < (unsigned)si) {
                    if (*(volatile int *)a.err != 0) break;
                    if (clock64() - t0 > a.timeout_cycles) {
                        atomicExch(a.err, 1);
                        break;
                    }
                    __nanosleep(32);
                }
                __threadfence();
            }
            named_barrier(bar_id, bar_n);
        }
        // the state written by other SMs, read next by the copy engine
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        const float *h = reinterpret_cast<const float *>(a.buf[s & 1]);
        float *hn = reinterpret_cast<float *>(a.buf[(s + 1) & 1]);
        const bool resid = ((s + 1) % a.resid_every) == 0;
        march_item<M, G, MODE>(a, mi, s, h, hn, resid, sh, rs);
        named_barrier(bar_id, bar_n);          // the group's stores and sums are issued
        if (fetcher) {
            __threadfence();
            const unsigned done = atomicAdd(a.ifin + inst, 1u) + 1u;
            if (done == (unsigned)((si + 1) * __ldg(a.iitems + inst))) {
                if (resid) residual_decision<MODE>(a, inst, s);
                __threadfence();
                atomicExch(a.idone + inst, (unsigned)(si + 1));
            }
        }
    }
}

// six linearised moments of one instance (rho, ux, uy, pxx, pxy, pyy per cell), FP64
template <typename T>
__global__ void inst_moments_kernel(const T *h, const BatchInst I, int m, const BatchArgs a, double u_ref, double *out)
{
    const long ncells = I.ncells;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (long)gridDim.x * blockDim.x) {
        const int yc = (int)(c / I.nx), xc = (int)(c - (long)yc * I.nx);
        double s0 = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
        for (int iy = 0; iy < m; ++iy) {
            const double ey = a.xi[iy];
            for (int ix = 0; ix < m; ++ix) {
                const double ex = a.xi[ix];
                const double v = (double)h[inst_index(I, m * m, iy * m + ix, xc, yc)];
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
}

template <typename TS, typename TC, int M, int G, int MODE>
void *kernel_ptr() { return (void *)batch_kernel<TS, TC, M, G, MODE>; }

// A march kernel and its correction-mode twin per (precision, M, warps per segment); the
// FP64 defect pass has one shape per M (any item list runs with any warps per segment).
struct Variant {
    int prec, m, g;
    void *fn, *fn_correct;
    int threads;
};

template <int M, int G>
Variant make_variant()
{
    return {LBM_FP32_PERTURB, M, G, kernel_ptr<float, float, M, G, BATCH_MARCH>(),
            kernel_ptr<float, float, M, G, BATCH_CORRECT>(), lbmk::Shape<G>::THREADS};
}

const std::vector<Variant> &variants()
{
    static const std::vector<Variant> v = {make_variant<8, 1>(), make_variant<8, 2>(), make_variant<8, 4>(),
                                           make_variant<4, 1>(), make_variant<4, 2>()};
    return v;
}

// column-march kernels (cavity instances): M = 4 or 8 nodes per axis, G warps per item
// (one velocity row per warp with G = M, two with G = M / 2, four with G = M / 4); dynamic
// shared memory
struct MarchFns {
    void *march, *correct;
    int g;
    size_t smem;
};

template <int M, int G>
MarchFns march_fns_of()
{
    return {(void *)batch_march_kernel<M, G, BATCH_MARCH>, (void *)batch_march_kernel<M, G, BATCH_CORRECT>, G,
            sizeof(MarchShared<M, G>)};
}

// g <= 0: the default shape, four velocity rows per warp for M = 8 (G = 2: 5-6 % faster
// than two rows on 32 cavities of 128^2 and 8 of 256^2, equal on 128 of 128^2; two rows had
// been 21 % faster than one -- the per-row fixed costs and the moment exchange are shared by
// more updates), two rows for M = 4
MarchFns march_fns(int m, int g = 0)
{
    if (m == 8) return g == 8 ? march_fns_of<8, 8>() : (g == 4 ? march_fns_of<8, 4>() : march_fns_of<8, 2>());
    if (m == 4) return g == 4 ? march_fns_of<4, 4>() : march_fns_of<4, 2>();
    return {nullptr, nullptr, 0, 0};
}

bool march_shape_ok(int m, int g)
{
    return g <= 0 || (m == 8 && (g == 8 || g == 4 || g == 2)) || (m == 4 && (g == 4 || g == 2));
}

struct DefectShape {
    void *fn;
    int g, threads;
};

DefectShape defect_shape(int m)
{
    if (m == 8) return {kernel_ptr<float, double, 8, 4, BATCH_DEFECT>(), 4, lbmk::Shape<4>::THREADS};
    return {kernel_ptr<float, double, 4, 2, BATCH_DEFECT>(), 2, lbmk::Shape<2>::THREADS};
}

const Variant *find_variant(int prec, int m, int g)
{
    for (const auto &v : variants())
        if (v.prec == prec && v.m == m && v.g == g) return &v;
    return nullptr;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct lbm_batch {
    std::vector<lbm_problem> probs;
    std::vector<BatchInst> inst;
    int m, nv, prec;
    std::vector<double> nodes, weights;
    cudaStream_t stream;
    void *base;
    bool owns;
    size_t bytes;
    long total_vals;
    // device pointers
    void *buf[2];
    BatchInst *d_inst;
    BatchItem *d_items;
    MarchItem *d_mitems;        // column-march items (cavity instances when the march is on)
    unsigned char *d_kind;      // [count] 1: cavity instance marched by columns
    bool march;                 // cavity instances by the column-march kernel
    int nmitems, mgrid, mchunk; // march items, their co-resident grid, rows per chunk
    std::vector<int> iitems;    // march items per instance (host copy of d_iitems)
    int mchunk_fixed;           // rows per chunk set by the caller (0: planned per rebuild)
    int mg;                     // warps per march item (0: the default shape)
    std::vector<std::pair<void *, int>> occ;   // resident blocks per SM of each kernel used
    int nsm;
    std::vector<char> live;     // instances in the current item lists (not yet converged)
    double *d_acc, *d_last_r, *d_best;
    int *d_flat;
    long *d_frozen;
    unsigned *d_ifin;     // [ninst] column march: items finished / steps completed in a launch
    unsigned *d_idone;
    int *d_iitems;        // [ninst] column-march items per step
    unsigned *d_bar;
    int *d_err;
    double *d_tab;          // 1-D nodes [LBM_MAX_M] then weights [LBM_MAX_M]
    float *d_scratch;       // warm start: features and predictions of one instance
    // schedule
    int g, blocks_per_sm, order, nitems, nwall;
    int grid;
    const Variant *var;
    long step;
    int resid_every;
    cudaGraphExec_t graph;
    bool graph_ok;
    cudaStream_t cap_stream;   // private capture stream (created on first use)
    long long timeout_cycles;
    // refinement workspace (allocated by the first lbm_batch_refine): the states being
    // refined, the defect, two correction buffers, then per-instance sums and flags
    void *ref_base;
    float *r_h, *r_d, *r_c[2];
    double *r_acc, *r_last, *r_n2;
    long *r_frozen;
    int *r_list;
};

namespace {

lbm_status bfail(lbm_status s, const std::string &m) { return lbm_norms_fail(s, m.c_str()); }

void inst_coeffs(const lbm_problem &p, const std::vector<double> &nodes, BatchInst &I)
{
    double mx = 0;
    for (double v : nodes) mx = std::max(mx, std::fabs(v));
    double dx, dy;
    if (p.geom == LBM_COUETTE) {
        dy = 1.0 / p.ny;
        dx = dy;
    } else {
        dx = 1.0 / p.nx;
        dy = 1.0 / p.ny;
    }
    double rate = mx / dy;
    const bool column = p.geom == LBM_COUETTE && p.nx == 1;
    if (!column) rate += mx / dx;
    double dt = p.cfl / rate;
    if (std::isfinite(p.kn) && dt > p.kn) dt = p.kn;
    I.cx = column ? 0.0 : dt / dx;
    I.cy = dt / dy;
    I.omega = std::isfinite(p.kn) ? dt / p.kn : 0.0;
    I.b = 1.0 - I.omega;
    I.u_bottom = p.u_bottom;
    I.u_top = p.u_top;
    double ur = std::max(std::fabs(p.u_bottom), std::fabs(p.u_top));
    if (ur == 0) ur = 1.0;
    I.inv_u_ref = 1.0 / ur;
    I.nx = p.nx;
    I.ny = p.ny;
    I.cavity = p.geom == LBM_CAVITY;
    I.tiled = I.cavity;
    I.ncells = (long)p.nx * p.ny;
}

// true if the 32-cell segment sg of instance I contains a wall-adjacent cell
bool segment_has_wall(const BatchInst &I, int sg)
{
    for (long c = (long)sg * 32; c < std::min((long)sg * 32 + 32, I.ncells); ++c) {
        const int y = (int)(c / I.nx), x = (int)(c % I.nx);
        if (y == 0 || y == I.ny - 1 || (I.cavity && (x == 0 || x == I.nx - 1))) return true;
    }
    return false;
}

// Build the (instance, segment) lists (wall-free first list, wall second) in one of three
// orders:
//   0: instance by instance, in the given order;
//   1: instances by decreasing size;
//   2: segments interleaved round-robin across instances (largest first).
BatchItem make_item(const BatchInst &I, int inst, int seg)
{
    BatchItem t;
    std::memset(&t, 0, sizeof t);
    t.off = I.off;
    t.ncells = (int)I.ncells;
    t.inst = inst;
    t.seg = seg;
    t.nx = I.nx;
    t.ny = I.ny;
    t.cavity = I.cavity;
    t.cx = (float)I.cx;
    t.cy = (float)I.cy;
    t.omega = (float)I.omega;
    t.b = (float)I.b;
    t.u_bottom = (float)I.u_bottom;
    t.u_top = (float)I.u_top;
    t.drive_bottom = (float)(I.u_bottom * I.inv_u_ref);
    t.drive_top = (float)(I.u_top * I.inv_u_ref);
    return t;
}

bool marched(const lbm_batch *b, int i, bool march) { return march && b->inst[i].cavity; }

void build_items(const lbm_batch *b, int order, bool march, std::vector<BatchItem> &bulk, std::vector<BatchItem> &wall)
{
    const int ni = (int)b->inst.size();
    std::vector<int> idx;
    for (int i = 0; i < ni; ++i)
        if (b->live[i] && !marched(b, i, march)) idx.push_back(i);
    if (order >= 1)
        std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) { return b->inst[p].ncells > b->inst[q].ncells; });
    bulk.clear();
    wall.clear();
    auto add = [&](int i, int sgm) {
        (segment_has_wall(b->inst[i], sgm) ? wall : bulk).push_back(make_item(b->inst[i], i, sgm));
    };
    if (order <= 1) {
        for (int i : idx) {
            const int nseg = (int)((b->inst[i].ncells + 31) / 32);
            for (int sgm = 0; sgm < nseg; ++sgm) add(i, sgm);
        }
    } else {
        int maxseg = 0;
        for (int i : idx) maxseg = std::max(maxseg, (int)((b->inst[i].ncells + 31) / 32));
        for (int sgm = 0; sgm < maxseg; ++sgm)
            for (int i : idx)
                if (sgm < (int)((b->inst[i].ncells + 31) / 32)) add(i, sgm);
    }
}

// Column-march items of the live cavity instances with chunks of about `chunk` rows,
// instance by instance (within an instance chunk by chunk, strips side by side, so that
// neighbouring strips run at about the same time and their x halos are L2 hits): the items
// of a step are taken in this order, so the first instances complete the step first, and the
// warp groups that reach the next step find their instances ready (the kernel waits only for
// an item's own instance).
void build_march_items(const lbm_batch *b, double chunk, std::vector<MarchItem> &out)
{
    out.clear();
    const int ni = (int)b->inst.size();
    std::vector<std::vector<MarchItem>> per(ni);
    for (int i = 0; i < ni; ++i) {
        if (!b->live[i] || !b->inst[i].cavity) continue;
        const BatchInst &I = b->inst[i];
        const int nch = std::max(1, (int)std::lround(I.ny / chunk));   // near-equal chunks of about `chunk` rows
        for (int k = 0; k < nch; ++k)
            for (int x0 = 0; x0 < I.nx; x0 += 32) {
                MarchItem t;
                std::memset(&t, 0, sizeof t);
                t.off = I.off;
                t.inst = i;
                t.nx = I.nx;
                t.ny = I.ny;
                t.x0 = x0;
                t.y0 = (int)((long)I.ny * k / nch);
                t.y1 = (int)((long)I.ny * (k + 1) / nch);
                t.cx = (float)I.cx;
                t.cy = (float)I.cy;
                t.omega = (float)I.omega;
                t.b = (float)I.b;
                t.u_bottom = (float)I.u_bottom;
                t.u_top = (float)I.u_top;
                t.drive_bottom = (float)(I.u_bottom * I.inv_u_ref);
                t.drive_top = (float)(I.u_top * I.inv_u_ref);
                per[i].push_back(t);
            }
    }
    for (int i = 0; i < ni; ++i) out.insert(out.end(), per[i].begin(), per[i].end());
}

// Resident blocks per SM of a kernel of this batch (queried once per kernel) and the SM count.
cudaError_t occupancy(lbm_batch *b, void *fn, int threads, int *nsm, int *blocks, size_t smem = 0)
{
    if (b->nsm == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            b->nsm = 0;
            return e;
        }
    }
    *nsm = b->nsm;
    for (const auto &o : b->occ)
        if (o.first == fn) {
            *blocks = o.second;
            return cudaSuccess;
        }
    cudaError_t e = cudaSuccess;
    if (smem > 0) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
    if (e == cudaSuccess) b->occ.emplace_back(fn, *blocks);
    return e;
}

// Rows per chunk of the column march: items are fetched dynamically, so the chunks only
// have to be many enough to keep the warp groups busy and long enough to amortise an item's
// start (its first rows' copies and the wall prologue).
double march_chunk_plan(const lbm_batch *b, long slots)
{
    long strip_rows = 0;
    int cavities = 0;
    for (int i = 0; i < (int)b->inst.size(); ++i)
        if (b->live[i] && b->inst[i].cavity) {
            strip_rows += (long)((b->inst[i].nx + 31) / 32) * b->inst[i].ny;
            ++cavities;
        }
    // Items per warp group and step: about 1.3 with eight or more cavities, 1.7 with fewer.
    // Items are taken step after step, each waiting only for its own instance's previous
    // step, so a group that finishes early starts the next step's items: fewer, longer
    // items amortise each item's start (its first rows' copies, the wall prologue) as long
    // as every group still has one.  Measured over chunk lengths (ms per step, best against
    // the 1.7 rule): 16 x 128^2 0.0307 / 0.0321, 32 x 128^2 0.0534 / 0.0557, 64 x 128^2
    // 0.1015 / 0.1043, 8 x 256^2 0.0570 / 0.0582.  With few instances the end of each
    // instance's step, where its groups run out of items, costs more than the starts: two
    // 512^2 cavities run best at 1.7 (0.0570 ms; 0.0582 at 1.4).  Each chunk re-reads one
    // row, so chunks stay at least 4 rows.
    const double per_group = cavities >= 8 ? 1.3 : 1.7;
    const double h = (double)strip_rows / (per_group * (double)std::max(1L, slots));
    return std::max(4.0, std::min(128.0, h));
}

lbm_status apply_schedule_march(lbm_batch *b, int g, int bpsm, int order, bool march);

lbm_status apply_schedule(lbm_batch *b, int g, int bpsm, int order)
{
    return apply_schedule_march(b, g, bpsm, order, b->march);
}

lbm_status apply_schedule_march(lbm_batch *b, int g, int bpsm, int order, bool march)
{
    const Variant *v = find_variant(b->prec, b->m, g);
    if (!v) return bfail(LBM_EUNSUPPORTED, "no batched kernel for this precision / velocity set / warps per segment");
    int nsm = 0, maxb = 0, mb = 0;
    cudaError_t e = occupancy(b, v->fn, v->threads, &nsm, &maxb);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (maxb < 1) return bfail(LBM_EUNSUPPORTED, "batched kernel does not fit on an SM");
    if (bpsm < 1 || bpsm > maxb) bpsm = maxb;
    std::vector<BatchItem> items, wall;
    build_items(b, order, march, items, wall);
    std::vector<MarchItem> mitems;
    int mgrid = 0, mchunk = 0;
    const MarchFns mf = march_fns(b->m, b->mg);
    if (march && mf.march) {
        int mbc = 0;
        e = occupancy(b, mf.march, 256, &nsm, &mb, mf.smem);
        if (e == cudaSuccess) e = occupancy(b, mf.correct, 256, &nsm, &mbc, mf.smem);
        if (e != cudaSuccess || mb < 1 || mbc < 1)
            return bfail(LBM_EUNSUPPORTED, "column-march kernel does not fit on an SM");
        mb = std::min(mb, mbc);                // one grid serves the march and the correction
        const int sub = 8 / mf.g;
        const double rows = b->mchunk_fixed > 0 ? (double)b->mchunk_fixed : march_chunk_plan(b, (long)nsm * mb * sub);
        mchunk = (int)std::lround(rows);
        build_march_items(b, rows, mitems);
        mgrid = (int)std::min<long>((long)nsm * mb, std::max<long>(1, ((long)mitems.size() + sub - 1) / sub));
    }
    // stream-ordered uploads (pageable sources are staged before the calls return)
    e = cudaSuccess;
    if (!mitems.empty()) {
        b->iitems.assign(b->inst.size(), 0);
        for (const MarchItem &t : mitems) b->iitems[t.inst] += 1;
        e = cudaMemcpyAsync(b->d_mitems, mitems.data(), sizeof(MarchItem) * mitems.size(), cudaMemcpyHostToDevice,
                            b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_iitems, b->iitems.data(), sizeof(int) * b->iitems.size(), cudaMemcpyHostToDevice,
                                b->stream);
    }
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !wall.empty())
        e = cudaMemcpyAsync(b->d_items + items.size(), wall.data(), sizeof(BatchItem) * wall.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("uploading the schedule: ") + cudaGetErrorString(e));
    if (b->graph_ok) cudaGraphExecDestroy(b->graph);
    b->graph_ok = false;
    b->var = v;
    b->g = g;
    b->blocks_per_sm = bpsm;
    b->order = order;
    b->nitems = (int)items.size();
    b->nwall = (int)wall.size();
    b->nmitems = (int)mitems.size();
    b->mgrid = mgrid;
    b->mchunk = mchunk;
    const int spb = segs_per_block(g);
    const long groups = std::max(((long)b->nitems + spb - 1) / spb, ((long)b->nwall + spb - 1) / spb);
    b->grid = (int)std::min<long>((long)nsm * bpsm, std::max<long>(1, groups));
    return LBM_OK;
}

BatchArgs make_args(const lbm_batch *b, int nsteps, double tol)
{
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.buf[0] = b->buf[0];
    a.buf[1] = b->buf[1];
    a.inst = b->d_inst;
    a.ninst = (int)b->inst.size();
    a.items = b->d_items;
    a.nitems = b->nitems;
    a.wall_items = b->d_items + b->nitems;
    a.nwall = b->nwall;
    a.mitems = b->d_mitems;
    a.nmitems = b->nmitems;
    a.kind = b->d_kind;
    a.acc = b->d_acc;
    a.last_r = b->d_last_r;
    a.best_r = b->d_best;
    a.flat = b->d_flat;
    a.frozen = b->d_frozen;
    a.bar_count = b->d_bar;
    a.bar_gen = b->d_bar + 1;
    a.mcount = b->d_bar + 8;
    a.ifin = b->d_ifin;
    a.idone = b->d_idone;
    a.iitems = b->d_iitems;
    a.err = b->d_err;
    a.step0 = b->step;
    a.nsteps = nsteps;
    a.resid_every = b->resid_every;
    a.tol = tol;
    a.timeout_cycles = b->timeout_cycles;
    double sx = 0, sy = 0;
    const int m = b->m;
    for (int i = 0; i < m; ++i) {
        a.xi[i] = b->nodes[i];
        a.w1[i] = b->weights[i];
        a.xi_f[i] = (float)b->nodes[i];
        a.w1_f[i] = (float)b->weights[i];
    }
    for (int iy = 0; iy < m; ++iy)
        for (int ix = 0; ix < m; ++ix) {
            const double w = b->weights[ix] * b->weights[iy];
            if (b->nodes[ix] > 0) sx += b->nodes[ix] * w;
            if (b->nodes[iy] > 0) sy += b->nodes[iy] * w;
        }
    a.inv_dx_wall = 1.0 / sx;
    a.inv_dy_wall = 1.0 / sy;
    a.inv_dx_wall_f = (float)a.inv_dx_wall;
    a.inv_dy_wall_f = (float)a.inv_dy_wall;
    return a;
}

cudaError_t launch_coop(void *fn, int grid, int threads, const BatchArgs &a, cudaStream_t st, size_t smem = 0)
{
    void *args[] = {(void *)&a};
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// One advance: the column-march kernel over the cavity items, then the segment kernel over
// the other instances' items (each launched only when it has items).
cudaError_t launch_pair(lbm_batch *b, const BatchArgs &a0, void *mfn, void *sfn, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (b->nmitems > 0) {
        BatchArgs a = a0;
        a.kind_sel = 1;
        e = cudaMemsetAsync(a.mcount, 0, 2 * sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.ifin, 0, 2 * sizeof(unsigned) * b->inst.size(), st);
        if (e == cudaSuccess) e = launch_coop(mfn, b->mgrid, 256, a, st, march_fns(b->m, b->mg).smem);
    }
    if (e == cudaSuccess && (b->nitems > 0 || b->nwall > 0)) {
        BatchArgs a = a0;
        a.kind_sel = 0;
        e = launch_coop(sfn, b->grid, b->var->threads, a, st);
    }
    return e;
}

cudaError_t launch_batch(lbm_batch *b, const BatchArgs &a, cudaStream_t st)
{
    return launch_pair(b, a, march_fns(b->m, b->mg).march, b->var->fn, st);
}

// Co-resident grid of a kernel of this batch for the current item lists.
int coop_grid(lbm_batch *b, void *fn, int threads, int g)
{
    int nsm = 0, maxb = 0;
    if (occupancy(b, fn, threads, &nsm, &maxb) != cudaSuccess || maxb < 1) {
        cudaGetLastError();
        return 0;
    }
    const int spb = segs_per_block(g);
    const long groups = std::max(((long)b->nitems + spb - 1) / spb, ((long)b->nwall + spb - 1) / spb);
    return (int)std::min<long>((long)nsm * std::min(maxb, std::max(1, b->blocks_per_sm)), std::max<long>(1, groups));
}

// h[i] += c[parity of instance i's final correction step][i] for the instances in the list
__global__ void batch_apply_kernel(float *h, const float *c0, const float *c1, const BatchInst *inst,
                                   const long *frozen, const int *list, int nv)
{
    const int i = list[blockIdx.y];
    const long n = inst_vals(inst[i], nv), off = inst[i].off;
    const float *c = (frozen[i] & 1) ? c1 : c0;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        h[off + k] += c[off + k];
}

lbm_status refine_alloc(lbm_batch *b)
{
    if (b->ref_base) return LBM_OK;
    const int n = (int)b->inst.size();
    const size_t sb = align256(sizeof(float) * b->total_vals);
    const size_t bytes = 4 * sb + align256(sizeof(double) * 2 * n) + 2 * align256(sizeof(double) * n) +
                         align256(sizeof(long) * n) + align256(sizeof(int) * n);
    cudaError_t e = cudaMalloc(&b->ref_base, bytes);
    if (e != cudaSuccess) {
        b->ref_base = nullptr;
        return bfail(LBM_ENOMEM, std::string("cudaMalloc for the refinement workspace: ") + cudaGetErrorString(e));
    }
    char *p = (char *)b->ref_base;
    b->r_h = (float *)p;
    b->r_d = (float *)(p + sb);
    b->r_c[0] = (float *)(p + 2 * sb);
    b->r_c[1] = (float *)(p + 3 * sb);
    size_t o = 4 * sb;
    b->r_acc = (double *)(p + o);
    o += align256(sizeof(double) * 2 * n);
    b->r_last = (double *)(p + o);
    o += align256(sizeof(double) * n);
    b->r_n2 = (double *)(p + o);
    o += align256(sizeof(double) * n);
    b->r_frozen = (long *)(p + o);
    o += align256(sizeof(long) * n);
    b->r_list = (int *)(p + o);
    return LBM_OK;
}

lbm_status check_err(lbm_batch *b)
{
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("refinement: ") + cudaGetErrorString(e));
    if (err == 1) return bfail(LBM_ETIMEOUT, "a grid barrier of the batched kernel timed out");
    if (err == 2) return bfail(LBM_ENONFINITE, "non-finite residual in the batch");
    return LBM_OK;
}

// Instances in `sel` into the item lists (the schedule otherwise unchanged).
lbm_status select_items(lbm_batch *b, const std::vector<char> &sel, bool march)
{
    b->live = sel;
    return apply_schedule_march(b, b->g, b->blocks_per_sm, b->order, march);
}

// FP64 defect of the states in the workspace for the instances in the item lists:
// r_d = M64(r_h) - r_h (float); per-instance sums ||D||^2 and ||M64(H)||^2 to the host.
lbm_status refine_defect(lbm_batch *b, std::vector<double> &sums)
{
    const int n = (int)b->inst.size();
    std::vector<long> open(n, LONG_MAX);
    BatchArgs a = make_args(b, 1, 0.0);
    a.buf[0] = b->r_h;
    a.buf[1] = b->r_d;
    a.acc = b->r_acc;
    a.last_r = b->r_last;
    a.best_r = nullptr;          // the refinement keeps its own stagnation rule
    a.flat = nullptr;
    a.frozen = b->r_frozen;
    a.step0 = 0;
    const DefectShape ds = defect_shape(b->m);
    const int grid = coop_grid(b, ds.fn, ds.threads, ds.g);
    if (grid < 1) return bfail(LBM_EUNSUPPORTED, "defect kernel does not fit on an SM");
    cudaError_t e = cudaMemsetAsync(b->r_acc, 0, sizeof(double) * 2 * n, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->r_frozen, open.data(), sizeof(long) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && (b->nitems > 0 || b->nwall > 0)) e = launch_coop(ds.fn, grid, ds.threads, a, b->stream);
    sums.assign(2 * n, 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums.data(), b->r_acc, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("defect pass of the batch: ") + cudaGetErrorString(e));
    return check_err(b);
}

}  // namespace

extern "C" {

lbm_status lbm_batch_bytes(const lbm_vset *vs, const lbm_problem *insts, int count, size_t *bytes);
lbm_status lbm_batch_init(const lbm_vset *vs, const lbm_problem *insts, int count, void *device_buf,
                          size_t buf_bytes, void *stream, lbm_batch **out);

static lbm_status batch_layout(const lbm_vset *vs, const lbm_problem *insts, int count, int *prec,
                               long *total_vals, long *total_segs, long *total_mitems, size_t *bytes)
{
    int nv = 0, m = 0;
    lbm_status st = lbm_vset_query(vs, &nv, &m, nullptr, nullptr, nullptr);
    if (st != LBM_OK) return st;
    if (!insts || count < 1) return bfail(LBM_EINVAL, "batch needs at least one instance");
    const int p0 = insts[0].prec;
    long vals = 0, segs = 0, mits = 0;
    for (int i = 0; i < count; ++i) {
        size_t one;
        st = lbm_sim_bytes(vs, &insts[i], &one);   // validates the instance
        if (st != LBM_OK) return st;
        if (insts[i].prec != p0) return bfail(LBM_EINVAL, "all batch instances must share the precision");
        if (insts[i].residual_every != insts[0].residual_every)
            return bfail(LBM_EINVAL, "all batch instances must share residual_every");
        const long nc = (long)insts[i].nx * insts[i].ny;
        vals += insts[i].geom == LBM_CAVITY ? (long)((insts[i].nx + 31) / 32) * insts[i].ny * nv * 32 : (long)nv * nc;
        segs += (nc + 31) / 32;
        if (insts[i].geom == LBM_CAVITY)     // column-march items: chunks of at least 4 rows
            mits += (long)((insts[i].nx + 31) / 32) * ((insts[i].ny + 3) / 4);
    }
    if (p0 != LBM_FP32_PERTURB || !find_variant(p0, m, 1))
        return bfail(LBM_EUNSUPPORTED, "batched kernels exist for FP32 with 4 or 8 nodes per axis");
    const size_t es = p0 == LBM_FP64 ? 8 : 4;
    size_t off = 0;
    off = align256(off + vals * es);          // buffer 0
    off = align256(off + vals * es);          // buffer 1
    off = align256(off + sizeof(BatchInst) * count);
    off = align256(off + sizeof(BatchItem) * segs);
    off = align256(off + sizeof(MarchItem) * std::max(1L, mits));
    off = align256(off + (size_t)count);                        // instance kinds
    off = align256(off + sizeof(double) * 2 * count);
    off = align256(off + sizeof(double) * count);     // last residual
    off = align256(off + sizeof(double) * count);     // best residual
    off = align256(off + sizeof(int) * count);        // checks without improvement
    off = align256(off + sizeof(long) * count);
    off = align256(off + sizeof(unsigned) * 3 * count);        // march completion counters, items per step
    off = align256(off + 64);
    off = align256(off + sizeof(double) * 2 * LBM_MAX_M);      // 1-D nodes and weights
    long maxc = 0;
    for (int i = 0; i < count; ++i) maxc = std::max(maxc, (long)insts[i].nx * insts[i].ny);
    off = align256(off + 40 * (size_t)maxc);                    // warm-start scratch
    *prec = p0;
    *total_vals = vals;
    *total_segs = segs;
    *total_mitems = mits;
    *bytes = off;
    return LBM_OK;
}

lbm_status lbm_batch_bytes(const lbm_vset *vs, const lbm_problem *insts, int count, size_t *bytes)
{
    if (!bytes) return bfail(LBM_EINVAL, "bytes is NULL");
    int prec;
    long vals, segs, mits;
    return batch_layout(vs, insts, count, &prec, &vals, &segs, &mits, bytes);
}

lbm_status lbm_batch_init(const lbm_vset *vs, const lbm_problem *insts, int count, void *device_buf,
                          size_t buf_bytes, void *stream, lbm_batch **out)
{
    if (!out) return bfail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int prec;
    long vals, segs, mits;
    size_t bytes;
    lbm_status st = batch_layout(vs, insts, count, &prec, &vals, &segs, &mits, &bytes);
    if (st != LBM_OK) return st;
    if (device_buf && buf_bytes < bytes) return bfail(LBM_ENOMEM, "device buffer too small for the batch");
    if (device_buf && ((uintptr_t)device_buf & 255)) return bfail(LBM_EINVAL, "device buffer must be 256-byte aligned");
    lbm_batch *b = new (std::nothrow) lbm_batch;
    if (!b) return bfail(LBM_ENOMEM, "host allocation failed");
    int nv = 0, m = 0;
    lbm_vset_query(vs, &nv, &m, nullptr, nullptr, nullptr);
    std::vector<double> xx(nv), yy(nv), ww(nv);
    lbm_vset_query(vs, nullptr, nullptr, xx.data(), yy.data(), ww.data());
    b->m = m;
    b->nv = nv;
    b->prec = prec;
    b->nodes.assign(xx.begin(), xx.begin() + m);
    b->weights.resize(m);
    // 1-D weights from the tensor product: w[ix] = w(ix, iy0) / w1[iy0], w1 from the row sums
    for (int ix = 0; ix < m; ++ix) {
        double col = 0;
        for (int iy = 0; iy < m; ++iy) col += ww[iy * m + ix];
        b->weights[ix] = col;
    }
    b->probs.assign(insts, insts + count);
    b->inst.resize(count);
    b->live.assign(count, 1);
    long off = 0;
    for (int i = 0; i < count; ++i) {
        inst_coeffs(insts[i], b->nodes, b->inst[i]);
        b->inst[i].off = off;
        off += inst_vals(b->inst[i], nv);
    }
    b->stream = (cudaStream_t)stream;
    b->owns = device_buf == nullptr;
    b->bytes = bytes;
    b->total_vals = vals;
    b->step = 0;
    b->resid_every = insts[0].residual_every;
    b->graph_ok = false;
    b->cap_stream = nullptr;
    b->timeout_cycles = 4000000000LL;   // about 2 s at the GB300 SM clock
    b->ref_base = nullptr;
    b->march = march_fns(m).march != nullptr;
    b->nmitems = b->mgrid = b->mchunk = 0;
    b->nsm = 0;
    b->mchunk_fixed = 0;
    b->mg = 0;
    if (b->owns) {
        cudaError_t e = cudaMalloc(&b->base, bytes);
        if (e != cudaSuccess) {
            delete b;
            return bfail(LBM_ENOMEM, std::string("cudaMalloc for the batch: ") + cudaGetErrorString(e));
        }
    } else {
        b->base = device_buf;
    }
    const size_t es = prec == LBM_FP64 ? 8 : 4;
    char *p = (char *)b->base;
    size_t o = 0;
    b->buf[0] = p + o;
    o = align256(o + vals * es);
    b->buf[1] = p + o;
    o = align256(o + vals * es);
    b->d_inst = (BatchInst *)(p + o);
    o = align256(o + sizeof(BatchInst) * count);
    b->d_items = (BatchItem *)(p + o);
    o = align256(o + sizeof(BatchItem) * segs);
    b->d_mitems = (MarchItem *)(p + o);
    o = align256(o + sizeof(MarchItem) * std::max(1L, mits));
    b->d_kind = (unsigned char *)(p + o);
    o = align256(o + (size_t)count);
    b->d_acc = (double *)(p + o);
    o = align256(o + sizeof(double) * 2 * count);
    b->d_last_r = (double *)(p + o);
    o = align256(o + sizeof(double) * count);
    b->d_best = (double *)(p + o);
    o = align256(o + sizeof(double) * count);
    b->d_flat = (int *)(p + o);
    o = align256(o + sizeof(int) * count);
    b->d_frozen = (long *)(p + o);
    o = align256(o + sizeof(long) * count);
    b->d_ifin = (unsigned *)(p + o);
    b->d_idone = b->d_ifin + count;
    b->d_iitems = (int *)(b->d_ifin + 2 * count);
    o = align256(o + sizeof(unsigned) * 3 * count);
    b->d_bar = (unsigned *)(p + o);
    b->d_err = (int *)(p + o + 16);
    o = align256(o + 64);
    b->d_tab = (double *)(p + o);
    o = align256(o + sizeof(double) * 2 * LBM_MAX_M);
    b->d_scratch = (float *)(p + o);
    std::vector<long> frozen(count, LONG_MAX);
    std::vector<double> last(count, INFINITY);
    cudaError_t e = cudaMemsetAsync(b->buf[0], 0, vals * es, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[1], 0, vals * es, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_acc, 0, sizeof(double) * 2 * count, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_last_r, last.data(), sizeof(double) * count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_best, last.data(), sizeof(double) * count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flat, 0, sizeof(int) * count, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_frozen, frozen.data(), sizeof(long) * count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 64, b->stream);
    std::vector<unsigned char> kind(count);
    for (int i = 0; i < count; ++i) kind[i] = marched(b, i, b->march) ? 1 : 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_kind, kind.data(), count, cudaMemcpyHostToDevice, b->stream);
    std::vector<double> tab(2 * LBM_MAX_M, 0.0);
    for (int k = 0; k < m; ++k) {
        tab[k] = b->nodes[k];
        tab[LBM_MAX_M + k] = b->weights[k];
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return bfail(LBM_ECUDA, std::string("initialising the batch: ") + cudaGetErrorString(e));
    }
    st = apply_schedule(b, b->m == 8 ? 4 : 2, 0, 2);
    if (st != LBM_OK) {
        lbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->graph_ok) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ref_base) cudaFree(b->ref_base);
    if (b->owns && b->base) cudaFree(b->base);
    delete b;
}

lbm_status lbm_batch_set_schedule(lbm_batch *b, int warps_per_segment, int blocks_per_sm, int order)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (order < 0 || order > 2) return bfail(LBM_EINVAL, "order must be 0, 1 or 2");
    return apply_schedule(b, warps_per_segment, blocks_per_sm, order);
}

lbm_status lbm_batch_set_march(lbm_batch *b, int on, int rows_per_chunk, int warps_per_item)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (on && !march_fns(b->m).march) return bfail(LBM_EUNSUPPORTED, "no column-march kernel for this velocity set");
    if (rows_per_chunk != 0 && rows_per_chunk < 4) return bfail(LBM_EINVAL, "rows per chunk must be 0 or >= 4");
    if (!march_shape_ok(b->m, warps_per_item))
        return bfail(LBM_EINVAL, "warps per march item must be 0, M or M / 2 (M = 4 or 8)");
    b->march = on != 0;
    b->mchunk_fixed = rows_per_chunk;
    b->mg = warps_per_item;
    const int n = (int)b->inst.size();
    std::vector<unsigned char> kind(n);
    for (int i = 0; i < n; ++i) kind[i] = marched(b, i, b->march) ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync(b->d_kind, kind.data(), n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("setting the march: ") + cudaGetErrorString(e));
    return apply_schedule(b, b->g, b->blocks_per_sm, b->order);
}

lbm_status lbm_batch_get_march(const lbm_batch *b, int *on, int *rows_per_chunk, int *items, int *grid,
                               int *warps_per_item)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (on) *on = b->march;
    if (warps_per_item) *warps_per_item = march_fns(b->m, b->mg).g;
    if (rows_per_chunk) *rows_per_chunk = b->mchunk;
    if (items) *items = b->nmitems;
    if (grid) *grid = b->mgrid;
    return LBM_OK;
}

lbm_status lbm_batch_get_schedule(const lbm_batch *b, int *warps_per_segment, int *blocks_per_sm, int *order,
                                  int *grid)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (warps_per_segment) *warps_per_segment = b->g;
    if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
    if (order) *order = b->order;
    if (grid) *grid = b->grid;
    return LBM_OK;
}

lbm_status lbm_batch_set_timeout(lbm_batch *b, long long cycles)
{
    if (!b || cycles < 1) return bfail(LBM_EINVAL, "invalid timeout");
    b->timeout_cycles = cycles;
    return LBM_OK;
}

lbm_status lbm_batch_advance(lbm_batch *b, int nsteps, double tol)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (nsteps < 1 || !(tol >= 0)) return bfail(LBM_EINVAL, "nsteps must be >= 1 and tol >= 0");
    BatchArgs a = make_args(b, nsteps, tol);
    cudaError_t e;
    // the graph holds the launch arguments by value: re-capture whenever they change
    // (the start step does; the executable graph is updated in place).  The capture runs
    // on a stream private to the batch (a caller's stream may be shared with other
    // threads, whose work would otherwise land in the graph); the launch on the caller's.
    if (b->stream) {
        cudaGraph_t g = nullptr;
        e = cudaSuccess;
        if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) b->cap_stream = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = launch_batch(b, a, b->cap_stream);
            e = cudaStreamEndCapture(b->cap_stream, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) {
            if (b->graph_ok) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(b->graph, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(b->graph);
                    b->graph_ok = false;
                }
            }
            if (!b->graph_ok) {
                e = cudaGraphInstantiate(&b->graph, g, 0);
                if (e == cudaSuccess) b->graph_ok = true;
            }
        }
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) {        // fall back to a direct cooperative launch
            cudaGetLastError();
            e = launch_batch(b, a, b->stream);
        }
    } else {
        e = launch_batch(b, a, b->stream);
    }
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("launching the batched kernel: ") + cudaGetErrorString(e));
    b->step += nsteps;
    return LBM_OK;
}

lbm_status lbm_batch_reset(lbm_batch *b)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    const int n = (int)b->inst.size();
    const size_t es = b->prec == LBM_FP64 ? 8 : 4;
    std::vector<long> frozen(n, LONG_MAX);
    std::vector<double> last(n, INFINITY);
    cudaError_t e = cudaMemsetAsync(b->buf[0], 0, b->total_vals * es, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[1], 0, b->total_vals * es, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_acc, 0, sizeof(double) * 2 * n, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_last_r, last.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_best, last.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flat, 0, sizeof(int) * n, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_frozen, frozen.data(), sizeof(long) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 64, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("resetting the batch: ") + cudaGetErrorString(e));
    b->step = 0;
    if (std::count(b->live.begin(), b->live.end(), 0) > 0) {
        b->live.assign(n, 1);
        return apply_schedule(b, b->g, b->blocks_per_sm, b->order);
    }
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int steps_per_trial, int *best_g, int *best_bpsm, int *best_order,
                          double *best_ms_per_step)
{
    if (!b || steps_per_trial < 1) return bfail(LBM_EINVAL, "invalid tuning arguments");
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
        return bfail(LBM_ECUDA, "creating timing events");
    double best = INFINITY;
    int bg = b->g, bb = b->blocks_per_sm, bo = b->order;
    for (const auto &v : variants()) {
        if (v.prec != b->prec || v.m != b->m) continue;
        int maxb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, v.fn, v.threads, 0) != cudaSuccess) continue;
        for (int bpsm = 1; bpsm <= maxb; ++bpsm) {
            for (int order = 0; order <= 2; ++order) {
                if (apply_schedule(b, v.g, bpsm, order) != LBM_OK) continue;
                lbm_status st = lbm_batch_advance(b, 2, 0.0);      // warm-up (and graph capture)
                if (st != LBM_OK) continue;
                cudaEventRecord(t0, b->stream);
                st = lbm_batch_advance(b, steps_per_trial, 0.0);
                cudaEventRecord(t1, b->stream);
                if (st != LBM_OK || cudaEventSynchronize(t1) != cudaSuccess) continue;
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                int n_active;
                long step;
                if (lbm_batch_poll(b, &n_active, &step) != LBM_OK) {
                    cudaEventDestroy(t0);
                    cudaEventDestroy(t1);
                    return LBM_ETIMEOUT;
                }
                const double per = ms / steps_per_trial;
                if (per < best) {
                    best = per;
                    bg = v.g;
                    bb = bpsm;
                    bo = order;
                }
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    lbm_status st = apply_schedule(b, bg, bb, bo);
    if (st == LBM_OK) st = lbm_batch_reset(b);
    if (st != LBM_OK) return st;
    if (best_g) *best_g = bg;
    if (best_bpsm) *best_bpsm = bb;
    if (best_order) *best_order = bo;
    if (best_ms_per_step) *best_ms_per_step = best;
    return LBM_OK;
}

lbm_status lbm_batch_poll(lbm_batch *b, int *n_active, long *step)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    const int n = (int)b->inst.size();
    std::vector<long> frozen(n);
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(frozen.data(), b->d_frozen, sizeof(long) * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("polling the batch: ") + cudaGetErrorString(e));
    if (err == 1) return bfail(LBM_ETIMEOUT, "a grid barrier of the batched kernel timed out");
    if (err == 2) return bfail(LBM_ENONFINITE, "non-finite residual in the batch");
    int act = 0;
    bool changed = false;
    for (int i = 0; i < n; ++i) {
        const char l = frozen[i] == LONG_MAX;
        act += l;
        changed |= l != b->live[i];
    }
    if (n_active) *n_active = act;
    if (step) *step = b->step;
    // drop the items of instances that converged since the lists were built
    if (changed && act > 0) {
        for (int i = 0; i < n; ++i) b->live[i] = frozen[i] == LONG_MAX;
        return apply_schedule(b, b->g, b->blocks_per_sm, b->order);
    }
    return LBM_OK;
}

lbm_status lbm_batch_status(lbm_batch *b, int i, long *steps, double *residual, int *converged)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (i < 0 || i >= (int)b->inst.size()) return bfail(LBM_EINVAL, "instance index out of range");
    long f;
    double r;
    int flat = 0;
    cudaError_t e = cudaMemcpyAsync(&f, b->d_frozen + i, sizeof(long), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, b->d_last_r + i, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flat, b->d_flat + i, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("reading instance status: ") + cudaGetErrorString(e));
    if (steps) *steps = f == LONG_MAX ? b->step : f;
    if (residual) *residual = r;
    // frozen by the tolerance (the stagnation rule freezes at its 20th flat check and leaves
    // that count in place; a freeze by the tolerance happens with fewer)
    if (converged) *converged = f != LONG_MAX && flat < 20;
    return LBM_OK;
}

lbm_status lbm_batch_stalled(lbm_batch *b, int i, int *stalled)
{
    if (!b || !stalled) return bfail(LBM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) return bfail(LBM_EINVAL, "instance index out of range");
    long f;
    int flat = 0;
    cudaError_t e = cudaMemcpyAsync(&f, b->d_frozen + i, sizeof(long), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flat, b->d_flat + i, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("reading instance status: ") + cudaGetErrorString(e));
    *stalled = f != LONG_MAX && flat >= 20;
    return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch *b, int i, double *out_dev)
{
    if (!b || !out_dev) return bfail(LBM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) return bfail(LBM_EINVAL, "instance index out of range");
    long steps;
    lbm_status st = lbm_batch_status(b, i, &steps, nullptr, nullptr);
    if (st != LBM_OK) return st;
    const BatchArgs a = make_args(b, 1, 0.0);
    const BatchInst &I = b->inst[i];
    const int nb = (int)std::min<long>(1216, (I.ncells + 255) / 256);
    const float *h = (const float *)b->buf[steps & 1] + I.off;
    inst_moments_kernel<float><<<nb, 256, 0, b->stream>>>(h, I, b->m, a, 1.0 / I.inv_u_ref, out_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : bfail(LBM_ECUDA, std::string("instance moments: ") + cudaGetErrorString(e));
}

lbm_status lbm_batch_set_state(lbm_batch *b, int i, const double *h)
{
    if (!b || !h) return bfail(LBM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) return bfail(LBM_EINVAL, "instance index out of range");
    if (b->step != 0) return bfail(LBM_EINVAL, "initial states can be set before the first advance only");
    const BatchInst &I = b->inst[i];
    const long n = inst_vals(I, b->nv);
    std::vector<float> tmp(n, 0.f);
    for (int a = 0; a < b->nv; ++a)              // host order [n][ny][nx] into the instance's layout
        for (int y = 0; y < I.ny; ++y)
            for (int x = 0; x < I.nx; ++x)
                tmp[inst_index(I, b->nv, a, x, y)] = (float)h[((long)a * I.ny + y) * I.nx + x];
    cudaError_t e = cudaMemcpyAsync((float *)b->buf[0] + I.off, tmp.data(), sizeof(float) * n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? LBM_OK : bfail(LBM_ECUDA, std::string("setting an instance state: ") + cudaGetErrorString(e));
}

lbm_status lbm_batch_warm_start(lbm_batch *b, int i, lbm_mlp *mlp, double kn, double u_w)
{
    if (!b || !mlp) return bfail(LBM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) return bfail(LBM_EINVAL, "instance index out of range");
    if (b->step != 0) return bfail(LBM_EINVAL, "initial states can be set before the first advance only");
    const BatchInst &I = b->inst[i];
    if (!I.cavity) return bfail(LBM_EINVAL, "the warm-start network is trained on cavities");
    float *feat = b->d_scratch, *pred = b->d_scratch + 4 * I.ncells;
    lbm_status st = lbm_mlp_features(mlp, I.nx, I.ny, kn, u_w, feat);
    if (st == LBM_OK) st = lbm_mlp_forward(mlp, feat, (int)I.ncells, pred);
    if (st != LBM_OK) return st;
    // the MLP runs on its own stream: order the reconstruction after it
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = launch_warm_state(pred, I.nx, I.ny, I.ncells, I.nx, b->m, b->d_tab, b->d_tab + LBM_MAX_M,
                              u_w * I.inv_u_ref, (float *)b->buf[0] + I.off, LBM_FP32_PERTURB, b->stream,
                              I.tiled != 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? LBM_OK : bfail(LBM_ECUDA, std::string("warm start of an instance: ") + cudaGetErrorString(e));
}

lbm_status lbm_batch_get_state(lbm_batch *b, int i, double *h)
{
    if (!b || !h) return bfail(LBM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) return bfail(LBM_EINVAL, "instance index out of range");
    long steps;
    lbm_status st = lbm_batch_status(b, i, &steps, nullptr, nullptr);
    if (st != LBM_OK) return st;
    const BatchInst &I = b->inst[i];
    const long n = inst_vals(I, b->nv);
    const int par = (int)(steps & 1);
    // batches are FP32 (lbm_batch_init refuses FP64)
    std::vector<float> tmp(n);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), (float *)b->buf[par] + I.off, sizeof(float) * n,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess)                         // the instance's layout into host order [n][ny][nx]
        for (int a = 0; a < b->nv; ++a)
            for (int y = 0; y < I.ny; ++y)
                for (int x = 0; x < I.nx; ++x)
                    h[((long)a * I.ny + y) * I.nx + x] = tmp[inst_index(I, b->nv, a, x, y)];
    return e == cudaSuccess ? LBM_OK : bfail(LBM_ECUDA, std::string("reading instance state: ") + cudaGetErrorString(e));
}

lbm_status lbm_batch_refine(lbm_batch *b, double tol, int max_sweeps, double refine_tol, long max_steps,
                            lbm_batch_refine_info *info)
{
    if (!b) return bfail(LBM_EINVAL, "batch is NULL");
    if (!(tol > 0) || max_sweeps < 0 || max_steps < 1 || refine_tol < 0)
        return bfail(LBM_EINVAL, "invalid refinement arguments");
    const int n = (int)b->inst.size();
    lbm_status st = refine_alloc(b);
    if (st != LBM_OK) return st;
    // the step each instance stands at (its state is in buffer step & 1), into the workspace
    std::vector<long> fro(n), at(n);
    cudaError_t e = cudaMemcpyAsync(fro.data(), b->d_frozen, sizeof(long) * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        at[i] = fro[i] == LONG_MAX ? b->step : fro[i];
        const size_t bytes = sizeof(float) * inst_vals(b->inst[i], b->nv);
        e = cudaMemcpyAsync(b->r_h + b->inst[i].off, (const float *)b->buf[at[i] & 1] + b->inst[i].off, bytes,
                            cudaMemcpyDeviceToDevice, b->stream);
    }
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("refinement: ") + cudaGetErrorString(e));
    const std::vector<char> live0 = b->live;
    std::vector<double> sums, r64(n, 0.0), n2(n, 0.0);
    std::vector<int> sweeps(n, 0);
    std::vector<long> csteps(n, 0);
    std::vector<char> todo(n, 1);
    auto restore = [&](lbm_status s0) {
        lbm_status s1 = select_items(b, live0, b->march);
        return s0 != LBM_OK ? s0 : s1;
    };
    st = select_items(b, todo, false);      // the FP64 defect pass runs on segment items
    if (st == LBM_OK) st = refine_defect(b, sums);
    if (st != LBM_OK) return restore(st);
    for (int i = 0; i < n; ++i) {
        n2[i] = sums[2 * i + 1];
        r64[i] = n2[i] > 0 ? std::sqrt(sums[2 * i] / n2[i]) : 0.0;
        todo[i] = max_sweeps > 0 && n2[i] > 0 && r64[i] >= tol;
    }
    const double ctol = refine_tol > 0 ? refine_tol : 0.1 * tol;
    const int every = std::max(1, b->resid_every);
    const int chunk = 5 * every;
    const size_t state_bytes = sizeof(float) * b->total_vals;
    std::vector<double> last(n);
    std::vector<int> list;
    while (std::count(todo.begin(), todo.end(), 1) > 0) {
        // --- correction march delta <- L(delta) + D from delta = 0, all open instances at once ---
        std::vector<char> open = todo;
        for (int i = 0; i < n; ++i) fro[i] = todo[i] ? LONG_MAX : 0;
        std::vector<double> best(n, INFINITY);
        std::vector<int> flat(n, 0);
        st = select_items(b, open, b->march);
        if (st != LBM_OK) return restore(st);
        e = cudaMemsetAsync(b->r_c[0], 0, state_bytes, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->r_acc, 0, sizeof(double) * 2 * n, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->r_n2, n2.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->r_frozen, fro.data(), sizeof(long) * n, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return restore(bfail(LBM_ECUDA, std::string("refinement: ") + cudaGetErrorString(e)));
        long k = 0;
        for (;;) {
            BatchArgs a = make_args(b, chunk, ctol);
            a.buf[0] = b->r_c[0];
            a.buf[1] = b->r_c[1];
            a.src = b->r_d;
            a.ref_n2 = b->r_n2;
            a.acc = b->r_acc;
            a.last_r = b->r_last;
    a.best_r = nullptr;          // the refinement keeps its own stagnation rule
    a.flat = nullptr;
            a.frozen = b->r_frozen;
            a.step0 = k;
            e = launch_pair(b, a, march_fns(b->m, b->mg).correct, b->var->fn_correct, b->stream);
            k += chunk;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(fro.data(), b->r_frozen, sizeof(long) * n, cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(last.data(), b->r_last, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess)
                return restore(bfail(LBM_ECUDA, std::string("correction march of the batch: ") + cudaGetErrorString(e)));
            st = check_err(b);
            if (st != LBM_OK) return restore(st);
            // converged instances leave the lists; those whose change has not improved by 1 %
            // over 20 residual checks (the FP32 rounding floor), or that reached max_steps,
            // are stopped at the current step
            bool changed = false, forced = false;
            for (int i = 0; i < n; ++i) {
                if (!open[i]) continue;
                if (fro[i] != LONG_MAX) {
                    open[i] = 0;
                    changed = true;
                    continue;
                }
                if (last[i] < 0.99 * best[i]) {
                    best[i] = last[i];
                    flat[i] = 0;
                } else {
                    flat[i] += chunk / every;
                }
                if (flat[i] >= 20 || k >= max_steps) {
                    fro[i] = k;
                    open[i] = 0;
                    changed = forced = true;
                }
            }
            if (forced) {
                e = cudaMemcpyAsync(b->r_frozen, fro.data(), sizeof(long) * n, cudaMemcpyHostToDevice, b->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
                if (e != cudaSuccess) return restore(bfail(LBM_ECUDA, std::string("refinement: ") + cudaGetErrorString(e)));
            }
            if (std::count(open.begin(), open.end(), 1) == 0) break;
            if (changed) {
                st = select_items(b, open, b->march);
                if (st != LBM_OK) return restore(st);
            }
        }
        // --- h += delta, then the FP64 defect of the corrected states ---
        list.clear();
        long maxv = 0;
        for (int i = 0; i < n; ++i)
            if (todo[i]) {
                list.push_back(i);
                csteps[i] += fro[i];
                sweeps[i] += 1;
                maxv = std::max(maxv, inst_vals(b->inst[i], b->nv));
            }
        e = cudaMemcpyAsync(b->r_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) {
            const int bx = (int)std::min<long>(1024, (maxv + 1023) / 1024);
            batch_apply_kernel<<<dim3(bx, (unsigned)list.size()), 256, 0, b->stream>>>(
                b->r_h, b->r_c[0], b->r_c[1], b->d_inst, b->r_frozen, b->r_list, b->nv);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return restore(bfail(LBM_ECUDA, std::string("applying the corrections: ") + cudaGetErrorString(e)));
        st = select_items(b, todo, false);
        if (st == LBM_OK) st = refine_defect(b, sums);
        if (st != LBM_OK) return restore(st);
        for (int i : list) {
            const double prev = r64[i];
            r64[i] = sums[2 * i + 1] > 0 ? std::sqrt(sums[2 * i] / sums[2 * i + 1]) : 0.0;
            // done below tol, at the FP32 rounding floor (the defect stopped halving), or
            // after max_sweeps
            if (r64[i] < tol || r64[i] > 0.5 * prev || sweeps[i] >= max_sweeps) todo[i] = 0;
        }
    }
    // refined states back to the buffer each instance's step points at
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        if (sweeps[i] > 0)
            e = cudaMemcpyAsync((float *)b->buf[at[i] & 1] + b->inst[i].off, b->r_h + b->inst[i].off,
                                sizeof(float) * inst_vals(b->inst[i], b->nv), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return restore(bfail(LBM_ECUDA, std::string("refinement: ") + cudaGetErrorString(e)));
    if (info)
        for (int i = 0; i < n; ++i) {
            info[i].correction_steps = csteps[i];
            info[i].sweeps = sweeps[i];
            info[i].defect = r64[i];
        }
    return restore(LBM_OK);
}

}  // extern "C"
