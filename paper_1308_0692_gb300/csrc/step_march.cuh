// Interior of the FP32 step as a column march with TMA staging (sm_103a).
//
// The same update as the bulk path of step_kernel.cuh (first-order upwind transport, then
// relaxation towards w_a (rho' + xi_a . j'), Eqs. 5-7 with the scheme's discretisation),
// organised so that every value of the old state crosses the L2 -> SM path about once:
//
//   * A block owns a strip of 64 cells in x (lane = 2 neighbouring cells, packed FP32x2
//     arithmetic along x) and marches it row by row through a chunk of rows.  Its G warps
//     split the M velocity rows iy as in the segment kernels (warp g owns M/G rows, all
//     with the same sign of xi_y).
//   * Per row and velocity the warp copies one 288-byte line (the 64 cells and 4 cells of
//     x halo on each side) into shared memory with a 1-D bulk asynchronous copy
//     (cp.async.bulk ... mbarrier::complete_tx).  A ring of S row slots per warp keeps the
//     rows y-1, y, y+1 resident, so the upwind y neighbour of row y is a line that was
//     copied for row y-1 or y+1 anyway: no second read of it, unlike the segment kernels
//     (which read every line twice: once as own cells, once as a neighbour row).  S-2 rows
//     of copies stay in flight ahead of the arithmetic; with S = 2 none do, and two blocks
//     share an SM instead.
//   * The interior is cut into items (strip, chunk of rows), numbered chunk-major so that
//     blocks running at the same time work on neighbouring strips of the same rows (their
//     x halos are then L2 hits).  The grid is persistent (one or more blocks per SM); a
//     block's first three items are fixed (b, grid + b, 2 grid + b), later ones come from
//     an atomic counter as blocks finish items, and the copies of a block's next item are
//     issued while it finishes the current one.  The last block to finish resets the
//     counter for the next launch.
//
// Cells covered: x in [32, nx - 32), y in [1, ny - 2]; the wall kernel handles the rest
// (rows 0 and ny-1 and the 32-cell segments at x = 0 and x = nx - 32 of every inner row,
// exactly the wall-segment list when nx is a multiple of 32).  Host-checked requirements:
// FP32 state, cavity, nx a multiple of 64 and at least 128, chunks at least S rows long.
//
// Every wait on a copy is bounded: after the limit the warp sets the status word and a
// block-wide abort flag, all warps leave the march at the next row barrier, wait (again
// bounded) for the copies they still have in flight, and return.
//
// TILED (load path 8): the state is strip-tiled (lbm_internal.h): tile t holds x in
// [64 t - 32, 64 t + 32) as [y][a][64], so the march's strip s is exactly tile s + 1 and one
// row of it, all n velocities, is one contiguous stretch of n * 256 bytes.  Per row a warp
// then copies its NV velocity lines with ONE bulk copy of NV * 256 contiguous bytes; the
// upwind x halo of each velocity (the last cell of the left tile for xi_x > 0, the first
// cell of the right tile for xi_x < 0; those tiles' rows are being marched by the
// neighbouring blocks at about the same time, so these reads are mostly L2 hits) comes with
// one 4-byte asynchronous copy per lane (cp.async, the load/store unit's path: as bulk
// copies of 16 bytes, 24 per warp and row, they held the copy engine to 0.78 of the copy
// rate), whose completion the same mbarrier tracks (cp.async.mbarrier.arrive.noinc; the
// barrier expects 1 + NV arrivals).  Every DRAM access of the march is then part of a long
// contiguous stream instead of 144 separate 288-byte lines from planes 16.8 MB apart.
// With TILED = 2 (load path 9) the stores go the same way: each warp writes its relaxed row
// (NV lines, contiguous in the tiled layout) into a staging buffer in shared memory and one
// lane hands it to the copy engine as a single bulk asynchronous store
// (cp.async.bulk.global.shared::cta), so the warps issue no global store instructions; the
// staging buffer is reused only after the previous row's store has read it
// (cp.async.bulk.wait_group.read), and every store has completed before the block exits.
//
// ORDER = 2 (the second-order transport of step_so.cuh on the strip-tiled state): the
// march covers x in [32, nx - 32), y in [2, ny - 3], where no face flux reaches a wall, so
// every cell takes the plain upwind-biased (Beam-Warming) flux difference.  A warp reads
// its own row and its two upwind rows (an item copies its rows and the two upwind rows
// below or above it; ring of S >= 4 slots, S - 3 rows in flight), and the halo copy of each
// velocity is the pair of cells next to the strip on the upwind side (one 8-byte cp.async).
// The wall kernel beside it then covers rows 0, 1, ny - 2, ny - 1 and the side segments.
#pragma once

#include <cstdint>
#include <cstring>

#include "step_tma.cuh"

namespace lbmk {

template <int M, int G, int S, int TILED = 0>
struct MarchShape {
    static constexpr int RPL = M / G;              // velocity rows per warp
    static constexpr int NV = RPL * M;             // velocities per warp
    // planar: floats per staged line (64 + 4 + 4); tiled: dense 64-float lines, then a
    // 4-float halo per velocity
    static constexpr int LINE = TILED ? 64 : 72;
    static constexpr int SLOT = TILED ? NV * (64 + 4) : NV * LINE;   // floats of one warp's row slot
    static constexpr int THREADS = 32 * G;
    static constexpr int OUT = TILED == 2 ? NV * 64 : 0;       // floats of one warp's store staging
    static constexpr int SMEM = S * G * SLOT * 4 + S * G * 8 + G * OUT * 4;
    // a ring of two slots (the own row and its upwind row, nothing in flight ahead) is small
    // enough for two blocks per SM: the second block computes while the first waits
    static constexpr int MIN_BLOCKS = S == 2 ? 2 : 1;
};

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// first row of chunk k of the interior rows [first, first + rows) cut into nchunks
// near-equal chunks (first = 1 for the first-order transport, 2 for the second-order one)
__device__ __forceinline__ int march_row0(int k, int rows, int nchunks, int first = 1)
{
    return first + (int)(((long)k * rows) / nchunks);
}

template <int M, int G, int S, bool RESID, bool DEFER, int TILED = 0, int ORDER = 1>
__global__ void __launch_bounds__(MarchShape<M, G, S, TILED>::THREADS, MarchShape<M, G, S, TILED>::MIN_BLOCKS)
step_march_kernel(const StepArgs a)
{
    using Sh = MarchShape<M, G, S, TILED>;
    static_assert(!(TILED && DEFER), "the tiled march has no deferred-relaxation form");
    // deferred relaxation (steps without the residual): row t's moment partials are published
    // through an mbarrier phase and row t - 1 is relaxed after row t's transport, so a warp
    // meets the slowest warp's partials one transport later than at a block barrier
    constexpr bool DEF = DEFER && !RESID;
    constexpr int NMOM = DEF ? 4 : 2;
    constexpr int RPL = Sh::RPL, NV = Sh::NV, LINE = Sh::LINE, HALF = M / 2;
    static_assert(M % 2 == 0 && (M / 2) % 2 == 0, "even M with velocity pairs on one side of xi = 0");
    static_assert(HALF % RPL == 0, "the velocity rows of a warp share the sign of xi_y");
    static_assert(NV <= 32, "one bulk copy per lane and row");
    // the velocities of a warp share the sign of xi_y, so it reads two rows per step (y and
    // its upwind neighbour); a copy overwrites the slot of the row before those two, which the
    // warp finished reading in its previous row step
    static_assert(S >= 2, "own row and upwind row resident");
    // second order: the two upwind rows and the two upwind cells in x (8-byte halos) are
    // read; the tiled layout only, no deferred relaxation
    static_assert(ORDER == 1 || (ORDER == 2 && TILED != 0 && !DEFER && S >= 4), "second-order march form");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ float2 s_mom[NMOM][3][G][32];
    __shared__ uint64_t s_mbar[2];
    __shared__ int s_items[4];
    __shared__ int s_abort;
    __shared__ double s_red[2][G];

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long ncells = a.ncells;
    const int nx = a.nx;
    const int nstrips = a.march_strips, nchunks = a.march_chunks;
    const int nitems = nstrips * nchunks;
    const int rows = a.ny - 2 * ORDER;   // interior rows [ORDER, ny - 1 - ORDER]
    const bool ypos = g * RPL >= HALF;   // xi_y > 0: upwind row y - 1; else y + 1
    float *slots = reinterpret_cast<float *>(smem_raw) + (long)g * S * Sh::SLOT;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (long)S * G * Sh::SLOT * 4) + g * S;
    // staging of this warp's relaxed row for the bulk store (TILED = 2)
    float *outst = reinterpret_cast<float *>(smem_raw + (long)S * G * Sh::SLOT * 4 + (long)S * G * 8) + g * Sh::OUT;
    (void)outst;
    const float *__restrict__ h = reinterpret_cast<const float *>(a.h);
    float *__restrict__ hn = reinterpret_cast<float *>(a.hn);

    // the first three items of every block are fixed (block b takes b, grid + b, 2 grid + b),
    // so that the blocks start on consecutive items (neighbouring strips of the same rows);
    // items from 3 grid on are handed out by the counter as blocks finish items
    const int first_dyn = 3 * (int)gridDim.x;
    if (threadIdx.x == 0) {
        s_items[0] = (int)blockIdx.x;
        s_items[1] = (int)gridDim.x + (int)blockIdx.x;
        s_items[2] = 2 * (int)gridDim.x + (int)blockIdx.x;
        s_abort = 0;
        if (DEF) {
            mbar_init(&s_mbar[0], Sh::THREADS);
            mbar_init(&s_mbar[1], Sh::THREADS);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    if (lane == 0) {
        // tiled: lane 0's expect-tx arrival and the NV lanes' halo copies complete a phase
        for (int j = 0; j < S; ++j) mbar_init(&bars[j], TILED ? 1 + NV : 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    // the wall kernel of this step (a programmatic dependent launch) may start now and run
    // beside the march on the SM resources the march leaves free
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

    // coefficients as FP32x2 pairs (both halves equal: one coefficient, two cells), set
    // once: per velocity of the warp 1 - nu_x - nu_y (k = r*M + ix), per ix nu_x, xi, w
    float2 a0r[NV], nux2[M], xi2[M], w2[M];
    // second order (Beam-Warming face fluxes, no wall within two cells): per direction with
    // Courant number nu, P = nu (3 - nu) / 2 (own cell), B = nu (2 - nu) (first upwind
    // cell), C = nu (1 - nu) / 2 (second upwind cell; the host's tables hold -C), so that
    //     h* = (1 - P_x - P_y) h + B_x h_x1 - C_x h_x2 + B_y h_y1 - C_y h_y2;
    // a0r then holds 1 - P_x - P_y (formed in FP64, rounded once), cx2 and cy2 hold -C
    float2 bx2[ORDER == 2 ? M : 1], cx2[ORDER == 2 ? M : 1], by2[ORDER == 2 ? RPL : 1], cy2[ORDER == 2 ? RPL : 1];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int r = k / M, ix = k - r * M;
        float v;
        if constexpr (ORDER == 2) {
            v = (float)(1.0 - a.so_p[0][ix] - a.so_p[1][g * RPL + r]);
        } else {
            v = 1.f - a.nux_f[ix] - a.nuy_f[g * RPL + r];
        }
        a0r[k] = make_float2(v, v);
    }
    if constexpr (ORDER == 2) {
#pragma unroll
        for (int ix = 0; ix < M; ++ix) {
            const float b = a.so_b_f[0][ix], c = a.so_c_f[0][ix];
            bx2[ix] = make_float2(b, b);
            cx2[ix] = make_float2(c, c);
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const float b = a.so_b_f[1][g * RPL + r], c = a.so_c_f[1][g * RPL + r];
            by2[r] = make_float2(b, b);
            cy2[r] = make_float2(c, c);
        }
    }
#pragma unroll
    for (int ix = 0; ix < M; ++ix) {
        nux2[ix] = make_float2(a.nux_f[ix], a.nux_f[ix]);
        xi2[ix] = make_float2(a.xi_f[ix], a.xi_f[ix]);
        w2[ix] = make_float2(a.w1_f[ix], a.w1_f[ix]);
    }
    // plane offset of this lane's copy (lanes < NV issue one line each per row)
    const int kc = lane < NV ? lane : 0;
    const float *src_plane = h + (long)((g * RPL + kc / M) * M + (kc % M)) * ncells;
    // tiled: rows of a tile are NVALL * 64 floats apart; this warp's lines start at velocity
    // g * NV; lane kc's halo comes from the left tile (xi_x > 0) or the right tile (xi_x < 0),
    // as an offset from the left tile's row
    constexpr long TROW = (long)M * M * LBM_TILE_W;
    const long tp = a.tile_pitch;
    const bool left_halo = (kc % M) >= M - HALF;
    // (second order: the two cells next to the strip, 8 bytes, at halo slot floats 2-3 for
    // the left pair x0 - 2, x0 - 1 and 0-1 for the right pair x0 + 64, x0 + 65)
    const long halo_off = left_halo ? (long)(g * NV + kc) * LBM_TILE_W + (LBM_TILE_W - ORDER)
                                    : 2 * tp + (long)(g * NV + kc) * LBM_TILE_W;
    const int halo_dst = NV * LBM_TILE_W + 4 * kc + (left_halo ? 4 - ORDER : 0);   // where the kernel reads it
    // x-upwind neighbour of a lane's cell pair, as base + k * step floats from the own row
    // slot (velocity k of the warp): the neighbouring cell of the own line, or, for the
    // strip's edge lane, the halo copied from the neighbouring tile
    const int pl_base = lane > 0 ? 2 * lane - 1 : NV * LBM_TILE_W + 3, pl_step = lane > 0 ? LBM_TILE_W : 4;
    const int pr_base = lane < 31 ? 2 * lane + 2 : NV * LBM_TILE_W, pr_step = lane < 31 ? LBM_TILE_W : 4;
    // second order: the neighbouring cell pair on the upwind side (x - 2, x - 1 or x + 2,
    // x + 3 of the lane's first cell) as one 8-byte read at base + k * step
    const int ql_base = lane > 0 ? 2 * lane - 2 : NV * LBM_TILE_W + 2, ql_step = lane > 0 ? LBM_TILE_W : 4;
    const int qr_base = lane < 31 ? 2 * lane + 2 : NV * LBM_TILE_W, qr_step = lane < 31 ? LBM_TILE_W : 4;
    (void)tp; (void)halo_off; (void)halo_dst; (void)pl_base; (void)pl_step; (void)pr_base; (void)pr_step;
    (void)ql_base; (void)ql_step; (void)qr_base; (void)qr_step;

    // loader state (uniform within the warp)
    int l_pos = 0, l_item = s_items[0], l_i = 0;
    int l_row0 = 0, l_len = 0, l_strip = 0;
    auto l_decode = [&]() {
        const int k = l_item / nstrips;
        l_strip = l_item - k * nstrips;
        l_row0 = march_row0(k, rows, nchunks, ORDER);
        l_len = march_row0(k + 1, rows, nchunks, ORDER) - l_row0;
    };
    if (l_item < nitems) l_decode();
    long nl = 0;       // copies issued (row slots)
    long waited = 0;   // row slots [0, waited) have landed

    auto issue = [&]() {
        const int slot = (int)(nl % S);
        const int row = l_row0 - (ypos ? ORDER : 0) + l_i;   // an item's rows and ORDER upwind rows
        if constexpr (TILED) {
            // transaction bytes of the bulk copy only: the halo copies count as arrivals
            if (lane == 0) mbar_arrive_expect(&bars[slot], (unsigned)(NV * LBM_TILE_W * 4));
            __syncwarp();
            fence_proxy_async_smem();
            float *dst = slots + slot * Sh::SLOT;
            const float *left_row = h + (long)l_strip * tp + (long)row * TROW;
            if (lane < NV) {
                if constexpr (ORDER == 1)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n"
                                 "cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%2];\n" ::"r"(smem_addr(dst + halo_dst)),
                                 "l"(left_row + halo_off), "r"(smem_addr(&bars[slot]))
                                 : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n"
                                 "cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%2];\n" ::"r"(smem_addr(dst + halo_dst)),
                                 "l"(left_row + halo_off), "r"(smem_addr(&bars[slot]))
                                 : "memory");
            }
            if (lane == 0)
                bulk_copy(dst, left_row + tp + (long)g * NV * LBM_TILE_W, NV * LBM_TILE_W * 4, &bars[slot]);
        } else {
            if (lane == 0) mbar_arrive_expect(&bars[slot], (unsigned)(NV * LINE * 4));
            __syncwarp();
            fence_proxy_async_smem();   // this slot's earlier generic reads before the async writes
            if (lane < NV)
                bulk_copy(slots + slot * Sh::SLOT + lane * LINE,
                          src_plane + (long)row * nx + 28 + 64L * l_strip, LINE * 4, &bars[slot]);
        }
        ++nl;
        if (++l_i > l_len + ORDER - 1) {
            l_i = 0;
            ++l_pos;
            l_item = s_items[l_pos & 3];
            if (l_item < nitems) l_decode();
        }
    };
    bool ok = true;
    auto wait_through = [&](long j_last) {
        for (; waited <= j_last; ++waited) {
            if (!mbar_wait_bounded(&bars[waited % S], (unsigned)((waited / S) & 1), 2000000000LL)) {
                ok = false;
                return;
            }
        }
    };

    // compute state
    int c_pos = 0, c_item = s_items[0], c_u = 0;
    int c_row0 = 0, c_len = 0, c_strip = 0;
    auto c_decode = [&]() {
        const int k = c_item / nstrips;
        c_strip = c_item - k * nstrips;
        c_row0 = march_row0(k, rows, nchunks, ORDER);
        c_len = march_row0(k + 1, rows, nchunks, ORDER) - c_row0;
    };
    if (c_item < nitems) c_decode();
    long gb = 0;       // row-slot index of load 0 of the item being computed
    int par = 0;
    const float om = a.omega_f;
    const float2 b2 = make_float2(a.b_f, a.b_f);
    double psd = 0.0, psn = 0.0;
    // deferred relaxation: the transported row waiting for its moments, its first cell
    float2 hp[NV];
    long pcell = 0;
    long t = 0;        // rows transported by this block
    // relaxation and store of the deferred row from the moment partials in buffer bt
    auto relax_deferred = [&](int bt, long cell) {
        float2 r2 = make_float2(0.f, 0.f), x2 = r2, y2 = r2;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            r2 = __fadd2_rn(r2, s_mom[bt][0][q][lane]);
            x2 = __fadd2_rn(x2, s_mom[bt][1][q][lane]);
            y2 = __fadd2_rn(y2, s_mom[bt][2][q][lane]);
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const float wom = om * a.w1_f[iy];
            const float xiy = a.xi_f[iy];
            const float2 q2 = __fmul2_rn(make_float2(wom, wom), __ffma2_rn(make_float2(xiy, xiy), y2, r2));
            const float2 jj2 = __fmul2_rn(make_float2(wom, wom), x2);
            float *rowp = hn + (long)(iy * M) * ncells + cell;
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const int k = r * M + ix;
                const float2 tt = __ffma2_rn(xi2[ix], jj2, q2);
                *reinterpret_cast<float2 *>(rowp + (long)ix * ncells) = __ffma2_rn(w2[ix], tt, __fmul2_rn(b2, hp[k]));
            }
        }
    };

    while (c_item < nitems) {
        // keep S - 1 - ORDER rows of copies ahead of the rows being computed
        while (l_item < nitems && nl <= gb + c_u + S - 1) issue();
        if (ok) wait_through(gb + c_u + ORDER);
        ok = __all_sync(FULL, ok);      // one verdict per warp
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.status, 1);
                s_abort = 1;
            }
            // deferred: leave now (the other warps' next moment wait runs out and they leave)
            if (DEF) break;
        }
        const long jo = ypos ? gb + c_u + ORDER : gb + c_u;              // own row y
        const long jy = ypos ? gb + c_u + ORDER - 1 : gb + c_u + 1;      // upwind row y -/+ 1
        const long jq = ypos ? gb + c_u : gb + c_u + 2;                  // second order: y -/+ 2
        const float *own = slots + (int)(jo % S) * Sh::SLOT;
        const float *ynb = slots + (int)(jy % S) * Sh::SLOT;
        const float *ynb2 = slots + (int)(jq % S) * Sh::SLOT;
        (void)ynb2;

        // ---- transport + moment sums (two cells per lane) ----
        float2 hs[NV];
        float2 rho2 = make_float2(0.f, 0.f), jx2 = rho2, jy2 = rho2;
        if (ok) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int iy = g * RPL + r;
                const float nuy = a.nuy_f[iy];
                const float2 nuy2 = make_float2(nuy, nuy);
                // row sums in NACC independent partial sums (short dependency chains)
                constexpr int NACC = 4;
                float2 R2[NACC], X2[NACC];
#pragma unroll
                for (int q = 0; q < NACC; ++q) R2[q] = X2[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int ix = 0; ix < M; ++ix) {
                    const int k = r * M + ix;
                    float2 hc, hx, hy;
                    if constexpr (ORDER == 2) {
                        // the pair's upwind neighbours: in x the next pair on the upwind side
                        // (x -/+ 2 of the first cell, one 8-byte read) and the cell between,
                        // in y the same pair in the rows y -/+ 1 and y -/+ 2
                        hc = *reinterpret_cast<const float2 *>(own + k * LINE + 2 * lane);
                        const bool xpos = ix >= M - HALF;
                        const float2 nb = xpos ? *reinterpret_cast<const float2 *>(own + ql_base + k * ql_step)
                                               : *reinterpret_cast<const float2 *>(own + qr_base + k * qr_step);
                        const float2 h1x = xpos ? make_float2(nb.y, hc.x) : make_float2(hc.y, nb.x);
                        const float2 h1y = *reinterpret_cast<const float2 *>(ynb + k * LINE + 2 * lane);
                        const float2 h2y = *reinterpret_cast<const float2 *>(ynb2 + k * LINE + 2 * lane);
                        float2 v = __fmul2_rn(a0r[k], hc);
                        v = __ffma2_rn(bx2[ix], h1x, v);
                        v = __ffma2_rn(cx2[ix], nb, v);
                        v = __ffma2_rn(by2[r], h1y, v);
                        v = __ffma2_rn(cy2[r], h2y, v);
                        hs[k] = v;
                        R2[ix % NACC] = __fadd2_rn(R2[ix % NACC], v);
                        X2[ix % NACC] = __ffma2_rn(xi2[ix], v, X2[ix % NACC]);
                        continue;
                    }
                    if constexpr (TILED) {
                        hc = *reinterpret_cast<const float2 *>(own + k * LINE + 2 * lane);
                        hx = (ix >= M - HALF) ? make_float2(own[pl_base + k * pl_step], hc.x)   // xi_x > 0: x - 1
                                              : make_float2(hc.y, own[pr_base + k * pr_step]);  // xi_x < 0: x + 1
                        hy = *reinterpret_cast<const float2 *>(ynb + k * LINE + 2 * lane);
                    } else {
                        const float *lo = own + k * LINE;
                        hc = *reinterpret_cast<const float2 *>(lo + 4 + 2 * lane);
                        hx = (ix >= M - HALF) ? make_float2(lo[3 + 2 * lane], hc.x)     // xi_x > 0: x - 1
                                              : make_float2(hc.y, lo[6 + 2 * lane]);    // xi_x < 0: x + 1
                        hy = *reinterpret_cast<const float2 *>(ynb + k * LINE + 4 + 2 * lane);
                    }
                    float2 v;
                    if constexpr (DEF) {
                        // h + nu_x (h_x - h) + nu_y (h_y - h): no per-velocity coefficient held
                        // in registers (they hold the deferred row instead)
                        const float2 m1 = make_float2(-1.f, -1.f);     // x - h as fma(h, -1, x)
                        v = __ffma2_rn(nux2[ix], __ffma2_rn(hc, m1, hx), hc);
                        v = __ffma2_rn(nuy2, __ffma2_rn(hc, m1, hy), v);
                    } else {
                        v = __fmul2_rn(a0r[k], hc);
                        v = __ffma2_rn(nux2[ix], hx, v);
                        v = __ffma2_rn(nuy2, hy, v);
                    }
                    hs[k] = v;
                    R2[ix % NACC] = __fadd2_rn(R2[ix % NACC], v);
                    X2[ix % NACC] = __ffma2_rn(xi2[ix], v, X2[ix % NACC]);
                }
                const float2 R = __fadd2_rn(__fadd2_rn(R2[0], R2[1]), __fadd2_rn(R2[2], R2[3]));
                const float2 X = __fadd2_rn(__fadd2_rn(X2[0], X2[1]), __fadd2_rn(X2[2], X2[3]));
                const float xiy = a.xi_f[iy];
                rho2 = __fadd2_rn(rho2, R);
                jx2 = __fadd2_rn(jx2, X);
                jy2 = __ffma2_rn(make_float2(xiy, xiy), R, jy2);
            }
        }
        if constexpr (DEF) {
            // publish row t, then relax row t - 1 (its partials were published one transport ago)
            const int bt = (int)(t & 3);
            s_mom[bt][0][g][lane] = rho2;
            s_mom[bt][1][g][lane] = jx2;
            s_mom[bt][2][g][lane] = jy2;
            mbar_arrive(&s_mbar[t & 1]);
            if (t > 0) {
                const long tp = t - 1;
                ok = mbar_wait_bounded(&s_mbar[tp & 1], (unsigned)((tp >> 1) & 1), 2000000000LL);
                ok = __all_sync(FULL, ok);
                if (!ok) {
                    if (lane == 0) {
                        atomicExch(a.status, 1);
                        s_abort = 1;
                    }
                    break;
                }
                relax_deferred((int)(tp & 3), pcell);
            }
            const int y = c_row0 + c_u;
            pcell = (long)y * nx + 32 + 64L * c_strip + 2 * lane;
#pragma unroll
            for (int k = 0; k < NV; ++k) hp[k] = hs[k];
            ++t;
            if (++c_u == c_len) {
                gb += c_len + ORDER;
                c_u = 0;
                ++c_pos;
                c_item = s_items[c_pos & 3];
                if (c_item < nitems) c_decode();
                if (threadIdx.x == 0) s_items[(c_pos + 2) & 3] = first_dyn + atomicAdd(a.counters, 1);
            }
            continue;
        }
        s_mom[par][0][g][lane] = rho2;
        s_mom[par][1][g][lane] = jx2;
        s_mom[par][2][g][lane] = jy2;
        __syncthreads();
        if (s_abort) break;
        rho2 = jx2 = jy2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            rho2 = __fadd2_rn(rho2, s_mom[par][0][q][lane]);
            jx2 = __fadd2_rn(jx2, s_mom[par][1][q][lane]);
            jy2 = __fadd2_rn(jy2, s_mom[par][2][q][lane]);
        }
        par ^= 1;

        // ---- relaxation, store, residual ----
        const int y = c_row0 + c_u;
        const long cell = (long)y * nx + 32 + 64L * c_strip + 2 * lane;
        // tiled: this lane's cell pair in velocity 0 of the strip's tile row
        const long tcell = (long)(c_strip + 1) * tp + (long)y * TROW + 2 * lane;
        float2 psd2 = make_float2(0.f, 0.f), psn2 = psd2;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const float wom = om * a.w1_f[iy];
            const float xiy = a.xi_f[iy];
            const float2 q2 = __fmul2_rn(make_float2(wom, wom), __ffma2_rn(make_float2(xiy, xiy), jy2, rho2));
            const float2 jj2 = __fmul2_rn(make_float2(wom, wom), jx2);
            float *rowp = TILED ? hn + tcell + (long)(iy * M) * LBM_TILE_W : hn + (long)(iy * M) * ncells + cell;
            const long vstride = TILED ? (long)LBM_TILE_W : ncells;
            if constexpr (TILED == 2) {
                if (r == 0) {
                    // the previous row's bulk store must have read the staging buffer
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                    __syncwarp();
                }
            }
#pragma unroll
            for (int ix = 0; ix < M; ++ix) {
                const int k = r * M + ix;
                const float2 t = __ffma2_rn(xi2[ix], jj2, q2);
                const float2 v = __ffma2_rn(w2[ix], t, __fmul2_rn(b2, hs[k]));
                if (RESID) {
                    const float2 hc = *reinterpret_cast<const float2 *>(own + k * LINE + (TILED ? 0 : 4) + 2 * lane);
                    const float2 d = __fadd2_rn(v, make_float2(-hc.x, -hc.y));
                    psd2 = __ffma2_rn(d, d, psd2);
                    psn2 = __ffma2_rn(v, v, psn2);
                }
                if constexpr (TILED == 2)
                    *reinterpret_cast<float2 *>(outst + k * LBM_TILE_W + 2 * lane) = v;
                else
                    *reinterpret_cast<float2 *>(rowp + (long)ix * vstride) = v;
            }
        }
        if constexpr (TILED == 2) {
            // this warp's NV lines of the strip's tile row, one contiguous stretch
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                float *dst = hn + (tcell - 2 * lane) + (long)g * NV * LBM_TILE_W;
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                             "cp.async.bulk.commit_group;\n" ::"l"(dst), "r"(smem_addr(outst)),
                             "r"((unsigned)(NV * LBM_TILE_W * 4))
                             : "memory");
            }
        }
        if (RESID) {
            psd += (double)psd2.x + (double)psd2.y;
            psn += (double)psn2.x + (double)psn2.y;
        }

        // ---- next row / item ----
        if (++c_u == c_len) {
            gb += c_len + ORDER;
            c_u = 0;
            ++c_pos;
            c_item = s_items[c_pos & 3];
            if (c_item < nitems) c_decode();
            if (threadIdx.x == 0) s_items[(c_pos + 2) & 3] = first_dyn + atomicAdd(a.counters, 1);
        }
    }

    // the last deferred row
    if (DEF && ok && t > 0) {
        const long tp = t - 1;
        ok = __all_sync(FULL, mbar_wait_bounded(&s_mbar[tp & 1], (unsigned)((tp >> 1) & 1), 2000000000LL));
        if (ok) relax_deferred((int)(tp & 3), pcell);
        else if (lane == 0) atomicExch(a.status, 1);
    }

    // copies still in flight (abort path) must land before the block's shared memory goes
    for (; waited < nl; ++waited) mbar_wait_bounded(&bars[waited % S], (unsigned)((waited / S) & 1), 2000000000LL);
    // and the bulk stores must have completed (their source and the new state)
    if constexpr (TILED == 2)
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");

    if (RESID) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            psd += __shfl_xor_sync(FULL, psd, off);
            psn += __shfl_xor_sync(FULL, psn, off);
        }
        if (lane == 0) {
            s_red[0][g] = psd;
            s_red[1][g] = psn;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (RESID) {
            double td = 0.0, tn = 0.0;
            for (int q = 0; q < G; ++q) {
                td += s_red[0][q];
                tn += s_red[1][q];
            }
            a.partials[2 * blockIdx.x] = td;
            a.partials[2 * blockIdx.x + 1] = tn;
        }
        // the last block to finish resets the item counter for the next launch
        __threadfence();
        if (atomicAdd(a.counters + 1, 1) == (int)gridDim.x - 1) {
            a.counters[0] = 0;
            a.counters[1] = 0;
            __threadfence();
        }
    }
}

template <int M, int G, int S, bool DEFER, int TILED = 0, int ORDER = 1>
cudaError_t prepare_march(int *grid)
{
    constexpr int SMEM = MarchShape<M, G, S, TILED>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(step_march_kernel<M, G, S, true, DEFER, TILED, ORDER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_march_kernel<M, G, S, false, DEFER, TILED, ORDER>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    // the largest shared-memory carveout: otherwise the driver may pick the smallest one that
    // holds one march block (164 KB for the tiled ring) and leave no room for the wall blocks
    // that run beside it
    for (int r = 0; r < 2 && e == cudaSuccess; ++r)
        e = cudaFuncSetAttribute(r ? step_march_kernel<M, G, S, true, DEFER, TILED, ORDER>
                                   : step_march_kernel<M, G, S, false, DEFER, TILED, ORDER>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_march_kernel<M, G, S, false, DEFER, TILED, ORDER>,
                                                          MarchShape<M, G, S, TILED>::THREADS, SMEM);
    if (e == cudaSuccess && DEFER) {
        int per_sm_resid = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_resid, step_march_kernel<M, G, S, true, DEFER, TILED, ORDER>,
                                                          MarchShape<M, G, S, TILED>::THREADS, SMEM);
        if (per_sm_resid < per_sm) per_sm = per_sm_resid;
    }
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) *grid = per_sm > 0 ? per_sm * sms : 0;
    return e;
}

// Wall segments of a step whose interior is marched by step_march_kernel, launched as its
// programmatic dependent: the two grids run side by side (they read the same old state and
// write disjoint cells of the new one).  Block 0 waits for the march grid before it exits,
// so that this grid completes only after the march has completed and its writes are
// visible: work the stream orders after this launch sees the whole step.
template <int M, int G, bool RESID, int TILED = 0>
__global__ void __launch_bounds__(Shape<G>::THREADS) step_wall_beside_march_kernel(const StepArgs a)
{
    step_body<float, float, M, G, RESID, false, false, true, false, TILED != 0>(a, blockIdx.x);
    if (blockIdx.x == 0) asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// March kernel over `grid` persistent blocks, and beside it the wall kernel over the wall
// segments (programmatic dependent launch).
// The wall kernel `wall` over the wall segments as a programmatic dependent launch of the
// march grid just enqueued on `s` (its residual partials after the march's `grid` slots).
template <int G>
cudaError_t launch_wall_beside(void (*wall)(const StepArgs), const StepArgs &a, int grid, cudaStream_t s)
{
    StepArgs b = a;
    b.partials_offset = grid;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((a.n_wall_segs + Shape<G>::SPB - 1) / Shape<G>::SPB);
    cfg.blockDim = dim3(Shape<G>::THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, wall, b);
}

template <int M, int G, int S, bool DEFER, bool RESID, int TILED = 0>
cudaError_t launch_march(const StepArgs &a, int grid, cudaStream_t s)
{
    constexpr int SMEM = MarchShape<M, G, S, TILED>::SMEM;
    step_march_kernel<M, G, S, RESID, DEFER, TILED><<<grid, MarchShape<M, G, S, TILED>::THREADS, SMEM, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_wall_segs == 0) return e;
    return launch_wall_beside<G>(step_wall_beside_march_kernel<M, G, RESID, TILED>, a, grid, s);
}

}  // namespace lbmk
