// Bulk (wall-free) segments of the fused step with TMA staging of the upwind halo
// (sm_103a): the same arithmetic as the bulk path of step_kernel.cuh, but every warp first
// has the Tensor Memory Accelerator copy, with 1-D bulk asynchronous copies
// (cp.async.bulk ... mbarrier::complete_tx), all the data its velocity rows need into
// shared memory: per velocity the own-cell line widened by 4 cells on each side (the x
// upwind neighbours, 160 bytes) and the upwind y-neighbour line (128 bytes).  The copies
// hold no registers while in flight, so a warp keeps ~10 KB of loads outstanding instead
// of the few lines its registers allow, which is what the memory system needs to stay
// busy (the register-staged kernel was latency bound: long-scoreboard stalls, DRAM at
// half its peak).  The warp then waits on its mbarrier (a bounded wait: after the limit
// it sets the status word, waits again for its copies and skips the segment), computes
// from shared memory, and stores with ordinary coalesced stores.
//
// Requirements (checked by the host): number of cells and nx multiples of 4, so that
// every copied line starts on a 16-byte boundary; wall segments (and therefore the
// first and last segments of the grid) are left to the wall kernel.
#pragma once

#include <cstdint>

#include "step_kernel.cuh"

namespace lbmk {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Test for completion of the phase with the given parity; a thread whose phase is not
// complete may be suspended until it completes or for at most the time hint (10 ms), so
// a waiting warp does not spin on the issue slots the computing warps need.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_addr(bar)), "r"(phase), "r"(10000000u)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst_smem)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// wait for the phase of the given parity of a barrier, at most ~limit_cycles; false on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit_cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit_cycles) return false;
    }
    return true;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, long long limit_cycles)
{
    return mbar_wait_bounded(bar, 0u, limit_cycles);
}

template <int M, int G>
struct TmaShape {
    static constexpr int RPL = M / G;
    static constexpr int NV = RPL * M;               // velocities per warp
    static constexpr int CEN = 40;                   // floats per own-cell line (32 + 4 + 4)
    static constexpr int YN = 32;                    // floats per y-neighbour line
    static constexpr int WARP_FLOATS = NV * (CEN + YN);
    static constexpr int BYTES_PER_WARP = WARP_FLOATS * 4;
    static constexpr int SMEM = Shape<G>::WARPS * BYTES_PER_WARP + Shape<G>::WARPS * 8 + 16;
};

template <int M, int G, bool RESID>
__device__ __forceinline__ void tma_body(const StepArgs &a, const int bid)
{
    using TC = float;
    constexpr int SPB = Shape<G>::SPB;
    constexpr int WARPS = Shape<G>::WARPS;
    constexpr int RPL = M / G;
    constexpr int HALF = M / 2;
    constexpr int NVW = TmaShape<M, G>::NV;
    constexpr int CEN = TmaShape<M, G>::CEN, YN = TmaShape<M, G>::YN;
    static_assert(M % 2 == 0, "TMA path: even number of nodes per axis (no zero velocity)");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ TC s_mom[3][G][SPB][32];
    __shared__ double s_red[2][WARPS];

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = warp / G, g = warp - sl * G;
    const long ncells = a.ncells;
    const int nx = a.nx, ny = a.ny;
    float *cen = reinterpret_cast<float *>(smem_raw) + (long)warp * TmaShape<M, G>::WARP_FLOATS;
    float *yn = cen + NVW * CEN;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + WARPS * TmaShape<M, G>::BYTES_PER_WARP) + warp;

    const long seg = (long)bid * SPB + sl;
    const bool active = seg * 32 < ncells;
    const long c0 = seg * 32;
    const long cell0 = c0 + lane;
    const bool in_grid = cell0 < ncells;
    const long c = in_grid ? cell0 : ncells - 1;
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const bool cav = a.cavity != 0;
    const bool is_wall = in_grid && (y == 0 || y == ny - 1 || (cav && (x == 0 || x == nx - 1)));
    const bool work = active && !__any_sync(FULL, is_wall);
    const bool valid = work && in_grid;
    const float *__restrict__ h = reinterpret_cast<const float *>(a.h);

    // ---- issue the warp's bulk copies ----
    bool ok = true;
    if (work) {
        if (lane == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            mbar_arrive_expect(bar, (unsigned)(NVW * (CEN + YN) * 4));
        }
        __syncwarp();
        for (int k = lane; k < NVW; k += 32) {
            const int r = k / M, ix = k - r * M;
            const int iy = g * RPL + r;
            const float *plane = h + (long)(iy * M + ix) * ncells;
            bulk_copy(cen + k * CEN, plane + c0 - 4, CEN * 4, bar);
            const long ylin = (iy < HALF) ? c0 + nx : c0 - nx;      // upwind y row
            bulk_copy(yn + k * YN, plane + ylin, YN * 4, bar);
        }
        if (!mbar_wait_bounded(bar, 2000000000LL)) {
            ok = false;
            if (lane == 0) atomicExch(a.status, 1);
            mbar_wait_bounded(bar, 2000000000LL);   // let the copies land before leaving
        }
        __syncwarp();
    }
    const bool compute = work && ok;

    // ---- transport + moment row sums from shared memory ----
    // Velocities are processed in pairs (ix, ix+1) with the packed FP32x2 instructions of
    // sm_100+ (one FFMA2 does two updates), which halves the arithmetic instructions of this
    // issue-bound kernel.  Transport in the form (1 - nu_x - nu_y) h + nu_x h_x + nu_y h_y.
    // A pair never straddles the sign change of xi_x (M/2 is even for M = 8, 12).
    static_assert((M / 2) % 2 == 0, "velocity pairs must not straddle xi_x = 0");
    float2 hs[RPL * M / 2];
    TC rho = 0, jx = 0, jy = 0;
    if (compute) {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC xiy = a.xi_f[iy];
            const TC nuy = a.nuy_f[iy];
            const float2 nuy2 = make_float2(nuy, nuy);
            float2 R2 = make_float2(0.f, 0.f), X2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int pp = 0; pp < M / 2; ++pp) {
                const int ix = 2 * pp;
                const int k = r * M + ix;
                const int sx = (ix >= M - HALF) ? 3 : 5;          // upwind x neighbour in the line
                const float2 hc = make_float2(cen[k * CEN + 4 + lane], cen[(k + 1) * CEN + 4 + lane]);
                const float2 hx = make_float2(cen[k * CEN + sx + lane], cen[(k + 1) * CEN + sx + lane]);
                const float2 hy = make_float2(yn[k * YN + lane], yn[(k + 1) * YN + lane]);
                const float2 nux = make_float2(a.nux_f[ix], a.nux_f[ix + 1]);
                const float2 a0 = make_float2(1.f - a.nux_f[ix] - nuy, 1.f - a.nux_f[ix + 1] - nuy);
                float2 v = __fmul2_rn(a0, hc);
                v = __ffma2_rn(nux, hx, v);
                v = __ffma2_rn(nuy2, hy, v);
                hs[r * (M / 2) + pp] = v;
                R2 = __fadd2_rn(R2, v);
                X2 = __ffma2_rn(make_float2(a.xi_f[ix], a.xi_f[ix + 1]), v, X2);
            }
            const TC R = R2.x + R2.y, X = X2.x + X2.y;
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

    // ---- relaxation, store, residual ----
    TC psd = 0, psn = 0;
    if (compute) {
        const float2 b2 = make_float2(a.b_f, a.b_f);
        const TC om = a.omega_f;
        float *__restrict__ hn = reinterpret_cast<float *>(a.hn);
        float2 psd2 = make_float2(0.f, 0.f), psn2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int iy = g * RPL + r;
            const TC wom = om * a.w1_f[iy];
            const TC q = wom * (rho + a.xi_f[iy] * jy);
            const TC jj = wom * jx;
            const float2 q2 = make_float2(q, q), jj2 = make_float2(jj, jj);
            float *rowp = hn + (long)(iy * M) * ncells + c;
#pragma unroll
            for (int pp = 0; pp < M / 2; ++pp) {
                const int ix = 2 * pp;
                const int k = r * M + ix;
                const float2 t = __ffma2_rn(make_float2(a.xi_f[ix], a.xi_f[ix + 1]), jj2, q2);
                const float2 v = __ffma2_rn(make_float2(a.w1_f[ix], a.w1_f[ix + 1]), t,
                                            __fmul2_rn(b2, hs[r * (M / 2) + pp]));
                if (RESID) {
                    const float2 hc = make_float2(cen[k * CEN + 4 + lane], cen[(k + 1) * CEN + 4 + lane]);
                    const float2 d = __fadd2_rn(v, make_float2(-hc.x, -hc.y));
                    psd2 = __ffma2_rn(d, d, psd2);
                    psn2 = __ffma2_rn(v, v, psn2);
                }
                if (valid) {
                    rowp[(long)ix * ncells] = v.x;
                    rowp[(long)(ix + 1) * ncells] = v.y;
                }
            }
        }
        psd = psd2.x + psd2.y;
        psn = psn2.x + psn2.y;
    }

    if (RESID) {
        double sd = (valid && compute) ? (double)psd : 0.0, sn = (valid && compute) ? (double)psn : 0.0;
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
            a.partials[2 * bid] = td;
            a.partials[2 * bid + 1] = tn;
        }
    }
}

template <int M, int G, bool RESID>
__global__ void __launch_bounds__(Shape<G>::THREADS) step_tma_kernel(const StepArgs a)
{
    tma_body<M, G, RESID>(a, blockIdx.x);
}

// One launch for the whole step: the wall segments first (blocks [0, wall_blocks), the
// register-staged wall path), then the TMA-staged wall-free segments, so that the wall
// work overlaps the bulk instead of following it in a second launch.
template <int M, int G, bool RESID>
__global__ void __launch_bounds__(Shape<G>::THREADS) step_tma_merged_kernel(const StepArgs a)
{
    if ((int)blockIdx.x < a.wall_blocks)
        step_body<float, float, M, G, RESID, false, false, true, false>(a, blockIdx.x);
    else
        tma_body<M, G, RESID>(a, blockIdx.x - a.wall_blocks);
}

// Opt the kernels into their dynamic shared memory (once per process, before any launch
// or stream capture: lbm_set_variant calls it).
template <int M, int G>
cudaError_t prepare_tma()
{
    constexpr int SMEM = TmaShape<M, G>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<M, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_tma_kernel<M, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_tma_merged_kernel<M, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_tma_merged_kernel<M, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    return e;
}

// TMA bulk kernel, then the (register-staged) wall kernel over the wall segments.
template <int M, int G, bool RESID>
cudaError_t launch_tma(const StepArgs &a, int grid, cudaStream_t s, bool merged)
{
    constexpr int T = Shape<G>::THREADS;
    constexpr int SMEM = TmaShape<M, G>::SMEM;
    if (merged && a.n_wall_segs > 0) {
        StepArgs b = a;
        b.partials_offset = grid;        // wall partials after the bulk blocks' slots
        b.wall_blocks = (a.n_wall_segs + Shape<G>::SPB - 1) / Shape<G>::SPB;
        step_tma_merged_kernel<M, G, RESID><<<grid + b.wall_blocks, T, SMEM, s>>>(b);
        return cudaGetLastError();
    }
    step_tma_kernel<M, G, RESID><<<grid, T, SMEM, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n_wall_segs == 0) return e;
    StepArgs b = a;
    b.partials_offset = grid;
    const int wgrid = (a.n_wall_segs + Shape<G>::SPB - 1) / Shape<G>::SPB;
    step_kernel<float, float, M, G, RESID, false, false, true, false><<<wgrid, T, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace lbmk
