// Squared norms with no allocation at all: the variant of the norms reduction
// (lbm_norms) for callers that cannot call cudaMalloc -- code running inside a CUDA
// graph being built or replayed by someone else, allocator-less embedded hosts, signal or
// real-time paths where an allocation may block or fail -- and that cannot hand us a
// scratch buffer either.  The per-block partial sums live in a file-scope device array
// instead of caller memory.
//
// The array (LBM_NORMS_STATIC_PARTIALS pairs of doubles, 512 KiB) exists on every GPU
// that loads this library, from load until process exit.  In host code its name is only
// a host-side handle, so the kernels get its device address from cudaGetSymbolAddress,
// looked up with the call's device current.  A call whose stream is not being captured
// looks the address up afresh (a few microseconds), so the address stays right after a
// cudaDeviceReset; a call made while its stream is being captured reuses the address that
// the last uncaptured call on that device found, so make one uncaptured call on each
// device before capturing this entry point (and again after a cudaDeviceReset).  All calls
// share the array: every slot that a call reads is written by the same call first, so
// nothing needs clearing, but calls whose kernels overlap on the GPU (different streams,
// or overlapping graph launches) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

#define LBM_NORMS_STATIC_PARTIALS 32768
#define LBM_NORMS_STATIC_CHUNK (256L * 8L)   // elements per block (one partial pair)

static __device__ __align__(256) double g_norms_scratch[2 * LBM_NORMS_STATIC_PARTIALS];

namespace {

// One block per chunk of LBM_NORMS_STATIC_CHUNK consecutive elements; block k writes
// the pair (sum (a-b)^2, sum a^2) of its chunk to partials[2k], partials[2k+1].
template <typename T>
__global__ void __launch_bounds__(256) norms_chunk_kernel(const T *a, const T *b, long count,
                                                         double *partials)
{
    __shared__ double s_d[8], s_n[8];
    double sd = 0.0, sn = 0.0;
    const long base = (long)blockIdx.x * LBM_NORMS_STATIC_CHUNK;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const long i = base + (long)k * 256 + threadIdx.x;
        if (i < count) {
            const double va = (double)a[i];
            const double d = b ? va - (double)b[i] : va;
            sd += d * d;
            sn += va * va;
        }
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

std::mutex g_addr_mu;
void *g_addr[256];        // device address of g_norms_scratch found by the last uncaptured call
bool g_addr_ok[256];

}  // namespace

// error reporting shared with lbm_api.cu (sets the thread-local message)
lbm_status lbm_norms_fail(lbm_status s, const char *msg);

extern "C" lbm_status lbm_norms_noalloc(const void *a, const void *b, long count, int prec,
                                        double *out, void *stream)
{
    if (!a || !out) return lbm_norms_fail(LBM_EINVAL, "lbm_norms_noalloc: NULL argument");
    if (count < 0) return lbm_norms_fail(LBM_EINVAL, "lbm_norms_noalloc: count must be >= 0");
    if (prec != LBM_FP64 && prec != LBM_FP32_PERTURB)
        return lbm_norms_fail(LBM_EINVAL, "lbm_norms_noalloc: unknown precision");
    const long nblocks = (count + LBM_NORMS_STATIC_CHUNK - 1) / LBM_NORMS_STATIC_CHUNK;
    if (nblocks > LBM_NORMS_STATIC_PARTIALS)
        return lbm_norms_fail(LBM_EINVAL,
                              "lbm_norms_noalloc: count exceeds the 67108864-element limit of the "
                              "static scratch (use lbm_norms with caller scratch)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm_norms_fail(LBM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return lbm_norms_fail(LBM_EINVAL, "lbm_norms_noalloc: device ordinal");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return lbm_norms_fail(LBM_ECUDA, cudaGetErrorString(e));
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_addr_mu);
        if (cap == cudaStreamCaptureStatusNone || !g_addr_ok[dev]) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_norms_scratch);
            if (e != cudaSuccess) {
                g_addr_ok[dev] = false;
                return lbm_norms_fail(LBM_ECUDA, cudaGetErrorString(e));
            }
            g_addr[dev] = addr;
            g_addr_ok[dev] = true;
        }
        scratch = g_addr[dev];
    }
    double *partials = (double *)scratch;
    if (nblocks > 0) {
        if (prec == LBM_FP64)
            norms_chunk_kernel<double><<<(int)nblocks, 256, 0, s>>>((const double *)a, (const double *)b,
                                                                   count, partials);
        else
            norms_chunk_kernel<float><<<(int)nblocks, 256, 0, s>>>((const float *)a, (const float *)b,
                                                                  count, partials);
        e = cudaGetLastError();
        if (e != cudaSuccess) return lbm_norms_fail(LBM_ECUDA, cudaGetErrorString(e));
    }
    e = launch_finalize_pairs(partials, (int)nblocks, out, 2, s);
    if (e != cudaSuccess) return lbm_norms_fail(LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}
