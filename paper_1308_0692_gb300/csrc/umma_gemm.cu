// BF16 GEMM on the fifth-generation tensor cores (sm_103a): C[M][N] (FP32) = A[M][K] B[N][K]^T
// (+ bias[N]), both operands K-major BF16 in global memory -- the products of the warm-start
// network (forward z = a W^T, input gradient da = g W, weight gradient dW = g^T a).
//
// One CTA of four warps computes a 128 x BN tile of C (BN = 256 or 128 -- 128 when 256-wide
// tiles would leave most SMs idle -- or 16 for the narrow products with N <= 16):
//   * warp 0, one lane: the producer.  Per 64-wide K step it has the Tensor Memory
//     Accelerator copy the A tile [128][64] and the B tile [BN][64] into a ring of STAGES
//     shared-memory stages (cp.async.bulk.tensor.2d, 128-byte swizzle, completion counted in
//     bytes on the stage's "full" mbarrier; rows or columns beyond the matrix are zero-filled
//     by the copy);
//   * warp 1, one lane: the MMA issuer.  Per stage four tcgen05.mma.cta_group::1.kind::f16
//     (M = 128, N = BN, K = 16 each) accumulate into a 128 x BN FP32 accumulator in tensor
//     memory (TMEM); tcgen05.commit then frees the stage ("empty" mbarrier) once those MMAs
//     have read it, and after the last stage signals the accumulator;
//   * all four warps: the epilogue.  Warp w reads TMEM lanes 32w..32w+31 (rows of the tile),
//     32 columns at a time, with tcgen05.ld, passes them through shared memory (the pipeline
//     stages are free by then) so that each store instruction writes 32 consecutive columns
//     of one row, and adds the bias.
// Split-K (gridDim.z > 1): CTA z takes K steps [z*kper, (z+1)*kper) and writes its partial
// tile to C + z * M * ldc; a second kernel sums the partials in a fixed order (deterministic).
//
// Every mbarrier wait is bounded: after the limit the thread sets *status and the CTA
// winds down (the MMA issuer still commits, so the epilogue's wait ends once the issued
// MMAs are done; the producer waits, bounded, for the copies it issued; TMEM is freed).
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "lbm_internal.h"

namespace {

constexpr int UM = 128;         // rows of a CTA tile (TMEM lanes)
constexpr int UK = 64;          // K elements per stage: one 128-byte swizzle row of BF16
constexpr int STAGES = 4;
constexpr long long WAIT_LIMIT = 2000000000LL;     // cycles (about a second)

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void bar_expect(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *b, unsigned parity)
{
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(su32(b)), "r"(parity), "r"(1000000u)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ bool bar_wait(uint64_t *b, unsigned parity)
{
    const long long t0 = clock64();
    while (!bar_try(b, parity))
        if (clock64() - t0 > WAIT_LIMIT) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *b)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(su32(dst)), "l"(map), "r"(x), "r"(y), "r"(su32(b))
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzling: rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1, layout code 2.
__device__ __forceinline__ uint64_t smem_desc(const void *tile)
{
    const uint64_t addr = su32(tile);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int BN>
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(b))
                 : "memory");
}

template <int BN>
struct Smem {
    static constexpr int A_BYTES = UM * UK * 2;
    static constexpr int B_BYTES = BN * UK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;             // multiple of 1024
    static constexpr int TOTAL = STAGES * STAGE + 1024;         // + alignment slack
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;         // power of two >= 32
};

template <int BN>
__global__ void __launch_bounds__(128, 1) umma_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                          const __grid_constant__ CUtensorMap tb, float *C, int ldc,
                                                          const float *bias, int M, int N, int ktiles, int kper,
                                                          int *status)
{
    using S = Smem<BN>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accf;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * UM, n0 = blockIdx.x * BN;
    const int kt0 = blockIdx.z * kper;
    const int kt1 = min(ktiles, kt0 + kper);
    float *Cz = C + (size_t)blockIdx.z * M * ldc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        bar_init(&accf, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&ta) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tb) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&s_tmem)),
                     "r"(S::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        int issued = 0;
        for (int kt = kt0; kt < kt1; ++kt, ++issued) {
            const int s = issued % STAGES;
            if (issued >= STAGES && !bar_wait(&empty[s], ((issued / STAGES) - 1) & 1)) {
                atomicExch(status, 1);
                s_abort = 1;
                break;
            }
            unsigned char *st = smem + s * S::STAGE;
            bar_expect(&full[s], S::STAGE);
            tma_load_2d(st, &ta, kt * UK, m0, &full[s]);
            tma_load_2d(st + S::A_BYTES, &tb, kt * UK, n0, &full[s]);
        }
        // the copies still in flight land before the CTA can exit
        for (int j = issued > STAGES ? issued - STAGES : 0; j < issued; ++j)
            bar_wait(&full[j % STAGES], (j / STAGES) & 1);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        constexpr uint32_t idesc = instr_desc<BN>();
        int done = 0;
        for (int kt = kt0; kt < kt1; ++kt, ++done) {
            const int s = done % STAGES;
            if (!bar_wait(&full[s], (done / STAGES) & 1)) {
                atomicExch(status, 1);
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned char *st = smem + s * S::STAGE;
            const uint64_t da = smem_desc(st), db = smem_desc(st + S::A_BYTES);
#pragma unroll
            for (int k = 0; k < UK / 16; ++k)   // advance 16 BF16 = 32 bytes along K inside the swizzle row
                mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (done > 0 || k > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        mma_commit(&accf);
    }
    __syncwarp();
    __syncthreads();     // the producer's copies have all landed: the stages can take the staging

    // ---- epilogue: all four warps ----
    const bool ok = bar_wait(&accf, 0);
    if (!ok && lane == 0) atomicExch(status, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const bool any = kt1 > kt0;
    float *stg = reinterpret_cast<float *>(smem) + warp * 32 * 33;    // [32 rows][33], padded
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                           "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                           "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = any ? __uint_as_float(r[j]) : 0.f;
            __syncwarp();
            const int col = n0 + c0 + lane;
            const float bv = (bias && col < N) ? bias[col] : 0.f;
            if (col < N) {
#pragma unroll 4
                for (int rr = 0; rr < 32; ++rr) {
                    const int row = m0 + warp * 32 + rr;
                    if (row < M) Cz[(size_t)row * ldc + col] = stg[rr * 33 + lane] + bv;
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(S::TMEM_COLS));
    }
}

// C[r][c] (+ bias[c]) = sum over z of the split-K partials P[z][r][c], z ascending
__global__ void splitk_sum_kernel(const float *P, int splits, int M, int N, int ld, const float *bias, float *C,
                                  int ldc)
{
    const long n = (long)M * N;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / N), c = (int)(i - (long)r * N);
        float v = 0.f;
        for (int z = 0; z < splits; ++z) v += P[((size_t)z * M + r) * ld + c];
        if (bias) v += bias[c];
        C[(size_t)r * ldc + c] = v;
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

// tensor map of a row-major BF16 matrix [rows][cols] (row pitch ld elements), box [box_rows][64]
bool make_map(CUtensorMap *map, const __nv_bfloat16 *base, int rows, int cols, int ld, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)UK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap &ta, const CUtensorMap &tb, float *C, int ldc, const float *bias, int M,
                      int N, int ktiles, int splits, int *status, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(umma_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<BN>::TOTAL);
    });
    if (attr != cudaSuccess) return attr;
    const int kper = (ktiles + splits - 1) / splits;
    dim3 grid((N + BN - 1) / BN, (M + UM - 1) / UM, splits);
    umma_gemm_kernel<BN><<<grid, 128, Smem<BN>::TOTAL, s>>>(ta, tb, C, ldc, bias, M, N, ktiles, kper, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t umma_gemm_nt(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, float *C, int ldc,
                         const float *bias, int M, int N, int K, int splits, float *partials, int *status,
                         cudaStream_t s)
{
    if (M < 1 || N < 1 || K < 1 || N > 256 || lda % 8 || ldb % 8 || K > lda || K > ldb) return cudaErrorInvalidValue;
    if ((((uintptr_t)A) & 15) || (((uintptr_t)B) & 15)) return cudaErrorInvalidValue;
    const int ktiles = (K + UK - 1) / UK;
    if (splits < 1) splits = 1;
    if (splits > ktiles) splits = ktiles;
    const bool split = splits > 1 && partials;
    // 256-wide tiles unless they would leave most SMs idle
    int bn = N <= 16 ? 16 : 256;
    if (bn == 256 && (long)((M + UM - 1) / UM) * ((N + 255) / 256) * (split ? splits : 1) < 152) bn = 128;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, lda, UM) || !make_map(&tb, B, N, K, ldb, bn)) return cudaErrorInvalidValue;
    float *out = split ? partials : C;
    const int ldo = split ? N : ldc;
    const float *b = split ? nullptr : bias;
    const int z = split ? splits : 1;
    cudaError_t e = bn == 16    ? launch_bn<16>(ta, tb, out, ldo, b, M, N, ktiles, z, status, s)
                    : bn == 128 ? launch_bn<128>(ta, tb, out, ldo, b, M, N, ktiles, z, status, s)
                                : launch_bn<256>(ta, tb, out, ldo, b, M, N, ktiles, z, status, s);
    if (e != cudaSuccess || !split) return e;
    const long n = (long)M * N;
    const int nb = (int)std::min<long>(1216, (n + 255) / 256);
    splitk_sum_kernel<<<nb, 256, 0, s>>>(partials, splits, M, N, N, bias, C, ldc);
    return cudaGetLastError();
}
