// Cost of one tcgen05.mma (kind::f16: BF16 operands, FP32 accumulator in tensor memory) by shape and operand
// source, measured with clock64 on one SM, or on the SM pair of a two-CTA cluster for cta_group::2.  A diagnostic
// entry point (foe_mma_cost), not part of any solve: it gives the contraction ceiling that bounds the tensor-core
// step kernels whatever their pipeline, for the orientations those kernels use and for the ones they could use
// (pixels on the N = 256 side, the A operand in tensor memory, M = 256 over two SMs).
//
// One or two issuing warps each enqueue `count` MMAs into their own accumulator, cycling over four K = 16 steps of
// a K = 64 operand region; one commit per warp; warp 0 waits (bounded) for the commits.  The region is timed twice
// and the second pass reported, so that the first MMA's start-up is not in the figure.
#include <cstdint>
#include <cuda_runtime.h>

#include "foe.h"
#include "foe_ptx.cuh"

namespace foe {
namespace {

using namespace ptx;

constexpr int kRowCap = 256;                                   // rows per 16-byte K chunk of an operand region
constexpr uint32_t kChunkBytes = 16u * kRowCap;                // 4096: stride between K chunks (leading byte offset)
constexpr int kKSteps = 4;                                     // K = 64 per region: four K = 16 steps, cycled
constexpr uint32_t kRegionBytes = 2u * kChunkBytes * kKSteps;  // 32 KB per operand
constexpr uint32_t kATmemCol = 480;                            // A in tensor memory: 4 steps x 8 columns
constexpr uint32_t kTmemCols = 512;
constexpr size_t kSmem = 160 * 1024;                           // above half an SM's shared memory: one CTA per SM

struct CostArgs {
    int m, n, a_tmem, issuers, count;
    long long *cycles;   // [1]: cycles of the timed pass, CTA rank 0
    int *status;         // FOE_ETIMEOUT if a wait expired
};

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_pair_elect(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// arrive on the mbarrier at this offset in both CTAs of the pair once this thread's MMAs are complete
__device__ __forceinline__ void commit_pair_elect(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// PAIR: a cluster of two CTAs, every tcgen05 instruction of the kernel with cta_group::2 (M = 256: each CTA holds
// 128 rows of A, N / 2 rows of B and 128 lanes of the accumulator), issued by CTA rank 0.  Otherwise one CTA,
// cta_group::1 throughout.
template <bool PAIR>
__global__ void __launch_bounds__(128, 1) k_mma_cost(CostArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5;
    uint32_t rank = 0;
    if constexpr (PAIR) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));

    // operands: bf16 values in [0.125, 0.25), so that every accumulation stays finite
    uint32_t *w = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t i = threadIdx.x; i < 2u * kRegionBytes / 4u; i += blockDim.x) w[i] = (0x3E00u + 16u * (i % 7u)) * 0x10001u;
    fence_async_smem();
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        if constexpr (PAIR) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        if constexpr (PAIR)
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                         "r"(kTmemCols)
                         : "memory");
        else
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                         "r"(kTmemCols)
                         : "memory");
    }
    fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();
    fence_after();
    const uint32_t tmem = tmem_base;
    if (!PAIR && a.a_tmem) {
        // A operand in tensor memory: lanes 32 warp .. + 31, columns kATmemCol .. + 31
        uint32_t v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = (0x3E00u + 16u * ((threadIdx.x + i) % 7u)) * 0x10001u;
        tmem_st32(tmem + ((uint32_t)(32 * warp) << 16) + kATmemCol, v);
        tmem_wait_st();
        fence_before();
        __syncthreads();
        fence_after();
    }

    const uint32_t idesc = idesc_bf16((uint32_t)a.m, (uint32_t)a.n);
    const uint32_t sA = smem_u32(smem), sB = sA + kRegionBytes;
    const bool issuer = warp < a.issuers && rank == 0;
    for (int rep = 0; rep < 2; ++rep) {
        if constexpr (PAIR) cluster_sync();
        else __syncthreads();
        const long long t0 = clock64();
        if (issuer) {
            const uint32_t d = tmem + 256u * (uint32_t)warp;
            for (int i = 0; i < a.count; ++i) {
                const uint32_t s = (uint32_t)(i & (kKSteps - 1));
                const uint64_t bd = sdesc(sB + 2u * kChunkBytes * s, kChunkBytes, 128);
                const uint32_t acc = (rep > 0 || i > 0) ? 1u : 0u;
                if constexpr (PAIR) {
                    mma_pair_elect(d, sdesc(sA + 2u * kChunkBytes * s, kChunkBytes, 128), bd, idesc, acc);
                } else {
                    if (a.a_tmem) mma_ta_elect<false>(d, tmem + kATmemCol + 8u * s, bd, idesc, acc);
                    else mma_elect<false>(d, sdesc(sA + 2u * kChunkBytes * s, kChunkBytes, 128), bd, idesc, acc);
                }
            }
            if constexpr (PAIR) commit_pair_elect(&bar[warp]);
            else commit_elect(&bar[warp]);
        }
        if (warp == 0) {
            for (int k = 0; k < a.issuers; ++k) mbar_wait_drain(&bar[k], (uint32_t)rep, a.status);
            const long long t1 = clock64();
            if (rep == 1 && rank == 0 && threadIdx.x == 0) a.cycles[0] = t1 - t0;
        }
    }

    fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();
    if (warp == 0) {
        fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace
}  // namespace foe

extern "C" FOE_API foe_status foe_mma_cost(int m, int n, int a_in_tmem, int cta_pair, int issuers, int count,
                                           double *cycles_per_mma)
{
    using namespace foe;
    if (!cycles_per_mma || issuers < 1 || issuers > 2 || count < 1 || count > 65536) return FOE_EINVAL;
    if ((a_in_tmem != 0 && a_in_tmem != 1) || (cta_pair != 0 && cta_pair != 1)) return FOE_EINVAL;
    if (cta_pair) {
        if (m != 256 || a_in_tmem || n < 32 || n > 256 || n % 16) return FOE_EINVAL;
    } else {
        if (m == 64) {
            if (n < 8 || n > 256 || n % 8 || a_in_tmem) return FOE_EINVAL;
        } else if (m == 128) {
            if (n < 16 || n > 256 || n % 16) return FOE_EINVAL;
        } else {
            return FOE_EINVAL;
        }
        // accumulators at columns 0 and 256; the A operand at kATmemCol
        if (a_in_tmem && 256 * (issuers - 1) + n > (int)kATmemCol) return FOE_EINVAL;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FOE_ECUDA;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return FOE_EUNSUPPORTED;

    long long *d_cycles = nullptr;
    int *d_status = nullptr;
    if (cudaMalloc(&d_cycles, sizeof(long long)) != cudaSuccess) return FOE_ENOMEM;
    if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess) {
        cudaFree(d_cycles);
        return FOE_ENOMEM;
    }
    foe_status st = FOE_OK;
    cudaMemset(d_cycles, 0, sizeof(long long));
    cudaMemset(d_status, 0, sizeof(int));
    CostArgs args{m, n, a_in_tmem, issuers, count, d_cycles, d_status};
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = kSmem;
    cudaError_t e;
    if (cta_pair) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaFuncSetAttribute(k_mma_cost<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_mma_cost<true>, args);
    } else {
        cfg.gridDim = dim3(1);
        e = cudaFuncSetAttribute(k_mma_cost<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_mma_cost<false>, args);
    }
    long long cyc = 0;
    int dst = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&cyc, d_cycles, sizeof cyc, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&dst, d_status, sizeof dst, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = FOE_ECUDA;
    else if (dst != 0) st = (foe_status)dst;
    cudaFree(d_cycles);
    cudaFree(d_status);
    if (st == FOE_OK) *cycles_per_mma = (double)cyc / ((double)issuers * (double)count);
    return st;
}
