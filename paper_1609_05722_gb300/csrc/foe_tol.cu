// Stopping check of the iPiano solve (the relative change of the iterate, ||u^n - u^{n-1}|| <= tol ||u^n||; the
// paper runs to convergence and reports the iteration counts, Sec. 5.1, without fixing a rule).
//
// One launch checks every image of a step launch: kTolBlocks blocks per image each sum, in FP64, the squares of the
// delta plane (u^n - u^{n-1}) and of the iterate over rows b, b + kTolBlocks, ...; the last block of an image to
// finish (an atomic count) adds the kTolBlocks partials in block order, so the result does not depend on the
// blocks' schedule, and writes the stopping word.  Bytes per pixel: 8 (u_hi, delta), 12 with u_lo.
#include "foe_kernels.h"

namespace foe {
namespace {

constexpr int kTolThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kTolThreads) k_tol_check(const __grid_constant__ TolArgs A)
{
    const int j = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
    const TolImg &I = A.img[j];
    if (__ldcg(I.stop) != 0) return;  // stopped at an earlier check: every block of the image returns here
    double dd = 0.0, uu = 0.0;
    for (int r = b; r < I.H; r += kTolBlocks) {
        const size_t row = (size_t)r * I.ld;
        for (int c = tid; c < I.W; c += kTolThreads) {
            const double e = (double)I.delta[row + c];
            const double u = (double)I.u_hi[row + c] + (I.u_lo ? (double)I.u_lo[row + c] : 0.0);
            dd = fma(e, e, dd);
            uu = fma(u, u, uu);
        }
    }
    __shared__ double sd[kTolThreads / 32], su[kTolThreads / 32];
    __shared__ bool last;
    dd = warp_sum(dd);
    uu = warp_sum(uu);
    if ((tid & 31) == 0) {
        sd[tid >> 5] = dd;
        su[tid >> 5] = uu;
    }
    __syncthreads();
    if (tid == 0) {
        double bd = 0.0, bu = 0.0;
        for (int w = 0; w < kTolThreads / 32; ++w) {
            bd += sd[w];
            bu += su[w];
        }
        double *p = A.partials + ((size_t)j * kTolBlocks + b) * 2;
        p[0] = bd;
        p[1] = bu;
        __threadfence();
        last = atomicAdd(&A.count[j], 1u) == (unsigned)(kTolBlocks - 1);
    }
    __syncthreads();
    if (!last || tid != 0) return;
    __threadfence();
    const double *p = A.partials + (size_t)j * kTolBlocks * 2;
    double td = 0.0, tu = 0.0;
    for (int k = 0; k < kTolBlocks; ++k) {
        td += __ldcg(p + 2 * k);
        tu += __ldcg(p + 2 * k + 1);
    }
    A.count[j] = 0u;
    if (sqrt(td) <= A.tol * sqrt(tu)) *I.stop = A.n;
}

}  // namespace

cudaError_t launch_tol_check(const TolArgs &a, cudaStream_t s)
{
    if (a.nimg <= 0) return cudaSuccess;
    k_tol_check<<<dim3(kTolBlocks, a.nimg), kTolThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace foe
