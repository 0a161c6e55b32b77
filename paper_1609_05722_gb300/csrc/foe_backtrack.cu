// Reductions of the backtracking step control: the inner product <grad F(u^n), u^{n+1} - u^n> and the
// squared norm ||u^{n+1} - u^n||^2 of the sufficient-decrease test (Sec. 2.3, iPiano step sizes), in FP64.
#include "foe_kernels.h"

namespace foe {

namespace {

constexpr int kRowsPerBlock = 8;
constexpr int kThreads = 256;

__device__ __forceinline__ void block_sum2(double &a, double &b, double *sa, double *sb)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sa[w];
            b += sb[w];
        }
    }
}

__global__ void k_dot2(const float *g, const float *dl, int H, int W, int ld, double *partials)
{
    __shared__ double sa[kThreads / 32], sb[kThreads / 32];
    double a = 0.0, b = 0.0;
    const int y0 = blockIdx.x * kRowsPerBlock;
    for (int y = y0; y < y0 + kRowsPerBlock && y < H; ++y)
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const double gv = g[(size_t)y * ld + x], dv = dl[(size_t)y * ld + x];
            a += gv * dv;
            b += dv * dv;
        }
    block_sum2(a, b, sa, sb);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_dot2_final(const double *partials, int n, double *out)
{
    __shared__ double sa[kThreads / 32], sb[kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    block_sum2(a, b, sa, sb);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

}  // namespace

int dot2_blocks(int H) { return (H + kRowsPerBlock - 1) / kRowsPerBlock; }

cudaError_t launch_dot2(const float *g, const float *dl, int H, int W, int ld, double *partials, double *out,
                        cudaStream_t s)
{
    const int nb = dot2_blocks(H);
    k_dot2<<<nb, kThreads, 0, s>>>(g, dl, H, W, ld, partials);
    k_dot2_final<<<1, kThreads, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

}  // namespace foe
