// Conjugate gradients for the implicit-differentiation training gradient (Sec. 2.5, Eq. implicitdifferentiation):
// q = H_E(w*)^{-1} b per image, b = dL/dw, from q = 0.  The products H_E p come from the backward kernel in its
// Hessian-vector mode; these kernels do the rest of an iteration for a batch of equally sized images, with FP64
// dot products reduced in a fixed order (per (image, block) partials, summed in block order by whoever needs the
// value), so the result does not depend on scheduling.  Scalars stay on the device: an iteration is four launches
// (product, <p, Ap>, the q / r update with <r, r>, the p update) and no host synchronisation.
//   alpha = <r, r> / <p, Ap>;  q += alpha p;  r -= alpha Ap;  beta = <r', r'> / <r, r>;  p = r' + beta p.
// An image stops (alpha = 0 from then on) once ||r|| <= tol ||b||, or when <p, Ap> <= 0 (H_E not positive
// definite along p: recorded as a breakdown).  rr and the stop flag are double-buffered by iteration parity, so
// the blocks of one launch never see a value written in the same launch.
#include "foe_common.cuh"
#include "foe_kernels.h"

namespace foe {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;  // valid in thread 0
}

__device__ __forceinline__ double sum_parts(const double *part, int i)
{
    double t = 0.0;
    for (int b = 0; b < kCgBlocks; ++b) t += part[(size_t)i * kCgBlocks + b];
    return t;
}

// part[i][block] = partial sum of a . c over image i
__global__ void k_cg_dot(const float *a, const float *c, int H, int W, int ld, size_t plane, double *part)
{
    const int i = blockIdx.y;
    const float *ai = a + (size_t)i * plane, *ci = c + (size_t)i * plane;
    double acc = 0.0;
    const long n = (long)H * W;
    for (long e = blockIdx.x * (long)kThreads + threadIdx.x; e < n; e += (long)kCgBlocks * kThreads) {
        const size_t idx = (size_t)(e / W) * ld + (size_t)(e % W);
        acc += (double)ai[idx] * (double)ci[idx];
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[(size_t)i * kCgBlocks + blockIdx.x] = t;
}

// st[i] from <b, b>: rr[0] = rr0, stop flag if b = 0
__global__ void k_cg_init(const double *part, CgState *st, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double rr0 = sum_parts(part, i);
    st[i].rr[0] = st[i].rr[1] = rr0;
    st[i].rr0 = rr0;
    st[i].done[0] = st[i].done[1] = !(rr0 > 0.0);
    st[i].iters = 0;
    st[i].breakdown = 0;
}

// q += alpha p, r -= alpha Ap; part_rr[i][block] = partial sum of r . r after the update
__global__ void k_cg_qr(float *q, float *r, const float *p, const float *Ap, int H, int W, int ld, size_t plane,
                        const double *part_pap, const CgState *st, int k, double *part_rr)
{
    const int i = blockIdx.y;
    __shared__ double alpha_s;
    if (threadIdx.x == 0) {
        const double pap = sum_parts(part_pap, i);
        alpha_s = (st[i].done[k & 1] || !(pap > 0.0)) ? 0.0 : st[i].rr[k & 1] / pap;
    }
    __syncthreads();
    const float alpha = (float)alpha_s;
    float *qi = q + (size_t)i * plane, *ri = r + (size_t)i * plane;
    const float *pi = p + (size_t)i * plane, *ai = Ap + (size_t)i * plane;
    double acc = 0.0;
    const long n = (long)H * W;
    for (long e = blockIdx.x * (long)kThreads + threadIdx.x; e < n; e += (long)kCgBlocks * kThreads) {
        const size_t idx = (size_t)(e / W) * ld + (size_t)(e % W);
        const float rv = fmaf(-alpha, ai[idx], ri[idx]);
        qi[idx] = fmaf(alpha, pi[idx], qi[idx]);
        ri[idx] = rv;
        acc += (double)rv * (double)rv;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part_rr[(size_t)i * kCgBlocks + blockIdx.x] = t;
}

// p = r + beta p; block 0 records rr, the stop flag and the iteration count for iteration k + 1
__global__ void k_cg_p(float *p, const float *r, int H, int W, int ld, size_t plane, const double *part_pap,
                       const double *part_rr, CgState *st, int k, double tol2)
{
    const int i = blockIdx.y;
    __shared__ double beta_s;
    __shared__ int skip_s;
    if (threadIdx.x == 0) {
        const int done = st[i].done[k & 1];
        const double rr = st[i].rr[k & 1], rr1 = sum_parts(part_rr, i), pap = sum_parts(part_pap, i);
        const bool brk = !done && !(pap > 0.0);
        skip_s = done || brk;
        beta_s = skip_s ? 0.0 : rr1 / rr;
        if (blockIdx.x == 0) {
            CgState &s = st[i];
            if (done || brk) {
                s.rr[(k + 1) & 1] = rr;
                s.done[(k + 1) & 1] = 1;
                if (brk) s.breakdown = 1;
            } else {
                s.rr[(k + 1) & 1] = rr1;
                s.done[(k + 1) & 1] = rr1 <= tol2 * s.rr0;
                s.iters = k + 1;
            }
        }
    }
    __syncthreads();
    if (skip_s) return;
    const float beta = (float)beta_s;
    float *pi = p + (size_t)i * plane;
    const float *ri = r + (size_t)i * plane;
    const long n = (long)H * W;
    for (long e = blockIdx.x * (long)kThreads + threadIdx.x; e < n; e += (long)kCgBlocks * kThreads) {
        const size_t idx = (size_t)(e / W) * ld + (size_t)(e % W);
        pi[idx] = fmaf(beta, pi[idx], ri[idx]);
    }
}

}  // namespace

cudaError_t launch_cg_dot(const float *a, const float *c, int B, int H, int W, int ld, double *part, cudaStream_t s)
{
    k_cg_dot<<<dim3(kCgBlocks, B), kThreads, 0, s>>>(a, c, H, W, ld, (size_t)H * ld, part);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(const double *part, CgState *st, int B, cudaStream_t s)
{
    k_cg_init<<<(B + 63) / 64, 64, 0, s>>>(part, st, B);
    return cudaGetLastError();
}

cudaError_t launch_cg_update(float *q, float *r, float *p, const float *Ap, int B, int H, int W, int ld,
                             const double *part_pap, double *part_rr, CgState *st, int k, double tol2, cudaStream_t s)
{
    const size_t plane = (size_t)H * ld;
    k_cg_qr<<<dim3(kCgBlocks, B), kThreads, 0, s>>>(q, r, p, Ap, H, W, ld, plane, part_pap, st, k, part_rr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cg_p<<<dim3(kCgBlocks, B), kThreads, 0, s>>>(p, r, H, W, ld, plane, part_pap, part_rr, st, k, tol2);
    return cudaGetLastError();
}

}  // namespace foe
