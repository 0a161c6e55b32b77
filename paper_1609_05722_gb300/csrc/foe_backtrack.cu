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

// tau and the step constants of trial L (the same expressions as the host used, evaluated in IEEE double)
__device__ __forceinline__ void bt_set_trial(BtState *st)
{
    st->tau = (float)(2.0 * (1.0 - st->gam) / (st->L + st->c2));
    st->sc = make_step_consts(st->tau, st->gamma, st->lambda);
}

__global__ void k_bt_init(BtState *st, const double *F0, double L0, double gam, double c2, float gamma, float lambda,
                          int cap)
{
    st->L = L0;
    st->Fn = *F0;
    st->gam = gam;
    st->c2 = c2;
    st->gamma = gamma;
    st->lambda = lambda;
    st->trial = st->rejected = st->nlog = st->status = 0;
    st->cap = cap;
    st->tau_last = 0.0f;
    bt_set_trial(st);
}

__global__ void k_bt_decide(cudaGraphConditionalHandle h, BtState *st, const double *outs, float *log_tau,
                            unsigned char *log_acc, const int *stop)
{
    // a stopped image (stopping rule) or a failed solve: leave the state as it is and end the trial loop
    if (st->status != 0 || (stop && *(const volatile int *)stop != 0)) {
        cudaGraphSetConditional(h, 0u);
        return;
    }
    const double g_du = outs[0], du2 = outs[1], F1 = outs[2];
    if (!isfinite(g_du) || !isfinite(du2) || !isfinite(F1)) {
        st->status = kBtNonFinite;
        cudaGraphSetConditional(h, 0u);
        return;
    }
    const bool accept = F1 <= fma(0.5 * st->L, du2, st->Fn + g_du);
    if (st->nlog < st->cap) {
        log_tau[st->nlog] = st->tau;
        log_acc[st->nlog] = accept ? 1 : 0;
    }
    st->nlog++;
    if (accept) {
        st->Fn = F1;
        st->tau_last = st->tau;
        st->L /= 1.5;
        st->trial = 0;
        bt_set_trial(st);
        cudaGraphSetConditional(h, 0u);
        return;
    }
    st->L *= 2.0;
    st->rejected++;
    if (st->trial >= 60) {
        st->status = kBtNoStep;
        cudaGraphSetConditional(h, 0u);
        return;
    }
    st->trial++;
    bt_set_trial(st);
    cudaGraphSetConditional(h, 1u);
}

}  // namespace

cudaError_t launch_bt_init(BtState *st, const double *F0, double L0, double gam, double c2, float gamma, float lambda,
                           int cap, cudaStream_t s)
{
    k_bt_init<<<1, 1, 0, s>>>(st, F0, L0, gam, c2, gamma, lambda, cap);
    return cudaGetLastError();
}

cudaError_t launch_bt_decide(cudaGraphConditionalHandle h, BtState *st, const double *outs, float *log_tau,
                             unsigned char *log_acc, const int *stop, cudaStream_t s)
{
    k_bt_decide<<<1, 1, 0, s>>>(h, st, outs, log_tau, log_acc, stop);
    return cudaGetLastError();
}

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
