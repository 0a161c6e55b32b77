// Device-side definitions shared by the FoE kernels: launch descriptors, padding, the compensated
// FP32 iterate update and the pointwise proximal maps.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace foe {

constexpr int kNF = 48;     // filters (Sec. 2.5.3: 48 filters of 7x7)
constexpr int kKS = 7;      // filter side
constexpr int kKK = 49;     // taps
constexpr int kR = 3;       // filter radius
constexpr int kMaxBatch = 64;

enum Model : int { kDirect = 0, kAnsL2 = 1, kAnsIdiv = 2 };
enum Bc : int { kSymmetric = 0, kZero = 1 };
// kHess / kHvp (tensor-core kernel, TF32): the Hessian factors of the responses of u, then Hessian-vector products
enum Mode : int { kStep = 0, kGrad = 1, kEnergy = 2, kHvp = 3, kHess = 4 };

// Constants of one iPiano step (Eq. iPianoupdate) for one image.  Products that must stay
// accurate (tau*lambda and the quadratic prox weights) are carried as FP32 pairs hi + lo,
// computed on the host in FP64.
struct StepConsts {
    float tau, gamma, lambda;
    float c_hi, c_lo;          // c = tau * lambda
    float a1_hi, a1_lo;        // 1 / (1 + c)        (quadratic prox, Eq. subproblemGL2)
    float a2_hi, a2_lo;        // c / (1 + c)
};

// The constants of a step of size tau (host and device: the backtracking decides tau on the device and must
// reproduce the host's constants exactly, so no FMA contraction applies here: only products, sums and quotients).
__host__ __device__ inline StepConsts make_step_consts(float tau, float gamma, float lambda)
{
    StepConsts s;
    s.tau = tau;
    s.gamma = gamma;
    s.lambda = lambda;
    const double c = (double)tau * (double)lambda;  // exact: a product of two floats
    const double d = 1.0 + c;
    const double v[3] = {c, 1.0 / d, c / d};
    float *hi[3] = {&s.c_hi, &s.a1_hi, &s.a2_hi}, *lo[3] = {&s.c_lo, &s.a1_lo, &s.a2_lo};
    for (int i = 0; i < 3; ++i) {
        *hi[i] = (float)v[i];
        *lo[i] = (float)(v[i] - (double)*hi[i]);
    }
    return s;
}

// One image of a launch.  u_hi is double-buffered: a launch reads u_hi[parity] (with halos) and
// writes u_hi[parity ^ 1]; u_lo and delta are private to each pixel and updated in place.
struct ImgDesc {
    float *u_hi[2];
    float *u_lo;               // may be null in kGrad / kEnergy modes
    float *delta;              // u^n - u^{n-1}
    const float *d;            // data term: y (direct) or v (Anscombe models)
    float *out;                // kGrad: gradient; unused otherwise
    int H, W, ld;
    int tiles_x;
    int tile_h;                // tensor-core path: output rows of this image's tiles
    int model;
    StepConsts sc;
    float *hess;               // kHess writes, kHvp reads: per pixel the 48 factors (1 - r^2) / (1 + r^2)^2 of the
                               // responses r of u (the curvature rho'' / 2 of Sec. 2.5.2), [H][W][48] in the order
                               // of the tensor-core kernel's response columns
    const int *stop;           // nullable: the image's stopping word; non-zero once its stopping rule has held (the
                               // step count at that check), after which every step launch leaves the image as it is
};

struct LaunchArgs {
    int nimg;
    int parity;
    int bc;
    int nchunks;               // ceil(nf / 8)
    int prior_only;            // kGrad / kEnergy: the FoE prior term alone (no data term), 0 otherwise
    int withhold_arrival;      // failure-detection test: CTA 0 of the tensor-core step withholds one mbarrier
                               // arrival, so that a bounded wait expires (0 otherwise)
    const float *wts;          // device [48][49], correlation form w_i(a, b) = k_i(-a, -b)
    const float *alpha;        // device [48]
    double *partials;          // kEnergy: one FP64 partial per tile
    const void *tcops;         // tensor-core operand images (bf16): forward filters, then adjoint filters
    const void *tcops32;       // the same images in tf32
    const void *pairops;       // operand images of the pixel-pair kernel (bf16)
    const StepConsts *sc_dev;  // nullable: the step constants of every image of a kStep launch of the FP32 kernel,
                               // read from device memory (backtracking decides the step on the device)
    int tile_prefix[kMaxBatch + 1];
    ImgDesc img[kMaxBatch];
};

// Backward pass of the unrolled solve (training): one image of a launch.
struct BwdImg {
    const float *u;            // u^n
    const float *gb1;          // gbar^{n+1}
    const float *gb2;          // gbar^{n+2} (nullable: zero)
    float *gout;               // gbar^n
    int H, W, ld;
    int tiles_x;
};

constexpr int kBwdPartials = kNF * kKK + kNF;  // per-tile partial sums: filters (48 x 49), then weights (48)

struct BwdArgs {
    int nimg;
    int bc;
    int nchunks;
    int write_g;               // 0 at the last reverse step (gbar^0 is not needed)
    int hvp_only;              // 1: gout only (no parameter partials; partials may be null)
    float tau, gamma, c1;      // c1 = 1 / (1 + tau lambda)
    const float *wts;          // device [48][49], correlation form
    const float *alpha;        // device [48]
    float *partials;           // [tiles][kBwdPartials]
    int tile_prefix[kMaxBatch + 1];
    BwdImg img[kMaxBatch];
};

// Half-sample symmetric padding (edge repeated), any overshoot; -1 for zero padding outside.
__host__ __device__ inline int pad_index(int i, int n, int bc)
{
    if (bc == kZero) return (i >= 0 && i < n) ? i : -1;
    while (i < 0 || i >= n) {
        if (i < 0) i = -1 - i;
        if (i >= n) i = 2 * n - 1 - i;
    }
    return i;
}

// ---- error-free transformations on FP32 (Knuth two-sum, Dekker fast two-sum, FMA two-product) ----
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (ah + al) + (bh + bl)
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &rh, float &rl)
{
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, rh, rl);
}

// (ah + al) * (bh + bl), low-order cross term bl*al dropped
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &rh, float &rl)
{
    float p, e;
    two_prod(ah, bh, p, e);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    fast_two_sum(p, e, rh, rl);
}

// iPiano update of one pixel.  g = grad F(u^n) (FP32); the iterate is u = uh + ul, delta = u^n - u^{n-1}.
//   u~    = u - tau g + gamma delta                               (forward + inertial step)
//   u^{n+1} = prox(u~): quadratic (u~ + c d) / (1 + c)            (Eq. subproblemGL2)
//                      I-divergence (t + sqrt(t^2 + 4 c d)) / 2, t = u~ - c   (Eq. subproblemGIdiv)
// All in FP32 pair arithmetic so that rounding does not accumulate over hundreds of iterations.
__device__ __forceinline__ void ipiano_update(float g, float uh, float ul, float delta, float d, int model,
                                              const StepConsts &sc, float &nh, float &nl, float &ndelta)
{
    const float s = __fmaf_rn(sc.gamma, delta, -__fmul_rn(sc.tau, g));
    float th, tl;
    two_sum(uh, s, th, tl);
    tl = __fadd_rn(tl, ul);
    fast_two_sum(th, tl, th, tl);
    float ph, pl;
    if (model == kAnsL2) {
        float xh, xl, yh, yl;
        df_mul(th, tl, sc.a1_hi, sc.a1_lo, xh, xl);
        df_mul(d, 0.0f, sc.a2_hi, sc.a2_lo, yh, yl);
        df_add(xh, xl, yh, yl, ph, pl);
    } else {
        float qh, ql, sh, sl, mh, ml;
        df_add(th, tl, -sc.c_hi, -sc.c_lo, qh, ql);            // t = u~ - c
        df_mul(qh, ql, qh, ql, sh, sl);                        // t^2
        df_mul(4.0f * sc.c_hi, 4.0f * sc.c_lo, d, 0.0f, mh, ml);  // 4 c d
        float zh, zl;
        df_add(sh, sl, mh, ml, zh, zl);                        // t^2 + 4 c d >= 0
        float rh = 0.0f, rl = 0.0f;
        if (zh > 0.0f) {
            rh = __fsqrt_rn(zh);
            rl = __fdiv_rn(__fadd_rn(__fmaf_rn(-rh, rh, zh), zl), __fmul_rn(2.0f, rh));
        }
        df_add(qh, ql, rh, rl, ph, pl);
        ph *= 0.5f;
        pl *= 0.5f;
    }
    float dh, dl;
    df_add(ph, pl, -uh, -ul, dh, dl);
    nh = ph;
    nl = pl;
    ndelta = __fadd_rn(dh, dl);
}

// Gradient of the data term, FP32: lambda (1 - d / u) for the I-divergence forms, lambda (u - d) for the quadratic one.
__device__ __forceinline__ float data_grad(float u, float d, int model, float lambda)
{
    return model == kAnsL2 ? lambda * (u - d) : lambda * (1.0f - d / u);
}

// Data term energy of one pixel in FP64 (0 log 0 = 0).
__device__ __forceinline__ double data_energy(float u, float d, int model, float lambda)
{
    const double ud = u, dd = d;
    if (model == kAnsL2) return 0.5 * lambda * (ud - dd) * (ud - dd);
    if (dd == 0.0) return lambda * ud;
    return lambda * (ud - dd * log(ud));
}

// True when the image's stopping rule has held.  The word is written by the stopping check, a launch of its own
// between two step launches, and read here after any griddepcontrol.wait (L2, not a possibly stale L1 line).
__device__ __forceinline__ bool image_stopped(const ImgDesc &d) { return d.stop && __ldcg(d.stop) != 0; }

// Image index of a flat tile index (binary search over the launch's tile prefix).
__device__ __forceinline__ int tile_image(const LaunchArgs &a, int tile)
{
    int lo = 0, hi = a.nimg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.tile_prefix[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace foe
