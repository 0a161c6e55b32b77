// Host-side launchers of the FoE kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "foe_common.cuh"

namespace foe {

// Plain FP32 fused tile kernel (foe_f32.cu).
int f32_tile();
size_t f32_smem_bytes();
cudaError_t f32_setup();
cudaError_t f32_launch(const LaunchArgs &a, int mode, cudaStream_t s);

// Tensor-core (tcgen05, BF16 or TF32) fused tile kernels: 26 x 26 tiles (foe_tc.cu) and 58 x 58 pixel-pair tiles
// (foe_pair.cu, BF16 images of at least pair_min_rows() rows and pair_min_pixels() pixels).  tc_launch runs the
// images of a launch in the kernel their tiles belong to.
int tc_tile_h(bool tf32, int H, int W);  // output rows of the tensor-core tiles of an H x W image
int tc_tile_w(int tile_h);        // output columns of those tiles
cudaError_t tc_setup();
// A second stream and two events of the caller's context: a launch holding images of both tile sizes runs the
// 26 x 26 kernel on `stream`, forked from and joined back into the caller's stream, beside the pixel-pair kernel.
struct SideStream {
    cudaStream_t stream;
    cudaEvent_t fork, join;
};
cudaError_t tc_launch(const LaunchArgs &a, int mode, bool tf32, int *d_status, cudaStream_t s, const SideStream &side);
int pair_tile_w();  // output columns and rows of the pixel-pair tiles
int pair_tile_h();
int pair_min_rows();
long pair_min_pixels();
cudaError_t pair_setup();
// the images of `a` in pixel-pair tiles (all of them if `all`), one persistent CTA per SM
cudaError_t pair_launch(const LaunchArgs &a, int mode, bool all, int sms, int *d_status, cudaStream_t s);

// Backward pass of the unrolled solve (foe_train.cu).
int bwd_tile();
size_t bwd_smem_bytes();
cudaError_t bwd_setup();
cudaError_t bwd_launch(const BwdArgs &a, cudaStream_t s);
cudaError_t launch_train_loss(const float *u_hi, const float *u_lo, const float *clean, int H, int W, int ld, int cld,
                              float *gbar, double *partials, int nblocks, cudaStream_t s);
cudaError_t launch_reduce_partials(const float *partials, int tiles, double *acc, cudaStream_t s);
cudaError_t launch_train_finish(const double *acc, const float *alpha, float tau, int nf, float *dk, float *dla,
                                cudaStream_t s);
cudaError_t launch_copy(const float *src, float *dst, long n, cudaStream_t s);

cudaError_t launch_init(const float *y, int H, int W, int yld, int ld, int model, float zero_c, float *d, float *uh,
                        float *ul, float *delta, cudaStream_t s);
// x = the output map of the iterate; *nonfinite (nullable) += the number of non-finite outputs; x = NaN while
// *status (nullable: not checked) is non-zero.  With a stopping word (stop non-null) the iterate is read from uh when
// the step count, *stop if non-zero and `budget` otherwise, has the parity of `budget`, and from uh_alt when not.
cudaError_t launch_output(const float *uh, const float *ul, int H, int W, int ld, int xld, int model, float *x, int *nonfinite,
                          cudaStream_t s, const int *status = nullptr, const float *uh_alt = nullptr, int budget = 0,
                          const int *stop = nullptr);

// Stopping check (foe_tol.cu) after step n of the images of a launch: for every image whose word is still 0, in
// FP64 and a fixed summation order, dd = sum (u^n - u^{n-1})^2 (the delta plane) and uu = sum (u_hi + u_lo)^2; the
// word becomes n when sqrt(dd) <= tol sqrt(uu).
constexpr int kTolBlocks = 32;    // blocks per image (rows b, b + kTolBlocks, ...)
struct TolImg {
    const float *u_hi, *u_lo;     // u^n (u_lo nullable: 0)
    const float *delta;           // u^n - u^{n-1}
    int H, W, ld;
    int *stop;
};
struct TolArgs {
    int nimg, n;
    double tol;
    double *partials;             // [kMaxBatch][kTolBlocks][2]
    unsigned *count;              // [kMaxBatch], 0 between checks
    TolImg img[kMaxBatch];
};
cudaError_t launch_tol_check(const TolArgs &a, cudaStream_t s);
cudaError_t launch_anscombe(const float *y, float *v, long n, cudaStream_t s);
cudaError_t launch_inverse(const float *z, float *x, long n, cudaStream_t s);
cudaError_t launch_reduce(const double *p, int n, double *out, cudaStream_t s);

// Conjugate gradients of the implicit-differentiation gradient (foe_implicit.cu), B images of H x W (pitch ld,
// image stride H * ld).  part arrays hold kCgBlocks FP64 partials per image.
constexpr int kCgBlocks = 64;
struct CgState {
    double rr[2];      // <r, r> at iteration k (slot k & 1)
    double rr0;        // <b, b>
    int done[2];       // stopped before iteration k (slot k & 1)
    int iters;         // iterations taken
    int breakdown;     // stopped at <p, H_E p> <= 0
};
cudaError_t launch_cg_dot(const float *a, const float *c, int B, int H, int W, int ld, double *part, cudaStream_t s);
cudaError_t launch_cg_init(const double *part, CgState *st, int B, cudaStream_t s);
cudaError_t launch_cg_update(float *q, float *r, float *p, const float *Ap, int B, int H, int W, int ld,
                             const double *part_pap, double *part_rr, CgState *st, int k, double tol2, cudaStream_t s);

// Binning variant (foe_bin.cu): yb = ceil(H/3) x ceil(W/3) bin sums of y (pitch ldb); x = the bilinear upscaling of
// the bin image xb (pitch ldb) to H x W (pitch ld), divided by 9.
cudaError_t launch_bin3(const float *y, int H, int W, int ld, float *yb, int ldb, cudaStream_t s);
cudaError_t launch_upscale3(const float *xb, int ldb, float *x, int H, int W, int ld, cudaStream_t s);

// Step control (foe_backtrack.cu): out[0] = sum g * dl, out[1] = sum dl * dl over an H x W plane (pitch ld),
// FP64, in a fixed order (per-block partials in `partials`, 2 * dot2_blocks(H) doubles, then one block).
int dot2_blocks(int H);

// Device-side step decision (foe_backtrack.cu).  One trial of iteration n: the step with the trial's constants
// (st->sc), the two reductions above and F(u+); then k_bt_decide accepts it when
//   F(u+) <= F(u^n) + <grad F(u^n), u+ - u^n> + L/2 ||u+ - u^n||^2   (FP64, right side as fma(L/2, |du|^2, F + <g,du>))
// and sets the loop condition of the trial loop (a CUDA graph conditional node): 0 when accepted (L / 1.5 for the
// next iteration), 1 to retry with 2 L; more than 60 rejections in one iteration, or a non-finite scalar, end the
// solve with st->status set.
constexpr int kBtNoStep = 1, kBtNonFinite = 2;
struct BtState {
    double L, Fn;              // current estimate, F(u^n)
    double gam, c2;            // gamma (as a double), the 2 c2 term of tau = 2 (1 - gamma) / (L + 2 c2)
    float gamma, lambda;       // as the step constants take them
    float tau, tau_last;       // the current trial's step, the last accepted one
    int trial, rejected;       // trial index within the iteration, rejected trials so far
    int nlog, cap;             // trial log entries written (counting those past the capacity), capacity
    int status;                // 0, kBtNoStep, kBtNonFinite
    StepConsts sc;             // constants of the current trial
};
cudaError_t launch_bt_init(BtState *st, const double *F0, double L0, double gam, double c2, float gamma, float lambda,
                           int cap, cudaStream_t s);
cudaError_t launch_bt_decide(cudaGraphConditionalHandle h, BtState *st, const double *outs, float *log_tau,
                             unsigned char *log_acc, const int *stop, cudaStream_t s);
cudaError_t launch_dot2(const float *g, const float *dl, int H, int W, int ld, double *partials, double *out,
                        cudaStream_t s);

}  // namespace foe
