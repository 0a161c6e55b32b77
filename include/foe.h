/*
 * foe.h: C ABI of the GB300 FoE Poisson denoiser.
 *
 * Method: Feng, Qiao, Chen, "Poisson Noise Reduction with Higher-order Natural Image Prior Model"
 * (arXiv:1609.05722).  Each solve minimises
 *
 *     E(u) = sum_i alpha_i sum_p rho((k_i * u)_p) + D(u),   rho(z) = log(1 + z^2)   (Eq. FOEmodel, STfunc)
 *
 * with iPiano (Eq. iPianoupdate): u+ = prox_{tau D}(u - tau grad F(u) + gamma (u - u-)),
 * grad F(u) = sum_i alpha_i K_i^T rho'(K_i u) (Eq. FoEF).  Three data terms D:
 *   FOE_MODEL_DIRECT    lambda <x - y log x, 1> on the counts y           (Eq. straightforward, prox Eq. subproblemGIdiv)
 *   FOE_MODEL_ANS_L2    lambda/2 ||u - v||^2, v = 2 sqrt(y + 3/8)         (Eq. overallModel, prox Eq. subproblemGL2)
 *   FOE_MODEL_ANS_IDIV  lambda <u - v log u, 1> in the Anscombe domain    (Eq. lowcase)
 *   FOE_MODEL_AUTO      ANS_L2 if peak >= 5 else ANS_IDIV                 (Eq. FOEscheme)
 * The Anscombe models return x = I_C(max(u, sqrt(3/2))) (Eq. invAns); the direct model returns u.
 *
 * Conventions
 *   - Images are FP32, row-major, H rows x W columns, row pitch ld floats (ld >= W, ld % 4 == 0),
 *     device-resident unless a parameter says "host".  H, W >= 7.
 *   - Filters are 7x7 convolution kernels: filters[i*49 + (a+3)*7 + (b+3)] = k_i(a, b), a, b in -3..3,
 *     (k * u)_p = sum_{a,b} k(a, b) u(p - (a, b)).  Responses exist at the image pixels only, on the
 *     image padded by P: FOE_BC_SYMMETRIC = half-sample reflection (edge repeated), FOE_BC_ZERO = zeros.
 *     The gradient is the exact adjoint P^T K_valid^T.
 *   - Ownership: the caller owns every image buffer; the context owns its filter copies, its cached
 *     step size and its workspace (grown on demand with cudaMalloc; never shrunk until foe_destroy).
 *   - Execution: calls are stream-ordered on the given cudaStream_t (NULL = legacy default stream).
 *     Results written to host pointers (energies, reports) synchronise that stream first.
 *   - Errors: no call aborts or throws.  Each returns a foe_status; foe_last_error(ctx) gives text.
 *     Argument errors are detected on the host before any device work (FOE_EINVAL).
 *   - Threads: a context may be used by one host thread at a time.
 */
#ifndef FOE_H
#define FOE_H

#include <stddef.h>

#if defined(__GNUC__)
#define FOE_API __attribute__((visibility("default")))
#else
#define FOE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FOE_OK = 0,
    FOE_EINVAL = 1,       /* bad argument (detected on the host, nothing launched) */
    FOE_ENOMEM = 2,       /* device or host allocation failed */
    FOE_ECUDA = 3,        /* a CUDA runtime call failed; the text names it */
    FOE_ENONFINITE = 4,   /* a non-finite value was produced */
    FOE_ETIMEOUT = 5,     /* a bounded device-side wait expired */
    FOE_EBUSY = 6,        /* resource in use */
    FOE_EUNSUPPORTED = 7  /* option not implemented for this combination */
} foe_status;

typedef enum { FOE_MODEL_DIRECT = 0, FOE_MODEL_ANS_L2 = 1, FOE_MODEL_ANS_IDIV = 2, FOE_MODEL_AUTO = 3 } foe_model;

/* Arithmetic of the 96 convolutions per iteration: FP32 on the FFMA units, or tcgen05 tensor cores with
 * TF32 or BF16 operands and FP32 accumulation.  State, data term and prox are always FP32: the FP32 path
 * holds the iterate as an unevaluated FP32 pair hi + lo, the tensor-core paths as plain FP32 (their BF16 /
 * TF32 rounding of u and psi is orders of magnitude above the drift that the pair removes). */
typedef enum { FOE_PREC_FP32 = 0, FOE_PREC_TF32 = 1, FOE_PREC_BF16 = 2 } foe_precision;

typedef enum { FOE_BC_SYMMETRIC = 0, FOE_BC_ZERO = 1 } foe_bc;

typedef enum { FOE_STEP_FIXED = 0, FOE_STEP_BACKTRACK = 1 } foe_step_mode;

typedef struct foe_ctx foe_ctx;

/* FoE prior (Eq. FOEmodel): nf filters of ksize x ksize and their weights (host memory, copied). */
typedef struct {
    int nf;               /* 1..48 */
    int ksize;            /* must be 7 */
    const float *filters; /* host, [nf][49] convolution kernels as described above */
    const float *alpha;   /* host, [nf], > 0 (the weights themselves, i.e. e^{alpha} of Eq. learningmodel) */
} foe_prior;

typedef struct {
    foe_model model;
    float lambda;         /* data-term weight, > 0 */
    float gamma;          /* inertia, 0 <= gamma < 1 */
    float tau;            /* step size; 0 = the context's default for (bc, gamma) */
    float tol;            /* stopping rule, >= 0 (0: every solve runs its whole iteration budget).  The paper
                             runs iPiano to convergence and reports the iteration counts (Sec. 5.1) without
                             fixing a rule; the rule here: after step n, n a multiple of tol_every, an image
                             stops at u^n once ||u^n - u^{n-1}||_2 <= tol ||u^n||_2, both norms summed in
                             FP64 on the device in a fixed order.  The output is then the map of u^n; the
                             budget (`iters`, or the desc's) caps n.  foe_iters_done returns the counts. */
    int iters;            /* >= 0 */
    foe_step_mode step;   /* FIXED: constant tau.  BACKTRACK (foe_denoise with FOE_PREC_FP32 only; the other
                             entry points return FOE_EUNSUPPORTED): Lipschitz backtracking on the prior, see
                             foe_denoise */
    foe_bc bc;
    foe_precision prec;
    float zero_c;         /* direct model: zero counts are replaced by zero_c (Sec. 3.1.1), >= 0 */
    int use_graph;        /* foe_denoise_batch: 1 = capture the whole batch solve (initialisation, every
                             iteration launch, output maps) as one CUDA graph and replay it; needs a
                             non-default stream (on the legacy default stream the launches are issued
                             directly).  The instantiated graph is cached in the context and updated in
                             place when the next batch has the same launch structure. */
    int tol_every;        /* check interval of the stopping rule, >= 1 when tol > 0.  A check reads the
                             iterate and its last change once (8 bytes per pixel, 12 on the FP32 path). */
} foe_solve_opts;

typedef struct {
    int iters_done;
    int model_used;       /* resolved foe_model (never AUTO) */
    float tau_used;       /* FIXED: the step size; BACKTRACK: the last accepted one */
    foe_status status;
    int backtracks;       /* BACKTRACK: rejected trials (0 for FIXED) */
    double lipschitz_final; /* BACKTRACK: L after the last step; FIXED: the L that tau_used corresponds to */
    int nonfinite;        /* non-finite output pixels (NaN / Inf sentinel); the call then returns FOE_ENONFINITE */
} foe_report;

/* One image of a batch (foe_denoise_batch). */
typedef struct {
    const float *y;       /* device, noisy counts, H x W, pitch ld */
    float *x;             /* device, output, H x W, pitch ld (may alias y) */
    int H, W, ld;
    float peak;           /* used for FOE_MODEL_AUTO */
    int iters;            /* per-image iteration budget, >= 0 */
    int use_model;        /* 0: the image takes opts->model; 1: it takes `model` (images of different data
                             terms then share one batch).  Zero-initialised descriptors keep the first. */
    foe_model model;      /* read when use_model is 1: DIRECT, ANS_L2, ANS_IDIV or AUTO */
} foe_image_desc;

/* Fills *opts with the defaults: AUTO model, lambda 1, gamma 0.8, tau 0 (auto), no stopping rule (tol 0,
 * tol_every 10), 300 iterations, fixed steps, symmetric padding, BF16 convolutions, zero_c 0, no graph
 * capture. */
FOE_API foe_status foe_default_opts(foe_solve_opts *opts);

/* Creates a context for one prior: validates it, copies the filters to the device and precomputes
 * the Lipschitz bound of grad F used for the default step size.  Needs a current CUDA device. */
FOE_API foe_status foe_create(const foe_prior *prior, foe_ctx **out);

/* Releases the context and its device memory.  NULL is ignored.  The caller must make sure no
 * work that uses the context is still running. */
FOE_API void foe_destroy(foe_ctx *ctx);

/* Host-only: the step size used when opts.tau == 0.
 *   L   = 2 kappa max_w sum_i alpha_i |k_i^(w)|^2  (kappa = 4 symmetric, 1 zero padding; the maximum
 *         over a 512 x 512 DTFT grid, FP64), a bound on the Lipschitz constant of grad F
 *         (|rho''| <= 2, Sec. 2.5.2);
 *   tau = 0.99 * 2 (1 - gamma) / (L + 2e-3), inside iPiano's step condition tau < 2 (1 - gamma) / L.
 * Either output pointer may be NULL. */
FOE_API foe_status foe_step_size(const foe_ctx *ctx, foe_bc bc, float gamma, float *tau_out, double *lipschitz_out);

/* Host-only, needs no device: the Lipschitz bound L above for a prior that has no context yet. */
FOE_API foe_status foe_prior_lipschitz(const foe_prior *prior, foe_bc bc, double *lipschitz_out);

/* Trials of the context's last FOE_STEP_BACKTRACK solve, in order: tau[i] the trial's step size,
 * accepted[i] 1 if it was taken, 0 if it was rejected (L doubled).  Copies min(n, max_n) entries into the host
 * arrays (which may be NULL when max_n = 0) and returns n, the number of trials; -1 on invalid arguments.
 * Accepted trials are exactly one per iteration. */
FOE_API int foe_step_log(const foe_ctx *ctx, float *tau, unsigned char *accepted, int max_n);

/* Denoises one image (steps a1-a10 of the solve): data term from y, iPiano iterations, output map.
 *   y    device, noisy counts (non-negative integers stored as FP32), H x W, pitch ld
 *   x    device, output in the intensity domain, H x W, pitch ld (may alias y)
 *   peak the noise level (max of the clean image, Sec. 2.1); only FOE_MODEL_AUTO reads it
 *   rep  host, nullable; if given, the stream is synchronised and the report filled, and the call also returns
 *        FOE_ETIMEOUT for an expired device-side wait and FOE_ENONFINITE if any output pixel is not finite
 * opts.step = FOE_STEP_BACKTRACK (FP32 only; step a9): the step size of iPiano (Sec. 2.3, given there only as a
 * symbol) is found per iteration by Lipschitz backtracking on the smooth part F = E_FoE: a trial with estimate
 * L uses tau = 2 (1 - gamma) / (L + 2e-3) and is accepted when
 *   F(u+) <= F(u) + <grad F(u), u+ - u> + L/2 ||u+ - u||^2    (FP64 reductions on the GPU),
 * otherwise L doubles and the step is retried from the same u; after each accepted step L is divided by 1.5.
 * L starts at the bound of foe_step_size (or at the L implied by opts.tau when it is > 0).  Every decision is
 * taken on the device: an iteration is one CUDA graph launch (gradient, snapshot, then a conditional loop of
 * trials that a one-thread kernel ends by accepting), all iterations are queued without waiting, and the host
 * synchronises once at the end.  A trial costs a step, an energy evaluation and two reductions, so this mode is
 * for accuracy, not throughput.  Not on a stream under capture (FOE_EUNSUPPORTED).
 * foe_step_log returns the trials of the last such solve.
 * With opts.tol > 0 (fixed steps) the host reads the image's stopping word one check interval behind the
 * device (an event on the stream; the next interval is queued meanwhile), issues no launch past the interval
 * after the stop, and step launches after the stop leave the image unchanged.  On a stream under capture the
 * whole budget is queued and the launches past the stop do no work. */
FOE_API foe_status foe_denoise(foe_ctx *ctx, const float *y, float *x, int H, int W, int ld, float peak,
                       const foe_solve_opts *opts, void *stream, foe_report *rep);

/* The binning variant FoEPNRbin (Sec. 4: a 3x3 ones kernel raises the peak nine-fold before the solve, bilinear
 * interpolation upscales the low-resolution estimate after it).  y is summed over the non-overlapping 3x3 bins
 * starting at pixel (0, 0) (a bin cut by the image border, with n < 9 pixels, is scaled by 9 / n); the
 * ceil(H/3) x ceil(W/3) bin image is denoised exactly as foe_denoise does, with peak 9 * peak (FOE_MODEL_AUTO
 * applies the threshold 5 to that binned peak, Sec. 3.4); x(r, c) is the bilinear interpolation of the estimate
 * at ((r - 1) / 3, (c - 1) / 3), bin (I, J) being centred on pixel (3I + 1, 3J + 1) and coordinates clamped to the
 * edge bins, divided by 9.
 *   y, x   device, H x W, pitch ld (floats), 16-byte aligned; H, W >= 19 (the bin image is at least 7 x 7)
 *   peak   the peak of the full-resolution image
 * The bin image and its estimate live in context memory (allocated on first use, grown as needed).  opts, the
 * report and the errors are those of foe_denoise (the report describes the binned solve). */
FOE_API foe_status foe_denoise_binned(foe_ctx *ctx, const float *y, float *x, int H, int W, int ld, float peak,
                                      const foe_solve_opts *opts, void *stream, foe_report *rep);

/* foe_denoise for callers that cannot allocate device memory at the time of the call: code whose device
 * memory is owned entirely by another allocator (a framework's caching allocator or a fixed arena sized at
 * start-up, where a cudaMalloc from here would bypass its accounting or fail once the arena holds the
 * device), and real-time loops that cannot afford the implicit device synchronisation of cudaMalloc and
 * cudaFree.  It computes exactly what foe_denoise computes, but its workspace is a fixed 20 MiB device
 * array inside the library instead of context memory; it never calls cudaMalloc, cudaFree or any
 * allocating routine.  The paper has no counterpart of this entry point.
 *   - Size limit: H * ld <= 1048576 floats (e.g. 1024 x 1024); larger images return FOE_EINVAL with a
 *     message, before any device work.
 *   - The array is shared by every call in the process on a device and keeps the last call's contents;
 *     calls whose work overlaps on the GPU (other streams, other threads) race on it.  Serialise them.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress), with
 *     that device current; make that first call before any stream capture begins.
 *   - No report and no profiling: nothing is synchronised.  The context (created earlier, when
 *     allocation was possible) supplies the filters.  With opts.tol > 0 the whole budget is queued and
 *     the launches past the stop do no work; foe_iters_done gives the count afterwards.
 *   - A device-side wait of the tensor-core kernel that expired earlier in this context (FOE_ETIMEOUT,
 *     sticky until read) makes every later tensor-core step launch of the context return at once.  This
 *     call cannot read that status without synchronising, so on the BF16 / TF32 paths its output map then
 *     fills x with NaN instead of a stale iterate; call foe_device_status (which reads and clears the
 *     status) after a solve whose result matters.
 * Arguments and the other errors are those of foe_denoise. */
FOE_API foe_status foe_denoise_static(foe_ctx *ctx, const float *y, float *x, int H, int W, int ld, float peak,
                                      const foe_solve_opts *opts, void *stream);

/* Denoises n independent images of mixed sizes, iteration budgets and data terms in one stream-ordered pass:
 * every iteration advances all images whose budget is not yet spent, in one launch over the tiles
 * of all of them.  opts->iters is ignored (each desc carries its own); a desc with use_model = 1 carries its
 * own model too.  With opts->tol > 0 every image has
 * its own stopping word: the whole budget is queued (nothing is synchronised), and the step launches skip
 * the tiles of images that have stopped, so a launch in which every image has stopped does almost no work. */
FOE_API foe_status foe_denoise_batch(foe_ctx *ctx, const foe_image_desc *descs, int n, const foe_solve_opts *opts,
                             void *stream);

/* Iterations taken by the images of the context's last foe_denoise, foe_denoise_static or foe_denoise_batch
 * solve (fixed steps): out[i] for image i in the order of the call (n = 1 for the single-image calls), the
 * step of the stopping rule's first success, or the image's budget when it never held or opts.tol was 0.
 * Synchronises the stream the solve ran on (pass it), reads n words from the device.
 *   out  host, n ints; n must equal the last solve's image count (FOE_EINVAL otherwise, or before any solve) */
FOE_API foe_status foe_iters_done(foe_ctx *ctx, int *out, int n, void *stream);

/* Energy and gradient of E = F + D at u (Eq. FOEmodel + the model's data term; gradient Eq. FoEF plus
 * grad D).  model must be DIRECT, ANS_L2 or ANS_IDIV; data is y (DIRECT) or v (Anscombe models).
 *   energy_host  host, nullable: E(u), accumulated in FP64 on the device; synchronises the stream
 *   grad         device, nullable: H x W with pitch ld */
FOE_API foe_status foe_energy_grad(foe_ctx *ctx, const float *u, const float *data, int H, int W, int ld, foe_model model,
                           float lambda, foe_bc bc, foe_precision prec, double *energy_host, float *grad,
                           void *stream);

/* One evaluation of the prior-training objective (Sec. 2.5, Eq. learningmodel) with the loss of Sec. 3.2,
 *     L = sum_s 1/2 ||I_C(u_s^T) - g_s||^2,
 * where u_s^T is T = opts->iters unrolled iPiano steps of the Anscombe quadratic model (Eq. overallModel)
 * from u^0 = u^{-1} = v_s, and of its gradient with respect to the filters and the log-weights
 * a_i (alpha_i = e^{a_i}), by reverse-mode differentiation of the unrolled iteration with a hand-written
 * backward kernel (Hessian-vector products of the prior, Sec. 2.5.2).  Iterates are checkpointed every
 * ckpt_every steps (0: about sqrt(T)) and recomputed segment by segment in the reverse sweep.
 *   clean, noisy  device, B images of H x W, row pitch ld, image stride H * ld floats (g_s and y_s)
 *   opts          model must be FOE_MODEL_ANS_L2, prec FOE_PREC_FP32; lambda, gamma, tau (0: default), bc;
 *                 tol must be 0 (FOE_EUNSUPPORTED otherwise: the T steps are the differentiated function)
 *   loss_host     host, nullable: L (synchronises the stream)
 *   dfilters      device, [nf][49], dL/dk_i(a, b) in the filters' convolution orientation
 *   dlogalpha     device, [nf], dL/da_i
 * The step size tau is held fixed (it is not differentiated). */
FOE_API foe_status foe_train_step(foe_ctx *ctx, const float *clean, const float *noisy, int B, int H, int W, int ld,
                                  const foe_solve_opts *opts, int ckpt_every, double *loss_host, float *dfilters,
                                  float *dlogalpha, void *stream);

typedef struct {
    int cg_iters;       /* largest number of conjugate-gradient iterations over the images */
    double cg_relres;   /* largest final relative residual ||dL/dw - H_E q|| / ||dL/dw|| (CG recurrence, FP64) */
    int breakdowns;     /* images whose CG stopped at p^T H_E p <= 0 (H_E not positive definite there) */
} foe_implicit_report;

/* The paper's own gradient of the same objective (Sec. 2.5, Eq. implicitdifferentiation and Eq.
 * overallderivative): at the minimiser w* of the lower-level problem (approximated by u^T, T = opts->iters
 * iPiano steps from v),
 *     q = H_E(w*)^{-1} dL/dw,   H_E = sum_i alpha_i K_i^T diag(rho''(K_i w*)) K_i + lambda I,
 *     dL/da_i = -alpha_i <K_i q, rho'(K_i w*)>,
 *     dL/dk_i(a, b) = -alpha_i sum_p [ (P q)(p - (a,b)) rho'(r_i(p)) + (K_i q)_p rho''(r_i(p)) (P w*)(p - (a,b)) ],
 * with q by conjugate gradients on the device from q = 0 (FP32 vectors, FP64 dot products in a fixed order;
 * at most max_cg iterations, per image until ||dL/dw - H_E q|| <= cg_tol ||dL/dw||).  The filter coefficients
 * are the parameters (the basis of Eq. filtercoe is the identity).  Unlike foe_train_step this needs no stored
 * iterates: memory is 10 planes per image whatever T is.  It equals the unrolled gradient as T grows (when the
 * iteration converges) and is exact only at a minimiser.
 *   clean, noisy, opts, loss_host, dfilters, dlogalpha  as foe_train_step, except that opts->prec may also be
 *       FOE_PREC_TF32: the Hessian-vector products of the CG then run on the tensor cores (TF32 operands, FP32
 *       accumulation; the factors rho''(K_i w*) / 2 are computed once, 48 floats per pixel, 192 B per pixel and
 *       image of context memory), the lower-level solve and the final gradients stay FP32.  The CG then solves
 *       with the TF32 operator, whose products differ from the FP32 ones at TF32 rounding level (~5e-4), so the
 *       CG's residual is that of the TF32 operator; the gradients stay within 1e-3 of the FP32 route's (2e-4
 *       measured against the FP64 oracle).
 *   max_cg >= 1, cg_tol >= 0 (0: run max_cg iterations)
 *   rep      host, nullable: CG iterations and residuals (synchronises the stream) */
FOE_API foe_status foe_train_grad_implicit(foe_ctx *ctx, const float *clean, const float *noisy, int B, int H, int W,
                                           int ld, const foe_solve_opts *opts, int max_cg, float cg_tol,
                                           double *loss_host, float *dfilters, float *dlogalpha,
                                           foe_implicit_report *rep, void *stream);

/* One iPiano step (Eq. iPianoupdate) on a state given explicitly, for callers that drive the loop:
 *   u_hi, u_lo   device, the iterate u^n = u_hi + u_lo (u_lo may be NULL = zeros; written if not NULL)
 *   delta        device, u^n - u^{n-1} (read, then overwritten with u^{n+1} - u^n)
 *   d            device, the data term (y for DIRECT, v for the Anscombe models)
 *   u_next_hi    device, receives the high part of u^{n+1}; must not alias u_hi
 * model must not be AUTO.  All images H x W with pitch ld. */
FOE_API foe_status foe_ipiano_step(foe_ctx *ctx, const float *u_hi, float *u_lo, float *delta, const float *d,
                           float *u_next_hi, int H, int W, int ld, foe_model model, float lambda, float tau,
                           float gamma, foe_bc bc, foe_precision prec, void *stream);

/* Elementwise maps on n-element device arrays.
 *   foe_anscombe: v = 2 sqrt(y + 3/8)            (Eq. Anscombetransform)
 *   foe_inverse:  x = I_C(max(z, sqrt(3/2)))     (Eq. invAns) */
FOE_API foe_status foe_anscombe(const float *y, float *v, long n, void *stream);
FOE_API foe_status foe_inverse(const float *z, float *x, long n, void *stream);

/* ---- Continuous-batching server ----
 * Denoise requests of mixed sizes, peaks and iteration budgets are admitted as slots and device
 * memory free up, iterated together (one step launch per iteration over the tiles of every admitted
 * request) and retired when their budget is spent.  Every request's iterate state stays on the device
 * from admission to completion.  One host thread per server. */
typedef struct foe_server foe_server;

typedef struct {
    size_t hbm_budget_bytes;  /* device memory for request state; allocated once at creation (>= 1 MiB) */
    int max_active;           /* requests iterated together, 1..64 */
    int iters_per_tick;       /* iterations each admitted request advances per tick, >= 1 */
    int use_graphs;           /* 1: each tick's step launches are captured and replayed as a CUDA graph */
    foe_solve_opts opts;      /* model, lambda, gamma, tau, bc, prec, zero_c for every request; iters ignored;
                                 tol must be 0 (FOE_EUNSUPPORTED otherwise) */
} foe_server_config;

typedef struct {
    int queued, active;       /* waiting for admission / admitted and iterating */
    int finishing;            /* finished in the last round, completed by the next foe_server_tick */
    long long completed, ticks, launches;
    double pixel_iters;       /* pixel-iterations executed so far */
    size_t bytes_in_use, bytes_peak, bytes_budget;
} foe_server_stats;

/* Creates a server on a context: allocates the arena (hbm_budget_bytes) and a private stream. */
FOE_API foe_status foe_server_create(foe_ctx *ctx, const foe_server_config *cfg, foe_server **out);
/* Waits for the server's work, frees it.  Requests not yet completed are dropped. */
FOE_API void foe_server_destroy(foe_server *srv);
/* Queues one request.  y_host: host counts, H x W with row pitch y_pitch floats; x_host: host buffer
 * for the result (row pitch x_pitch), written by the tick that completes the request.  Both must stay
 * valid until then (page-locked memory keeps the copies asynchronous).  Never blocks.  FOE_ENOMEM if the
 * request's state (5 H x ld FP32 planes, ld = W rounded up to 4) exceeds the whole budget. */
FOE_API foe_status foe_server_submit(foe_server *srv, const float *y_host, int y_pitch, float *x_host, int x_pitch,
                                     int H, int W, float peak, int iters, long long *id_out);
/* One scheduling round: admit queued requests in FIFO order while a slot and arena memory are free
 * (upload + initialise them), advance every admitted request by up to iters_per_tick iterations, and
 * queue the finishing of the requests whose budget is then spent (output map, copy to x_host).  Rounds
 * are pipelined: the call queues this round's device work behind the previous round's and then waits
 * for the previous round only, whose finished requests it completes (memory returned, ids to poll,
 * x_host written); *n_completed (nullable) = requests completed by this call.  A request finishing in
 * round k is therefore reported by the call of round k + 1; a call with nothing to admit or iterate
 * only completes the previous round (stats.finishing counts the requests it would complete).
 * If a device-side wait of the step kernel expired (FOE_ETIMEOUT), the server stops: this and every
 * later tick return FOE_ETIMEOUT, the affected requests are never reported, and the caller destroys
 * the server and reads (and clears) the context's status with foe_device_status. */
FOE_API foe_status foe_server_tick(foe_server *srv, int *n_completed);
/* Ids of completed requests not yet polled (up to max_ids), oldest first. */
FOE_API foe_status foe_server_poll(foe_server *srv, long long *ids, int max_ids, int *n);
FOE_API foe_status foe_server_get_stats(const foe_server *srv, foe_server_stats *stats);

/* Step-kernel timing (tracing aid).  foe_profile(ctx, 1) clears the counters and starts recording a
 * CUDA event pair around every iteration loop that foe_denoise / foe_denoise_batch enqueue (on the
 * caller's stream); foe_profile(ctx, 0) stops recording.  foe_profile_read waits for the recorded
 * events and returns, since the last foe_profile(ctx, 1): the summed device time of those loops in
 * ms, the number of step-kernel launches inside them, and the pixel-iterations they processed.
 * Any output pointer may be NULL. */
FOE_API foe_status foe_profile(foe_ctx *ctx, int enable);
FOE_API foe_status foe_profile_read(foe_ctx *ctx, double *loop_ms, long *launches, double *pixel_iters);

/* Tensor-core cost probe (diagnostic, no context): SM cycles per tcgen05.mma of kind::f16 (BF16 operands, FP32
 * accumulator in tensor memory, K = 16 per MMA) for an M x N shape: the contraction ceiling of the kernels that
 * compute the responses K_i u and their adjoint (Eq. FoEF) as implicit GEMMs.  Measured with clock64 over `count`
 * MMAs per issuing warp (1 or 2 warps, each into its own accumulator; operands cycle over a K = 64 region); the
 * second of two passes is reported.
 *   m, n            one CTA: m = 64 (n a multiple of 8 in 8..256) or m = 128 (n a multiple of 16 in 16..256);
 *                   cta_pair = 1: m = 256 over the two SMs of a two-CTA cluster (cta_group::2; each SM holds 128
 *                   rows of A and n / 2 rows of B), n a multiple of 16 in 32..256
 *   a_in_tmem       1: the A operand is read from tensor memory (m = 128, one CTA), else from shared memory
 *   issuers, count  1 or 2 issuing warps; MMAs per warp, 1..65536
 *   cycles_per_mma  host, out: elapsed cycles / (issuers x count)
 * FOE_EINVAL for other arguments, FOE_EUNSUPPORTED on a device of another compute capability than 10.3,
 * FOE_ETIMEOUT if the bounded wait for the MMAs expired.  Synchronises the current device. */
FOE_API foe_status foe_mma_cost(int m, int n, int a_in_tmem, int cta_pair, int issuers, int count,
                                double *cycles_per_mma);

FOE_API const char *foe_status_string(foe_status s);

/* Device-side status of the context: every wait of the tensor-core kernel is bounded, and one that expires records
 * FOE_ETIMEOUT in a status word that makes every later launch of the context return at once (a sticky failure).
 * A call with a report reads and clears it; foe_device_status does the same for calls without one: it
 * synchronises the stream, returns FOE_OK or the recorded status, and clears it so that the context is usable
 * again. */
FOE_API foe_status foe_device_status(foe_ctx *ctx, void *stream);

/* Failure-detection test aid: the next tensor-core launch of the context withholds one mbarrier arrival in one CTA,
 * so that its bounded waits expire (after about 2 s) and the launch records FOE_ETIMEOUT.  Nothing faults, traps or
 * hangs: the CTA drains its MMAs, frees its tensor memory and returns; the other CTAs finish normally. */
FOE_API foe_status foe_debug_withhold_arrival(foe_ctx *ctx);

/* Last error text of the context (never NULL). */
FOE_API const char *foe_last_error(const foe_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FOE_H */
