// Internal to the library: the context object and the host helpers shared by the C ABI entry points
// (argument checks, step constants, launch descriptors, workspace).
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/foe.h"
#include "foe_kernels.h"

using foe::ImgDesc;
using foe::LaunchArgs;

struct foe_ctx {
    int nf = 0;
    float kconv[foe::kNF * foe::kKK] = {};  // host copy, convolution orientation, zero padded to 48
    float alpha[foe::kNF] = {};
    double symbol_max = 0.0;                // max_w sum_i alpha_i |k_i^(w)|^2
    float *d_wts = nullptr;                 // device [48][49], correlation orientation
    float *d_alpha = nullptr;               // device [48]
    void *d_tcops = nullptr;                // device, bf16 operand images of the tensor-core kernel (12 KB)
    void *d_tcops32 = nullptr;              // device, the same in tf32 (24 KB)
    void *d_pairops = nullptr;              // device, bf16 operand images of the pixel-pair kernel (24 KB)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    float *d_bin = nullptr;                 // foe_denoise_binned: the bin image and its estimate
    size_t bin_bytes = 0;
    double *d_partials = nullptr;
    int partials_cap = 0;
    double *d_energy = nullptr;
    int *d_status = nullptr;
    int *d_nonfinite = nullptr;             // non-finite outputs of the last reporting solve
    int withhold_arrival = 0;               // foe_debug_withhold_arrival: applies to the next tensor-core launch
    // stopping rule (opts.tol): one word per image of a solve, the check's FP64 partials and block counts, and two
    // pinned words with events through which foe_denoise reads its word one check interval behind the device
    int *d_stop = nullptr;                  // [kMaxBatch]
    double *d_tol_part = nullptr;           // [kMaxBatch][kTolBlocks][2]
    unsigned *d_tol_count = nullptr;        // [kMaxBatch], 0 between checks
    int *h_stop = nullptr;                  // pinned [2]
    // second stream of the tensor-core launches that hold both tile sizes (foe::tc_launch)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    cudaEvent_t tol_ev[2] = {nullptr, nullptr};
    // the last fixed-step solve (foe_iters_done): per image of the call, its budget and its word (-1: none)
    std::vector<int> last_budget, last_word;
    LaunchArgs args;
    // step-loop timing (foe_profile)
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    cudaGraphExec_t batch_exec = nullptr;   // cached graph of the last captured foe_denoise_batch
    long prof_launches = 0;
    double prof_pixel_iters = 0.0;
    // trial log of the last FOE_STEP_BACKTRACK solve (foe_step_log), and its device-side state and log
    std::vector<float> bt_tau;
    std::vector<unsigned char> bt_accepted;
    foe::BtState *d_bt = nullptr;
    float *d_bt_tau = nullptr;
    unsigned char *d_bt_acc = nullptr;
    int bt_cap = 0;
    // Hessian factors of foe_train_grad_implicit's tensor-core Hessian-vector products ([B][H][W][48] floats)
    float *d_hess = nullptr;
    size_t hess_bytes = 0;
    char err[512] = {};
};

namespace foe_internal {

// NVTX range over a C-ABI call: a named span on a profiler's timeline (no cost when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline void set_err(foe_ctx *c, const char *fmt, ...)
{
    if (!c) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
}

#define FOE_CUDA(ctx, call)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            set_err(ctx, "%s failed: %s", #call, cudaGetErrorString(e_));                      \
            return e_ == cudaErrorMemoryAllocation ? FOE_ENOMEM : FOE_ECUDA;                   \
        }                                                                                      \
    } while (0)

// max over an n x n DTFT grid of sum_i alpha_i |k^_i(w)|^2, FP64, separable evaluation:
// k^(wy, wx) = sum_a e^{-i wy a} sum_b k(a, b) e^{-i wx b}.  |k^(-w)| = |k^(w)| halves the grid.
inline double symbol_max(const float *k, const float *alpha, int nf, int n)
{
    using cd = std::complex<double>;
    std::vector<cd> E((size_t)n * foe::kKS);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < foe::kKS; ++a) {
            const double ph = -2.0 * M_PI * (double)i * (a - foe::kR) / n;
            E[(size_t)i * foe::kKS + a] = cd(std::cos(ph), std::sin(ph));
        }
    std::vector<cd> R((size_t)nf * foe::kKS * n);
    for (int f = 0; f < nf; ++f)
        for (int a = 0; a < foe::kKS; ++a)
            for (int ix = 0; ix < n; ++ix) {
                cd s = 0.0;
                for (int b = 0; b < foe::kKS; ++b)
                    s += (double)k[f * foe::kKK + a * foe::kKS + b] * E[(size_t)ix * foe::kKS + b];
                R[((size_t)f * foe::kKS + a) * n + ix] = s;
            }
    double best = 0.0;
    for (int iy = 0; iy <= n / 2; ++iy)
        for (int ix = 0; ix < n; ++ix) {
            double s = 0.0;
            for (int f = 0; f < nf; ++f) {
                cd v = 0.0;
                for (int a = 0; a < foe::kKS; ++a) v += E[(size_t)iy * foe::kKS + a] * R[((size_t)f * foe::kKS + a) * n + ix];
                s += (double)alpha[f] * std::norm(v);
            }
            best = std::max(best, s);
        }
    return best;
}

inline uint16_t f32_to_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even (inputs are finite)
    return (uint16_t)(u >> 16);
}

// bf16 operand images of the tensor-core kernel, from correlation weights w[48][49] and alpha:
//   forward B  [tap row a (8)][filter (48)][tap col b (8)] = w_f(a, b)          (0 for a or b = 7)
//   adjoint B  [filter group (6)][tap 8a+b (64)][filter in group (8)] = 2 alpha_f w_f(a, b)
inline std::vector<uint16_t> tc_operands(const float *w, const float *alpha)
{
    std::vector<uint16_t> out(8 * 48 * 8 + 6 * 64 * 8, 0);
    for (int a = 0; a < 8; ++a)
        for (int f = 0; f < 48; ++f)
            for (int b = 0; b < 8; ++b)
                out[(a * 48 + f) * 8 + b] = (a < 7 && b < 7) ? f32_to_bf16(w[f * foe::kKK + a * 7 + b]) : 0;
    uint16_t *adj = out.data() + 8 * 48 * 8;
    for (int g = 0; g < 6; ++g)
        for (int n = 0; n < 64; ++n)
            for (int e = 0; e < 8; ++e) {
                const int f = 8 * g + e, a = n / 8, b = n % 8;
                adj[(g * 64 + n) * 8 + e] = (a < 7 && b < 7) ? f32_to_bf16(2.0f * alpha[f] * w[f * foe::kKK + a * 7 + b]) : 0;
            }
    return out;
}

// bf16 operand images of the pixel-pair kernel (foe_pair.cu), from correlation weights w[48][49] and alpha.  Within
// each group of four filters the tensor-memory (and K) order is f0, f2, f1, f3 (sigma = {0, 2, 1, 3}), so that
// one reciprocal serves the pair (f0, f1) and the pair (f2, f3) with aligned f32x2 operands.
//   forward B  [tap row a (8)][n = 48 s + e (96)][column c (8)] = w_f(a, c - s), f = 4 (e / 4) + sigma(e % 4)
//              (s: pixel of the pair; 0 unless a < 7 and 0 <= c - s < 7)
//   adjoint B  [K chunk h (12)][n' = 8 a + slot (64)][K value e8 (8)] = 2 alpha_f w_f(a, c - s) with s = h / 6,
//              e = 8 (h % 6) + e8, f as above, c = {3, 4, 1, 2, 5, 6, 7, 0}[slot] (the column offset 2j + c - 3
//              of the output that pair j feeds; 0 unless a < 7 and 0 <= c - s < 7)
inline std::vector<uint16_t> pair_operands(const float *w, const float *alpha)
{
    static const int sigma[4] = {0, 2, 1, 3};
    static const int slot_c[8] = {3, 4, 1, 2, 5, 6, 7, 0};
    auto filt = [&](int e) { return 4 * (e / 4) + sigma[e % 4]; };
    std::vector<uint16_t> out(8 * 96 * 8 + 12 * 64 * 8, 0);
    for (int a = 0; a < 8; ++a)
        for (int n = 0; n < 96; ++n)
            for (int c = 0; c < 8; ++c) {
                const int s = n / 48, f = filt(n % 48), b = c - s;
                out[(a * 96 + n) * 8 + c] = (a < 7 && b >= 0 && b < 7) ? f32_to_bf16(w[f * foe::kKK + a * 7 + b]) : 0;
            }
    uint16_t *adj = out.data() + 8 * 96 * 8;
    for (int h = 0; h < 12; ++h)
        for (int n = 0; n < 64; ++n)
            for (int e8 = 0; e8 < 8; ++e8) {
                const int s = h / 6, f = filt(8 * (h % 6) + e8), a = n / 8, b = slot_c[n % 8] - s;
                adj[(h * 64 + n) * 8 + e8] =
                    (a < 7 && b >= 0 && b < 7) ? f32_to_bf16(2.0f * alpha[f] * w[f * foe::kKK + a * 7 + b]) : 0;
            }
    return out;
}

inline uint32_t f32_to_tf32_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0xFFFu + ((u >> 13) & 1u);  // round to nearest even at 10 mantissa bits (inputs are finite)
    return u & ~0x1FFFu;
}

// tf32 operand images (32-bit containers), 4 values per 16-byte entry:
//   forward B  [tap row a (8)][column chunk (2)][filter (48)][tap cols 4c..4c+3] = w_f(a, b)  (0 for a or b = 7)
//   adjoint B  [filter chunk (12)][tap 8a+b (64)][filters 4c..4c+3] = 2 alpha_f w_f(a, b)
inline std::vector<uint32_t> tc_operands_tf32(const float *w, const float *alpha)
{
    std::vector<uint32_t> out(8 * 2 * 48 * 4 + 12 * 64 * 4, 0);
    for (int a = 0; a < 8; ++a)
        for (int ch = 0; ch < 2; ++ch)
            for (int f = 0; f < 48; ++f)
                for (int e = 0; e < 4; ++e) {
                    const int b = 4 * ch + e;
                    out[((a * 2 + ch) * 48 + f) * 4 + e] = (a < 7 && b < 7) ? f32_to_tf32_bits(w[f * foe::kKK + a * 7 + b]) : 0;
                }
    uint32_t *adj = out.data() + 8 * 2 * 48 * 4;
    for (int ch = 0; ch < 12; ++ch)
        for (int n = 0; n < 64; ++n)
            for (int e = 0; e < 4; ++e) {
                const int f = 4 * ch + e, a = n / 8, b = n % 8;
                adj[(ch * 64 + n) * 4 + e] =
                    (a < 7 && b < 7) ? f32_to_tf32_bits(2.0f * alpha[f] * w[f * foe::kKK + a * 7 + b]) : 0;
            }
    return out;
}

inline foe_status check_prior(const foe_prior *p)
{
    if (!p || !p->filters || !p->alpha) return FOE_EINVAL;
    if (p->nf < 1 || p->nf > foe::kNF || p->ksize != foe::kKS) return FOE_EINVAL;
    for (int i = 0; i < p->nf; ++i)
        if (!(p->alpha[i] > 0.0f) || !std::isfinite(p->alpha[i])) return FOE_EINVAL;
    for (int i = 0; i < p->nf * foe::kKK; ++i)
        if (!std::isfinite(p->filters[i])) return FOE_EINVAL;
    return FOE_OK;
}

inline double kappa(int bc) { return bc == foe::kZero ? 1.0 : 4.0; }

inline float default_tau(double symbol, int bc, float gamma)
{
    const double L = 2.0 * kappa(bc) * symbol;
    return (float)(0.99 * 2.0 * (1.0 - (double)gamma) / (L + 2e-3));
}

inline foe_status check_opts(foe_ctx *c, const foe_solve_opts *o)
{
    if (!o) { set_err(c, "opts is NULL"); return FOE_EINVAL; }
    if (o->model < FOE_MODEL_DIRECT || o->model > FOE_MODEL_AUTO) { set_err(c, "bad model"); return FOE_EINVAL; }
    if (!(o->lambda > 0.0f) || !std::isfinite(o->lambda)) { set_err(c, "lambda must be > 0"); return FOE_EINVAL; }
    if (!(o->gamma >= 0.0f && o->gamma < 1.0f)) { set_err(c, "gamma must be in [0, 1)"); return FOE_EINVAL; }
    if (!(o->tau >= 0.0f) || !std::isfinite(o->tau)) { set_err(c, "tau must be >= 0"); return FOE_EINVAL; }
    if (o->iters < 0) { set_err(c, "iters must be >= 0"); return FOE_EINVAL; }
    if (o->step != FOE_STEP_FIXED && o->step != FOE_STEP_BACKTRACK) { set_err(c, "bad step mode"); return FOE_EINVAL; }
    if (o->bc != FOE_BC_SYMMETRIC && o->bc != FOE_BC_ZERO) { set_err(c, "bad bc"); return FOE_EINVAL; }
    if (o->prec != FOE_PREC_FP32 && o->prec != FOE_PREC_BF16 && o->prec != FOE_PREC_TF32) {
        set_err(c, "bad precision");
        return FOE_EINVAL;
    }
    if (!(o->zero_c >= 0.0f) || !std::isfinite(o->zero_c)) { set_err(c, "zero_c must be >= 0"); return FOE_EINVAL; }
    if (!(o->tol >= 0.0f) || !std::isfinite(o->tol)) { set_err(c, "tol must be >= 0"); return FOE_EINVAL; }
    if (o->tol > 0.0f && o->tol_every < 1) { set_err(c, "tol_every must be >= 1 when tol > 0"); return FOE_EINVAL; }
    return FOE_OK;
}

// Entry points that run every iteration of their budget (training, serving) take no stopping rule.
inline foe_status check_no_tol(foe_ctx *c, const foe_solve_opts *o, const char *entry)
{
    if (o && o->tol > 0.0f) {
        set_err(c, "%s: opts.tol > 0 is not supported here (every iteration of the budget runs)", entry);
        return FOE_EUNSUPPORTED;
    }
    return FOE_OK;
}

// Entry points other than foe_denoise run fixed steps only.
inline foe_status check_opts_fixed(foe_ctx *c, const foe_solve_opts *o, const char *entry)
{
    const foe_status st = check_opts(c, o);
    if (st != FOE_OK) return st;
    if (o->step != FOE_STEP_FIXED) {
        set_err(c, "%s: FOE_STEP_BACKTRACK is implemented in foe_denoise only", entry);
        return FOE_EUNSUPPORTED;
    }
    return FOE_OK;
}

inline foe_status check_image(foe_ctx *c, const void *p, int H, int W, int ld, const char *what)
{
    if (!p) { set_err(c, "%s is NULL", what); return FOE_EINVAL; }
    if (H < 7 || W < 7) { set_err(c, "%s: H and W must be >= 7 (got %d x %d)", what, H, W); return FOE_EINVAL; }
    if (ld < W || ld % 4 != 0) { set_err(c, "%s: ld must be >= W and a multiple of 4 (got %d)", what, ld); return FOE_EINVAL; }
    if ((reinterpret_cast<uintptr_t>(p) & 15) != 0) { set_err(c, "%s must be 16-byte aligned", what); return FOE_EINVAL; }
    return FOE_OK;
}

inline int resolve_model(int model, float peak) { return model == FOE_MODEL_AUTO ? (peak >= 5.0f ? foe::kAnsL2 : foe::kAnsIdiv) : model; }

inline foe::StepConsts step_consts(float tau, float gamma, float lambda) { return foe::make_step_consts(tau, gamma, lambda); }

inline void tile_dims(int prec, int H, int W, int &th, int &tw)
{
    if (prec == FOE_PREC_BF16 || prec == FOE_PREC_TF32) {
        th = foe::tc_tile_h(prec == FOE_PREC_TF32, H, W);
        tw = foe::tc_tile_w(th);
    } else {
        th = tw = foe::f32_tile();
    }
}

inline void args_begin(foe_ctx *c, int bc)
{
    LaunchArgs &A = c->args;
    A.nimg = 0;
    A.parity = 0;
    A.bc = bc;
    A.nchunks = (c->nf + 7) / 8;
    A.prior_only = 0;
    A.withhold_arrival = 0;
    A.wts = c->d_wts;
    A.alpha = c->d_alpha;
    A.partials = c->d_partials;
    A.tcops = c->d_tcops;
    A.tcops32 = c->d_tcops32;
    A.pairops = c->d_pairops;
    A.sc_dev = nullptr;
    A.tile_prefix[0] = 0;
}

inline void args_add(foe_ctx *c, int prec, const ImgDesc &d)
{
    LaunchArgs &A = c->args;
    int th, tw;
    tile_dims(prec, d.H, d.W, th, tw);
    ImgDesc e = d;
    e.tiles_x = (d.W + tw - 1) / tw;
    e.tile_h = th;
    const int tiles = e.tiles_x * ((d.H + th - 1) / th);
    A.img[A.nimg] = e;
    A.tile_prefix[A.nimg + 1] = A.tile_prefix[A.nimg] + tiles;
    A.nimg++;
}

inline foe_status launch(foe_ctx *c, int prec, int mode, cudaStream_t s)
{
    cudaError_t e;
    if (prec == FOE_PREC_FP32) {
        e = foe::f32_launch(c->args, mode, s);
    } else {
        c->args.withhold_arrival = c->withhold_arrival;
        c->withhold_arrival = 0;
        e = foe::tc_launch(c->args, mode, prec == FOE_PREC_TF32, c->d_status, s,
                           foe::SideStream{c->side_stream, c->side_fork, c->side_join});
        c->args.withhold_arrival = 0;
    }
    if (e != cudaSuccess) {
        set_err(c, "kernel launch failed: %s", cudaGetErrorString(e));
        return e == cudaErrorNotSupported ? FOE_EUNSUPPORTED : FOE_ECUDA;
    }
    return FOE_OK;
}

inline foe_status ensure_ws(foe_ctx *c, size_t bytes)
{
    if (bytes <= c->ws_bytes) return FOE_OK;
    if (c->ws) FOE_CUDA(c, cudaFree(c->ws));
    c->ws = nullptr;
    c->ws_bytes = 0;
    FOE_CUDA(c, cudaMalloc(&c->ws, bytes));
    c->ws_bytes = bytes;
    return FOE_OK;
}

inline foe_status ensure_bin(foe_ctx *c, size_t bytes)
{
    if (bytes <= c->bin_bytes) return FOE_OK;
    if (c->d_bin) FOE_CUDA(c, cudaFree(c->d_bin));
    c->d_bin = nullptr;
    c->bin_bytes = 0;
    FOE_CUDA(c, cudaMalloc(&c->d_bin, bytes));
    c->bin_bytes = bytes;
    return FOE_OK;
}

// Device state and a trial log of `cap` entries for FOE_STEP_BACKTRACK.
inline foe_status ensure_bt(foe_ctx *c, int cap)
{
    if (!c->d_bt) FOE_CUDA(c, cudaMalloc(&c->d_bt, sizeof(foe::BtState)));
    if (cap <= c->bt_cap) return FOE_OK;
    if (c->d_bt_tau) FOE_CUDA(c, cudaFree(c->d_bt_tau));
    if (c->d_bt_acc) FOE_CUDA(c, cudaFree(c->d_bt_acc));
    c->d_bt_tau = nullptr;
    c->d_bt_acc = nullptr;
    c->bt_cap = 0;
    FOE_CUDA(c, cudaMalloc(&c->d_bt_tau, sizeof(float) * (size_t)cap));
    FOE_CUDA(c, cudaMalloc(&c->d_bt_acc, (size_t)cap));
    c->bt_cap = cap;
    return FOE_OK;
}

inline foe_status ensure_partials(foe_ctx *c, int n)
{
    if (n <= c->partials_cap) return FOE_OK;
    if (c->d_partials) FOE_CUDA(c, cudaFree(c->d_partials));
    c->d_partials = nullptr;
    c->partials_cap = 0;
    FOE_CUDA(c, cudaMalloc(&c->d_partials, sizeof(double) * (size_t)n));
    c->partials_cap = n;
    return FOE_OK;
}

inline foe_status prof_begin(foe_ctx *c, cudaStream_t s, cudaEvent_t *ev)
{
    ev[0] = ev[1] = nullptr;
    if (!c->prof) return FOE_OK;
    FOE_CUDA(c, cudaEventCreate(&ev[0]));
    FOE_CUDA(c, cudaEventCreate(&ev[1]));
    FOE_CUDA(c, cudaEventRecord(ev[0], s));
    return FOE_OK;
}

inline foe_status prof_end(foe_ctx *c, cudaStream_t s, cudaEvent_t *ev, long launches, double pixel_iters)
{
    if (!ev[0]) return FOE_OK;
    FOE_CUDA(c, cudaEventRecord(ev[1], s));
    c->prof_events.emplace_back(ev[0], ev[1]);
    c->prof_launches += launches;
    c->prof_pixel_iters += pixel_iters;
    return FOE_OK;
}

inline void prof_clear(foe_ctx *c)
{
    for (auto &p : c->prof_events) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    c->prof_events.clear();
    c->prof_launches = 0;
    c->prof_pixel_iters = 0.0;
}

// The FP32 path keeps the iterate as an unevaluated pair u_hi + u_lo; the tensor-core paths (whose BF16 / TF32
// operand rounding dominates the error) keep a plain FP32 u_hi, so their u_lo plane is left out everywhere.
inline float *lo_plane(int prec, float *ul) { return prec == FOE_PREC_FP32 ? ul : nullptr; }

// Per-image workspace: u_hi[2], u_lo, delta, d, each H x ld floats.
struct Slot {
    float *uh0, *uh1, *ul, *delta, *d;
};

// Stopping check after step n: the iterate u^n (plane n & 1) and its change of the listed images.
inline foe::TolImg tol_img(const ImgDesc &d, int n)
{
    foe::TolImg t;
    t.u_hi = d.u_hi[n & 1];
    t.u_lo = d.u_lo;
    t.delta = d.delta;
    t.H = d.H;
    t.W = d.W;
    t.ld = d.ld;
    t.stop = const_cast<int *>(d.stop);
    return t;
}

// Checks the images 0 .. nimg - 1 of the context's launch arguments that carry a stopping word.
inline foe_status tol_check(foe_ctx *c, int nimg, int n, float tol, cudaStream_t s)
{
    foe::TolArgs t;
    t.nimg = 0;
    t.n = n;
    t.tol = (double)tol;
    t.partials = c->d_tol_part;
    t.count = c->d_tol_count;
    for (int j = 0; j < nimg; ++j)
        if (c->args.img[j].stop) t.img[t.nimg++] = tol_img(c->args.img[j], n);
    FOE_CUDA(c, foe::launch_tol_check(t, s));
    return FOE_OK;
}

// Records the images of a fixed-step solve for foe_iters_done.
inline void note_solve(foe_ctx *c, int n, const int *budget, const int *word)
{
    c->last_budget.assign(budget, budget + n);
    c->last_word.assign(word, word + n);
}

inline Slot carve(float *base, size_t plane)
{
    return Slot{base, base + plane, base + 2 * plane, base + 3 * plane, base + 4 * plane};
}

}  // namespace foe_internal

using namespace foe_internal;
