// C ABI of the FoE denoiser: argument checks, context and workspace, step size, launch sequencing.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

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
    void *ws = nullptr;
    size_t ws_bytes = 0;
    double *d_partials = nullptr;
    int partials_cap = 0;
    double *d_energy = nullptr;
    int *d_status = nullptr;
    LaunchArgs args;
    // step-loop timing (foe_profile)
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    long prof_launches = 0;
    double prof_pixel_iters = 0.0;
    char err[512] = {};
};

namespace {

void set_err(foe_ctx *c, const char *fmt, ...)
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
double symbol_max(const float *k, const float *alpha, int nf, int n)
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

uint16_t f32_to_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even (inputs are finite)
    return (uint16_t)(u >> 16);
}

// bf16 operand images of the tensor-core kernel, from correlation weights w[48][49] and alpha:
//   forward B  [tap row a (8)][filter (48)][tap col b (8)] = w_f(a, b)          (0 for a or b = 7)
//   adjoint B  [filter group (6)][tap 8a+b (64)][filter in group (8)] = 2 alpha_f w_f(a, b)
std::vector<uint16_t> tc_operands(const float *w, const float *alpha)
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

foe_status check_prior(const foe_prior *p)
{
    if (!p || !p->filters || !p->alpha) return FOE_EINVAL;
    if (p->nf < 1 || p->nf > foe::kNF || p->ksize != foe::kKS) return FOE_EINVAL;
    for (int i = 0; i < p->nf; ++i)
        if (!(p->alpha[i] > 0.0f) || !std::isfinite(p->alpha[i])) return FOE_EINVAL;
    for (int i = 0; i < p->nf * foe::kKK; ++i)
        if (!std::isfinite(p->filters[i])) return FOE_EINVAL;
    return FOE_OK;
}

double kappa(int bc) { return bc == foe::kZero ? 1.0 : 4.0; }

float default_tau(double symbol, int bc, float gamma)
{
    const double L = 2.0 * kappa(bc) * symbol;
    return (float)(0.99 * 2.0 * (1.0 - (double)gamma) / (L + 2e-3));
}

foe_status check_opts(foe_ctx *c, const foe_solve_opts *o)
{
    if (!o) { set_err(c, "opts is NULL"); return FOE_EINVAL; }
    if (o->model < FOE_MODEL_DIRECT || o->model > FOE_MODEL_AUTO) { set_err(c, "bad model"); return FOE_EINVAL; }
    if (!(o->lambda > 0.0f) || !std::isfinite(o->lambda)) { set_err(c, "lambda must be > 0"); return FOE_EINVAL; }
    if (!(o->gamma >= 0.0f && o->gamma < 1.0f)) { set_err(c, "gamma must be in [0, 1)"); return FOE_EINVAL; }
    if (!(o->tau >= 0.0f) || !std::isfinite(o->tau)) { set_err(c, "tau must be >= 0"); return FOE_EINVAL; }
    if (o->iters < 0) { set_err(c, "iters must be >= 0"); return FOE_EINVAL; }
    if (o->step != FOE_STEP_FIXED) { set_err(c, "only FOE_STEP_FIXED is implemented"); return FOE_EUNSUPPORTED; }
    if (o->bc != FOE_BC_SYMMETRIC && o->bc != FOE_BC_ZERO) { set_err(c, "bad bc"); return FOE_EINVAL; }
    if (o->prec != FOE_PREC_FP32 && o->prec != FOE_PREC_BF16 && o->prec != FOE_PREC_TF32) {
        set_err(c, "bad precision");
        return FOE_EINVAL;
    }
    if (o->prec == FOE_PREC_TF32) { set_err(c, "TF32 convolutions are not implemented"); return FOE_EUNSUPPORTED; }
    if (!(o->zero_c >= 0.0f) || !std::isfinite(o->zero_c)) { set_err(c, "zero_c must be >= 0"); return FOE_EINVAL; }
    return FOE_OK;
}

foe_status check_image(foe_ctx *c, const void *p, int H, int W, int ld, const char *what)
{
    if (!p) { set_err(c, "%s is NULL", what); return FOE_EINVAL; }
    if (H < 7 || W < 7) { set_err(c, "%s: H and W must be >= 7 (got %d x %d)", what, H, W); return FOE_EINVAL; }
    if (ld < W || ld % 4 != 0) { set_err(c, "%s: ld must be >= W and a multiple of 4 (got %d)", what, ld); return FOE_EINVAL; }
    if ((reinterpret_cast<uintptr_t>(p) & 15) != 0) { set_err(c, "%s must be 16-byte aligned", what); return FOE_EINVAL; }
    return FOE_OK;
}

int resolve_model(int model, float peak) { return model == FOE_MODEL_AUTO ? (peak >= 5.0f ? foe::kAnsL2 : foe::kAnsIdiv) : model; }

foe::StepConsts step_consts(float tau, float gamma, float lambda)
{
    foe::StepConsts s;
    s.tau = tau;
    s.gamma = gamma;
    s.lambda = lambda;
    const double c = (double)tau * (double)lambda;
    auto split = [](double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    split(c, s.c_hi, s.c_lo);
    split(1.0 / (1.0 + c), s.a1_hi, s.a1_lo);
    split(c / (1.0 + c), s.a2_hi, s.a2_lo);
    return s;
}

void tile_dims(int prec, int &th, int &tw)
{
    if (prec == FOE_PREC_BF16) {
        th = foe::tc_tile_h();
        tw = foe::tc_tile_w();
    } else {
        th = tw = foe::f32_tile();
    }
}

void args_begin(foe_ctx *c, int bc)
{
    LaunchArgs &A = c->args;
    A.nimg = 0;
    A.parity = 0;
    A.bc = bc;
    A.nchunks = (c->nf + 7) / 8;
    A.wts = c->d_wts;
    A.alpha = c->d_alpha;
    A.partials = c->d_partials;
    A.tcops = c->d_tcops;
    A.tile_prefix[0] = 0;
}

void args_add(foe_ctx *c, int prec, const ImgDesc &d)
{
    LaunchArgs &A = c->args;
    int th, tw;
    tile_dims(prec, th, tw);
    ImgDesc e = d;
    e.tiles_x = (d.W + tw - 1) / tw;
    const int tiles = e.tiles_x * ((d.H + th - 1) / th);
    A.img[A.nimg] = e;
    A.tile_prefix[A.nimg + 1] = A.tile_prefix[A.nimg] + tiles;
    A.nimg++;
}

foe_status launch(foe_ctx *c, int prec, int mode, cudaStream_t s)
{
    cudaError_t e = prec == FOE_PREC_BF16 ? foe::tc_launch(c->args, mode, c->d_status, s) : foe::f32_launch(c->args, mode, s);
    if (e != cudaSuccess) {
        set_err(c, "kernel launch failed: %s", cudaGetErrorString(e));
        return e == cudaErrorNotSupported ? FOE_EUNSUPPORTED : FOE_ECUDA;
    }
    return FOE_OK;
}

foe_status ensure_ws(foe_ctx *c, size_t bytes)
{
    if (bytes <= c->ws_bytes) return FOE_OK;
    if (c->ws) FOE_CUDA(c, cudaFree(c->ws));
    c->ws = nullptr;
    c->ws_bytes = 0;
    FOE_CUDA(c, cudaMalloc(&c->ws, bytes));
    c->ws_bytes = bytes;
    return FOE_OK;
}

foe_status ensure_partials(foe_ctx *c, int n)
{
    if (n <= c->partials_cap) return FOE_OK;
    if (c->d_partials) FOE_CUDA(c, cudaFree(c->d_partials));
    c->d_partials = nullptr;
    c->partials_cap = 0;
    FOE_CUDA(c, cudaMalloc(&c->d_partials, sizeof(double) * (size_t)n));
    c->partials_cap = n;
    return FOE_OK;
}

foe_status prof_begin(foe_ctx *c, cudaStream_t s, cudaEvent_t *ev)
{
    ev[0] = ev[1] = nullptr;
    if (!c->prof) return FOE_OK;
    FOE_CUDA(c, cudaEventCreate(&ev[0]));
    FOE_CUDA(c, cudaEventCreate(&ev[1]));
    FOE_CUDA(c, cudaEventRecord(ev[0], s));
    return FOE_OK;
}

foe_status prof_end(foe_ctx *c, cudaStream_t s, cudaEvent_t *ev, long launches, double pixel_iters)
{
    if (!ev[0]) return FOE_OK;
    FOE_CUDA(c, cudaEventRecord(ev[1], s));
    c->prof_events.emplace_back(ev[0], ev[1]);
    c->prof_launches += launches;
    c->prof_pixel_iters += pixel_iters;
    return FOE_OK;
}

void prof_clear(foe_ctx *c)
{
    for (auto &p : c->prof_events) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    c->prof_events.clear();
    c->prof_launches = 0;
    c->prof_pixel_iters = 0.0;
}

// Per-image workspace: u_hi[2], u_lo, delta, d, each H x ld floats.
struct Slot {
    float *uh0, *uh1, *ul, *delta, *d;
};

Slot carve(float *base, size_t plane)
{
    return Slot{base, base + plane, base + 2 * plane, base + 3 * plane, base + 4 * plane};
}

}  // namespace

extern "C" {

const char *foe_status_string(foe_status s)
{
    switch (s) {
    case FOE_OK: return "ok";
    case FOE_EINVAL: return "invalid argument";
    case FOE_ENOMEM: return "out of memory";
    case FOE_ECUDA: return "CUDA error";
    case FOE_ENONFINITE: return "non-finite value";
    case FOE_ETIMEOUT: return "device wait timed out";
    case FOE_EBUSY: return "busy";
    case FOE_EUNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char *foe_last_error(const foe_ctx *ctx) { return ctx ? ctx->err : "no context"; }

foe_status foe_default_opts(foe_solve_opts *o)
{
    if (!o) return FOE_EINVAL;
    o->model = FOE_MODEL_AUTO;
    o->lambda = 1.0f;
    o->gamma = 0.8f;
    o->tau = 0.0f;
    o->tol = 0.0f;
    o->iters = 300;
    o->step = FOE_STEP_FIXED;
    o->bc = FOE_BC_SYMMETRIC;
    o->prec = FOE_PREC_BF16;
    o->zero_c = 0.0f;
    return FOE_OK;
}

foe_status foe_prior_lipschitz(const foe_prior *prior, foe_bc bc, double *lipschitz_out)
{
    if (check_prior(prior) != FOE_OK || !lipschitz_out || (bc != FOE_BC_SYMMETRIC && bc != FOE_BC_ZERO))
        return FOE_EINVAL;
    *lipschitz_out = 2.0 * kappa(bc) * symbol_max(prior->filters, prior->alpha, prior->nf, 512);
    return FOE_OK;
}

foe_status foe_create(const foe_prior *prior, foe_ctx **out)
{
    if (!out) return FOE_EINVAL;
    *out = nullptr;
    if (check_prior(prior) != FOE_OK) return FOE_EINVAL;
    foe_ctx *c = new (std::nothrow) foe_ctx();
    if (!c) return FOE_ENOMEM;
    c->nf = prior->nf;
    std::memcpy(c->kconv, prior->filters, sizeof(float) * prior->nf * foe::kKK);
    std::memcpy(c->alpha, prior->alpha, sizeof(float) * prior->nf);
    c->symbol_max = symbol_max(c->kconv, c->alpha, c->nf, 512);
    // correlation form for the kernels: w_i(a, b) = k_i(-a, -b)
    float w[foe::kNF * foe::kKK] = {};
    for (int f = 0; f < c->nf; ++f)
        for (int t = 0; t < foe::kKK; ++t) w[f * foe::kKK + t] = c->kconv[f * foe::kKK + (foe::kKK - 1 - t)];
    foe_status st = FOE_OK;
    auto fail = [&](foe_status s) {
        foe_destroy(c);
        return s;
    };
    const std::vector<uint16_t> ops = tc_operands(w, c->alpha);
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_wts, sizeof(w))) || (e = cudaMalloc(&c->d_alpha, sizeof(c->alpha))) ||
        (e = cudaMalloc(&c->d_tcops, ops.size() * sizeof(uint16_t))) ||
        (e = cudaMemcpy(c->d_tcops, ops.data(), ops.size() * sizeof(uint16_t), cudaMemcpyHostToDevice)) ||
        (e = cudaMalloc(&c->d_energy, sizeof(double))) || (e = cudaMalloc(&c->d_status, sizeof(int))) ||
        (e = cudaMemcpy(c->d_wts, w, sizeof(w), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_alpha, c->alpha, sizeof(c->alpha), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->d_status, 0, sizeof(int))) || (e = foe::f32_setup()) || (e = foe::tc_setup()))
        return fail(e == cudaErrorMemoryAllocation ? FOE_ENOMEM : FOE_ECUDA);
    (void)st;
    if (ensure_partials(c, 1024) != FOE_OK) return fail(FOE_ENOMEM);
    *out = c;
    return FOE_OK;
}

void foe_destroy(foe_ctx *c)
{
    if (!c) return;
    prof_clear(c);
    cudaFree(c->d_wts);
    cudaFree(c->d_alpha);
    cudaFree(c->d_tcops);
    cudaFree(c->d_energy);
    cudaFree(c->d_status);
    cudaFree(c->d_partials);
    cudaFree(c->ws);
    delete c;
}

foe_status foe_step_size(const foe_ctx *ctx, foe_bc bc, float gamma, float *tau_out, double *lipschitz_out)
{
    if (!ctx || (bc != FOE_BC_SYMMETRIC && bc != FOE_BC_ZERO) || !(gamma >= 0.0f && gamma < 1.0f)) return FOE_EINVAL;
    if (tau_out) *tau_out = default_tau(ctx->symbol_max, bc, gamma);
    if (lipschitz_out) *lipschitz_out = 2.0 * kappa(bc) * ctx->symbol_max;
    return FOE_OK;
}

foe_status foe_denoise(foe_ctx *c, const float *y, float *x, int H, int W, int ld, float peak,
                       const foe_solve_opts *o, void *stream, foe_report *rep)
{
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts(c, o)) != FOE_OK) return st;
    if ((st = check_image(c, y, H, W, ld, "y")) != FOE_OK) return st;
    if ((st = check_image(c, x, H, W, ld, "x")) != FOE_OK) return st;
    if (o->model == FOE_MODEL_AUTO && !(peak > 0.0f && std::isfinite(peak))) {
        set_err(c, "peak must be > 0 for FOE_MODEL_AUTO");
        return FOE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int model = resolve_model(o->model, peak);
    const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
    const size_t plane = (size_t)H * ld;
    if ((st = ensure_ws(c, 5 * plane * sizeof(float))) != FOE_OK) return st;
    Slot sl = carve((float *)c->ws, plane);
    FOE_CUDA(c, foe::launch_init(y, H, W, ld, ld, model, o->zero_c, sl.d, sl.uh0, sl.ul, sl.delta, s));
    args_begin(c, o->bc);
    ImgDesc d{};
    d.u_hi[0] = sl.uh0;
    d.u_hi[1] = sl.uh1;
    d.u_lo = sl.ul;
    d.delta = sl.delta;
    d.d = sl.d;
    d.out = nullptr;
    d.H = H;
    d.W = W;
    d.ld = ld;
    d.model = model;
    d.sc = step_consts(tau, o->gamma, o->lambda);
    args_add(c, o->prec, d);
    cudaEvent_t ev[2];
    if ((st = prof_begin(c, s, ev)) != FOE_OK) return st;
    for (int n = 0; n < o->iters; ++n) {
        c->args.parity = n & 1;
        if ((st = launch(c, o->prec, foe::kStep, s)) != FOE_OK) return st;
    }
    if ((st = prof_end(c, s, ev, o->iters, (double)H * W * o->iters)) != FOE_OK) return st;
    const float *uf = (o->iters & 1) ? sl.uh1 : sl.uh0;
    FOE_CUDA(c, foe::launch_output(uf, sl.ul, H, W, ld, ld, model, x, s));
    if (rep) {
        int dev_status = 0;
        FOE_CUDA(c, cudaMemcpyAsync(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
        rep->iters_done = o->iters;
        rep->model_used = model;
        rep->tau_used = tau;
        rep->status = dev_status ? (foe_status)dev_status : FOE_OK;
        if (dev_status) {
            FOE_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_err(c, "a device-side wait expired during the solve");
            return (foe_status)dev_status;
        }
    }
    return FOE_OK;
}

foe_status foe_denoise_batch(foe_ctx *c, const foe_image_desc *descs, int n, const foe_solve_opts *o, void *stream)
{
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts(c, o)) != FOE_OK) return st;
    if (!descs || n < 1 || n > foe::kMaxBatch) {
        set_err(c, "batch size must be in 1..%d", foe::kMaxBatch);
        return FOE_EINVAL;
    }
    std::vector<int> order(n);
    size_t total = 0;
    int max_iters = 0;
    for (int i = 0; i < n; ++i) {
        const foe_image_desc &d = descs[i];
        if ((st = check_image(c, d.y, d.H, d.W, d.ld, "desc.y")) != FOE_OK) return st;
        if ((st = check_image(c, d.x, d.H, d.W, d.ld, "desc.x")) != FOE_OK) return st;
        if (d.iters < 0) { set_err(c, "desc.iters must be >= 0"); return FOE_EINVAL; }
        if (o->model == FOE_MODEL_AUTO && !(d.peak > 0.0f && std::isfinite(d.peak))) {
            set_err(c, "desc.peak must be > 0 for FOE_MODEL_AUTO");
            return FOE_EINVAL;
        }
        order[i] = i;
        total += 5 * (size_t)d.H * d.ld;
        max_iters = std::max(max_iters, d.iters);
    }
    // images with larger budgets first: the active set of every iteration is a prefix
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return descs[a].iters > descs[b].iters; });
    if ((st = ensure_ws(c, total * sizeof(float))) != FOE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Slot> slots(n);
    std::vector<int> models(n);
    float *base = (float *)c->ws;
    args_begin(c, o->bc);
    for (int j = 0; j < n; ++j) {
        const foe_image_desc &d = descs[order[j]];
        const size_t plane = (size_t)d.H * d.ld;
        slots[j] = carve(base, plane);
        base += 5 * plane;
        models[j] = resolve_model(o->model, d.peak);
        FOE_CUDA(c, foe::launch_init(d.y, d.H, d.W, d.ld, d.ld, models[j], o->zero_c, slots[j].d, slots[j].uh0,
                                     slots[j].ul, slots[j].delta, s));
        const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
        ImgDesc e{};
        e.u_hi[0] = slots[j].uh0;
        e.u_hi[1] = slots[j].uh1;
        e.u_lo = slots[j].ul;
        e.delta = slots[j].delta;
        e.d = slots[j].d;
        e.H = d.H;
        e.W = d.W;
        e.ld = d.ld;
        e.model = models[j];
        e.sc = step_consts(tau, o->gamma, o->lambda);
        args_add(c, o->prec, e);
    }
    const int nall = c->args.nimg;
    cudaEvent_t ev[2];
    if ((st = prof_begin(c, s, ev)) != FOE_OK) return st;
    double pix = 0.0;
    for (int it = 0; it < max_iters; ++it) {
        int active = 0;
        while (active < nall && descs[order[active]].iters > it) {
            pix += (double)descs[order[active]].H * descs[order[active]].W;
            ++active;
        }
        c->args.nimg = active;
        c->args.parity = it & 1;
        if ((st = launch(c, o->prec, foe::kStep, s)) != FOE_OK) {
            c->args.nimg = nall;
            return st;
        }
    }
    c->args.nimg = nall;
    if ((st = prof_end(c, s, ev, max_iters, pix)) != FOE_OK) return st;
    for (int j = 0; j < n; ++j) {
        const foe_image_desc &d = descs[order[j]];
        const float *uf = (d.iters & 1) ? slots[j].uh1 : slots[j].uh0;
        FOE_CUDA(c, foe::launch_output(uf, slots[j].ul, d.H, d.W, d.ld, d.ld, models[j], d.x, s));
    }
    return FOE_OK;
}

foe_status foe_energy_grad(foe_ctx *c, const float *u, const float *data, int H, int W, int ld, foe_model model,
                           float lambda, foe_bc bc, foe_precision prec, double *energy_host, float *grad, void *stream)
{
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_image(c, u, H, W, ld, "u")) != FOE_OK) return st;
    if ((st = check_image(c, data, H, W, ld, "data")) != FOE_OK) return st;
    if (grad && (st = check_image(c, grad, H, W, ld, "grad")) != FOE_OK) return st;
    if (model != FOE_MODEL_DIRECT && model != FOE_MODEL_ANS_L2 && model != FOE_MODEL_ANS_IDIV) {
        set_err(c, "model must be DIRECT, ANS_L2 or ANS_IDIV");
        return FOE_EINVAL;
    }
    if (!(lambda > 0.0f)) { set_err(c, "lambda must be > 0"); return FOE_EINVAL; }
    if (bc != FOE_BC_SYMMETRIC && bc != FOE_BC_ZERO) { set_err(c, "bad bc"); return FOE_EINVAL; }
    if (prec != FOE_PREC_FP32 && prec != FOE_PREC_BF16) { set_err(c, "precision not supported"); return FOE_EUNSUPPORTED; }
    cudaStream_t s = (cudaStream_t)stream;
    ImgDesc d{};
    d.u_hi[0] = const_cast<float *>(u);
    d.u_hi[1] = nullptr;
    d.d = data;
    d.out = grad;
    d.H = H;
    d.W = W;
    d.ld = ld;
    d.model = model;
    d.sc = step_consts(0.0f, 0.0f, lambda);
    if (grad) {
        args_begin(c, bc);
        args_add(c, prec, d);
        if ((st = launch(c, prec, foe::kGrad, s)) != FOE_OK) return st;
    }
    if (energy_host) {
        // the energy always uses the FP32 path (its responses are evaluated once, not iterated)
        args_begin(c, bc);
        args_add(c, FOE_PREC_FP32, d);
        const int tiles = c->args.tile_prefix[1];
        if ((st = ensure_partials(c, tiles)) != FOE_OK) return st;
        c->args.partials = c->d_partials;
        if ((st = launch(c, FOE_PREC_FP32, foe::kEnergy, s)) != FOE_OK) return st;
        FOE_CUDA(c, foe::launch_reduce(c->d_partials, tiles, c->d_energy, s));
        FOE_CUDA(c, cudaMemcpyAsync(energy_host, c->d_energy, sizeof(double), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
    }
    return FOE_OK;
}

foe_status foe_ipiano_step(foe_ctx *c, const float *u_hi, float *u_lo, float *delta, const float *d,
                           float *u_next_hi, int H, int W, int ld, foe_model model, float lambda, float tau,
                           float gamma, foe_bc bc, foe_precision prec, void *stream)
{
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_image(c, u_hi, H, W, ld, "u_hi")) != FOE_OK) return st;
    if (u_lo && (st = check_image(c, u_lo, H, W, ld, "u_lo")) != FOE_OK) return st;
    if ((st = check_image(c, delta, H, W, ld, "delta")) != FOE_OK) return st;
    if ((st = check_image(c, d, H, W, ld, "d")) != FOE_OK) return st;
    if ((st = check_image(c, u_next_hi, H, W, ld, "u_next_hi")) != FOE_OK) return st;
    if (u_next_hi == u_hi) { set_err(c, "u_next_hi must not alias u_hi"); return FOE_EINVAL; }
    if (model != FOE_MODEL_DIRECT && model != FOE_MODEL_ANS_L2 && model != FOE_MODEL_ANS_IDIV) {
        set_err(c, "model must be DIRECT, ANS_L2 or ANS_IDIV");
        return FOE_EINVAL;
    }
    if (!(lambda > 0.0f) || !(tau > 0.0f) || !(gamma >= 0.0f && gamma < 1.0f)) {
        set_err(c, "need lambda > 0, tau > 0, 0 <= gamma < 1");
        return FOE_EINVAL;
    }
    if (bc != FOE_BC_SYMMETRIC && bc != FOE_BC_ZERO) { set_err(c, "bad bc"); return FOE_EINVAL; }
    if (prec != FOE_PREC_FP32 && prec != FOE_PREC_BF16) { set_err(c, "precision not supported"); return FOE_EUNSUPPORTED; }
    ImgDesc e{};
    e.u_hi[0] = const_cast<float *>(u_hi);
    e.u_hi[1] = u_next_hi;
    e.u_lo = u_lo;
    e.delta = delta;
    e.d = d;
    e.H = H;
    e.W = W;
    e.ld = ld;
    e.model = model;
    e.sc = step_consts(tau, gamma, lambda);
    args_begin(c, bc);
    args_add(c, prec, e);
    return launch(c, prec, foe::kStep, (cudaStream_t)stream);
}

foe_status foe_profile(foe_ctx *c, int enable)
{
    if (!c) return FOE_EINVAL;
    if (enable) prof_clear(c);
    c->prof = enable != 0;
    return FOE_OK;
}

foe_status foe_profile_read(foe_ctx *c, double *loop_ms, long *launches, double *pixel_iters)
{
    if (!c) return FOE_EINVAL;
    double ms = 0.0;
    for (auto &p : c->prof_events) {
        FOE_CUDA(c, cudaEventSynchronize(p.second));
        float t = 0.0f;
        FOE_CUDA(c, cudaEventElapsedTime(&t, p.first, p.second));
        ms += t;
    }
    if (loop_ms) *loop_ms = ms;
    if (launches) *launches = c->prof_launches;
    if (pixel_iters) *pixel_iters = c->prof_pixel_iters;
    return FOE_OK;
}

foe_status foe_anscombe(const float *y, float *v, long n, void *stream)
{
    if (n < 0 || (n > 0 && (!y || !v))) return FOE_EINVAL;
    return foe::launch_anscombe(y, v, n, (cudaStream_t)stream) == cudaSuccess ? FOE_OK : FOE_ECUDA;
}

foe_status foe_inverse(const float *z, float *x, long n, void *stream)
{
    if (n < 0 || (n > 0 && (!z || !x))) return FOE_EINVAL;
    return foe::launch_inverse(z, x, n, (cudaStream_t)stream) == cudaSuccess ? FOE_OK : FOE_ECUDA;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Denoising without any allocation: the workspace of foe_denoise_static lives in a fixed device array
// of this file instead of memory obtained with cudaMalloc.
// ------------------------------------------------------------------------------------------------

// Five planes (u_hi[2], u_lo, delta, d) of at most kStaticMaxPlane floats each: 20 MiB, held on every
// device that loads the library until the process exits.
static constexpr size_t kStaticMaxPlane = (size_t)1 << 20;
static __device__ __align__(256) float g_static_ws[5 * kStaticMaxPlane];

namespace {

constexpr int kStaticMaxDevices = 64;
float *g_static_ws_ptr[kStaticMaxDevices] = {};
std::mutex g_static_ws_mu;

// Device address of g_static_ws on the current device, looked up once per device.  In host code the
// name g_static_ws is only a host-side stand-in, so kernels must be given this address instead.
foe_status static_workspace(foe_ctx *c, float **out)
{
    int dev = 0;
    FOE_CUDA(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) {
        set_err(c, "device ordinal %d is beyond the %d devices foe_denoise_static supports", dev, kStaticMaxDevices);
        return FOE_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_static_ws_mu);
    if (!g_static_ws_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || !p) {
            set_err(c, "cudaGetSymbolAddress(g_static_ws) failed: %s", cudaGetErrorString(e));
            return FOE_ECUDA;
        }
        g_static_ws_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_static_ws_ptr[dev];
    return FOE_OK;
}

}  // namespace

extern "C" foe_status foe_denoise_static(foe_ctx *c, const float *y, float *x, int H, int W, int ld, float peak,
                                         const foe_solve_opts *o, void *stream)
{
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts(c, o)) != FOE_OK) return st;
    if ((st = check_image(c, y, H, W, ld, "y")) != FOE_OK) return st;
    if ((st = check_image(c, x, H, W, ld, "x")) != FOE_OK) return st;
    if ((size_t)H * (size_t)ld > kStaticMaxPlane) {
        set_err(c, "image of %d x %d with pitch %d needs H * ld = %zu floats per plane; the static workspace "
                   "holds at most %zu (e.g. 1024 x 1024)", H, W, ld, (size_t)H * (size_t)ld, kStaticMaxPlane);
        return FOE_EINVAL;
    }
    if (o->model == FOE_MODEL_AUTO && !(peak > 0.0f && std::isfinite(peak))) {
        set_err(c, "peak must be > 0 for FOE_MODEL_AUTO");
        return FOE_EINVAL;
    }
    float *ws = nullptr;
    if ((st = static_workspace(c, &ws)) != FOE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int model = resolve_model(o->model, peak);
    const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
    // every plane that the solve reads is written first by k_init (d, u_hi[0], u_lo, delta) or by the
    // step that precedes the read (u_hi[1]), so the previous call's contents need no clearing
    Slot sl = carve(ws, (size_t)H * ld);
    FOE_CUDA(c, foe::launch_init(y, H, W, ld, ld, model, o->zero_c, sl.d, sl.uh0, sl.ul, sl.delta, s));
    args_begin(c, o->bc);
    ImgDesc d{};
    d.u_hi[0] = sl.uh0;
    d.u_hi[1] = sl.uh1;
    d.u_lo = sl.ul;
    d.delta = sl.delta;
    d.d = sl.d;
    d.H = H;
    d.W = W;
    d.ld = ld;
    d.model = model;
    d.sc = step_consts(tau, o->gamma, o->lambda);
    args_add(c, o->prec, d);
    for (int n = 0; n < o->iters; ++n) {
        c->args.parity = n & 1;
        if ((st = launch(c, o->prec, foe::kStep, s)) != FOE_OK) return st;
    }
    const float *uf = (o->iters & 1) ? sl.uh1 : sl.uh0;
    FOE_CUDA(c, foe::launch_output(uf, sl.ul, H, W, ld, ld, model, x, s));
    return FOE_OK;
}
