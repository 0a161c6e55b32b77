// Host side of the prior training step: forward solve with checkpoints, loss, reverse sweep.
#include <cmath>

#include "foe_internal.h"

namespace {

// Launches one iteration of the FP32 step kernel for images [i0, i1), with the image's read / write
// planes given explicitly (parity 0).
foe_status forward_group(foe_ctx *c, const std::vector<ImgDesc> &descs, int i0, int i1, int bc, cudaStream_t s)
{
    args_begin(c, bc);
    for (int i = i0; i < i1; ++i) args_add(c, FOE_PREC_FP32, descs[i]);
    c->args.parity = 0;
    return launch(c, FOE_PREC_FP32, foe::kStep, s);
}

}  // namespace

extern "C" foe_status foe_train_step(foe_ctx *c, const float *clean, const float *noisy, int B, int H, int W, int ld,
                                     const foe_solve_opts *o, int ckpt_every, double *loss_host, float *dfilters,
                                     float *dlogalpha, void *stream)
{
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts_fixed(c, o, "foe_train_step")) != FOE_OK) return st;
    if (o->model != FOE_MODEL_ANS_L2) { set_err(c, "training needs FOE_MODEL_ANS_L2"); return FOE_EUNSUPPORTED; }
    if (o->prec != FOE_PREC_FP32) { set_err(c, "training runs in FP32"); return FOE_EUNSUPPORTED; }
    if (B < 1 || !dfilters || !dlogalpha) { set_err(c, "need B >= 1 and gradient buffers"); return FOE_EINVAL; }
    if ((st = check_image(c, clean, H, W, ld, "clean")) != FOE_OK) return st;
    if ((st = check_image(c, noisy, H, W, ld, "noisy")) != FOE_OK) return st;
    const int T = o->iters;
    if (T < 1) { set_err(c, "iters must be >= 1"); return FOE_EINVAL; }
    const int C = ckpt_every > 0 ? ckpt_every : std::max(1, (int)std::lround(std::sqrt((double)T)));
    const int ncp = (T + C - 1) / C;
    const size_t plane = (size_t)H * ld;
    const int tiles_per = ((H + foe::bwd_tile() - 1) / foe::bwd_tile()) * ((W + foe::bwd_tile() - 1) / foe::bwd_tile());
    const int group = foe::kMaxBatch;
    const int max_group_tiles = std::min(B, group) * tiles_per;
    constexpr int kLossBlocks = 64;
    // workspace: state 5, checkpoints 3 * ncp, segment C, gbar 3 (planes per image); partials; FP64 accumulators
    const size_t nplanes = (size_t)B * (5 + 3 * ncp + C + 3);
    const size_t bytes = nplanes * plane * sizeof(float) + (size_t)max_group_tiles * foe::kBwdPartials * sizeof(float) +
                         (foe::kBwdPartials + (size_t)B * kLossBlocks) * sizeof(double) + 256;
    if ((st = ensure_ws(c, bytes)) != FOE_OK) return st;
    float *base = (float *)c->ws;
    auto P = [&](size_t k) { return base + k * plane; };
    std::vector<Slot> slot(B);
    for (int i = 0; i < B; ++i) slot[i] = carve(P((size_t)i * 5), plane);
    auto ckpt = [&](int cp, int i, int which) { return P((size_t)B * 5 + ((size_t)cp * B + i) * 3 + which); };
    auto seg = [&](int k, int i) { return P((size_t)B * (5 + 3 * ncp) + (size_t)k * B + i); };
    auto gbp = [&](int r, int i) { return P((size_t)B * (5 + 3 * ncp + C) + (size_t)r * B + i); };
    float *partials = P(nplanes);
    double *acc = reinterpret_cast<double *>(((uintptr_t)(partials + (size_t)max_group_tiles * foe::kBwdPartials) + 255) &
                                             ~(uintptr_t)255);
    double *loss_part = acc + foe::kBwdPartials;
    cudaStream_t s = (cudaStream_t)stream;
    const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
    const foe::StepConsts sc = step_consts(tau, o->gamma, o->lambda);
    const float c1 = (float)(1.0 / (1.0 + (double)tau * (double)o->lambda));

    // ---- forward: u^0 = u^{-1} = v, T steps, checkpoints of (u_hi, u_lo, delta) at n = 0, C, 2C, ... ----
    std::vector<ImgDesc> d(B);
    for (int i = 0; i < B; ++i) {
        FOE_CUDA(c, foe::launch_init(noisy + (size_t)i * plane, H, W, ld, ld, foe::kAnsL2, 0.0f, slot[i].d, slot[i].uh0,
                                     slot[i].ul, slot[i].delta, s));
        d[i] = ImgDesc{};
        d[i].u_lo = slot[i].ul;
        d[i].delta = slot[i].delta;
        d[i].d = slot[i].d;
        d[i].H = H;
        d[i].W = W;
        d[i].ld = ld;
        d[i].model = foe::kAnsL2;
        d[i].sc = sc;
    }
    for (int n = 0; n < T; ++n) {
        for (int i = 0; i < B; ++i) {
            float *un = (n & 1) ? slot[i].uh1 : slot[i].uh0;
            if (n % C == 0) {
                FOE_CUDA(c, foe::launch_copy(un, ckpt(n / C, i, 0), (long)plane, s));
                FOE_CUDA(c, foe::launch_copy(slot[i].ul, ckpt(n / C, i, 1), (long)plane, s));
                FOE_CUDA(c, foe::launch_copy(slot[i].delta, ckpt(n / C, i, 2), (long)plane, s));
            }
            d[i].u_hi[0] = un;
            d[i].u_hi[1] = (n & 1) ? slot[i].uh0 : slot[i].uh1;
        }
        for (int i0 = 0; i0 < B; i0 += group)
            if ((st = forward_group(c, d, i0, std::min(B, i0 + group), o->bc, s)) != FOE_OK) return st;
    }
    // ---- loss and gbar^T ----
    for (int i = 0; i < B; ++i) {
        const float *uT = (T & 1) ? slot[i].uh1 : slot[i].uh0;
        FOE_CUDA(c, foe::launch_train_loss(uT, slot[i].ul, clean + (size_t)i * plane, H, W, ld, ld, gbp(0, i),
                                           loss_part + (size_t)i * kLossBlocks, kLossBlocks, s));
    }
    FOE_CUDA(c, cudaMemsetAsync(acc, 0, foe::kBwdPartials * sizeof(double), s));

    // ---- reverse sweep, one checkpoint segment at a time ----
    int r1 = 0, r2 = -1, rout = 1;  // gbar ring: gbar^{n+1} in r1, gbar^{n+2} in r2 (none yet), gbar^n -> rout
    for (int cp = ncp - 1; cp >= 0; --cp) {
        const int n0 = cp * C, n1 = std::min(T, n0 + C);
        // recompute u^{n0} .. u^{n1-1} into the segment planes
        for (int i = 0; i < B; ++i) {
            FOE_CUDA(c, foe::launch_copy(ckpt(cp, i, 0), seg(0, i), (long)plane, s));
            FOE_CUDA(c, foe::launch_copy(ckpt(cp, i, 1), slot[i].ul, (long)plane, s));
            FOE_CUDA(c, foe::launch_copy(ckpt(cp, i, 2), slot[i].delta, (long)plane, s));
        }
        for (int n = n0; n < n1 - 1; ++n) {
            for (int i = 0; i < B; ++i) {
                d[i].u_hi[0] = seg(n - n0, i);
                d[i].u_hi[1] = seg(n + 1 - n0, i);
            }
            for (int i0 = 0; i0 < B; i0 += group)
                if ((st = forward_group(c, d, i0, std::min(B, i0 + group), o->bc, s)) != FOE_OK) return st;
        }
        for (int n = n1 - 1; n >= n0; --n) {
            for (int i0 = 0; i0 < B; i0 += group) {
                const int i1 = std::min(B, i0 + group);
                foe::BwdArgs a{};
                a.nimg = 0;
                a.bc = o->bc;
                a.nchunks = (c->nf + 7) / 8;
                a.write_g = n >= 1;
                a.tau = tau;
                a.gamma = o->gamma;
                a.c1 = c1;
                a.wts = c->d_wts;
                a.alpha = c->d_alpha;
                a.partials = partials;
                a.tile_prefix[0] = 0;
                for (int i = i0; i < i1; ++i) {
                    foe::BwdImg &e = a.img[a.nimg];
                    e.u = seg(n - n0, i);
                    e.gb1 = gbp(r1, i);
                    e.gb2 = r2 >= 0 ? gbp(r2, i) : nullptr;
                    e.gout = gbp(rout, i);
                    e.H = H;
                    e.W = W;
                    e.ld = ld;
                    e.tiles_x = (W + foe::bwd_tile() - 1) / foe::bwd_tile();
                    a.tile_prefix[a.nimg + 1] = a.tile_prefix[a.nimg] + tiles_per;
                    a.nimg++;
                }
                FOE_CUDA(c, foe::bwd_launch(a, s));
                FOE_CUDA(c, foe::launch_reduce_partials(partials, a.tile_prefix[a.nimg], acc, s));
            }
            // rotate: gbar^{n+2} <- gbar^{n+1}, gbar^{n+1} <- gbar^n
            const int free_buf = r2 >= 0 ? r2 : 3 - r1 - rout;
            r2 = r1;
            r1 = rout;
            rout = free_buf;
        }
    }
    FOE_CUDA(c, foe::launch_train_finish(acc, c->d_alpha, tau, c->nf, dfilters, dlogalpha, s));
    if (loss_host) {
        std::vector<double> lp((size_t)B * kLossBlocks);
        FOE_CUDA(c, cudaMemcpyAsync(lp.data(), loss_part, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
        double L = 0.0;
        for (double v : lp) L += v;
        *loss_host = L;
    }
    return FOE_OK;
}
