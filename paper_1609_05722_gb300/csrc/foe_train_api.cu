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
    NvtxRange nvtx_range("foe_train_step");
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts_fixed(c, o, "foe_train_step")) != FOE_OK) return st;
    if ((st = check_no_tol(c, o, "foe_train_step")) != FOE_OK) return st;
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

extern "C" foe_status foe_train_grad_implicit(foe_ctx *c, const float *clean, const float *noisy, int B, int H, int W,
                                              int ld, const foe_solve_opts *o, int max_cg, float cg_tol,
                                              double *loss_host, float *dfilters, float *dlogalpha,
                                              foe_implicit_report *rep, void *stream)
{
    NvtxRange nvtx_range("foe_train_grad_implicit");
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts_fixed(c, o, "foe_train_grad_implicit")) != FOE_OK) return st;
    if ((st = check_no_tol(c, o, "foe_train_grad_implicit")) != FOE_OK) return st;
    if (o->model != FOE_MODEL_ANS_L2) { set_err(c, "training needs FOE_MODEL_ANS_L2"); return FOE_EUNSUPPORTED; }
    if (o->prec != FOE_PREC_FP32 && o->prec != FOE_PREC_TF32) {
        set_err(c, "foe_train_grad_implicit runs in FP32, or with TF32 tensor-core Hessian-vector products");
        return FOE_EUNSUPPORTED;
    }
    const bool tc_hvp = o->prec == FOE_PREC_TF32;
    if (B < 1 || !dfilters || !dlogalpha) { set_err(c, "need B >= 1 and gradient buffers"); return FOE_EINVAL; }
    if (max_cg < 1 || !(cg_tol >= 0.0f) || !std::isfinite(cg_tol)) {
        set_err(c, "need max_cg >= 1 and a finite cg_tol >= 0");
        return FOE_EINVAL;
    }
    if ((st = check_image(c, clean, H, W, ld, "clean")) != FOE_OK) return st;
    if ((st = check_image(c, noisy, H, W, ld, "noisy")) != FOE_OK) return st;
    const int T = o->iters;
    const size_t plane = (size_t)H * ld;
    const int tiles_per = ((H + foe::bwd_tile() - 1) / foe::bwd_tile()) * ((W + foe::bwd_tile() - 1) / foe::bwd_tile());
    const int group = foe::kMaxBatch;
    const int max_group_tiles = std::min(B, group) * tiles_per;
    constexpr int kLossBlocks = 64;
    // workspace: state 5 planes per image, then b, q, r, p, Ap (B planes each); partials; FP64 accumulators; CG state
    const size_t nplanes = (size_t)B * 10;
    const size_t bytes = nplanes * plane * sizeof(float) + (size_t)max_group_tiles * foe::kBwdPartials * sizeof(float) +
                         (foe::kBwdPartials + (size_t)B * (kLossBlocks + 2 * foe::kCgBlocks)) * sizeof(double) +
                         (size_t)B * sizeof(foe::CgState) + 512;
    if ((st = ensure_ws(c, bytes)) != FOE_OK) return st;
    float *base = (float *)c->ws;
    std::vector<Slot> slot(B);
    for (int i = 0; i < B; ++i) slot[i] = carve(base + (size_t)i * 5 * plane, plane);
    float *bv = base + (size_t)B * 5 * plane, *qv = bv + (size_t)B * plane, *rv = qv + (size_t)B * plane,
          *pv = rv + (size_t)B * plane, *Apv = pv + (size_t)B * plane;
    float *partials = Apv + (size_t)B * plane;
    double *acc = reinterpret_cast<double *>(((uintptr_t)(partials + (size_t)max_group_tiles * foe::kBwdPartials) + 255) &
                                             ~(uintptr_t)255);
    double *loss_part = acc + foe::kBwdPartials;
    double *part_pap = loss_part + (size_t)B * kLossBlocks, *part_rr = part_pap + (size_t)B * foe::kCgBlocks;
    foe::CgState *cgs = reinterpret_cast<foe::CgState *>(part_rr + (size_t)B * foe::kCgBlocks);
    cudaStream_t s = (cudaStream_t)stream;
    const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
    const foe::StepConsts sc = step_consts(tau, o->gamma, o->lambda);

    // ---- lower-level solve: u^0 = u^{-1} = v, T iPiano steps (w* ~ u^T) ----
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
            d[i].u_hi[0] = (n & 1) ? slot[i].uh1 : slot[i].uh0;
            d[i].u_hi[1] = (n & 1) ? slot[i].uh0 : slot[i].uh1;
        }
        for (int i0 = 0; i0 < B; i0 += group)
            if ((st = forward_group(c, d, i0, std::min(B, i0 + group), o->bc, s)) != FOE_OK) return st;
    }
    auto wstar = [&](int i) -> const float * { return (T & 1) ? slot[i].uh1 : slot[i].uh0; };

    // ---- TF32 path: the Hessian factors (1 - r^2) / (1 + r^2)^2 of the responses of w*, once ----
    const size_t hess_per = (size_t)H * W * 48;
    std::vector<ImgDesc> hd;
    if (tc_hvp) {
        const size_t hb = (size_t)B * hess_per * sizeof(float);
        if (hb > c->hess_bytes) {
            if (c->d_hess) FOE_CUDA(c, cudaFree(c->d_hess));
            c->d_hess = nullptr;
            c->hess_bytes = 0;
            FOE_CUDA(c, cudaMalloc(&c->d_hess, hb));
            c->hess_bytes = hb;
        }
        hd.resize(B);
        for (int i = 0; i < B; ++i) {
            hd[i] = ImgDesc{};
            hd[i].u_hi[0] = const_cast<float *>(wstar(i));
            hd[i].H = H;
            hd[i].W = W;
            hd[i].ld = ld;
            hd[i].model = foe::kAnsL2;
            hd[i].sc = sc;
            hd[i].hess = c->d_hess + (size_t)i * hess_per;
        }
        for (int i0 = 0; i0 < B; i0 += group) {
            args_begin(c, o->bc);
            for (int i = i0; i < std::min(B, i0 + group); ++i) args_add(c, FOE_PREC_TF32, hd[i]);
            if ((st = launch(c, FOE_PREC_TF32, foe::kHess, s)) != FOE_OK) return st;
        }
    }
    // H_E x on the tensor cores: the direction's responses (TF32), times the stored factors, the adjoint, + lambda x
    auto tc_hvp_launch = [&](const float *x, float *out) -> foe_status {
        for (int i0 = 0; i0 < B; i0 += group) {
            args_begin(c, o->bc);
            for (int i = i0; i < std::min(B, i0 + group); ++i) {
                ImgDesc e = hd[i];
                e.u_hi[0] = const_cast<float *>(x + (size_t)i * plane);
                e.out = out + (size_t)i * plane;
                args_add(c, FOE_PREC_TF32, e);
            }
            foe_status r = launch(c, FOE_PREC_TF32, foe::kHvp, s);
            if (r != FOE_OK) return r;
        }
        return FOE_OK;
    };

    // ---- loss and b = dL/dw at w* ----
    for (int i = 0; i < B; ++i)
        FOE_CUDA(c, foe::launch_train_loss(wstar(i), slot[i].ul, clean + (size_t)i * plane, H, W, ld, ld,
                                           bv + (size_t)i * plane, loss_part + (size_t)i * kLossBlocks, kLossBlocks, s));

    // one backward-kernel launch per group of images: Hessian-vector products (hvp_only) or parameter partials
    auto bwd = [&](bool hvp, const float *x, float *out) -> foe_status {
        for (int i0 = 0; i0 < B; i0 += group) {
            const int i1 = std::min(B, i0 + group);
            foe::BwdArgs a{};
            a.bc = o->bc;
            a.nchunks = (c->nf + 7) / 8;
            a.write_g = hvp ? 1 : 0;
            a.hvp_only = hvp ? 1 : 0;
            a.tau = -1.0f;                // gout = (1 + gamma) x - tau H x = lambda x + H x
            a.gamma = o->lambda - 1.0f;
            a.c1 = 1.0f;
            a.wts = c->d_wts;
            a.alpha = c->d_alpha;
            a.partials = partials;
            a.tile_prefix[0] = 0;
            for (int i = i0; i < i1; ++i) {
                foe::BwdImg &e = a.img[a.nimg];
                e.u = wstar(i);
                e.gb1 = x + (size_t)i * plane;
                e.gb2 = nullptr;
                e.gout = hvp ? out + (size_t)i * plane : nullptr;
                e.H = H;
                e.W = W;
                e.ld = ld;
                e.tiles_x = (W + foe::bwd_tile() - 1) / foe::bwd_tile();
                a.tile_prefix[a.nimg + 1] = a.tile_prefix[a.nimg] + tiles_per;
                a.nimg++;
            }
            FOE_CUDA(c, foe::bwd_launch(a, s));
            if (!hvp) FOE_CUDA(c, foe::launch_reduce_partials(partials, a.tile_prefix[a.nimg], acc, s));
        }
        return FOE_OK;
    };

    // ---- q = H_E(w*)^{-1} b by conjugate gradients from q = 0 ----
    FOE_CUDA(c, cudaMemsetAsync(qv, 0, (size_t)B * plane * sizeof(float), s));
    FOE_CUDA(c, cudaMemcpyAsync(rv, bv, (size_t)B * plane * sizeof(float), cudaMemcpyDeviceToDevice, s));
    FOE_CUDA(c, cudaMemcpyAsync(pv, bv, (size_t)B * plane * sizeof(float), cudaMemcpyDeviceToDevice, s));
    FOE_CUDA(c, foe::launch_cg_dot(bv, bv, B, H, W, ld, part_pap, s));
    FOE_CUDA(c, foe::launch_cg_init(part_pap, cgs, B, s));
    const double tol2 = (double)cg_tol * (double)cg_tol;
    std::vector<foe::CgState> hs(B);
    auto all_done = [&](int k) -> bool {
        if (cudaMemcpyAsync(hs.data(), cgs, B * sizeof(foe::CgState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return false;
        for (const auto &x : hs)
            if (!x.done[k & 1]) return false;
        return true;
    };
    int K = 0;  // iterations launched; every image's final <r, r> is then in slot K & 1
    for (int k = 0; k < max_cg; ++k) {
        if (k % 32 == 0 && all_done(k)) break;
        if ((st = tc_hvp ? tc_hvp_launch(pv, Apv) : bwd(true, pv, Apv)) != FOE_OK) return st;
        FOE_CUDA(c, foe::launch_cg_dot(pv, Apv, B, H, W, ld, part_pap, s));
        FOE_CUDA(c, foe::launch_cg_update(qv, rv, pv, Apv, B, H, W, ld, part_pap, part_rr, cgs, k, tol2, s));
        K = k + 1;
    }

    // ---- dL/dk, dL/da from (w*, q): Eq. overallderivative (partials of the backward kernel, factor -alpha_i) ----
    FOE_CUDA(c, cudaMemsetAsync(acc, 0, foe::kBwdPartials * sizeof(double), s));
    if ((st = bwd(false, qv, nullptr)) != FOE_OK) return st;
    FOE_CUDA(c, foe::launch_train_finish(acc, c->d_alpha, 1.0f, c->nf, dfilters, dlogalpha, s));
    if (rep || loss_host) {
        std::vector<double> lp((size_t)B * kLossBlocks);
        FOE_CUDA(c, cudaMemcpyAsync(lp.data(), loss_part, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaMemcpyAsync(hs.data(), cgs, B * sizeof(foe::CgState), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
        if (loss_host) {
            double L = 0.0;
            for (double v : lp) L += v;
            *loss_host = L;
        }
        if (rep) {
            rep->cg_iters = 0;
            rep->cg_relres = 0.0;
            rep->breakdowns = 0;
            for (const auto &x : hs) {
                rep->cg_iters = std::max(rep->cg_iters, x.iters);
                const double rel = x.rr0 > 0.0 ? std::sqrt(x.rr[K & 1] / x.rr0) : 0.0;
                rep->cg_relres = std::max(rep->cg_relres, rel);
                rep->breakdowns += x.breakdown;
            }
        }
    }
    return FOE_OK;
}
