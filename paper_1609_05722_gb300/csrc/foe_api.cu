// C ABI of the FoE denoiser: argument checks, context and workspace, step size, launch sequencing.
#include <mutex>

#include "foe_internal.h"

// Enqueues a whole batch solve on s: initialisation, the iteration launches, the output maps.
static foe_status enqueue_batch(foe_ctx *c, const foe_image_desc *descs, int n, const foe_solve_opts *o,
                                cudaStream_t s, const std::vector<int> &order, int max_iters, bool profile)
{
    foe_status st;
    std::vector<Slot> slots(n);
    std::vector<int> models(n);
    float *base = (float *)c->ws;
    const bool tol_on = o->tol > 0.0f;
    if (tol_on) FOE_CUDA(c, cudaMemsetAsync(c->d_stop, 0, sizeof(int) * n, s));
    args_begin(c, o->bc);
    for (int j = 0; j < n; ++j) {
        const foe_image_desc &d = descs[order[j]];
        const size_t plane = (size_t)d.H * d.ld;
        slots[j] = carve(base, plane);
        base += 5 * plane;
        models[j] = resolve_model(d.use_model ? d.model : o->model, d.peak);
        FOE_CUDA(c, foe::launch_init(d.y, d.H, d.W, d.ld, d.ld, models[j], o->zero_c, slots[j].d, slots[j].uh0,
                                     lo_plane(o->prec, slots[j].ul), slots[j].delta, s));
        const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
        ImgDesc e{};
        e.u_hi[0] = slots[j].uh0;
        e.u_hi[1] = slots[j].uh1;
        e.u_lo = lo_plane(o->prec, slots[j].ul);
        e.delta = slots[j].delta;
        e.d = slots[j].d;
        e.H = d.H;
        e.W = d.W;
        e.ld = d.ld;
        e.model = models[j];
        e.sc = step_consts(tau, o->gamma, o->lambda);
        e.stop = tol_on ? c->d_stop + j : nullptr;
        args_add(c, o->prec, e);
    }
    const int nall = c->args.nimg;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (profile && (st = prof_begin(c, s, ev)) != FOE_OK) return st;
    double pix = 0.0;
    for (int it = 0; it < max_iters; ++it) {
        int active = 0;
        while (active < nall && descs[order[active]].iters > it) {
            pix += (double)descs[order[active]].H * descs[order[active]].W;
            ++active;
        }
        c->args.nimg = active;
        c->args.parity = it & 1;
        if ((st = launch(c, o->prec, foe::kStep, s)) != FOE_OK ||
            (tol_on && (it + 1) % o->tol_every == 0 && (st = tol_check(c, active, it + 1, o->tol, s)) != FOE_OK)) {
            c->args.nimg = nall;
            return st;
        }
    }
    c->args.nimg = nall;
    if (profile && (st = prof_end(c, s, ev, max_iters, pix)) != FOE_OK) return st;
    for (int j = 0; j < n; ++j) {
        const foe_image_desc &d = descs[order[j]];
        const float *uf = (d.iters & 1) ? slots[j].uh1 : slots[j].uh0, *ua = (d.iters & 1) ? slots[j].uh0 : slots[j].uh1;
        FOE_CUDA(c, foe::launch_output(uf, lo_plane(o->prec, slots[j].ul), d.H, d.W, d.ld, d.ld, models[j], d.x, nullptr, s,
                                       nullptr, ua, d.iters, tol_on ? c->d_stop + j : nullptr));
    }
    return FOE_OK;
}


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
    o->use_graph = 0;
    o->tol_every = 10;
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
    auto fail = [&](foe_status s) {
        foe_destroy(c);
        return s;
    };
    const std::vector<uint16_t> ops = tc_operands(w, c->alpha);
    const std::vector<uint32_t> ops32 = tc_operands_tf32(w, c->alpha);
    const std::vector<uint16_t> pops = pair_operands(w, c->alpha);
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_wts, sizeof(w))) || (e = cudaMalloc(&c->d_alpha, sizeof(c->alpha))) ||
        (e = cudaMalloc(&c->d_tcops, ops.size() * sizeof(uint16_t))) ||
        (e = cudaMemcpy(c->d_tcops, ops.data(), ops.size() * sizeof(uint16_t), cudaMemcpyHostToDevice)) ||
        (e = cudaMalloc(&c->d_tcops32, ops32.size() * sizeof(uint32_t))) ||
        (e = cudaMemcpy(c->d_tcops32, ops32.data(), ops32.size() * sizeof(uint32_t), cudaMemcpyHostToDevice)) ||
        (e = cudaMalloc(&c->d_pairops, pops.size() * sizeof(uint16_t))) ||
        (e = cudaMemcpy(c->d_pairops, pops.data(), pops.size() * sizeof(uint16_t), cudaMemcpyHostToDevice)) ||
        (e = cudaMalloc(&c->d_energy, sizeof(double))) || (e = cudaMalloc(&c->d_status, sizeof(int))) || (e = cudaMalloc(&c->d_nonfinite, sizeof(int))) ||
        (e = cudaMemcpy(c->d_wts, w, sizeof(w), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_alpha, c->alpha, sizeof(c->alpha), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->d_status, 0, sizeof(int))) || (e = foe::f32_setup()) || (e = foe::tc_setup()) || (e = foe::bwd_setup()))
        return fail(e == cudaErrorMemoryAllocation ? FOE_ENOMEM : FOE_ECUDA);
    if ((e = cudaMalloc(&c->d_stop, sizeof(int) * foe::kMaxBatch)) ||
        (e = cudaMalloc(&c->d_tol_part, sizeof(double) * 2 * foe::kTolBlocks * foe::kMaxBatch)) ||
        (e = cudaMalloc(&c->d_tol_count, sizeof(unsigned) * foe::kMaxBatch)) ||
        (e = cudaMemset(c->d_stop, 0, sizeof(int) * foe::kMaxBatch)) ||
        (e = cudaMemset(c->d_tol_count, 0, sizeof(unsigned) * foe::kMaxBatch)) ||
        (e = cudaHostAlloc(&c->h_stop, 2 * sizeof(int), cudaHostAllocDefault)) ||
        (e = cudaEventCreateWithFlags(&c->tol_ev[0], cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->tol_ev[1], cudaEventDisableTiming)) ||
        (e = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&c->side_fork, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->side_join, cudaEventDisableTiming)))
        return fail(e == cudaErrorMemoryAllocation ? FOE_ENOMEM : FOE_ECUDA);
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
    cudaFree(c->d_tcops32);
    cudaFree(c->d_pairops);
    cudaFree(c->d_energy);
    cudaFree(c->d_status);
    cudaFree(c->d_nonfinite);
    cudaFree(c->d_partials);
    cudaFree(c->ws);
    cudaFree(c->d_bin);
    cudaFree(c->d_stop);
    cudaFree(c->d_bt);
    cudaFree(c->d_bt_tau);
    cudaFree(c->d_bt_acc);
    cudaFree(c->d_hess);
    cudaFree(c->d_tol_part);
    cudaFree(c->d_tol_count);
    if (c->h_stop) cudaFreeHost(c->h_stop);
    for (cudaEvent_t e : c->tol_ev)
        if (e) cudaEventDestroy(e);
    if (c->side_fork) cudaEventDestroy(c->side_fork);
    if (c->side_join) cudaEventDestroy(c->side_join);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
    delete c;
}

foe_status foe_step_size(const foe_ctx *ctx, foe_bc bc, float gamma, float *tau_out, double *lipschitz_out)
{
    if (!ctx || (bc != FOE_BC_SYMMETRIC && bc != FOE_BC_ZERO) || !(gamma >= 0.0f && gamma < 1.0f)) return FOE_EINVAL;
    if (tau_out) *tau_out = default_tau(ctx->symbol_max, bc, gamma);
    if (lipschitz_out) *lipschitz_out = 2.0 * kappa(bc) * ctx->symbol_max;
    return FOE_OK;
}

// iPiano (Sec. 2.3, Eq. iPianoupdate) with Lipschitz backtracking on the smooth part F = E_FoE (the prior; the
// data term is the proximal part).  A trial with constant L uses tau = 2 (1 - gamma) / (L + 2 c2), c2 = 1e-3, and is
// accepted when F(u+) <= F(u) + <grad F(u), u+ - u> + L / 2 ||u+ - u||^2 (FP64 reductions on the GPU, decided on
// the host); otherwise L doubles and the trial is repeated from the same u.  After an accepted step L is divided
// by 1.5.  L starts at the context's certified bound (or at the L implied by opts->tau when it is set).  Every
// trial is one fused FP32 step launch, so rejected trials restore u_lo and delta from a snapshot.
// Owns the graphs of a backtracking solve (destroyed on every return path).
struct BtGraphs {
    cudaGraph_t g[2] = {nullptr, nullptr};
    cudaGraphExec_t x[2] = {nullptr, nullptr};
    ~BtGraphs()
    {
        for (int i = 0; i < 2; ++i) {
            if (x[i]) cudaGraphExecDestroy(x[i]);
            if (g[i]) cudaGraphDestroy(g[i]);
        }
    }
};

// FOE_STEP_BACKTRACK (FP32): every accept / reject decision is taken on the device.  An iteration is one launch of
// a CUDA graph: the prior gradient at u^n and a snapshot of u_lo and delta, then a conditional WHILE node whose body
// is one trial (restore the snapshot, the step with the trial's constants read from device memory, the FP64
// reductions, F(u+), k_bt_decide, which sets the loop condition).  Two graphs alternate the iterate planes.  The
// host queues all iterations without waiting and reads the state and the trial log once at the end.
static foe_status denoise_backtrack(foe_ctx *c, const float *y, float *x, int H, int W, int ld, int model,
                                    const foe_solve_opts *o, cudaStream_t s, foe_report *rep)
{
    if (o->prec != FOE_PREC_FP32) {
        set_err(c, "FOE_STEP_BACKTRACK needs FOE_PREC_FP32");
        return FOE_EUNSUPPORTED;
    }
    {
        // the iterations are graphs with conditional nodes, which cannot become part of another graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        FOE_CUDA(c, cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            set_err(c, "FOE_STEP_BACKTRACK cannot run on a stream under capture");
            return FOE_EUNSUPPORTED;
        }
    }
    foe_status st;
    const size_t plane = (size_t)H * ld;
    if ((st = ensure_ws(c, 8 * plane * sizeof(float))) != FOE_OK) return st;
    Slot sl = carve((float *)c->ws, plane);
    float *gpl = (float *)c->ws + 5 * plane, *snap_lo = gpl + plane, *snap_dl = snap_lo + plane;
    const double c2 = 1e-3, gam = o->gamma;
    const bool tol_on = o->tol > 0.0f;
    int tiles = 0;
    // launch arguments for one image: read u0 (parity 0), write u1; prior_only for the gradient / energy
    auto set_args = [&](float *u0, float *u1, int prior_only) {
        args_begin(c, o->bc);
        ImgDesc d{};
        d.u_hi[0] = u0;
        d.u_hi[1] = u1;
        d.u_lo = sl.ul;
        d.delta = sl.delta;
        d.d = sl.d;
        d.out = gpl;
        d.H = H;
        d.W = W;
        d.ld = ld;
        d.model = model;
        d.sc = step_consts(0.0f, o->gamma, o->lambda);  // the step launches read the trial's constants on the device
        d.stop = tol_on ? c->d_stop : nullptr;
        args_add(c, FOE_PREC_FP32, d);
        c->args.prior_only = prior_only;
        tiles = c->args.tile_prefix[1];
    };
    set_args(sl.uh0, nullptr, 1);
    const int nb = foe::dot2_blocks(H);
    if ((st = ensure_partials(c, tiles + 2 * nb + 4)) != FOE_OK) return st;
    double *dot_part = c->d_partials + tiles, *outs = dot_part + 2 * nb;  // outs: <g, du>, |du|^2, F(u+)
    const int cap = std::max(1, std::min(o->iters * 61, 1 << 20));     // trial log entries kept
    if ((st = ensure_bt(c, cap)) != FOE_OK) return st;
    auto prior_energy = [&](float *u, double *dst, cudaStream_t q) -> foe_status {
        set_args(u, nullptr, 1);
        c->args.partials = c->d_partials;
        foe_status e = launch(c, FOE_PREC_FP32, foe::kEnergy, q);
        if (e != FOE_OK) return e;
        FOE_CUDA(c, foe::launch_reduce(c->d_partials, tiles, dst, q));
        return FOE_OK;
    };

    FOE_CUDA(c, foe::launch_init(y, H, W, ld, ld, model, o->zero_c, sl.d, sl.uh0, sl.ul, sl.delta, s));
    const double L0 = o->tau > 0.0f ? 2.0 * (1.0 - gam) / (double)o->tau - 2.0 * c2 : 2.0 * kappa(o->bc) * c->symbol_max;
    if (!(L0 > 0.0)) {
        set_err(c, "opts->tau implies a non-positive Lipschitz estimate");
        return FOE_EINVAL;
    }
    if (tol_on) FOE_CUDA(c, cudaMemsetAsync(c->d_stop, 0, sizeof(int), s));
    if ((st = prior_energy(sl.uh0, outs + 2, s)) != FOE_OK) return st;
    FOE_CUDA(c, foe::launch_bt_init(c->d_bt, outs + 2, L0, gam, 2.0 * c2, o->gamma, o->lambda, cap, s));

    // the two iteration graphs, captured on the context's side stream (capture only: they run on s)
    BtGraphs G;
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    FOE_CUDA(c, cudaStreamIsCapturing(c->side_stream, &cap_status));
    if (cap_status != cudaStreamCaptureStatusNone) {
        set_err(c, "FOE_STEP_BACKTRACK: the context's side stream is being captured");
        return FOE_EINVAL;
    }
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    for (int par = 0; par < 2; ++par) {
        float *cur = par ? sl.uh1 : sl.uh0, *nxt = par ? sl.uh0 : sl.uh1;
        FOE_CUDA(c, cudaGraphCreate(&G.g[par], 0));
        // gradient at u^n and the snapshot
        FOE_CUDA(c, cudaStreamBeginCaptureToGraph(c->side_stream, G.g[par], nullptr, nullptr, 0, mode));
        set_args(cur, nullptr, 1);
        st = launch(c, FOE_PREC_FP32, foe::kGrad, c->side_stream);
        cudaError_t ce = cudaSuccess;
        if (st == FOE_OK) ce = cudaMemcpyAsync(snap_lo, sl.ul, plane * sizeof(float), cudaMemcpyDeviceToDevice, c->side_stream);
        if (st == FOE_OK && ce == cudaSuccess)
            ce = cudaMemcpyAsync(snap_dl, sl.delta, plane * sizeof(float), cudaMemcpyDeviceToDevice, c->side_stream);
        cudaGraph_t got = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->side_stream, &got);
        if (st != FOE_OK) return st;
        FOE_CUDA(c, ce);
        FOE_CUDA(c, ee);
        size_t npre = 0;
        FOE_CUDA(c, cudaGraphGetNodes(G.g[par], nullptr, &npre));
        std::vector<cudaGraphNode_t> pre(npre);
        FOE_CUDA(c, cudaGraphGetNodes(G.g[par], pre.data(), &npre));
        // the trial loop
        cudaGraphConditionalHandle h;
        FOE_CUDA(c, cudaGraphConditionalHandleCreate(&h, G.g[par], 1u, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop;
        FOE_CUDA(c, cudaGraphAddNode(&loop, G.g[par], pre.data(), nullptr, npre, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        FOE_CUDA(c, cudaStreamBeginCaptureToGraph(c->side_stream, body, nullptr, nullptr, 0, mode));
        ce = cudaMemcpyAsync(sl.ul, snap_lo, plane * sizeof(float), cudaMemcpyDeviceToDevice, c->side_stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sl.delta, snap_dl, plane * sizeof(float), cudaMemcpyDeviceToDevice, c->side_stream);
        if (ce == cudaSuccess) {
            set_args(cur, nxt, 0);
            c->args.sc_dev = &c->d_bt->sc;
            st = launch(c, FOE_PREC_FP32, foe::kStep, c->side_stream);  // u+ (delta = u+ - u^n)
            c->args.sc_dev = nullptr;
        }
        if (ce == cudaSuccess && st == FOE_OK) ce = foe::launch_dot2(gpl, sl.delta, H, W, ld, dot_part, outs, c->side_stream);
        if (ce == cudaSuccess && st == FOE_OK) st = prior_energy(nxt, outs + 2, c->side_stream);
        if (ce == cudaSuccess && st == FOE_OK)
            ce = foe::launch_bt_decide(h, c->d_bt, outs, c->d_bt_tau, c->d_bt_acc, tol_on ? c->d_stop : nullptr,
                                       c->side_stream);
        got = nullptr;
        const cudaError_t eb = cudaStreamEndCapture(c->side_stream, &got);
        if (st != FOE_OK) return st;
        FOE_CUDA(c, ce);
        FOE_CUDA(c, eb);
        FOE_CUDA(c, cudaGraphInstantiate(&G.x[par], G.g[par], 0));
    }

    // the iterations: queued without waiting; the stopping rule is checked between them
    ImgDesc td{};
    td.u_hi[0] = sl.uh0;
    td.u_hi[1] = sl.uh1;
    td.u_lo = sl.ul;
    td.delta = sl.delta;
    td.H = H;
    td.W = W;
    td.ld = ld;
    td.stop = c->d_stop;
    for (int n = 0; n < o->iters; ++n) {
        FOE_CUDA(c, cudaGraphLaunch(G.x[n & 1], s));
        if (tol_on && (n + 1) % o->tol_every == 0) {
            foe::TolArgs t;
            t.nimg = 1;
            t.n = n + 1;
            t.tol = (double)o->tol;
            t.partials = c->d_tol_part;
            t.count = c->d_tol_count;
            t.img[0] = tol_img(td, n + 1);
            FOE_CUDA(c, foe::launch_tol_check(t, s));
        }
    }
    foe::BtState bs{};
    int stop = 0;
    FOE_CUDA(c, cudaMemcpyAsync(&bs, c->d_bt, sizeof(bs), cudaMemcpyDeviceToHost, s));
    if (tol_on) FOE_CUDA(c, cudaMemcpyAsync(&stop, c->d_stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    FOE_CUDA(c, cudaStreamSynchronize(s));
    const int nlog = std::min(bs.nlog, cap);
    c->bt_tau.resize(nlog);
    c->bt_accepted.resize(nlog);
    if (nlog > 0) {
        FOE_CUDA(c, cudaMemcpy(c->bt_tau.data(), c->d_bt_tau, sizeof(float) * nlog, cudaMemcpyDeviceToHost));
        FOE_CUDA(c, cudaMemcpy(c->bt_accepted.data(), c->d_bt_acc, nlog, cudaMemcpyDeviceToHost));
    }
    if (bs.status == foe::kBtNonFinite) {
        set_err(c, "non-finite energy or step during backtracking");
        return FOE_ENONFINITE;
    }
    if (bs.status == foe::kBtNoStep) {
        set_err(c, "backtracking did not find an accepted step within 61 trials");
        return FOE_ENONFINITE;
    }
    const int done = stop ? stop : o->iters;
    const int word = tol_on ? 0 : -1;
    note_solve(c, 1, &o->iters, &word);
    const float *uf = (o->iters & 1) ? sl.uh1 : sl.uh0, *ua = (o->iters & 1) ? sl.uh0 : sl.uh1;
    if (rep) FOE_CUDA(c, cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), s));
    FOE_CUDA(c, foe::launch_output(uf, sl.ul, H, W, ld, ld, model, x, rep ? c->d_nonfinite : nullptr, s, nullptr, ua,
                                   o->iters, tol_on ? c->d_stop : nullptr));
    if (rep) {
        int dev_status = 0, nonfinite = 0;
        FOE_CUDA(c, cudaMemcpyAsync(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaMemcpyAsync(&nonfinite, c->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
        rep->nonfinite = nonfinite;
        rep->iters_done = done;
        rep->model_used = model;
        rep->tau_used = bs.tau_last;
        rep->status = dev_status ? (foe_status)dev_status : FOE_OK;
        rep->backtracks = bs.rejected;
        rep->lipschitz_final = bs.L;
        if (nonfinite) {
            set_err(c, "%d non-finite output pixels", nonfinite);
            return FOE_ENONFINITE;
        }
    }
    return FOE_OK;
}

foe_status foe_denoise(foe_ctx *c, const float *y, float *x, int H, int W, int ld, float peak,
                       const foe_solve_opts *o, void *stream, foe_report *rep)
{
    NvtxRange nvtx_range("foe_denoise");
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
    if (o->step == FOE_STEP_BACKTRACK) return denoise_backtrack(c, y, x, H, W, ld, model, o, s, rep);
    const float tau = o->tau > 0.0f ? o->tau : default_tau(c->symbol_max, o->bc, o->gamma);
    const size_t plane = (size_t)H * ld;
    if ((st = ensure_ws(c, 5 * plane * sizeof(float))) != FOE_OK) return st;
    Slot sl = carve((float *)c->ws, plane);
    FOE_CUDA(c, foe::launch_init(y, H, W, ld, ld, model, o->zero_c, sl.d, sl.uh0, lo_plane(o->prec, sl.ul), sl.delta, s));
    args_begin(c, o->bc);
    ImgDesc d{};
    d.u_hi[0] = sl.uh0;
    d.u_hi[1] = sl.uh1;
    d.u_lo = lo_plane(o->prec, sl.ul);
    d.delta = sl.delta;
    d.d = sl.d;
    d.out = nullptr;
    d.H = H;
    d.W = W;
    d.ld = ld;
    d.model = model;
    d.sc = step_consts(tau, o->gamma, o->lambda);
    const bool tol_on = o->tol > 0.0f;
    if (tol_on) {
        FOE_CUDA(c, cudaMemsetAsync(c->d_stop, 0, sizeof(int), s));
        d.stop = c->d_stop;
    }
    args_add(c, o->prec, d);
    // the host follows the stopping word one check interval behind the device, unless the stream is captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (tol_on) FOE_CUDA(c, cudaStreamIsCapturing(s, &cap));
    const bool follow = tol_on && cap == cudaStreamCaptureStatusNone;
    cudaEvent_t ev[2];
    if ((st = prof_begin(c, s, ev)) != FOE_OK) return st;
    int launched = 0, checks = 0;
    for (int n = 0; n < o->iters; ++n) {
        c->args.parity = n & 1;
        if ((st = launch(c, o->prec, foe::kStep, s)) != FOE_OK) return st;
        ++launched;
        if (!tol_on || (n + 1) % o->tol_every != 0) continue;
        if ((st = tol_check(c, 1, n + 1, o->tol, s)) != FOE_OK) return st;
        if (!follow) continue;
        const int slot = checks++ & 1;
        FOE_CUDA(c, cudaMemcpyAsync(c->h_stop + slot, c->d_stop, sizeof(int), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaEventRecord(c->tol_ev[slot], s));
        if (checks > 1) {
            // the previous check's word (this interval's launches keep the device busy meanwhile)
            FOE_CUDA(c, cudaEventSynchronize(c->tol_ev[slot ^ 1]));
            if (c->h_stop[slot ^ 1] != 0) break;
        }
    }
    if ((st = prof_end(c, s, ev, launched, (double)H * W * launched)) != FOE_OK) return st;
    const int word = tol_on ? 0 : -1;
    note_solve(c, 1, &o->iters, &word);
    const float *uf = (o->iters & 1) ? sl.uh1 : sl.uh0, *ua = (o->iters & 1) ? sl.uh0 : sl.uh1;
    if (rep) FOE_CUDA(c, cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), s));
    FOE_CUDA(c, foe::launch_output(uf, lo_plane(o->prec, sl.ul), H, W, ld, ld, model, x, rep ? c->d_nonfinite : nullptr, s,
                                   nullptr, ua, o->iters, tol_on ? c->d_stop : nullptr));
    if (rep) {
        int dev_status = 0, nonfinite = 0, stop = 0;
        FOE_CUDA(c, cudaMemcpyAsync(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaMemcpyAsync(&nonfinite, c->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (tol_on) FOE_CUDA(c, cudaMemcpyAsync(&stop, c->d_stop, sizeof(int), cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
        rep->nonfinite = nonfinite;
        rep->iters_done = stop ? stop : o->iters;
        rep->model_used = model;
        rep->tau_used = tau;
        rep->status = dev_status ? (foe_status)dev_status : FOE_OK;
        rep->backtracks = 0;
        rep->lipschitz_final = 2.0 * (1.0 - (double)o->gamma) / (double)tau - 2e-3;
        if (dev_status) {
            FOE_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_err(c, "a device-side wait expired during the solve");
            return (foe_status)dev_status;
        }
        if (nonfinite) {
            set_err(c, "%d non-finite output pixels", nonfinite);
            return FOE_ENONFINITE;
        }
    }
    return FOE_OK;
}

foe_status foe_device_status(foe_ctx *c, void *stream)
{
    if (!c) return FOE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev_status = 0;
    FOE_CUDA(c, cudaMemcpyAsync(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    FOE_CUDA(c, cudaStreamSynchronize(s));
    if (!dev_status) return FOE_OK;
    FOE_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    FOE_CUDA(c, cudaStreamSynchronize(s));
    set_err(c, "a device-side wait expired");
    return (foe_status)dev_status;
}

foe_status foe_debug_withhold_arrival(foe_ctx *c)
{
    if (!c) return FOE_EINVAL;
    c->withhold_arrival = 1;
    return FOE_OK;
}

foe_status foe_denoise_binned(foe_ctx *c, const float *y, float *x, int H, int W, int ld, float peak,
                              const foe_solve_opts *o, void *stream, foe_report *rep)
{
    NvtxRange nvtx_range("foe_denoise_binned");
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts(c, o)) != FOE_OK) return st;
    if ((st = check_image(c, y, H, W, ld, "y")) != FOE_OK) return st;
    if ((st = check_image(c, x, H, W, ld, "x")) != FOE_OK) return st;
    const int Hb = (H + 2) / 3, Wb = (W + 2) / 3, ldb = (Wb + 3) / 4 * 4;
    if (Hb < 7 || Wb < 7) {
        set_err(c, "foe_denoise_binned: the binned image must be at least 7 x 7 (H, W >= 19; got %d x %d)", H, W);
        return FOE_EINVAL;
    }
    if (o->model == FOE_MODEL_AUTO && !(peak > 0.0f && std::isfinite(peak))) {
        set_err(c, "peak must be > 0 for FOE_MODEL_AUTO");
        return FOE_EINVAL;
    }
    const size_t plane = (size_t)Hb * ldb;
    if ((st = ensure_bin(c, 2 * plane * sizeof(float))) != FOE_OK) return st;
    float *yb = c->d_bin, *xb = c->d_bin + plane;
    cudaStream_t s = (cudaStream_t)stream;
    FOE_CUDA(c, foe::launch_bin3(y, H, W, ld, yb, ldb, s));
    if ((st = foe_denoise(c, yb, xb, Hb, Wb, ldb, 9.0f * peak, o, stream, rep)) != FOE_OK) return st;
    FOE_CUDA(c, foe::launch_upscale3(xb, ldb, x, H, W, ld, s));
    return FOE_OK;
}

foe_status foe_denoise_batch(foe_ctx *c, const foe_image_desc *descs, int n, const foe_solve_opts *o, void *stream)
{
    NvtxRange nvtx_range("foe_denoise_batch");
    if (!c) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts_fixed(c, o, "foe_denoise_batch")) != FOE_OK) return st;
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
        if (d.use_model != 0 && d.use_model != 1) { set_err(c, "desc.use_model must be 0 or 1"); return FOE_EINVAL; }
        const int m = d.use_model ? d.model : o->model;
        if (m < FOE_MODEL_DIRECT || m > FOE_MODEL_AUTO) { set_err(c, "desc.model: bad model"); return FOE_EINVAL; }
        if (m == FOE_MODEL_AUTO && !(d.peak > 0.0f && std::isfinite(d.peak))) {
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
    {
        // image order[j] of the call holds stopping word j
        std::vector<int> budget(n), word(n, -1);
        for (int j = 0; j < n; ++j) {
            budget[order[j]] = descs[order[j]].iters;
            if (o->tol > 0.0f) word[order[j]] = j;
        }
        note_solve(c, n, budget.data(), word.data());
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FOE_CUDA(c, cudaStreamIsCapturing(s, &cap));
    const bool graph = o->use_graph && s != nullptr && cap == cudaStreamCaptureStatusNone;
    if (!graph) return enqueue_batch(c, descs, n, o, s, order, max_iters, !cap);
    // capture the whole solve, then replay it (updating the cached executable graph when possible)
    cudaEvent_t ev[2];
    if ((st = prof_begin(c, s, ev)) != FOE_OK) return st;
    FOE_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    st = enqueue_batch(c, descs, n, o, s, order, max_iters, false);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st != FOE_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    FOE_CUDA(c, ec);
    bool updated = false;
    if (c->batch_exec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(c->batch_exec, g, &info) == cudaSuccess;
        if (!updated) {
            (void)cudaGetLastError();
            cudaGraphExecDestroy(c->batch_exec);
            c->batch_exec = nullptr;
        }
    }
    if (!updated) {
        const cudaError_t ei = cudaGraphInstantiate(&c->batch_exec, g, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(g);
            FOE_CUDA(c, ei);
        }
    }
    cudaGraphDestroy(g);
    FOE_CUDA(c, cudaGraphLaunch(c->batch_exec, s));
    double pix = 0.0;
    for (int j = 0; j < n; ++j) pix += (double)descs[j].H * descs[j].W * descs[j].iters;
    return prof_end(c, s, ev, max_iters, pix);
}

foe_status foe_iters_done(foe_ctx *c, int *out, int n, void *stream)
{
    if (!c) return FOE_EINVAL;
    if (!out || n < 1 || (size_t)n != c->last_budget.size()) {
        set_err(c, "foe_iters_done: n must equal the image count of the last solve (%zu)", c->last_budget.size());
        return FOE_EINVAL;
    }
    int words = 0;
    for (int w : c->last_word) words = std::max(words, w + 1);
    std::vector<int> stop(std::max(words, 1), 0);
    if (words > 0) {
        cudaStream_t s = (cudaStream_t)stream;
        FOE_CUDA(c, cudaMemcpyAsync(stop.data(), c->d_stop, sizeof(int) * words, cudaMemcpyDeviceToHost, s));
        FOE_CUDA(c, cudaStreamSynchronize(s));
    }
    for (int i = 0; i < n; ++i) {
        const int w = c->last_word[i];
        out[i] = (w >= 0 && stop[w] != 0) ? stop[w] : c->last_budget[i];
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
    if (prec != FOE_PREC_FP32 && prec != FOE_PREC_BF16 && prec != FOE_PREC_TF32) {
        set_err(c, "bad precision");
        return FOE_EINVAL;
    }
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
    if (prec != FOE_PREC_FP32 && prec != FOE_PREC_BF16 && prec != FOE_PREC_TF32) {
        set_err(c, "bad precision");
        return FOE_EINVAL;
    }
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
    if ((st = check_opts_fixed(c, o, "foe_denoise_static")) != FOE_OK) return st;
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
    FOE_CUDA(c, foe::launch_init(y, H, W, ld, ld, model, o->zero_c, sl.d, sl.uh0, lo_plane(o->prec, sl.ul), sl.delta, s));
    args_begin(c, o->bc);
    ImgDesc d{};
    d.u_hi[0] = sl.uh0;
    d.u_hi[1] = sl.uh1;
    d.u_lo = lo_plane(o->prec, sl.ul);
    d.delta = sl.delta;
    d.d = sl.d;
    d.H = H;
    d.W = W;
    d.ld = ld;
    d.model = model;
    d.sc = step_consts(tau, o->gamma, o->lambda);
    const bool tol_on = o->tol > 0.0f;
    if (tol_on) {
        FOE_CUDA(c, cudaMemsetAsync(c->d_stop, 0, sizeof(int), s));
        d.stop = c->d_stop;
    }
    args_add(c, o->prec, d);
    for (int n = 0; n < o->iters; ++n) {
        c->args.parity = n & 1;
        if ((st = launch(c, o->prec, foe::kStep, s)) != FOE_OK) return st;
        if (tol_on && (n + 1) % o->tol_every == 0 && (st = tol_check(c, 1, n + 1, o->tol, s)) != FOE_OK) return st;
    }
    const int word = tol_on ? 0 : -1;
    note_solve(c, 1, &o->iters, &word);
    const float *uf = (o->iters & 1) ? sl.uh1 : sl.uh0, *ua = (o->iters & 1) ? sl.uh0 : sl.uh1;
    // no status is read back here (nothing is synchronised): on the tensor-core paths, whose step launches do
    // nothing while the context's device status is set, an expired device wait shows as a NaN output
    const int *guard = o->prec == FOE_PREC_FP32 ? nullptr : c->d_status;
    FOE_CUDA(c, foe::launch_output(uf, lo_plane(o->prec, sl.ul), H, W, ld, ld, model, x, nullptr, s, guard, ua, o->iters,
                                   tol_on ? c->d_stop : nullptr));
    return FOE_OK;
}


extern "C" int foe_step_log(const foe_ctx *c, float *tau, unsigned char *accepted, int max_n)
{
    if (!c || max_n < 0 || (max_n > 0 && (!tau || !accepted))) return -1;
    const int n = (int)c->bt_tau.size();
    for (int i = 0; i < n && i < max_n; ++i) {
        tau[i] = c->bt_tau[i];
        accepted[i] = c->bt_accepted[i];
    }
    return n;
}
