// Continuous-batching denoise server over the FoE step kernels.
//
// Requests (one noisy image each, any size, its own peak and iteration budget) wait in a FIFO until
// both a slot (at most max_active, the batch capacity of one launch) and device memory for their state
// (five planes of H x ld floats, taken from one arena allocated at creation within the HBM budget)
// are free.  Each tick admits what fits, uploads and initialises the new requests, then advances every
// admitted request by up to iters_per_tick iterations with one step launch per iteration over the
// tiles of all of them (captured as a CUDA graph when enabled), and finishes the requests whose budget
// is spent: output map, copy back, memory returned to the arena.  Requests that arrive while others
// are iterating join at the next tick: that is the continuous batching.  Every request's iterate state
// stays on the device from admission to completion.
//
// Ticks are pipelined: tick k queues its work behind tick k - 1's on the server's stream and only then waits
// for tick k - 1 (an event), so the host's admission, uploads and graph update for tick k overlap tick k - 1 on
// the GPU and the GPU does not idle between ticks.  A request that finishes in tick k is reported (and its memory
// returned) by tick k + 1; a tick with nothing left to admit or iterate only completes the previous one.
#include <deque>
#include <map>

#include "foe_internal.h"

namespace {

// First-fit allocator over one device allocation; blocks are 256-byte aligned; freed blocks coalesce.
class Arena {
public:
    void reset(size_t bytes)
    {
        free_.clear();
        free_[0] = bytes;
        cap_ = bytes;
        used_ = peak_ = 0;
    }

    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t o = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[o + bytes] = rem;
            *off = o;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }

    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
};

struct Request {
    long long id = 0;
    int H = 0, W = 0, ld = 0;
    int iters = 0, done = 0, model = 0;
    const float *y_host = nullptr;
    float *x_host = nullptr;
    int y_pitch = 0, x_pitch = 0;
    size_t off = 0, bytes = 0;
    foe::StepConsts sc{};
};

}  // namespace

struct foe_server {
    foe_ctx *ctx = nullptr;
    foe_server_config cfg{};
    float tau = 0.0f;
    char *arena_base = nullptr;
    Arena arena;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};  // tick k uses exec[k & 1]: the one being updated is idle
    cudaEvent_t done_ev[2] = {nullptr, nullptr};   // end of tick k's device work: done_ev[k & 1]
    int *h_status = nullptr;                       // pinned [2]: the context's device status after tick k
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::vector<Request *> finishing;              // finished in the last queued tick, not yet complete
    bool pending = false;                          // a queued tick not yet waited for
    foe_status failed = FOE_OK;                    // sticky: a device wait expired in some tick
    std::vector<long long> completed_ids;
    long long next_id = 1, completed = 0, ticks = 0, launches = 0;
    double pixel_iters = 0.0;
};

namespace {

Slot request_slot(foe_server *sv, const Request *r)
{
    return carve(reinterpret_cast<float *>(sv->arena_base + r->off), (size_t)r->H * r->ld);
}

// Enqueues the step launches of one tick on sv->stream.
foe_status enqueue_iterations(foe_server *sv)
{
    foe_ctx *c = sv->ctx;
    const foe_solve_opts &o = sv->cfg.opts;
    for (int it = 0; it < sv->cfg.iters_per_tick; ++it) {
        args_begin(c, o.bc);
        double pix = 0.0;
        for (Request *r : sv->active) {
            if (r->done + it >= r->iters) continue;
            const Slot sl = request_slot(sv, r);
            const bool odd = ((r->done + it) & 1) != 0;
            ImgDesc d{};
            d.u_hi[0] = odd ? sl.uh1 : sl.uh0;  // this request's own parity: read buffer first
            d.u_hi[1] = odd ? sl.uh0 : sl.uh1;
            d.u_lo = lo_plane(o.prec, sl.ul);
            d.delta = sl.delta;
            d.d = sl.d;
            d.H = r->H;
            d.W = r->W;
            d.ld = r->ld;
            d.model = r->model;
            d.sc = r->sc;
            args_add(c, o.prec, d);
            pix += (double)r->H * r->W;
        }
        if (c->args.nimg == 0) break;
        c->args.parity = 0;
        foe_status st = launch(c, o.prec, foe::kStep, sv->stream);
        if (st != FOE_OK) return st;
        sv->launches++;
        sv->pixel_iters += pix;
    }
    return FOE_OK;
}

}  // namespace

extern "C" {

foe_status foe_server_create(foe_ctx *ctx, const foe_server_config *cfg, foe_server **out)
{
    if (!out) return FOE_EINVAL;
    *out = nullptr;
    if (!ctx || !cfg) return FOE_EINVAL;
    foe_status st;
    if ((st = check_opts_fixed(ctx, &cfg->opts, "foe_server_create")) != FOE_OK) return st;
    if ((st = check_no_tol(ctx, &cfg->opts, "foe_server_create")) != FOE_OK) return st;
    if (cfg->max_active < 1 || cfg->max_active > foe::kMaxBatch || cfg->iters_per_tick < 1 ||
        cfg->hbm_budget_bytes < ((size_t)1 << 20)) {
        set_err(ctx, "server config: need 1 <= max_active <= %d, iters_per_tick >= 1, budget >= 1 MiB",
                foe::kMaxBatch);
        return FOE_EINVAL;
    }
    foe_server *sv = new (std::nothrow) foe_server();
    if (!sv) return FOE_ENOMEM;
    sv->ctx = ctx;
    sv->cfg = *cfg;
    sv->tau = cfg->opts.tau > 0.0f ? cfg->opts.tau : default_tau(ctx->symbol_max, cfg->opts.bc, cfg->opts.gamma);
    cudaError_t e;
    if ((e = cudaMalloc(&sv->arena_base, cfg->hbm_budget_bytes)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sv->done_ev[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sv->done_ev[1], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaHostAlloc(&sv->h_status, 2 * sizeof(int), cudaHostAllocDefault)) != cudaSuccess) {
        set_err(ctx, "server create: %s", cudaGetErrorString(e));
        foe_server_destroy(sv);
        return e == cudaErrorMemoryAllocation ? FOE_ENOMEM : FOE_ECUDA;
    }
    sv->arena.reset(cfg->hbm_budget_bytes);
    *out = sv;
    return FOE_OK;
}

void foe_server_destroy(foe_server *sv)
{
    if (!sv) return;
    if (sv->stream) cudaStreamSynchronize(sv->stream);
    for (cudaGraphExec_t x : sv->exec)
        if (x) cudaGraphExecDestroy(x);
    for (cudaEvent_t e : sv->done_ev)
        if (e) cudaEventDestroy(e);
    if (sv->h_status) cudaFreeHost(sv->h_status);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    cudaFree(sv->arena_base);
    for (Request *r : sv->queue) delete r;
    for (Request *r : sv->active) delete r;
    for (Request *r : sv->finishing) delete r;
    delete sv;
}

foe_status foe_server_submit(foe_server *sv, const float *y_host, int y_pitch, float *x_host, int x_pitch, int H,
                             int W, float peak, int iters, long long *id_out)
{
    if (!sv) return FOE_EINVAL;
    foe_ctx *c = sv->ctx;
    if (!y_host || !x_host || !id_out) { set_err(c, "submit: NULL pointer"); return FOE_EINVAL; }
    if (H < 7 || W < 7 || y_pitch < W || x_pitch < W || iters < 0) {
        set_err(c, "submit: need H, W >= 7, pitches >= W, iters >= 0");
        return FOE_EINVAL;
    }
    if (sv->cfg.opts.model == FOE_MODEL_AUTO && !(peak > 0.0f && std::isfinite(peak))) {
        set_err(c, "submit: peak must be > 0 for FOE_MODEL_AUTO");
        return FOE_EINVAL;
    }
    Request *r = new (std::nothrow) Request();
    if (!r) return FOE_ENOMEM;
    r->id = sv->next_id++;
    r->H = H;
    r->W = W;
    r->ld = (W + 3) / 4 * 4;
    r->iters = iters;
    r->model = resolve_model(sv->cfg.opts.model, peak);
    r->y_host = y_host;
    r->x_host = x_host;
    r->y_pitch = y_pitch;
    r->x_pitch = x_pitch;
    r->bytes = 5 * (size_t)H * r->ld * sizeof(float);
    r->sc = step_consts(sv->tau, sv->cfg.opts.gamma, sv->cfg.opts.lambda);
    if (Arena::round(r->bytes) > sv->arena.capacity()) {
        set_err(c, "submit: request needs %zu bytes, more than the whole budget of %zu", r->bytes, sv->arena.capacity());
        delete r;
        return FOE_ENOMEM;
    }
    sv->queue.push_back(r);
    *id_out = r->id;
    return FOE_OK;
}

// Waits for the queued tick, then completes its finished requests (memory back to the arena, ids to poll).
static foe_status complete_pending(foe_server *sv, int *n_completed)
{
    foe_ctx *c = sv->ctx;
    if (!sv->pending) return FOE_OK;
    const int slot = (int)((sv->ticks - 1) & 1);
    FOE_CUDA(c, cudaEventSynchronize(sv->done_ev[slot]));
    sv->pending = false;
    if (sv->h_status[slot] != 0) {
        // the tick's results are not valid: the server stops here (every later call returns this status); its
        // requests stay owned by it until foe_server_destroy, and the context's status is left for
        // foe_device_status to read and clear
        sv->failed = (foe_status)sv->h_status[slot];
        set_err(c, "a device-side wait expired during a server tick; the server has stopped");
        return sv->failed;
    }
    for (Request *r : sv->finishing) {
        sv->arena.release(r->off, r->bytes);
        sv->completed_ids.push_back(r->id);
        sv->completed++;
        delete r;
    }
    if (n_completed) *n_completed = (int)sv->finishing.size();
    sv->finishing.clear();
    return FOE_OK;
}

foe_status foe_server_tick(foe_server *sv, int *n_completed)
{
    NvtxRange nvtx_range("foe_server_tick");
    if (!sv) return FOE_EINVAL;
    foe_ctx *c = sv->ctx;
    const foe_solve_opts &o = sv->cfg.opts;
    foe_status st;
    if (n_completed) *n_completed = 0;
    if (sv->failed != FOE_OK) {
        set_err(c, "the server stopped after an expired device-side wait; destroy it");
        return sv->failed;
    }
    if (sv->queue.empty() && sv->active.empty()) return complete_pending(sv, n_completed);
    // 1. admission: FIFO order, while a slot and arena memory are free (the memory of the requests that finish
    // in the queued tick comes back when it completes, below)
    while (!sv->queue.empty() && (int)sv->active.size() < sv->cfg.max_active) {
        Request *r = sv->queue.front();
        size_t off;
        if (!sv->arena.alloc(r->bytes, &off)) break;
        r->off = off;
        sv->queue.pop_front();
        sv->active.push_back(r);
        const Slot sl = request_slot(sv, r);
        FOE_CUDA(c, cudaMemcpy2DAsync(sl.d, r->ld * sizeof(float), r->y_host, r->y_pitch * sizeof(float),
                                      r->W * sizeof(float), r->H, cudaMemcpyHostToDevice, sv->stream));
        FOE_CUDA(c, foe::launch_init(sl.d, r->H, r->W, r->ld, r->ld, r->model, o.zero_c, sl.d, sl.uh0, lo_plane(o.prec, sl.ul), sl.delta,
                                     sv->stream));
    }
    if (sv->active.empty()) {
        // nothing fits until the queued tick's memory comes back (with nothing queued on the device the whole
        // arena is free and the first request fits, so this retries once)
        if (!sv->pending) {
            set_err(c, "server: no request fits the free arena");
            return FOE_ENOMEM;
        }
        if ((st = complete_pending(sv, n_completed)) != FOE_OK) return st;
        int more = 0;
        st = sv->queue.empty() ? FOE_OK : foe_server_tick(sv, &more);
        if (n_completed) *n_completed += more;
        return st;
    }
    // 2. iterations of every admitted request
    const int slot = (int)(sv->ticks & 1);
    if (sv->cfg.use_graphs) {
        FOE_CUDA(c, cudaStreamBeginCapture(sv->stream, cudaStreamCaptureModeThreadLocal));
        st = enqueue_iterations(sv);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(sv->stream, &graph);
        if (st != FOE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        FOE_CUDA(c, ec);
        // exec[slot] was last launched two ticks ago, which has completed
        cudaGraphExec_t &exec = sv->exec[slot];
        bool updated = false;
        if (exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess;
            if (!updated) {
                (void)cudaGetLastError();
                cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
        }
        if (!updated) {
            const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(graph);
                FOE_CUDA(c, ei);
            }
        }
        cudaGraphDestroy(graph);
        FOE_CUDA(c, cudaGraphLaunch(exec, sv->stream));
    } else if ((st = enqueue_iterations(sv)) != FOE_OK) {
        return st;
    }
    // 3. requests whose budget is spent: output map into the delta plane, copy back
    std::vector<Request *> finished, still;
    for (Request *r : sv->active) {
        r->done = std::min(r->iters, r->done + sv->cfg.iters_per_tick);
        if (r->done < r->iters) {
            still.push_back(r);
            continue;
        }
        const Slot sl = request_slot(sv, r);
        const float *uf = (r->iters & 1) ? sl.uh1 : sl.uh0;
        FOE_CUDA(c, foe::launch_output(uf, lo_plane(o.prec, sl.ul), r->H, r->W, r->ld, r->ld, r->model, sl.delta, nullptr, sv->stream));
        FOE_CUDA(c, cudaMemcpy2DAsync(r->x_host, r->x_pitch * sizeof(float), sl.delta, r->ld * sizeof(float),
                                      r->W * sizeof(float), r->H, cudaMemcpyDeviceToHost, sv->stream));
        finished.push_back(r);
    }
    FOE_CUDA(c, cudaMemcpyAsync(sv->h_status + slot, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, sv->stream));
    FOE_CUDA(c, cudaEventRecord(sv->done_ev[slot], sv->stream));
    sv->active.swap(still);
    // 4. the previous tick (queued before this one) completes while this one runs
    st = complete_pending(sv, n_completed);
    sv->finishing.insert(sv->finishing.end(), finished.begin(), finished.end());
    sv->pending = true;
    sv->ticks++;
    return st;
}

foe_status foe_server_poll(foe_server *sv, long long *ids, int max_ids, int *n)
{
    if (!sv || !n || (max_ids > 0 && !ids)) return FOE_EINVAL;
    const int k = std::min(max_ids, (int)sv->completed_ids.size());
    for (int i = 0; i < k; ++i) ids[i] = sv->completed_ids[i];
    sv->completed_ids.erase(sv->completed_ids.begin(), sv->completed_ids.begin() + k);
    *n = k;
    return FOE_OK;
}

foe_status foe_server_get_stats(const foe_server *sv, foe_server_stats *s)
{
    if (!sv || !s) return FOE_EINVAL;
    s->queued = (int)sv->queue.size();
    s->active = (int)sv->active.size();
    s->finishing = (int)sv->finishing.size();
    s->completed = sv->completed;
    s->ticks = sv->ticks;
    s->launches = sv->launches;
    s->pixel_iters = sv->pixel_iters;
    s->bytes_in_use = sv->arena.used();
    s->bytes_peak = sv->arena.peak();
    s->bytes_budget = sv->arena.capacity();
    return FOE_OK;
}

}  // extern "C"
