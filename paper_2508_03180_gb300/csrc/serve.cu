// Continuous-batching request loop (serving workload; the paper has no
// serving layer).  Requests (one view of a resident scene each) queue on the
// host; a worker thread admits the oldest pending requests into a batch --
// views of mixed scenes and resolutions rendered by ONE launch chain -- as
// soon as one of kServeStreams chain slots is free and the batch's memory
// estimate fits the HBM budget.  While one chain runs on the GPU the next
// batch is binned on the other stream, so arrivals during a render join the
// next batch instead of waiting for a drain.  Device outputs are written by
// the blend kernel in place; host outputs are copied after the chain.
#include <chrono>
#include <cstring>

#include "runtime.h"

using namespace dgs;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int64_t request_bytes(const Scene &sc, const dgs_camera &c) {
    const int64_t px = (int64_t)c.W * c.H;
    const int64_t tiles = (int64_t)((c.W + 15) / 16) * ((c.H + 15) / 16);
    // per pixel: image, D, count; per Gaussian: one record; per cell: binning
    // arrays and sort scratch; per tile: a generous 64 (tile, cell) pairs
    return px * 20 + sc.G * 48 + sc.N * 40 + tiles * 64 * 24 + (1 << 20);
}

void finish(ServeState &S, InflightBatch &b, dgs_status st) {
    const double t = now_ms();
    std::lock_guard<std::mutex> lk(S.m);
    for (auto &r : b.reqs) {
        dgs_result res;
        res.status = st;
        res.batch_size = (int32_t)b.reqs.size();
        res.t_submit_ms = r.t_submit;
        res.t_start_ms = b.t_start;
        res.t_done_ms = t;
        S.finished[r.ticket] = res;
    }
    S.reserved -= b.bytes;
    S.cv_done.notify_all();
}

// Launch one batch on stream slot `si` (holding ctx->mu).
dgs_status launch_batch(dgs_ctx *ctx, ServeState &S, InflightBatch &b, int si) {
    cudaStream_t st = S.streams[si];
    dgs_status s;
    b.ws = acquire_ws(ctx, st, &s);
    if (!b.ws) return s;
    std::vector<ChainView> views;
    for (auto &r : b.reqs) {
        ChainView cv;
        cv.scene_id = r.req.scene_id;
        cv.cam = r.req.camera;
        cv.out = r.req.out_location == DGS_DEVICE ? r.req.out_rgb : nullptr;
        views.push_back(cv);
    }
    s = chain_forward(ctx, *b.ws, views, nullptr, false, false, st);
    if (s) return s;
    const float *rgb = (const float *)b.ws->rgb.p;
    for (size_t v = 0; v < b.reqs.size(); ++v) {
        const dgs_request &r = b.reqs[v].req;
        if (r.out_location != DGS_HOST) continue;
        const ViewDesc &vd = b.ws->hviews[v];
        cudaError_t e = cudaMemcpyAsync(r.out_rgb, rgb + 3 * vd.pix_base, 12LL * vd.W * vd.H, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_error(e, "copying a served image to host memory");
    }
    cudaError_t e = cudaEventRecord(S.events[si], st);
    if (e == cudaSuccess) e = cudaEventRecord(b.ws->done, st);
    if (e != cudaSuccess) return cuda_error(e, "recording batch completion");
    return DGS_OK;
}

void worker_main(dgs_ctx *ctx) {
    ServeState &S = *ctx->serve;
    cudaSetDevice(ctx->cfg.device);
    InflightBatch slot[kServeStreams];
    for (;;) {
        bool progressed = false;
        // retire finished chains
        for (int si = 0; si < kServeStreams; ++si) {
            if (!S.busy[si]) continue;
            const cudaError_t q = cudaEventQuery(S.events[si]);
            if (q == cudaErrorNotReady) continue;
            finish(S, slot[si], q == cudaSuccess ? DGS_OK : cuda_error(q, "served batch"));
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                ctx->pool.push_back(std::move(slot[si].ws));
            }
            slot[si].reqs.clear();
            S.busy[si] = false;
            progressed = true;
        }
        // admit the oldest pending requests into a free chain slot
        int free_si = -1;
        for (int si = 0; si < kServeStreams; ++si)
            if (!S.busy[si]) { free_si = si; break; }
        InflightBatch nb;
        {
            std::unique_lock<std::mutex> lk(S.m);
            if (S.stop && S.pending.empty() && !S.busy[0] && !S.busy[1]) break;
            if (free_si >= 0) {
                while (!S.pending.empty() && (int)nb.reqs.size() < S.max_batch) {
                    const PendingReq &r = S.pending.front();
                    const bool first = nb.reqs.empty() && S.reserved == 0;
                    if (!first && S.reserved + nb.bytes + r.bytes > S.budget) break;  // wait for memory
                    nb.bytes += r.bytes;
                    nb.reqs.push_back(r);
                    S.pending.pop_front();
                }
                S.reserved += nb.bytes;
            }
            if (nb.reqs.empty() && !progressed) {
                const bool any_busy = S.busy[0] || S.busy[1];
                if (any_busy) S.cv_work.wait_for(lk, std::chrono::microseconds(50));
                else S.cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        if (!nb.reqs.empty()) {
            nb.t_start = now_ms();
            nb.stream_idx = free_si;
            dgs_status s;
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                s = launch_batch(ctx, S, nb, free_si);
                if (s && nb.ws) ctx->pool.push_back(std::move(nb.ws));
            }
            if (s) {
                finish(S, nb, s);
            } else {
                slot[free_si] = std::move(nb);
                S.busy[free_si] = true;
            }
        }
    }
}

}  // namespace

extern "C" dgs_status dgs_serve_start(dgs_ctx *ctx, int32_t max_batch, int32_t queue_cap) {
    if (!ctx || max_batch < 1 || queue_cap < 1) return set_error(DGS_ERR_INVALID_ARG, "bad argument");
    if (ctx->serve) return DGS_OK;
    cudaError_t e = cudaSetDevice(ctx->cfg.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    auto S = std::make_unique<ServeState>();
    S->max_batch = max_batch;
    S->queue_cap = queue_cap;
    int64_t scene_bytes = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto &kv : ctx->scenes) scene_bytes += kv.second->cell.cap + kv.second->gauss.cap + kv.second->sh.cap;
    }
    S->budget = ctx->cfg.hbm_budget_bytes - scene_bytes;
    for (int i = 0; i < kServeStreams; ++i) {
        if ((e = cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_error(e, "creating a serving stream");
        if ((e = cudaEventCreateWithFlags(&S->events[i], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_error(e, "creating a serving event");
    }
    ctx->serve = std::move(S);
    ctx->serve->worker = std::thread(worker_main, ctx);
    return DGS_OK;
}

extern "C" dgs_status dgs_serve_stop(dgs_ctx *ctx) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    if (!ctx->serve) return DGS_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->serve->m);
        ctx->serve->stop = true;
        ctx->serve->cv_work.notify_all();
    }
    if (ctx->serve->worker.joinable()) ctx->serve->worker.join();
    for (int i = 0; i < kServeStreams; ++i) {
        if (ctx->serve->streams[i]) cudaStreamDestroy(ctx->serve->streams[i]);
        if (ctx->serve->events[i]) cudaEventDestroy(ctx->serve->events[i]);
    }
    ctx->serve.reset();
    return DGS_OK;
}

extern "C" dgs_status dgs_submit(dgs_ctx *ctx, const dgs_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->serve) return set_error(DGS_ERR_INVALID_ARG, "serving is not started");
    if (!req->out_rgb || (req->out_location != DGS_HOST && req->out_location != DGS_DEVICE))
        return set_error(DGS_ERR_INVALID_ARG, "bad output");
    const dgs_camera &c = req->camera;
    if (c.W <= 0 || c.H <= 0 || c.W > 32768 || c.H > 32768 || !(c.fx > 0.f) || !(c.fy > 0.f) || !(c.znear > 0.f))
        return set_error(DGS_ERR_INVALID_ARG, "bad camera");
    int64_t bytes;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->scenes.find(req->scene_id);
        if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
        bytes = request_bytes(*it->second, c);
    }
    ServeState &S = *ctx->serve;
    std::lock_guard<std::mutex> lk(S.m);
    if ((int)S.pending.size() >= S.queue_cap) return set_error(DGS_ERR_BUSY, "request queue is full");
    PendingReq p;
    p.ticket = S.next_ticket++;
    p.req = *req;
    p.t_submit = now_ms();
    p.bytes = bytes;
    S.pending.push_back(p);
    S.open.insert(p.ticket);
    *ticket = p.ticket;
    S.cv_work.notify_one();
    return DGS_OK;
}

extern "C" dgs_status dgs_poll(dgs_ctx *ctx, uint64_t ticket, int64_t timeout_us, dgs_result *out) {
    if (!ctx || !out) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->serve) return set_error(DGS_ERR_INVALID_ARG, "serving is not started");
    ServeState &S = *ctx->serve;
    std::unique_lock<std::mutex> lk(S.m);
    if (!S.open.count(ticket)) return set_error(DGS_ERR_NOT_FOUND, "unknown or consumed ticket");
    auto ready = [&] { return S.finished.count(ticket) > 0; };
    if (timeout_us < 0) S.cv_done.wait(lk, ready);
    else if (timeout_us > 0) S.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (!ready()) return set_error(DGS_ERR_TIMEOUT, "request not finished yet");
    *out = S.finished[ticket];
    S.finished.erase(ticket);
    S.open.erase(ticket);
    return DGS_OK;
}
