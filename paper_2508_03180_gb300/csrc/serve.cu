// Continuous-batching request loop (serving workload; the paper has no
// serving layer).  Requests (one view of a resident scene each) queue on the
// host; a worker thread admits the oldest pending requests into a batch --
// views of mixed scenes and resolutions rendered by ONE launch chain -- as
// soon as one of kServeStreams chain slots is free and the batch's memory
// estimate fits the HBM budget.  While one chain runs on the GPU the next
// batch is binned on the other stream, so arrivals during a render join the
// next batch instead of waiting for a drain.  Device outputs are written by
// the blend kernel in place; host outputs are copied after the chain.  A
// host callback behind each chain wakes the worker when the chain completes.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <stdexcept>
#include <string>

#include "runtime.h"

using namespace dgs;

void dgs::GraphSlot::drop() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
}

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int64_t request_bytes(const Scene &sc, const dgs_camera &c) {
    const int64_t px = (int64_t)c.W * c.H;
    const int64_t tiles = (int64_t)((c.W + 15) / 16) * ((c.H + 15) / 16);
    // per pixel: image, D, count; per Gaussian: one record (and its decoded
    // values for neural cells); per cell: binning arrays and sort scratch (and
    // the decode's sample record); per tile: a generous 64 (tile, cell) pairs
    const int64_t neural = sc.F > 0 ? sc.G * 4 * kDecF + sc.N * 96 : 0;
    return px * 20 + sc.G * 48 + sc.N * 40 + tiles * 64 * 24 + neural + (1 << 20);
}

// Host function enqueued behind every chain: wakes the worker.
void CUDART_CB on_chain_done(void *arg) {
    ServeState *S = static_cast<ServeState *>(arg);
    std::lock_guard<std::mutex> lk(S->m);
    S->gpu_signal = true;
    S->cv_work.notify_all();
}

void finish(ServeState &S, InflightBatch &b, dgs_status st) {
    const double t = now_ms();
    std::lock_guard<std::mutex> lk(S.m);
    for (auto &r : b.reqs) {
        dgs_result res;
        res.status = S.cancelled.erase(r.ticket) ? DGS_ERR_CANCELLED : st;
        res.batch_size = (int32_t)b.reqs.size();
        res.t_submit_ms = r.t_submit;
        res.t_start_ms = b.t_start;
        res.t_done_ms = t;
        S.finished[r.ticket] = res;
    }
    S.reserved -= b.bytes;
    S.cv_done.notify_all();
}

// Host description of one batch: views in request order, scenes as a sorted
// set (slot k = k-th smallest scene id).
struct BatchPlan {
    std::vector<uint32_t> scene_set;
    std::vector<const Scene *> scenes;
    std::vector<ViewDesc> views;
    ChainCaps need;
    int K_all = 0;
};

dgs_status plan_batch(dgs_ctx *ctx, const std::vector<PendingReq> &reqs, BatchPlan &p) {
    for (auto &r : reqs) p.scene_set.push_back(r.req.scene_id);
    std::sort(p.scene_set.begin(), p.scene_set.end());
    p.scene_set.erase(std::unique(p.scene_set.begin(), p.scene_set.end()), p.scene_set.end());
    for (uint32_t id : p.scene_set) {
        auto it = ctx->scenes.find(id);
        if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
        p.scenes.push_back(it->second.get());
    }
    p.K_all = p.scenes[0]->K;
    for (const Scene *sc : p.scenes)
        if (sc->K != p.K_all) p.K_all = 0;
    long long tiles = 0, px = 0, cells = 0, recs = 0;
    for (auto &r : reqs) {
        const int slot = (int)(std::lower_bound(p.scene_set.begin(), p.scene_set.end(), r.req.scene_id) -
                               p.scene_set.begin());
        const Scene &sc = *p.scenes[slot];
        ViewDesc v = make_view(r.req.camera, (int)tiles, px, slot, sc, cells, recs);
        v.out = r.req.out_location == DGS_DEVICE ? r.req.out_rgb : nullptr;
        p.views.push_back(v);
        tiles += (long long)v.Tx * v.Ty;
        px += (long long)v.W * v.H;
        cells += sc.N;
        recs += sc.G;
    }
    if (cells >= (1LL << 32) - 1 || tiles >= (1LL << 31)) return set_error(DGS_ERR_CAPACITY, "batch too large");
    p.need.V = (int)reqs.size();
    p.need.S = (int)p.scenes.size();
    p.need.E = cells;
    p.need.R = recs;
    p.need.T = tiles;
    p.need.P = px;
    return DGS_OK;
}

// Device bytes of a slot workspace with capacities c.
long long slot_bytes(const ChainCaps &c) {
    const long long n = std::max(c.E, c.L);
    return (long long)sizeof(ViewDesc) * c.V + (long long)sizeof(SceneDev) * c.S + 36 * c.E + 4 * c.E / 1024 +
           8 * n + 1024 * (n / 4096 + 1) + 8 * c.L + 8 * c.T + 48 * c.R + 20 * c.P +
           (c.W > 0 ? 4 * c.W + 4LL * kDecF * c.R : 0);
}

long long grown(long long have, long long need) {
    return need <= have ? have : std::max(need + need / 4, have + have / 2);
}

// Size the slot for the plan; any change of capacity drops the slot's graphs
// (they hold the old buffer addresses).
dgs_status fit_slot(dgs_ctx *ctx, ServeState &S, GraphSlot &g, const BatchPlan &p, cudaStream_t st) {
    if (g.scene_epoch != ctx->scene_epoch) {
        g.drop();
        g.scene_epoch = ctx->scene_epoch;
    }
    // capacities for max_batch views of the largest resident scene at the
    // largest resolution seen, so batch composition alone never recaptures
    long long maxN = 0, maxG = 0;
    for (auto &kv : ctx->scenes) {
        maxN = std::max<long long>(maxN, kv.second->N);
        maxG = std::max<long long>(maxG, kv.second->G);
    }
    // the decode's scratch for the resident neural scenes, for E samples
    auto decode_floats = [&](long long E) {
        long long w = 0;
        for (auto &kv : ctx->scenes) {
            const Scene &sc = *kv.second;
            if (sc.F > 0) w = std::max(w, decode_scratch_floats(sc.F, sc.H, sc.K, E, sc.G, false));
        }
        return w;
    };
    for (const ViewDesc &v : p.views) {
        g.view_tiles = std::max(g.view_tiles, (long long)v.Tx * v.Ty);
        g.view_px = std::max(g.view_px, (long long)v.W * v.H);
    }
    auto target = [&](long long B) {
        ChainCaps c = g.caps;
        c.V = std::max(c.V, S.max_batch);
        c.S = std::max(c.S, S.max_batch);
        c.G = std::max(c.G, maxG);
        c.E = grown(c.E, std::max(p.need.E, B * maxN));
        c.R = grown(c.R, std::max(p.need.R, B * maxG));
        c.T = grown(c.T, std::max(p.need.T, B * g.view_tiles));
        c.P = grown(c.P, std::max(p.need.P, B * g.view_px));
        c.W = std::max(c.W, decode_floats(c.E));
        // pairs: sized from the estimate when the tile capacity changes,
        // otherwise grown only by an overflow (g.L_need)
        c.L = grown(c.L, g.L_need);
        if (c.T != g.caps.T) c.L = grown(c.L, (long long)(S.pairs_per_tile * (double)c.T));
        return c;
    };
    // within the HBM budget's share of this slot, else just what the batch needs
    ChainCaps c = target(S.max_batch);
    if (slot_bytes(c) > S.budget / kServeStreams) c = target(0);
    if (g.ws && c.V == g.caps.V && c.S == g.caps.S && c.E == g.caps.E && c.R == g.caps.R && c.T == g.caps.T &&
        c.P == g.caps.P && c.L == g.caps.L && c.G == g.caps.G && c.W == g.caps.W)
        return DGS_OK;
    g.drop();
    dgs_status s;
    if (!g.ws) {
        g.ws = std::make_unique<Workspace>();
        if ((s = g.ws->init())) return s;
    }
    // a graph of this slot may still run (it is retired before the next
    // launch, but the previous chain's copies may be pending): wait for it
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "serving stream");
    Workspace &ws = *g.ws;
    if ((s = ws.views.ensure(sizeof(ViewDesc) * c.V)) || (s = ws.scenes.ensure(sizeof(SceneDev) * c.S)) ||
        (s = ws.sizes.ensure(sizeof(ChainSizes))) || (s = ws.small.ensure(256)) || (s = ws.zkey.ensure(4 * c.E)) ||
        (s = ws.zval.ensure(4 * c.E)) || (s = ws.rect.ensure(8 * c.E)) || (s = ws.depth.ensure(4 * c.E)) ||
        (s = ws.count.ensure(4 * c.E)) || (s = ws.cnt_sorted.ensure(4 * c.E)) || (s = ws.offs.ensure(4 * c.E)) ||
        (s = ws.scan.ensure(4 * scan_scratch_words(c.E))) || (s = ensure_sort_scratch(ws, std::max(c.E, c.L))) ||
        (s = ws.tkey.ensure(4 * c.L)) || (s = ws.tval.ensure(4 * c.L)) || (s = ws.ranges.ensure(8 * c.T)) ||
        (s = ws.rec.ensure(sizeof(float4) * kRecF4 * c.R)) || (s = ws.Dpix.ensure(4 * c.P)) ||
        (s = ws.ndpix.ensure(4 * c.P)) || (s = ws.rgb.ensure(12 * c.P)) || (s = ws.vview.ensure(4 * c.E)) ||
        (c.W > 0 && ((s = ws.dec.ensure(sizeof(float) * kDecF * c.R)) || (s = ws.wpack.ensure(sizeof(float) * c.W)))))
        return s;
    if (ws.h_views_cap < (size_t)c.V) {
        if (ws.h_views) cudaFreeHost(ws.h_views);
        ws.h_views = nullptr;
        ws.h_views_cap = 0;
        if ((e = cudaMallocHost(&ws.h_views, sizeof(ViewDesc) * c.V)) != cudaSuccess)
            return cuda_error(e, "pinned view descriptors");
        ws.h_views_cap = c.V;
    }
    if (ws.h_scenes_cap < (size_t)c.S) {
        if (ws.h_scenes) cudaFreeHost(ws.h_scenes);
        ws.h_scenes = nullptr;
        ws.h_scenes_cap = 0;
        if ((e = cudaMallocHost(&ws.h_scenes, sizeof(SceneDev) * c.S)) != cudaSuccess)
            return cuda_error(e, "pinned scene descriptors");
        ws.h_scenes_cap = c.S;
    }
    g.caps = c;
    return DGS_OK;
}

#define CKR(x)                                                \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_error(e_, #x);     \
    } while (0)

// The whole forward chain with every size read on the device: the stream
// work a serving graph is captured from.  Descriptors and sizes come from the
// workspace's pinned staging, copied by the graph's first nodes.
dgs_status record_chain(dgs_ctx *ctx, Workspace &ws, const ChainCaps &c, const BatchPlan &p, cudaStream_t st) {
    const BlendParams bp = blend_params(ctx->cfg);
    uint32_t *small = (uint32_t *)ws.small.p;
    const ChainSizes *dsz = (const ChainSizes *)ws.sizes.p;
    const uint32_t *d_E = (const uint32_t *)ws.sizes.p;  // ChainSizes::n_entries
    const uint32_t *d_L = small + kSmallPairs;
    const ViewDesc *dv = (const ViewDesc *)ws.views.p;
    const SortScratch sc = sort_scratch_of(ws);
    CKR(cudaMemcpyAsync(ws.views.p, ws.h_views, sizeof(ViewDesc) * c.V, cudaMemcpyHostToDevice, st));
    CKR(cudaMemcpyAsync(ws.scenes.p, ws.h_scenes, sizeof(SceneDev) * c.S, cudaMemcpyHostToDevice, st));
    CKR(cudaMemcpyAsync(ws.sizes.p, ws.h_sizes, sizeof(ChainSizes), cudaMemcpyHostToDevice, st));
    CKR(cudaMemsetAsync(small, 0, 256, st));
    launch_cell_project(dv, c.V, (const SceneDev *)ws.scenes.p, c.E, (uint32_t *)ws.zkey.p, (uint32_t *)ws.zval.p,
                        (short4 *)ws.rect.p, (float *)ws.depth.p, (uint32_t *)ws.count.p, small + kSmallVisible,
                        (float *)ws.vview.p, ctx->cfg.flags, st, dsz);
    radix_sort_pairs((uint32_t *)ws.zkey.p, (uint32_t *)ws.zval.p, c.E, 32, sc, st, d_E);
    launch_gather_counts((const uint32_t *)ws.zval.p, (const uint32_t *)ws.count.p, c.E, (uint32_t *)ws.cnt_sorted.p,
                         st, d_E);
    exclusive_scan_u32((const uint32_t *)ws.cnt_sorted.p, (uint32_t *)ws.offs.p, c.E, small + kSmallTotal,
                       (uint32_t *)ws.scan.p, st, d_E);
    launch_clamp_pairs(small, kSmallTotal, kSmallPairs, kSmallOverflow, dsz, st);
    launch_emit((const uint32_t *)ws.offs.p, (const uint32_t *)ws.zval.p, (const short4 *)ws.rect.p, dv, c.V, c.E,
                c.L, (uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, st, dsz, d_L);
    int bits = 1;
    while ((1LL << bits) < c.T) ++bits;
    radix_sort_pairs((uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, c.L, bits, sc, st, d_L);
    CKR(cudaMemsetAsync(ws.ranges.p, 0, 8 * (size_t)c.T, st));
    launch_tile_ranges((const uint32_t *)ws.tkey.p, c.L, (uint2 *)ws.ranges.p, st, d_L);
    // neural scenes: the decode writes their records (slot k's samples of the
    // visible entries, counted on the device); the table projection skips them
    for (size_t k = 0; k < p.scenes.size(); ++k) {
        const Scene &scn = *p.scenes[k];
        if (scn.F == 0) continue;
        launch_decode(dv, c.V, (int)k, scn.dev(), (const uint32_t *)ws.zval.p, c.E, small + kSmallVisible,
                      (float *)ws.dec.p, (float *)ws.wpack.p, (const float *)ws.vview.p, bp, (float4 *)ws.rec.p,
                      nullptr, small + kSmallTcErr, st);
    }
    launch_project_fwd_table(dv, (const SceneDev *)ws.scenes.p, c.G, (const uint32_t *)ws.count.p,
                             (const float *)ws.vview.p, bp, (float4 *)ws.rec.p, st, dsz);
    launch_blend_fwd(dv, c.V, (int)c.T, (const uint2 *)ws.ranges.p, (const uint32_t *)ws.tval.p,
                     (const float4 *)ws.rec.p, bp, (float *)ws.rgb.p, nullptr, (float *)ws.Dpix.p, (int *)ws.ndpix.p,
                     p.K_all, st, dsz, small + kSmallWork);
    CKR(cudaMemcpyAsync(ws.h_small, small, 64, cudaMemcpyDeviceToHost, st));
    CKR(cudaGetLastError());
    return DGS_OK;
}

dgs_status capture_chain(dgs_ctx *ctx, GraphSlot &g, const BatchPlan &p, cudaStream_t st, cudaGraphExec_t *out) {
    CKR(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const dgs_status s = record_chain(ctx, *g.ws, g.caps, p, st);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return s ? s : cuda_error(e, "capturing the serving chain");
    }
    const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_error(ei, "instantiating the serving chain");
    return DGS_OK;
}

// Launch one batch on stream slot `si` (holding ctx->mu): one replay of the
// slot's graph for the batch's scene set, then copies of host outputs.
dgs_status launch_batch_graph(dgs_ctx *ctx, ServeState &S, InflightBatch &b, int si) {
    cudaStream_t st = S.streams[si];
    GraphSlot &g = S.gslot[si];
    BatchPlan p;
    dgs_status s;
    if ((s = plan_batch(ctx, b.reqs, p)) || (s = fit_slot(ctx, S, g, p, st))) return s;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint32_t> key{(uint32_t)p.K_all};
    for (size_t k = 0; k < p.scenes.size(); ++k)
        if (p.scenes[k]->F > 0) {
            key.push_back((uint32_t)k);
            key.push_back(p.scene_set[k]);
        }
    auto it = g.graphs.find(key);
    if (it != g.graphs.end()) {
        exec = it->second;
    } else {
        if ((s = capture_chain(ctx, g, p, st, &exec))) return s;
        g.graphs[key] = exec;
        ++S.graphs_captured;
    }
    Workspace &ws = *g.ws;
    memcpy(ws.h_views, p.views.data(), sizeof(ViewDesc) * p.views.size());
    // the capacity's unused view slots: past every entry, in no scene slot
    // (the decode's search over the views' first entries never picks them)
    for (size_t v = p.views.size(); v < (size_t)g.caps.V; ++v) {
        ws.h_views[v] = p.views.back();
        ws.h_views[v].cell_base = (long long)1 << 62;
        ws.h_views[v].scene_slot = -1;
    }
    for (size_t k = 0; k < p.scenes.size(); ++k) ws.h_scenes[k] = p.scenes[k]->dev();
    ws.h_sizes->n_entries = (uint32_t)p.need.E;
    ws.h_sizes->n_views = p.need.V;
    ws.h_sizes->total_tiles = (int32_t)p.need.T;
    ws.h_sizes->L_cap = (uint32_t)g.caps.L;
    ws.h_sizes->n_scenes = (int32_t)p.scenes.size();
    ws.total_tiles = (int)p.need.T;
    CKR(cudaGraphLaunch(exec, st));
    const float *rgb = (const float *)ws.rgb.p;
    for (size_t v = 0; v < b.reqs.size(); ++v) {
        const dgs_request &r = b.reqs[v].req;
        if (r.out_location != DGS_HOST) continue;
        const ViewDesc &vd = p.views[v];
        CKR(cudaMemcpyAsync(r.out_rgb, rgb + 3 * vd.pix_base, 12LL * vd.W * vd.H, cudaMemcpyDeviceToHost, st));
    }
    CKR(cudaEventRecord(S.events[si], st));
    CKR(cudaLaunchHostFunc(st, on_chain_done, &S));
    ++S.batches;
    b.graph = true;
    return DGS_OK;
}

// The same batch as a plain launch chain (host-synchronised sizes); used
// when serving was started without graphs.
dgs_status launch_batch_chain(dgs_ctx *ctx, ServeState &S, InflightBatch &b, int si) {
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
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_chain_done, &S);
    if (e != cudaSuccess) return cuda_error(e, "recording batch completion");
    ++S.batches;
    return DGS_OK;
}

dgs_status launch_batch(dgs_ctx *ctx, ServeState &S, InflightBatch &b, int si) {
    return S.use_graphs ? launch_batch_graph(ctx, S, b, si) : launch_batch_chain(ctx, S, b, si);
}

// After a graph batch finished: DGS_OK, or a retry after growing the pair
// capacity (returns 1), or an error.
int check_graph_batch(ServeState &S, int si, dgs_status *err) {
    GraphSlot &g = S.gslot[si];
    const uint32_t *hs = g.ws->h_small;
    if (hs[kSmallSortErr] || hs[kSmallTcErr]) {
        *err = set_error(DGS_ERR_TIMEOUT, hs[kSmallSortErr] ? "radix sort look-back wait gave up"
                                                            : "a tensor-core completion wait of the decode gave up");
        return 0;
    }
    const double L = (double)hs[kSmallTotal];
    if (g.ws->total_tiles > 0) S.pairs_per_tile = std::max(S.pairs_per_tile, 1.25 * L / g.ws->total_tiles);
    if (hs[kSmallOverflow]) {  // fit_slot grows the pair buffers to L_need
        g.L_need = (long long)(1.25 * L) + 1024;
        ++S.overflow_retries;
        return 1;
    }
    *err = DGS_OK;
    return 0;
}

void worker_loop(dgs_ctx *ctx) {
    ServeState &S = *ctx->serve;
    cudaSetDevice(ctx->cfg.device);
    InflightBatch *slot = S.slot;
    for (;;) {
        bool progressed = false;
        {
            std::lock_guard<std::mutex> lk(S.m);
            S.gpu_signal = false;  // the checks below see every chain completed so far
        }
        // retire finished chains
        for (int si = 0; si < kServeStreams; ++si) {
            if (!S.busy[si]) continue;
            const cudaError_t q = cudaEventQuery(S.events[si]);
            if (q == cudaErrorNotReady) continue;
            dgs_status bs = q == cudaSuccess ? DGS_OK : cuda_error(q, "served batch");
            if (!bs && slot[si].graph) {
                std::lock_guard<std::mutex> lk(ctx->mu);
                if (check_graph_batch(S, si, &bs)) {
                    // pair buffers overflowed: grow them and run the batch again
                    bs = launch_batch(ctx, S, slot[si], si);
                    if (!bs) continue;
                    S.gslot[si].drop();
                }
            }
            finish(S, slot[si], bs);
            if (slot[si].ws) {
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
            const uint64_t seen = S.submits;
            if (S.inject_fault > 0 && !S.pending.empty()) {
                --S.inject_fault;
                throw std::runtime_error("injected host-side fault in the serving worker");
            }
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
                // sleep until a chain completes (host callback), a request
                // arrives or serving stops; the timeout is only a safety net
                S.cv_work.wait_for(lk, std::chrono::milliseconds(20),
                                   [&] { return S.stop || S.gpu_signal || S.submits != seen; });
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
                if (s && S.use_graphs) S.gslot[free_si].drop();  // a failed capture leaves nothing usable
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

// The worker's top level: a host-side fault (an exception) stops the worker,
// but first its streams finish the chains in flight (their buffers go back to
// the pool only then), and every request it had not finished -- in flight or
// pending -- completes with DGS_ERR_WORKER, so no poll waits for it.
void worker_main(dgs_ctx *ctx) {
    ServeState &S = *ctx->serve;
    std::string why;
    try {
        worker_loop(ctx);
        return;
    } catch (const std::exception &e) {
        why = e.what();
    } catch (...) {
        why = "unknown exception";
    }
    for (int si = 0; si < kServeStreams; ++si)
        if (S.streams[si]) cudaStreamSynchronize(S.streams[si]);
    for (int si = 0; si < kServeStreams; ++si) {
        if (S.busy[si]) {
            finish(S, S.slot[si], DGS_ERR_WORKER);
            S.busy[si] = false;
        }
        if (S.slot[si].ws) {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->pool.push_back(std::move(S.slot[si].ws));
        }
        S.slot[si].reqs.clear();
    }
    std::lock_guard<std::mutex> lk(S.m);
    const double t = now_ms();
    for (const PendingReq &r : S.pending) {
        dgs_result res;
        res.status = DGS_ERR_WORKER;
        res.batch_size = 0;
        res.t_submit_ms = r.t_submit;
        res.t_start_ms = res.t_done_ms = t;
        S.finished[r.ticket] = res;
    }
    S.pending.clear();
    S.dead = true;
    S.dead_msg = "serving worker stopped: " + why;
    S.cv_done.notify_all();
}

}  // namespace

dgs_status dgs::serve_inject_fault(dgs_ctx *ctx, int count) {
    if (!ctx || !ctx->serve) return set_error(DGS_ERR_INVALID_ARG, "serving is not started");
    ServeState &S = *ctx->serve;
    std::lock_guard<std::mutex> lk(S.m);
    S.inject_fault = std::max(0, count);
    S.cv_work.notify_all();
    return DGS_OK;
}

extern "C" dgs_status dgs_serve_start(dgs_ctx *ctx, int32_t max_batch, int32_t queue_cap, int32_t flags) {
    if (!ctx || max_batch < 1 || queue_cap < 1 || (flags & ~DGS_SERVE_NO_GRAPHS))
        return set_error(DGS_ERR_INVALID_ARG, "bad argument");
    if (ctx->serve) return DGS_OK;
    cudaError_t e = cudaSetDevice(ctx->cfg.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    auto S = std::make_unique<ServeState>();
    S->max_batch = max_batch;
    S->queue_cap = queue_cap;
    S->use_graphs = !(flags & DGS_SERVE_NO_GRAPHS);
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
    // completion callbacks still queued behind the last chains refer to the
    // serving state: let them run before it goes away
    for (int i = 0; i < kServeStreams; ++i)
        if (ctx->serve->streams[i]) cudaStreamSynchronize(ctx->serve->streams[i]);
    for (int i = 0; i < kServeStreams; ++i) {
        if (ctx->serve->streams[i]) cudaStreamDestroy(ctx->serve->streams[i]);
        if (ctx->serve->events[i]) cudaEventDestroy(ctx->serve->events[i]);
    }
    ctx->serve.reset();
    return DGS_OK;
}

extern "C" dgs_status dgs_serve_read_stats(dgs_ctx *ctx, dgs_serve_stats *out) {
    if (!ctx || !out) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->serve) return set_error(DGS_ERR_INVALID_ARG, "serving is not started");
    std::lock_guard<std::mutex> lk(ctx->mu);  // the worker updates these under ctx->mu
    const ServeState &S = *ctx->serve;
    out->batches = S.batches;
    out->graphs_captured = S.graphs_captured;
    out->overflow_retries = S.overflow_retries;
    out->pairs_per_tile = S.pairs_per_tile;
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
    if (S.dead) return set_error(DGS_ERR_WORKER, S.dead_msg);
    if ((int)S.pending.size() >= S.queue_cap) return set_error(DGS_ERR_BUSY, "request queue is full");
    PendingReq p;
    p.ticket = S.next_ticket++;
    p.req = *req;
    p.t_submit = now_ms();
    p.bytes = bytes;
    S.pending.push_back(p);
    ++S.submits;
    S.open.insert(p.ticket);
    *ticket = p.ticket;
    S.cv_work.notify_one();
    return DGS_OK;
}

extern "C" dgs_status dgs_cancel(dgs_ctx *ctx, uint64_t ticket) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    if (!ctx->serve) return set_error(DGS_ERR_INVALID_ARG, "serving is not started");
    ServeState &S = *ctx->serve;
    std::lock_guard<std::mutex> lk(S.m);
    if (!S.open.count(ticket)) return set_error(DGS_ERR_NOT_FOUND, "unknown or consumed ticket");
    if (S.finished.count(ticket)) return DGS_OK;  // too late: the result keeps its own status
    for (auto it = S.pending.begin(); it != S.pending.end(); ++it) {
        if (it->ticket != ticket) continue;
        dgs_result res;
        res.status = DGS_ERR_CANCELLED;
        res.batch_size = 0;
        res.t_submit_ms = it->t_submit;
        res.t_start_ms = res.t_done_ms = now_ms();
        S.pending.erase(it);
        S.finished[ticket] = res;
        S.cv_done.notify_all();
        return DGS_OK;
    }
    S.cancelled.insert(ticket);  // admitted: its batch reports it cancelled when it completes
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
