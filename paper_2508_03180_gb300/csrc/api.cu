// Host runtime behind include/dgs.h: contexts, resident scenes, camera
// slots, per-render workspaces, and the launch chains of render and
// render_backward.  Every step of the hot path runs in this library's own
// kernels (binning.cu, sort.cu, project.cu, blend.cu, misc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dgs.h"
#include "internal.cuh"
#include "runtime.h"

using namespace dgs;

static thread_local std::string g_last_error;

namespace dgs {

dgs_status set_error(dgs_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

dgs_status cuda_error(cudaError_t e, const char *what) {
    return set_error(e == cudaErrorMemoryAllocation ? DGS_ERR_OOM : DGS_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}


// ---------------------------------------------------------------- device buffers
// Debug mode pads every new device buffer with kGuardBytes of kGuardByte on
// each side and keeps it in a process-wide registry, so that
// dgs_debug_check_guards can find writes next to any buffer.  Fault injection
// (dgs_debug_inject_fault) makes allocations fail or overwrites one guard
// byte, both on the host.
namespace {
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
std::atomic<int> g_guards{-1};        // -1: not decided yet (DGS_DEBUG is read at the first allocation)
std::atomic<int> g_fail_allocs{0};    // injected allocation failures still to make
std::atomic<int> g_corrupt_next{0};   // overwrite a guard byte of the next padded buffer
std::mutex g_guard_mu;
std::set<const DevBuf *> g_guarded;   // live padded buffers

bool guards_on() {
    int v = g_guards.load();
    if (v < 0) {
        const char *e = std::getenv("DGS_DEBUG");
        const int want = e && e[0] == '1' && e[1] == 0 ? 1 : 0;
        g_guards.compare_exchange_strong(v, want);
        v = g_guards.load();
    }
    return v == 1;
}

bool take_injected(std::atomic<int> &counter) {
    int n = counter.load();
    while (n > 0)
        if (counter.compare_exchange_weak(n, n - 1)) return true;
    return false;
}
}  // namespace

dgs_status DevBuf::ensure(size_t bytes) {
    if (bytes <= cap) return DGS_OK;
    release();
    if (take_injected(g_fail_allocs)) return set_error(DGS_ERR_OOM, "device allocation failed (injected fault)");
    const size_t want = bytes + bytes / 8 + 256;
    const bool guard = guards_on();
    const size_t pad = guard ? kGuardBytes : 0;
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, want + 2 * pad);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(DGS_ERR_OOM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    if (guard) {
        char *b = static_cast<char *>(base);
        e = cudaMemset(b, kGuardByte, pad);
        if (e == cudaSuccess) e = cudaMemset(b + pad + want, kGuardByte, pad);
        if (e == cudaSuccess && take_injected(g_corrupt_next)) e = cudaMemset(b + pad + want + 7, 0, 1);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();  // the fill lands before any stream uses the buffer
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e != cudaSuccess) {
            cudaFree(base);
            return cuda_error(e, "filling guard words");
        }
        std::lock_guard<std::mutex> lk(g_guard_mu);
        g_guarded.insert(this);
    }
    p = static_cast<char *>(base) + pad;
    cap = want;
    guarded = guard;
    return DGS_OK;
}

void DevBuf::release() {
    if (p) {
        if (guarded) {
            {
                std::lock_guard<std::mutex> lk(g_guard_mu);
                g_guarded.erase(this);
            }
            cudaFree(static_cast<char *>(p) - kGuardBytes);
        } else {
            cudaFree(p);
        }
    }
    p = nullptr;
    cap = 0;
    guarded = false;
}

Workspace::~Workspace() {
    for (DevBuf *b : all()) b->release();
    if (h_small) cudaFreeHost(h_small);
    if (h_views) cudaFreeHost(h_views);
    if (h_scenes) cudaFreeHost(h_scenes);
    if (h_sizes) cudaFreeHost(h_sizes);
    if (done) cudaEventDestroy(done);
}

std::vector<DevBuf *> Workspace::all() {
    return {&views, &scenes, &zkey, &zval, &rect, &depth, &count, &cnt_sorted, &offs, &tkey, &tval, &ranges, &rec,
            &Dpix, &ndpix, &rgb, &g2d, &gstage, &sort_k, &sort_v, &sort_hist, &sort_status, &sort_ctr, &small, &scan, &sizes, &vview, &gvview, &dec};
}

dgs_status Workspace::init() {
    CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    CK(cudaMallocHost(&h_small, 256));
    memset(h_small, 0, 256);
    CK(cudaMallocHost(&h_sizes, sizeof(ChainSizes)));
    memset(h_sizes, 0, sizeof(ChainSizes));
    return DGS_OK;
}

dgs_status ensure_sort_scratch(Workspace &ws, long long n) {
    dgs_status s;
    if ((s = ws.sort_k.ensure(sizeof(uint32_t) * std::max(1LL, n)))) return s;
    if ((s = ws.sort_v.ensure(sizeof(uint32_t) * std::max(1LL, n)))) return s;
    if ((s = ws.sort_hist.ensure(sizeof(uint32_t) * 4 * 256))) return s;
    if ((s = ws.sort_status.ensure(sizeof(uint32_t) * 2 * 256 * std::max(1LL, sort_parts_for(n))))) return s;
    if ((s = ws.sort_ctr.ensure(sizeof(uint32_t) * 4))) return s;
    return DGS_OK;
}

SortScratch sort_scratch_of(Workspace &ws) {
    SortScratch s;
    s.keys_alt = (uint32_t *)ws.sort_k.p;
    s.vals_alt = (uint32_t *)ws.sort_v.p;
    s.hist = (uint32_t *)ws.sort_hist.p;
    s.status = (uint32_t *)ws.sort_status.p;
    s.counters = (uint32_t *)ws.sort_ctr.p;
    s.err = (uint32_t *)ws.small.p + kSmallSortErr;
    s.cap_items = (long long)(ws.sort_k.cap / 4);
    s.cap_parts = (long long)(ws.sort_status.cap / 2048);
    return s;
}

cudaEvent_t Profiler::take() {
    if (!spare.empty()) {
        cudaEvent_t e = spare.back();
        spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Profiler::drain() {
    for (auto &q : pending) {
        float ms_ = 0.f;
        if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms_, q.a, q.b) == cudaSuccess) {
            ms[q.stage] += ms_;
            launches[q.stage] += 1;
        }
        spare.push_back(q.a);
        spare.push_back(q.b);
    }
    pending.clear();
}

Profiler::~Profiler() {
    for (auto &q : pending) {
        cudaEventDestroy(q.a);
        cudaEventDestroy(q.b);
    }
    for (auto e : spare) cudaEventDestroy(e);
}

// NVTX names of the stages (dgs_stage order): the host-side range around each
// stage's launches, seen by nsys/ncu (--nvtx); a no-op without a tool attached.
static const char *const kStageNames[] = {"dgs.cell_project", "dgs.depth_sort", "dgs.count_scan", "dgs.emit",
                                          "dgs.tile_sort",    "dgs.tile_ranges", "dgs.project_fwd", "dgs.blend_fwd",
                                          "dgs.blend_bwd",    "dgs.project_bwd", "dgs.decode",      "dgs.decode_bwd"};

StageTimer::StageTimer(Profiler &p_, int s, cudaStream_t st_) : p(p_), stage(s), st(st_) {
    if (s >= 0 && s < (int)(sizeof(kStageNames) / sizeof(kStageNames[0]))) nvtxRangePushA(kStageNames[s]);
    if (!p.on) return;
    a = p.take();
    cudaEventRecord(a, st);
}

StageTimer::~StageTimer() {
    if (stage >= 0 && stage < (int)(sizeof(kStageNames) / sizeof(kStageNames[0]))) nvtxRangePop();
    if (!p.on || !a) return;
    cudaEvent_t b = p.take();
    cudaEventRecord(b, st);
    p.pending.push_back({stage, a, b});
}

SceneDev Scene::dev() const {
    SceneDev d;
    d.cell = (const float *)cell.p;
    d.gauss = (const float *)gauss.p;
    d.sh = (const float *)sh.p;
    d.vsh = vdeg >= 0 ? (const float *)vsh.p : nullptr;
    d.N = N;
    d.G = G;
    d.K = K;
    d.sh_degree = deg;
    d.v_sh_degree = vdeg;
    d.feat = F > 0 ? (const float *)feat.p : nullptr;
    d.goff = F > 0 ? (const float *)goff.p : nullptr;
    d.mlp = F > 0 ? (const float *)mlp.p : nullptr;
    d.F = F;
    d.H = H;
    d.pad = 0;
    return d;
}

}  // namespace dgs

// ------------------------------------------------------------------ context

extern "C" void dgs_config_default(dgs_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->eps = 1e-4f;
    c->alpha_max = 0.99f;
    c->d_min = 1e-10f;
    c->dilation = 0.3f;
    c->ksigma = 3.0f;
    c->device = 0;
}

extern "C" dgs_status dgs_create(const dgs_config *cfg, dgs_ctx **out) {
    if (!out) return set_error(DGS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    dgs_config c;
    if (cfg) c = *cfg; else dgs_config_default(&c);
    if (!(c.eps >= 0.f) || !(c.alpha_max > 0.f && c.alpha_max < 1.f) || !(c.ksigma > 0.f) || !(c.dilation >= 0.f) ||
        !(c.w_bg >= 0.f) || (c.flags & ~(DGS_FLAG_ALPHA_SKIP | DGS_FLAG_TERM_EXCLUDE | DGS_FLAG_AABB_SQUARE |
                                         DGS_FLAG_NUMERATOR | DGS_FLAG_NEAR_FULL)) != 0)
        return set_error(DGS_ERR_INVALID_ARG,
                         "config out of range (need eps >= 0, 0 < alpha_max < 1, ksigma > 0, w_bg >= 0, known flags)");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (c.device < 0 || c.device >= ndev) return set_error(DGS_ERR_INVALID_ARG, "no such CUDA device");
    CK(cudaSetDevice(c.device));
    dgs_ctx *ctx = new dgs_ctx();
    ctx->cfg = c;
    ctx->cams.resize(kMaxCamSlots);
    ctx->cam_set.assign(kMaxCamSlots, 0);
    if (c.hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        ctx->cfg.hbm_budget_bytes = (int64_t)(0.9 * (double)fr);
    }
    *out = ctx;
    return DGS_OK;
}

extern "C" void dgs_destroy(dgs_ctx *ctx) {
    if (!ctx) return;
    dgs_serve_stop(ctx);
    cudaSetDevice(ctx->cfg.device);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto *st : ctx->live_states) delete st;
        ctx->live_states.clear();
        ctx->pool.clear();
        ctx->scenes.clear();
        ctx->aux.release();
        ctx->sort_ws.reset();
    }
    delete ctx;
}

extern "C" const char *dgs_last_error(dgs_ctx *) { return g_last_error.c_str(); }

// ------------------------------------------------------------------ scenes

// Device address of host memory the GPU reaches directly (page-locked by
// cudaHostAlloc / cudaMallocHost or registered with cudaHostRegister, hence
// mapped into the device's address space), else nullptr (pageable memory).
// Kernels read and write such memory over the host link themselves, so a
// transfer overlaps the kernel's own work and needs no device staging copy.
static const void *mapped_host(const void *h) {
    if (!h) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// One parameter array (rows x cols, row-major, in `location` memory) into
// its structure-of-arrays planes.  Mapped host arrays are read by the
// transposing kernel over the host link; other host arrays go through
// `stage` (device, rows x cols floats).  The caller synchronises before the
// host memory or the staging is reused.
static dgs_status upload_param(const float *src, int location, int64_t rows, int cols, float *dst_planes,
                               int64_t plane_stride, float *stage, cudaStream_t st) {
    const size_t bytes = sizeof(float) * (size_t)rows * cols;
    if (bytes == 0) return DGS_OK;
    const float *dsrc = src;
    if (location == DGS_HOST) {
        if (const void *m = mapped_host(src)) {
            dsrc = (const float *)m;
        } else {
            CK(cudaMemcpyAsync(stage, src, bytes, cudaMemcpyHostToDevice, st));
            dsrc = stage;
        }
    }
    launch_aos_to_soa(dsrc, rows, cols, dst_planes, plane_stride, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

// Packed decoder weights of a neural scene (four decoders, outputs K, 3K, 3K, 4K).
static int neural_weights(const Scene &sc) {
    const int outs[4] = {sc.K, 3 * sc.K, 3 * sc.K, 4 * sc.K};
    int n = 0;
    for (int o : outs) n += sc.H * (sc.F + 4) + sc.H + o * sc.H + o;
    return n;
}

static dgs_status fill_scene(dgs_ctx *ctx, Scene &sc, const dgs_scene_desc *d, cudaStream_t st, bool cells_too) {
    const int64_t N = sc.N, G = sc.G;
    float *cell = (float *)sc.cell.p, *gs = (float *)sc.gauss.p, *sh = (float *)sc.sh.p;
    struct Part { const float *src; int64_t rows; int cols; float *dst; int64_t stride; };
    std::vector<Part> parts;
    if (cells_too) {
        parts.push_back({d->cell_center, N, 3, cell, N});
        parts.push_back({d->cell_axes, N, 3, cell + 3 * N, N});
        parts.push_back({d->cell_quat, N, 4, cell + 6 * N, N});
    }
    if (d->cell_v) parts.push_back({d->cell_v, N, 1, cell + 10 * N, N});
    if (sc.vdeg >= 0 && d->cell_v_sh) parts.push_back({d->cell_v_sh, N, sc.Cv, (float *)sc.vsh.p, N});
    if (sc.F > 0) {  // neural cells: features and offsets as planes, the weights as given (one row)
        parts.push_back({d->neural->cell_feat, N * sc.F, 1, (float *)sc.feat.p, N * sc.F});  // rows [N][F]
        parts.push_back({d->neural->g_offset, G, 3, (float *)sc.goff.p, G});
        parts.push_back({d->neural->mlp, 1, neural_weights(sc), (float *)sc.mlp.p, 1});
    } else {
        parts.push_back({d->g_mean, G, 3, gs, G});
        parts.push_back({d->g_scale, G, 3, gs + 3 * G, G});
        parts.push_back({d->g_quat, G, 4, gs + 6 * G, G});
        parts.push_back({d->g_logit, G, 1, gs + 10 * G, G});
        parts.push_back({d->g_sh, G, 3 * sc.C, sh, G});
    }
    // host inputs that are not mapped: every such array gets its own staging
    // region; one synchronisation at the end
    float *stage = nullptr;
    if (d->location == DGS_HOST) {
        int64_t total = 0;
        for (auto &p : parts)
            if (p.src && !mapped_host(p.src)) total += p.rows * p.cols;
        if (total) {
            dgs_status s = ctx->aux.ensure(sizeof(float) * total);
            if (s) return s;
            stage = (float *)ctx->aux.p;
        }
    }
    if (!d->cell_v && cells_too) launch_fill_f32(cell + 10 * N, N, 1.0f, st);
    for (auto &p : parts) {
        if (!p.src) continue;
        const bool staged = d->location == DGS_HOST && !mapped_host(p.src);
        dgs_status s = upload_param(p.src, d->location, p.rows, p.cols, p.dst, p.stride, stage, st);
        if (s) return s;
        if (staged) stage += p.rows * p.cols;
    }
    CK(cudaGetLastError());
    if (d->location == DGS_HOST) CK(cudaStreamSynchronize(st));  // host arrays and staging free again
    return DGS_OK;
}

static dgs_status check_desc(const dgs_scene_desc *d, bool need_cells = true) {
    if (!d) return set_error(DGS_ERR_INVALID_ARG, "scene desc is NULL");
    if (d->num_cells < 0 || d->K < 1 || d->K > kMaxK || d->sh_degree < 0 || d->sh_degree > 3)
        return set_error(DGS_ERR_INVALID_ARG, "need num_cells >= 0, 1 <= K <= 32, 0 <= sh_degree <= 3");
    if (d->location != DGS_HOST && d->location != DGS_DEVICE) return set_error(DGS_ERR_INVALID_ARG, "bad location");
    if (d->num_cells * (int64_t)d->K >= (1LL << 31)) return set_error(DGS_ERR_CAPACITY, "more than 2^31 Gaussians");
    const bool explicit_g = d->neural == nullptr;
    if (d->num_cells > 0 && ((need_cells && (!d->cell_center || !d->cell_axes || !d->cell_quat)) ||
                             (explicit_g && (!d->g_mean || !d->g_scale || !d->g_quat || !d->g_logit || !d->g_sh))))
        return set_error(DGS_ERR_INVALID_ARG, "a scene array is NULL");
    if (!explicit_g) {
        const dgs_neural_desc *n = d->neural;
        if (n->feat_dim < 1 || n->feat_dim > 64 || n->hidden < 1 || n->hidden > 64)
            return set_error(DGS_ERR_INVALID_ARG, "neural cells need 1 <= feat_dim, hidden <= 64");
        if (d->num_cells > 0 && (!n->cell_feat || !n->g_offset || !n->mlp))
            return set_error(DGS_ERR_INVALID_ARG, "a neural scene array is NULL");
    }
    if (d->cell_v_sh && (d->v_sh_degree < 0 || d->v_sh_degree > 3))
        return set_error(DGS_ERR_INVALID_ARG, "v_sh_degree must be in 0..3 with cell_v_sh");
    return DGS_OK;
}

// ------------------------------------------------------------------ scene files
struct DgsFileHeader {
    char magic[4];
    uint32_t version;
    int64_t num_cells;
    int32_t K, sh_degree, v_sh_degree, feat_dim, hidden;
    uint32_t reserved;
};
static_assert(sizeof(DgsFileHeader) == 40, "the scene file header is 40 bytes");

extern "C" dgs_status dgs_scene_save(dgs_ctx *ctx, uint32_t scene_id, const char *path) {
    if (!ctx || !path) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
    const Scene &sc = *it->second;
    const int64_t N = sc.N, G = sc.G;
    DgsFileHeader h{};
    memcpy(h.magic, "DGS1", 4);
    h.version = 1;
    h.num_cells = N;
    h.K = sc.K;
    h.sh_degree = sc.deg;
    h.v_sh_degree = sc.vdeg;
    h.feat_dim = sc.F;
    h.hidden = sc.H;
    // every array back to its row-major layout (the inverse of fill_scene's transposes)
    struct Part { const float *planes; int64_t rows; int cols; int64_t stride; };
    const float *cell = (const float *)sc.cell.p;
    std::vector<Part> parts = {
        {cell, N, 3, N}, {cell + 3 * N, N, 3, N}, {cell + 6 * N, N, 4, N}, {cell + 10 * N, N, 1, N}};
    if (sc.F > 0) {
        parts.push_back({(const float *)sc.feat.p, N * sc.F, 1, N * sc.F});
        parts.push_back({(const float *)sc.goff.p, G, 3, G});
        parts.push_back({(const float *)sc.mlp.p, 1, neural_weights(sc), 1});
    } else {
        const float *gs = (const float *)sc.gauss.p;
        parts.push_back({gs, G, 3, G});
        parts.push_back({gs + 3 * G, G, 3, G});
        parts.push_back({gs + 6 * G, G, 4, G});
        parts.push_back({gs + 10 * G, G, 1, G});
        parts.push_back({(const float *)sc.sh.p, G, 3 * sc.C, G});
    }
    if (sc.vdeg >= 0) parts.push_back({(const float *)sc.vsh.p, N, sc.Cv, N});
    int64_t total = 0;
    for (const Part &q : parts) total += q.rows * q.cols;
    std::vector<float> host((size_t)total);
    if (total > 0) {
        dgs_status s = ctx->aux.ensure(sizeof(float) * total);
        if (s) return s;
        float *stage = (float *)ctx->aux.p;
        int64_t o = 0;
        for (const Part &q : parts) {
            launch_soa_to_aos(q.planes, q.rows, q.cols, q.stride, stage + o, 0);
            o += q.rows * q.cols;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpy(host.data(), stage, sizeof(float) * total, cudaMemcpyDeviceToHost));
    }
    FILE *f = fopen(path, "wb");
    if (!f) return set_error(DGS_ERR_NOT_FOUND, std::string("cannot open ") + path + " for writing");
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 &&
                    (total == 0 || fwrite(host.data(), sizeof(float), (size_t)total, f) == (size_t)total);
    const bool closed = fclose(f) == 0;
    if (!ok || !closed) return set_error(DGS_ERR_INVALID_ARG, std::string("writing ") + path + " failed");
    return DGS_OK;
}

extern "C" dgs_status dgs_scene_load(dgs_ctx *ctx, const char *path, uint32_t *scene_id) {
    if (!ctx || !path || !scene_id) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return set_error(DGS_ERR_NOT_FOUND, std::string("cannot open ") + path);
    DgsFileHeader h{};
    const bool got = fread(&h, sizeof(h), 1, f) == 1;
    const bool shape_ok = got && memcmp(h.magic, "DGS1", 4) == 0 && h.version == 1 && h.num_cells >= 0 &&
                          h.num_cells < (1LL << 31) && h.K >= 1 && h.K <= kMaxK && h.sh_degree >= 0 &&
                          h.sh_degree <= 3 && h.v_sh_degree >= -1 && h.v_sh_degree <= 3 &&
                          ((h.feat_dim == 0 && h.hidden == 0) ||
                           (h.feat_dim >= 1 && h.feat_dim <= 64 && h.hidden >= 1 && h.hidden <= 64));
    if (!shape_ok) {
        fclose(f);
        return set_error(DGS_ERR_INVALID_ARG, std::string(path) + " is not a version-1 scene file");
    }
    const int64_t N = h.num_cells, G = N * h.K;
    const int64_t C = (h.sh_degree + 1) * (h.sh_degree + 1);
    const int64_t Cv = h.v_sh_degree >= 0 ? (h.v_sh_degree + 1) * (h.v_sh_degree + 1) : 0;
    Scene probe;  // sizes only: the packed weight count of a neural scene
    probe.K = h.K;
    probe.F = h.feat_dim;
    probe.H = h.hidden;
    const int64_t P = h.feat_dim > 0 ? neural_weights(probe) : 0;
    const int64_t sizes_cells[4] = {3 * N, 3 * N, 4 * N, N};
    std::vector<int64_t> sizes(sizes_cells, sizes_cells + 4);
    if (h.feat_dim > 0) {
        sizes.push_back(N * h.feat_dim);
        sizes.push_back(3 * G);
        sizes.push_back(P);
    } else {
        for (int64_t n : {3 * G, 3 * G, 4 * G, G, 3 * C * G}) sizes.push_back(n);
    }
    if (Cv) sizes.push_back(Cv * N);
    int64_t total = 0;
    for (int64_t n : sizes) total += n;
    // the file's length must match its header before anything is allocated for it
    const bool sized = fseek(f, 0, SEEK_END) == 0 && (int64_t)ftell(f) == (int64_t)sizeof(h) + 4 * total &&
                       fseek(f, (long)sizeof(h), SEEK_SET) == 0;
    if (!sized) {
        fclose(f);
        return set_error(DGS_ERR_INVALID_ARG, std::string(path) + ": size does not match its header");
    }
    std::vector<float> data((size_t)total);
    const bool body = total == 0 || fread(data.data(), sizeof(float), (size_t)total, f) == (size_t)total;
    fclose(f);
    if (!body) return set_error(DGS_ERR_INVALID_ARG, std::string("reading ") + path + " failed");
    std::vector<const float *> arr;
    int64_t o = 0;
    for (int64_t n : sizes) {
        arr.push_back(data.data() + o);
        o += n;
    }
    dgs_scene_desc d{};
    d.num_cells = N;
    d.K = h.K;
    d.sh_degree = h.sh_degree;
    d.location = DGS_HOST;
    d.cell_center = arr[0];
    d.cell_axes = arr[1];
    d.cell_quat = arr[2];
    d.cell_v = arr[3];
    dgs_neural_desc nd{};
    size_t k = 4;
    if (h.feat_dim > 0) {
        nd.feat_dim = h.feat_dim;
        nd.hidden = h.hidden;
        nd.cell_feat = arr[k++];
        nd.g_offset = arr[k++];
        nd.mlp = arr[k++];
        d.neural = &nd;
    } else {
        d.g_mean = arr[k++];
        d.g_scale = arr[k++];
        d.g_quat = arr[k++];
        d.g_logit = arr[k++];
        d.g_sh = arr[k++];
    }
    if (Cv) {
        d.cell_v_sh = arr[k++];
        d.v_sh_degree = h.v_sh_degree;
    }
    return dgs_scene_upload(ctx, &d, scene_id);
}

extern "C" dgs_status dgs_scene_upload(dgs_ctx *ctx, const dgs_scene_desc *d, uint32_t *scene_id) {
    if (!ctx || !scene_id) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    dgs_status s = check_desc(d);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    auto sc = std::make_unique<Scene>();
    sc->N = d->num_cells;
    sc->K = d->K;
    sc->G = sc->N * sc->K;
    sc->deg = d->sh_degree;
    sc->C = (sc->deg + 1) * (sc->deg + 1);
    sc->vdeg = d->cell_v_sh ? d->v_sh_degree : -1;
    sc->Cv = sc->vdeg >= 0 ? (sc->vdeg + 1) * (sc->vdeg + 1) : 0;
    if (d->neural) {
        sc->F = d->neural->feat_dim;
        sc->H = d->neural->hidden;
        if ((s = sc->feat.ensure(sizeof(float) * sc->F * std::max<int64_t>(1, sc->N))) ||
            (s = sc->goff.ensure(sizeof(float) * 3 * std::max<int64_t>(1, sc->G))) ||
            (s = sc->mlp.ensure(sizeof(float) * neural_weights(*sc))))
            return s;
    }
    if (sc->vdeg >= 0 && (s = sc->vsh.ensure(sizeof(float) * sc->Cv * std::max<int64_t>(1, sc->N)))) return s;
    if ((s = sc->cell.ensure(sizeof(float) * 11 * std::max<int64_t>(1, sc->N)))) return s;
    if ((s = sc->gauss.ensure(sizeof(float) * 11 * std::max<int64_t>(1, sc->G)))) return s;
    if ((s = sc->sh.ensure(sizeof(float) * 3 * sc->C * std::max<int64_t>(1, sc->G)))) return s;
    cudaStream_t st = 0;
    if ((s = fill_scene(ctx, *sc, d, st, true))) return s;
    CK(cudaStreamSynchronize(st));
    const uint32_t id = ctx->next_scene++;
    ctx->scenes[id] = std::move(sc);
    *scene_id = id;
    return DGS_OK;
}

extern "C" dgs_status dgs_scene_update(dgs_ctx *ctx, uint32_t scene_id, const dgs_scene_desc *d, dgs_stream stream) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    dgs_status s = check_desc(d, false);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
    Scene &sc = *it->second;
    if (d->num_cells != sc.N || d->K != sc.K || d->sh_degree != sc.deg ||
        (d->cell_v_sh && d->v_sh_degree != sc.vdeg) || ((d->neural != nullptr) != (sc.F > 0)) ||
        (d->neural && (d->neural->feat_dim != sc.F || d->neural->hidden != sc.H)))
        return set_error(DGS_ERR_INVALID_ARG, "update must keep N, K, sh_degree, v_sh_degree and the neural widths");
    return fill_scene(ctx, sc, d, (cudaStream_t)stream, false);
}

extern "C" dgs_status dgs_scene_release(dgs_ctx *ctx, uint32_t scene_id) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
    for (auto *st : ctx->live_states)
        if (st->scene_id == scene_id) return set_error(DGS_ERR_BUSY, "a forward state still refers to this scene");
    CK(cudaDeviceSynchronize());
    ctx->scenes.erase(it);
    ++ctx->scene_epoch;  // captured serving graphs may hold its pointers
    return DGS_OK;
}

extern "C" dgs_status dgs_camera_set(dgs_ctx *ctx, uint32_t slot, const dgs_camera *cam) {
    if (!ctx || !cam) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    if (slot >= (uint32_t)kMaxCamSlots) return set_error(DGS_ERR_INVALID_ARG, "camera slot out of range");
    if (cam->W <= 0 || cam->H <= 0 || cam->W > 32768 || cam->H > 32768 || !(cam->fx > 0.f) || !(cam->fy > 0.f) ||
        !(cam->znear > 0.f))
        return set_error(DGS_ERR_INVALID_ARG, "camera needs 0 < W,H <= 32768, fx, fy > 0, znear > 0");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->cams[slot] = *cam;
    ctx->cam_set[slot] = 1;
    return DGS_OK;
}

// ------------------------------------------------------------------ render

namespace dgs {

ViewDesc make_view(const dgs_camera &c, int tile_base, long long pix_base, int slot, const Scene &sc,
                          long long cell_base, long long rec_base) {
    ViewDesc v;
    memset(&v, 0, sizeof(v));
    v.W = c.W;
    v.H = c.H;
    v.Tx = (c.W + kTile - 1) / kTile;
    v.Ty = (c.H + kTile - 1) / kTile;
    v.tile_base = tile_base;
    v.scene_slot = slot;
    v.pix_base = pix_base;
    v.cell_base = cell_base;
    v.rec_base = rec_base;
    v.N = sc.N;
    v.K = sc.K;
    v.fx = c.fx;
    v.fy = c.fy;
    v.cx = c.cx;
    v.cy = c.cy;
    v.znear = c.znear;
    memcpy(v.R, c.R, sizeof(v.R));
    memcpy(v.t, c.t, sizeof(v.t));
    memcpy(v.eye, c.eye, sizeof(v.eye));
    return v;
}

BlendParams blend_params(const dgs_config &c) {
    BlendParams b;
    b.eps = c.eps;
    b.alpha_max = c.alpha_max;
    b.d_min = c.d_min;
    b.bg0 = c.bg[0];
    b.bg1 = c.bg[1];
    b.bg2 = c.bg[2];
    b.dilation = c.dilation;
    b.ksigma = c.ksigma;
    b.w_bg = c.w_bg;
    b.flags = c.flags;
    return b;
}

std::unique_ptr<Workspace> acquire_ws(dgs_ctx *ctx, cudaStream_t st, dgs_status *err) {
    std::unique_ptr<Workspace> ws;
    if (!ctx->pool.empty()) {
        ws = std::move(ctx->pool.back());
        ctx->pool.pop_back();
        // the previous chain on this workspace may still run on another stream
        cudaError_t e = cudaStreamWaitEvent(st, ws->done, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(ws->done);  // pinned host mirrors are rewritten next
        if (e != cudaSuccess) {
            *err = cuda_error(e, "waiting for a workspace");
            return nullptr;
        }
        if ((*err = observe_chain(ctx, *ws, true))) return nullptr;
    } else {
        ws = std::make_unique<Workspace>();
        if ((*err = ws->init())) return nullptr;
    }
    ws->bwd_done = false;
    *err = DGS_OK;
    return ws;
}

dgs_status observe_chain(dgs_ctx *ctx, Workspace &ws, bool wait) {
    if (!ws.async_pending && !ws.check_tc) return DGS_OK;
    if (wait) {
        CK(cudaEventSynchronize(ws.done));
    } else {
        const cudaError_t q = cudaEventQuery(ws.done);
        if (q == cudaErrorNotReady) return DGS_OK;
        if (q != cudaSuccess) return cuda_error(q, "a render's launch chain");
    }
    const uint32_t *h = ws.h_small;
    if (ws.check_tc && h[kSmallTcErr]) {
        ctx->pending_status = DGS_ERR_TIMEOUT;
        ctx->pending_msg = "an earlier call's tensor-core completion wait gave up: its results are not valid";
    }
    ws.check_tc = false;
    if (!ws.async_pending) return DGS_OK;
    ws.async_pending = false;
    const long long L = h[kSmallTotal];
    ws.L = std::min(L, ws.L_cap);
    ws.n_vis = h[kSmallVisible];
    if (ws.total_tiles > 0) ctx->pairs_per_tile = std::max(ctx->pairs_per_tile, (double)L / ws.total_tiles);
    if (h[kSmallSortErr]) {
        ctx->pending_status = DGS_ERR_TIMEOUT;
        ctx->pending_msg = "an earlier render's radix sort look-back wait gave up: its image and state are not valid";
    } else if (h[kSmallOverflow]) {
        ctx->pending_status = DGS_ERR_CAPACITY;
        ctx->pending_msg = "an earlier render's " + std::to_string(L) + " (tile, cell) pairs exceeded its capacity of " +
                           std::to_string(ws.L_cap) +
                           ": its image and state are incomplete; the capacity has grown, render it again";
    }
    return DGS_OK;
}

// Pair capacity of a device-sized chain: 1.5 times the largest pairs per tile
// seen in this context, at least 64 Ki pairs.
static long long pair_capacity(const dgs_ctx *ctx, const Workspace &ws) {
    const double want = 1.5 * ctx->pairs_per_tile * (double)std::max(1, ws.total_tiles);
    return std::max<long long>(1LL << 16, (long long)std::ceil(want));
}

// Binning of all views of the chain (steps a1-a5): cell projection and cull,
// depth sort over cells, count scan, key emission, tile sort, tile ranges.
// Synchronises the stream once to learn the sort length L, unless
// device_sized: then the pair count stays on the device, the pair buffers
// are sized by pair_capacity and the kernels stop at that capacity (a
// k_clamp_pairs flag records an overflow).
static dgs_status run_binning(dgs_ctx *ctx, Workspace &ws, cudaStream_t st, bool device_sized) {
    Profiler &pf = ctx->prof;
    const int V = ws.V;
    const long long n = ws.n_entries;
    const long long n1 = std::max(1LL, n);
    dgs_status s;
    if ((s = ws.small.ensure(256))) return s;
    CK(cudaMemsetAsync(ws.small.p, 0, 256, st));
    if ((s = ws.zkey.ensure(4 * n1)) || (s = ws.zval.ensure(4 * n1)) || (s = ws.rect.ensure(8 * n1)) ||
        (s = ws.depth.ensure(4 * n1)) || (s = ws.count.ensure(4 * n1)) || (s = ws.cnt_sorted.ensure(4 * n1)) ||
        (s = ws.offs.ensure(4 * n1)) || (s = ws.scan.ensure(4 * scan_scratch_words(n1))) ||
        (s = ws.vview.ensure(4 * n1)))
        return s;
    if ((s = ensure_sort_scratch(ws, n))) return s;
    // a device-sized chain sizes every buffer before its first launch, so no
    // buffer is reallocated under the kernels in flight
    const long long cap = device_sized ? pair_capacity(ctx, ws) : 0;
    if (device_sized &&
        ((s = ws.tkey.ensure(4 * cap)) || (s = ws.tval.ensure(4 * cap)) || (s = ensure_sort_scratch(ws, cap)) ||
         (s = ws.ranges.ensure(8 * (size_t)std::max(1, ws.total_tiles))) || (s = ws.sizes.ensure(sizeof(ChainSizes)))))
        return s;
    uint32_t *small = (uint32_t *)ws.small.p;
    const ViewDesc *dv = (const ViewDesc *)ws.views.p;
    {
        StageTimer t(pf, DGS_STAGE_CELL_PROJECT, st);
        launch_cell_project(dv, V, (const SceneDev *)ws.scenes.p, n, (uint32_t *)ws.zkey.p, (uint32_t *)ws.zval.p,
                            (short4 *)ws.rect.p, (float *)ws.depth.p, (uint32_t *)ws.count.p, small + kSmallVisible,
                            (float *)ws.vview.p, ctx->cfg.flags, st);
    }
    {
        StageTimer t(pf, DGS_STAGE_DEPTH_SORT, st);
        radix_sort_pairs((uint32_t *)ws.zkey.p, (uint32_t *)ws.zval.p, n, 32, sort_scratch_of(ws), st);
    }
    {
        StageTimer t(pf, DGS_STAGE_COUNT_SCAN, st);
        launch_gather_counts((const uint32_t *)ws.zval.p, (const uint32_t *)ws.count.p, n, (uint32_t *)ws.cnt_sorted.p,
                             st);
        exclusive_scan_u32((const uint32_t *)ws.cnt_sorted.p, (uint32_t *)ws.offs.p, n, small + kSmallTotal,
                           (uint32_t *)ws.scan.p, st);
    }
    CK(cudaGetLastError());
    int bits = 1;
    while ((1LL << bits) < ws.total_tiles) ++bits;
    if (device_sized) {
        ws.L_cap = cap;
        ws.L = -1;
        ws.n_vis = -1;
        *ws.h_sizes = ChainSizes{};
        ws.h_sizes->n_entries = (uint32_t)n;
        ws.h_sizes->n_views = V;
        ws.h_sizes->total_tiles = ws.total_tiles;
        ws.h_sizes->L_cap = (uint32_t)cap;
        ws.h_sizes->n_scenes = (int32_t)ws.scene_ids.size();
        CK(cudaMemcpyAsync(ws.sizes.p, ws.h_sizes, sizeof(ChainSizes), cudaMemcpyHostToDevice, st));
        const uint32_t *d_L = small + kSmallPairs;  // min(L, cap), written on the device
        launch_clamp_pairs(small, kSmallTotal, kSmallPairs, kSmallOverflow, (const ChainSizes *)ws.sizes.p, st);
        {
            StageTimer t(pf, DGS_STAGE_EMIT, st);
            launch_emit((const uint32_t *)ws.offs.p, (const uint32_t *)ws.zval.p, (const short4 *)ws.rect.p, dv, V,
                        n, cap, (uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, st, nullptr, d_L);
        }
        {
            StageTimer t(pf, DGS_STAGE_TILE_SORT, st);
            radix_sort_pairs((uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, cap, bits, sort_scratch_of(ws), st, d_L);
        }
        {
            StageTimer t(pf, DGS_STAGE_TILE_RANGES, st);
            CK(cudaMemsetAsync(ws.ranges.p, 0, 8 * (size_t)std::max(1, ws.total_tiles), st));
            launch_tile_ranges((const uint32_t *)ws.tkey.p, cap, (uint2 *)ws.ranges.p, st, d_L);
        }
        CK(cudaGetLastError());
        ws.async_pending = true;
        return DGS_OK;
    }
    CK(cudaMemcpyAsync(ws.h_small, small, 64, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ws.h_small[kSmallSortErr]) return set_error(DGS_ERR_TIMEOUT, "radix sort look-back wait gave up");
    const long long L = ws.h_small[kSmallTotal];
    ws.L = L;
    ws.n_vis = ws.h_small[kSmallVisible];
    if (ws.total_tiles > 0) ctx->pairs_per_tile = std::max(ctx->pairs_per_tile, (double)L / ws.total_tiles);
    if ((s = ws.tkey.ensure(4 * std::max(1LL, L))) || (s = ws.tval.ensure(4 * std::max(1LL, L)))) return s;
    if ((s = ensure_sort_scratch(ws, L))) return s;
    if ((s = ws.ranges.ensure(8 * (size_t)std::max(1, ws.total_tiles)))) return s;
    {
        StageTimer t(pf, DGS_STAGE_EMIT, st);
        launch_emit((const uint32_t *)ws.offs.p, (const uint32_t *)ws.zval.p, (const short4 *)ws.rect.p, dv, V, n, L,
                    (uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, st);
    }
    {
        StageTimer t(pf, DGS_STAGE_TILE_SORT, st);
        radix_sort_pairs((uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, L, bits, sort_scratch_of(ws), st);
    }
    {
        StageTimer t(pf, DGS_STAGE_TILE_RANGES, st);
        CK(cudaMemsetAsync(ws.ranges.p, 0, 8 * (size_t)std::max(1, ws.total_tiles), st));
        launch_tile_ranges((const uint32_t *)ws.tkey.p, L, (uint2 *)ws.ranges.p, st);
    }
    CK(cudaGetLastError());
    return DGS_OK;
}

dgs_status chain_forward(dgs_ctx *ctx, Workspace &ws, const std::vector<ChainView> &req, float *out_img,
                         bool keep_rgb, bool grad_buffers, cudaStream_t st, bool device_sized) {
    const int V = (int)req.size();
    ws.V = V;
    ws.hviews.clear();
    ws.scene_ids.clear();
    std::vector<const Scene *> slots;
    int tiles = 0;
    long long px = 0, cell_base = 0, rec_base = 0;
    for (int v = 0; v < V; ++v) {
        auto it = ctx->scenes.find(req[v].scene_id);
        if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
        int slot = -1;
        for (size_t k = 0; k < ws.scene_ids.size(); ++k)
            if (ws.scene_ids[k] == req[v].scene_id) slot = (int)k;
        if (slot < 0) {
            slot = (int)ws.scene_ids.size();
            ws.scene_ids.push_back(req[v].scene_id);
            slots.push_back(it->second.get());
        }
        const Scene &sc = *it->second;
        ws.hviews.push_back(make_view(req[v].cam, tiles, px, slot, sc, cell_base, rec_base));
        ws.hviews.back().out = req[v].out;
        tiles += ws.hviews.back().Tx * ws.hviews.back().Ty;
        px += (long long)req[v].cam.W * req[v].cam.H;
        cell_base += sc.N;
        rec_base += sc.G;
    }
    if (cell_base >= (1LL << 32) - 1) return set_error(DGS_ERR_CAPACITY, "views x cells exceeds 2^32");
    ws.total_tiles = tiles;
    ws.total_px = px;
    ws.n_entries = cell_base;
    ws.n_records = rec_base;
    const int S = (int)slots.size();
    dgs_status s;
    if ((s = ws.views.ensure(sizeof(ViewDesc) * V)) || (s = ws.scenes.ensure(sizeof(SceneDev) * S))) return s;
    if (ws.h_views_cap < (size_t)V) {
        if (ws.h_views) cudaFreeHost(ws.h_views);
        ws.h_views = nullptr;
        CK(cudaMallocHost(&ws.h_views, sizeof(ViewDesc) * V));
        ws.h_views_cap = V;
    }
    if (ws.h_scenes_cap < (size_t)S) {
        if (ws.h_scenes) cudaFreeHost(ws.h_scenes);
        ws.h_scenes = nullptr;
        CK(cudaMallocHost(&ws.h_scenes, sizeof(SceneDev) * S));
        ws.h_scenes_cap = S;
    }
    memcpy(ws.h_views, ws.hviews.data(), sizeof(ViewDesc) * V);
    for (int k = 0; k < S; ++k) ws.h_scenes[k] = slots[k]->dev();
    CK(cudaMemcpyAsync(ws.views.p, ws.h_views, sizeof(ViewDesc) * V, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws.scenes.p, ws.h_scenes, sizeof(SceneDev) * S, cudaMemcpyHostToDevice, st));
    if ((s = run_binning(ctx, ws, st, device_sized))) return s;
    const BlendParams bp = blend_params(ctx->cfg);
    const long long nrec = std::max(1LL, ws.n_records), px1 = std::max(1LL, px);
    bool any_neural = false;
    for (const Scene *sc : slots) any_neural = any_neural || sc->F > 0;
    // the decode's samples: the visible (view, cell) entries, counted on the
    // device (a device-sized chain knows only their capacity on the host)
    const long long n_samp = device_sized ? ws.n_entries : ws.n_vis;
    long long npk = 0;
    for (const Scene *sc : slots)
        if (sc->F > 0) npk = std::max(npk, decode_scratch_floats(sc->F, sc->H, sc->K, n_samp, sc->G, false));
    if ((any_neural && (s = ws.dec.ensure(sizeof(float) * kDecF * nrec))) ||
        (any_neural && (s = ws.wpack.ensure(sizeof(float) * npk))) ||
        (s = ws.rec.ensure(sizeof(float4) * kRecF4 * nrec)) ||
        (grad_buffers && (s = ws.g2d.ensure(sizeof(float) * kGradF * nrec))) || (s = ws.Dpix.ensure(4 * px1)) ||
        (s = ws.ndpix.ensure(4 * px1)) || ((keep_rgb || !out_img) && (s = ws.rgb.ensure(12 * px1))))
        return s;
    const ViewDesc *dv = (const ViewDesc *)ws.views.p;
    for (int k = 0; k < S; ++k) {
        const SceneDev sd = slots[k]->dev();
        if (slots[k]->F > 0) {  // neural cells: decode the visible cells' Gaussians for every view first
            // the decode writes the records too (the projection fused into it)
            StageTimer t(ctx->prof, DGS_STAGE_DECODE, st);
            launch_decode(dv, V, k, sd, (const uint32_t *)ws.zval.p, n_samp,
                          (const uint32_t *)ws.small.p + kSmallVisible, (float *)ws.dec.p, (float *)ws.wpack.p, (const float *)ws.vview.p, bp, (float4 *)ws.rec.p,
                          grad_buffers ? (float *)ws.g2d.p : nullptr, (uint32_t *)ws.small.p + kSmallTcErr, st);
            ws.check_tc = true;
        } else {
            StageTimer t(ctx->prof, DGS_STAGE_PROJECT_FWD, st);
            launch_project_fwd(dv, V, k, sd, (const uint32_t *)ws.count.p, (const float *)ws.vview.p, bp,
                               (float4 *)ws.rec.p, grad_buffers ? (float *)ws.g2d.p : nullptr, st);
        }
    }
    float *img = out_img ? out_img : (float *)ws.rgb.p;
    float *img2 = (keep_rgb && out_img) ? (float *)ws.rgb.p : nullptr;
    {
        StageTimer t(ctx->prof, DGS_STAGE_BLEND_FWD, st);
        int K_all = slots[0]->K;
        for (int k = 1; k < S; ++k)
            if (slots[k]->K != K_all) K_all = 0;
        launch_blend_fwd(dv, V, ws.total_tiles, (const uint2 *)ws.ranges.p, (const uint32_t *)ws.tval.p,
                         (const float4 *)ws.rec.p, bp, img, img2, (float *)ws.Dpix.p, (int *)ws.ndpix.p, K_all, st);
    }
    CK(cudaGetLastError());
    if (device_sized || ws.check_tc)  // the chain's sizes and flags, read once it has completed (observe_chain)
        CK(cudaMemcpyAsync(ws.h_small, ws.small.p, 64, cudaMemcpyDeviceToHost, st));
    ws.stream = st;
    return DGS_OK;
}

static dgs_status render_impl(dgs_ctx *ctx, uint32_t scene_id, int n_views, const uint32_t *cam_slots, float *out_rgb,
                              int out_location, dgs_fwd_state **state, cudaStream_t st, dgs_stats *stats) {
    if (n_views <= 0 || !cam_slots || !out_rgb) return set_error(DGS_ERR_INVALID_ARG, "need n_views > 0, cams, output");
    if (out_location != DGS_HOST && out_location != DGS_DEVICE) return set_error(DGS_ERR_INVALID_ARG, "bad location");
    if (!ctx->scenes.count(scene_id)) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
    std::vector<ChainView> req;
    for (int v = 0; v < n_views; ++v) {
        if (cam_slots[v] >= (uint32_t)kMaxCamSlots || !ctx->cam_set[cam_slots[v]])
            return set_error(DGS_ERR_NOT_FOUND, "camera slot not set");
        req.push_back({scene_id, ctx->cams[cam_slots[v]]});
    }
    dgs_status s;
    std::unique_ptr<Workspace> ws = acquire_ws(ctx, st, &s);
    if (!ws) return s;
    if (ctx->pending_status) {  // a completed earlier render overflowed (or its sort gave up)
        s = set_error(ctx->pending_status, ctx->pending_msg);
        ctx->pending_status = DGS_OK;
        ctx->pool.push_back(std::move(ws));
        return s;
    }
    // No host synchronisation unless stats are asked for or this context has
    // not rendered yet (no pairs-per-tile estimate to size the pair buffers);
    // a neural scene's decode reads its visible-cell count on the device.
    const bool device_sized = !stats && ctx->pairs_per_tile > 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timing = stats && stats->timing;
    if (timing) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    const bool keep = state != nullptr;
    s = chain_forward(ctx, *ws, req, out_location == DGS_DEVICE ? out_rgb : nullptr, keep, keep, st,
                      device_sized && out_location == DGS_DEVICE);
    if (!s && out_location == DGS_HOST) {
        cudaError_t e = cudaMemcpyAsync(out_rgb, ws->rgb.p, 12 * ws->total_px, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "copying the image to host memory");
    }
    if (timing) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&stats->ms_total, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (stats && !s) {
        stats->sort_length = ws->L;
        stats->num_tiles = ws->total_tiles;
        stats->visible_cells = ws->h_small[kSmallVisible];
    }
    cudaEventRecord(ws->done, st);
    if (s || !keep) {
        ctx->pool.push_back(std::move(ws));
        return s;
    }
    auto *fs = new dgs_fwd_state();
    fs->ws = std::move(ws);
    fs->scene_id = scene_id;
    ctx->live_states.insert(fs);
    *state = fs;
    return DGS_OK;
}

}  // namespace dgs

extern "C" dgs_status dgs_render(dgs_ctx *ctx, uint32_t scene_id, int32_t n_views, const uint32_t *cam_slots,
                                 float *out_rgb, int32_t out_location, dgs_fwd_state **state, dgs_stream stream,
                                 dgs_stats *stats) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    if (state) *state = nullptr;
    return render_impl(ctx, scene_id, n_views, cam_slots, out_rgb, out_location, state, (cudaStream_t)stream, stats);
}

extern "C" dgs_status dgs_render_backward(dgs_ctx *ctx, dgs_fwd_state *state, const float *dL_drgb, int32_t location,
                                          const dgs_grads *out, dgs_stream stream) {
    if (!ctx || !state || !dL_drgb || !out) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    if ((location != DGS_HOST && location != DGS_DEVICE) || (out->location != DGS_HOST && out->location != DGS_DEVICE))
        return set_error(DGS_ERR_INVALID_ARG, "bad location");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    if (!ctx->live_states.count(state)) return set_error(DGS_ERR_NOT_FOUND, "unknown or released forward state");
    auto it = ctx->scenes.find(state->scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "scene of this state was released");
    const Scene &sc = *it->second;
    const bool neural = sc.F > 0;
    if (neural && (out->g_mean || out->g_scale || out->g_log_scale || out->g_quat || out->g_logit || out->g_sh))
        return set_error(DGS_ERR_INVALID_ARG, "a neural scene has no explicit Gaussian parameters to differentiate");
    if (!neural && (out->g_mlp || out->g_feat || out->g_offset))
        return set_error(DGS_ERR_INVALID_ARG, "g_mlp, g_feat and g_offset need a neural scene");
    Workspace &ws = *state->ws;
    cudaStream_t st = (cudaStream_t)stream;
    dgs_status s;
    if ((s = observe_chain(ctx, ws, false))) return s;
    if (ctx->pending_status) {  // this state's render, or an earlier one, overflowed (see dgs_render)
        s = set_error(ctx->pending_status, ctx->pending_msg);
        ctx->pending_status = DGS_OK;
        return s;
    }
    CK(cudaStreamWaitEvent(st, ws.done, 0));
    const long long px = ws.total_px, G = sc.G, N = sc.N;
    const int C = sc.C, Cv = sc.Cv;
    if (out->g_cell_v_sh && sc.vdeg < 0)
        return set_error(DGS_ERR_INVALID_ARG, "g_cell_v_sh given for a scene without view-dependent v");
    // Host memory: mapped arrays are read (dL/drgb, by the blend adjoint) or
    // written (the explicit Gaussians' gradients, by the projection adjoint)
    // by the kernels over the host link; the others are staged in device
    // memory: dL/drgb (3 px), then the gradient outputs, copied at the end.
    const bool hin = location == DGS_HOST, hout = out->location == DGS_HOST;
    const float *dl_mapped = hin ? (const float *)mapped_host(dL_drgb) : nullptr;
    struct Out { float *user; long long n; bool direct; float *dev; };
    const long long P = neural ? neural_weights(sc) : 0, NF = neural ? N * sc.F : 0, GO = neural ? 3 * G : 0;
    Out o[] = {{out->g_mean, 3 * G, true, nullptr},     {out->g_scale, 3 * G, true, nullptr},
               {out->g_log_scale, 3 * G, true, nullptr}, {out->g_quat, 4 * G, true, nullptr},
               {out->g_logit, G, true, nullptr},         {out->g_sh, 3LL * C * G, true, nullptr},
               {out->g_cell_v, N, false, nullptr},       {out->g_cell_v_sh, (long long)Cv * N, false, nullptr},
               {out->g_mlp, P, false, nullptr},          {out->g_feat, NF, false, nullptr},
               {out->g_offset, GO, false, nullptr},      {out->g_cell_center, 3 * N, false, nullptr},
               {out->g_cell_axes, 3 * N, false, nullptr}, {out->g_cell_quat, 4 * N, false, nullptr}};
    long long n_stage = (hin && !dl_mapped ? 3 * px : 0) + 1;
    for (auto &q : o) {
        if (!q.user) continue;
        if (!hout) { q.dev = q.user; continue; }
        if (q.direct) q.dev = (float *)mapped_host(q.user);
        if (!q.dev) { q.direct = false; n_stage += q.n; }
    }
    if ((s = ws.gstage.ensure(sizeof(float) * n_stage))) return s;
    float *stage = (float *)ws.gstage.p;
    const float *dl = dL_drgb;
    if (hin) {
        if (dl_mapped) {
            dl = dl_mapped;
        } else {
            CK(cudaMemcpyAsync(stage, dL_drgb, 12 * px, cudaMemcpyHostToDevice, st));
            dl = stage;
            stage += 3 * px;
        }
    }
    for (auto &q : o)
        if (q.user && !q.dev) { q.dev = stage; stage += q.n; }
    float *o_mean = o[0].dev, *o_s = o[1].dev, *o_ls = o[2].dev, *o_q = o[3].dev, *o_lg = o[4].dev,
          *o_sh = o[5].dev, *o_v = o[6].dev, *o_vsh = o[7].dev, *o_mlp = o[8].dev, *o_f = o[9].dev,
          *o_off = o[10].dev, *o_cc = o[11].dev, *o_ca = o[12].dev, *o_cq = o[13].dev;
    // the cell gradients are sums of several kernels' contributions
    if (o_cc) CK(cudaMemsetAsync(o_cc, 0, sizeof(float) * 3 * N, st));
    if (o_ca) CK(cudaMemsetAsync(o_ca, 0, sizeof(float) * 3 * N, st));
    if (o_cq) CK(cudaMemsetAsync(o_cq, 0, sizeof(float) * 4 * N, st));
    // dL/dv per (view, cell) entry, chained to the outputs after the blend adjoint
    float *gv = nullptr;
    if (o_v || o_vsh || (o_cc && sc.vdeg >= 0)) {
        if ((s = ws.gvview.ensure(sizeof(float) * std::max(1LL, ws.n_entries)))) return s;
        gv = (float *)ws.gvview.p;
        CK(cudaMemsetAsync(gv, 0, sizeof(float) * ws.n_entries, st));
    }
    const BlendParams bp = blend_params(ctx->cfg);
    if (ws.bwd_done) {  // a second backward on the same state: clear the screen-space accumulators
        CK(cudaMemsetAsync(ws.g2d.p, 0, sizeof(float) * kGradF * (size_t)ws.n_records, st));
    }
    {
        StageTimer t(ctx->prof, DGS_STAGE_BLEND_BWD, st);
        launch_blend_bwd((const ViewDesc *)ws.views.p, ws.V, ws.total_tiles, sc.K, (const uint2 *)ws.ranges.p,
                         (const uint32_t *)ws.tval.p, (const float4 *)ws.rec.p, bp, (const float *)ws.rgb.p,
                         (const float *)ws.Dpix.p, (const int *)ws.ndpix.p, dl, (float *)ws.g2d.p, gv, st);
        if (gv) launch_cell_v_grad((const ViewDesc *)ws.views.p, ws.V, sc.dev(), gv, o_v, o_vsh, o_cc, st);
    }
    if (neural && (o_mlp || o_f || o_off || o_cc || o_ca || o_cq)) {
        if ((s = ws.gdec.ensure(sizeof(float) * kDecF * std::max(1LL, ws.n_records)))) return s;
        // the decode adjoint forms every output; unrequested ones go to scratch after its rows
        // the samples as the forward counted them on the device (their count may not be on the host yet)
        const long long n_samp = ws.n_vis >= 0 ? ws.n_vis : ws.n_entries;
        if ((s = ws.gscratch.ensure(sizeof(float) * std::max(1LL, P + NF + GO))) ||
            (s = ws.wpack.ensure(sizeof(float) * decode_scratch_floats(sc.F, sc.H, sc.K, n_samp, G, true))))
            return s;
        float *gscr = (float *)ws.gscratch.p;
        float *m = o_mlp ? o_mlp : gscr, *f = o_f ? o_f : gscr + P, *off = o_off ? o_off : gscr + P + NF;
        {
            StageTimer t(ctx->prof, DGS_STAGE_PROJECT_BWD, st);
            launch_project_bwd_neural((const ViewDesc *)ws.views.p, ws.V, 0, sc.dev(), (const uint32_t *)ws.count.p,
                                      bp, (const float *)ws.dec.p, (const float *)ws.g2d.p, (float *)ws.gdec.p, st);
        }
        StageTimer t(ctx->prof, DGS_STAGE_DECODE_BWD, st);
        CK(cudaMemsetAsync(m, 0, sizeof(float) * P, st));
        CK(cudaMemsetAsync(f, 0, sizeof(float) * NF, st));
        CK(cudaMemsetAsync(off, 0, sizeof(float) * GO, st));
        launch_decode_bwd((const ViewDesc *)ws.views.p, ws.V, 0, sc.dev(), (const uint32_t *)ws.zval.p, n_samp,
                          (const uint32_t *)ws.small.p + kSmallVisible, (const float *)ws.gdec.p, m, f, off,
                          CellGrads{o_cc, o_ca, o_cq}, (float *)ws.wpack.p, st);
    } else if (!neural) {
        StageTimer t(ctx->prof, DGS_STAGE_PROJECT_BWD, st);
        launch_project_bwd((const ViewDesc *)ws.views.p, ws.V, 0, sc.dev(), (const uint32_t *)ws.count.p, bp,
                           (const float *)ws.g2d.p, o_mean, o_s, o_ls, o_q, o_lg, o_sh, st);
    }
    CK(cudaGetLastError());
    ws.bwd_done = true;
    if (hin || hout) {
        for (auto &q : o)
            if (hout && q.user && q.n && !q.direct)
                CK(cudaMemcpyAsync(q.user, q.dev, sizeof(float) * q.n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));  // host arrays complete (and free again) on return
    }
    CK(cudaEventRecord(ws.done, st));
    return DGS_OK;
}

extern "C" dgs_status dgs_state_release(dgs_ctx *ctx, dgs_fwd_state *state) {
    if (!ctx || !state) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->live_states.count(state)) return set_error(DGS_ERR_NOT_FOUND, "unknown or released forward state");
    ctx->live_states.erase(state);
    state->ws->bwd_done = false;
    ctx->pool.push_back(std::move(state->ws));
    delete state;
    return DGS_OK;
}

extern "C" dgs_status dgs_state_read(dgs_ctx *ctx, const dgs_fwd_state *state, int32_t what, void *dst, int64_t bytes,
                                     int64_t *needed) {
    if (!ctx || !state) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    if (!ctx->live_states.count(const_cast<dgs_fwd_state *>(state)))
        return set_error(DGS_ERR_NOT_FOUND, "unknown or released forward state");
    auto it = ctx->scenes.find(state->scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "scene released");
    const Scene &sc = *it->second;
    Workspace &ws = *state->ws;
    dgs_status s = observe_chain(ctx, ws, true);  // L of a device-sized chain
    if (s) return s;
    const long long VN = ws.n_entries, VG = ws.n_records;
    (void)sc;
    int64_t need = 0;
    switch (what) {
        case DGS_BUF_CELL_RECT: need = 16 * VN; break;
        case DGS_BUF_CELL_DEPTH: need = 4 * VN; break;
        case DGS_BUF_TILE_CELLS: need = 4 * ws.L; break;
        case DGS_BUF_TILE_RANGES: need = 8LL * ws.total_tiles; break;
        case DGS_BUF_GAUSS_REC: need = 48 * VG; break;
        case DGS_BUF_PIX_D: need = 4 * ws.total_px; break;
        case DGS_BUF_PIX_NDONE: need = 4 * ws.total_px; break;
        case DGS_BUF_GRAD2D: need = ws.g2d.p ? 48 * VG : 0; break;
        case DGS_BUF_CELL_V: need = 4 * VN; break;
        case DGS_BUF_DECODED: need = ws.dec.p ? 4LL * kDecF * VG : 0; break;
        default: return set_error(DGS_ERR_INVALID_ARG, "unknown buffer id");
    }
    if (needed) *needed = need;
    if (!dst || bytes < need) return DGS_OK;
    CK(cudaEventSynchronize(ws.done));
    if (need == 0) return DGS_OK;
    if (what == DGS_BUF_CELL_RECT) {
        std::vector<short4> tmp(VN);
        CK(cudaMemcpy(tmp.data(), ws.rect.p, 8 * VN, cudaMemcpyDeviceToHost));
        int32_t *o = (int32_t *)dst;
        for (long long i = 0; i < VN; ++i) {
            o[4 * i] = tmp[i].x; o[4 * i + 1] = tmp[i].y; o[4 * i + 2] = tmp[i].z; o[4 * i + 3] = tmp[i].w;
        }
        return DGS_OK;
    }
    const void *src = nullptr;
    switch (what) {
        case DGS_BUF_CELL_DEPTH: src = ws.depth.p; break;
        case DGS_BUF_TILE_CELLS: src = ws.tval.p; break;
        case DGS_BUF_TILE_RANGES: src = ws.ranges.p; break;
        case DGS_BUF_GAUSS_REC: src = ws.rec.p; break;
        case DGS_BUF_PIX_D: src = ws.Dpix.p; break;
        case DGS_BUF_PIX_NDONE: src = ws.ndpix.p; break;
        case DGS_BUF_GRAD2D: src = ws.g2d.p; break;
        case DGS_BUF_CELL_V: src = ws.vview.p; break;
        case DGS_BUF_DECODED: src = ws.dec.p; break;
    }
    CK(cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost));
    return DGS_OK;
}

extern "C" dgs_status dgs_loss_l1(dgs_ctx *ctx, const float *rgb, const float *target, int64_t n, float *dL_drgb,
                                  float *loss, dgs_stream stream) {
    if (!ctx || !rgb || !target || !dL_drgb || !loss || n < 0) return set_error(DGS_ERR_INVALID_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    const int nb = loss_l1_blocks(n);
    dgs_status s = ctx->loss_partial.ensure(sizeof(float) * nb);
    if (s) return s;
    launch_loss_l1(rgb, target, n, dL_drgb, (float *)ctx->loss_partial.p, nb, loss, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return DGS_OK;
}

extern "C" dgs_status dgs_sort_pairs(dgs_ctx *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int32_t bits,
                                     dgs_stream stream) {
    if (!ctx || (n > 0 && (!keys || !vals)) || n < 0 || bits < 0 || bits > 32)
        return set_error(DGS_ERR_INVALID_ARG, "bad argument");
    if (n >= (1LL << 30)) return set_error(DGS_ERR_CAPACITY, "sort supports fewer than 2^30 items");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->sort_ws) {
        dgs_status e;
        ctx->sort_ws = acquire_ws(ctx, st, &e);
        if (!ctx->sort_ws) return e;
    }
    Workspace &ws = *ctx->sort_ws;
    dgs_status s;
    if ((s = ensure_sort_scratch(ws, n)) || (s = ws.small.ensure(256))) return s;
    CK(cudaMemsetAsync(ws.small.p, 0, 256, st));
    radix_sort_pairs(keys, vals, n, bits, sort_scratch_of(ws), st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ws.h_small, ws.small.p, 64, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ws.h_small[kSmallSortErr]) return set_error(DGS_ERR_TIMEOUT, "radix sort look-back wait gave up");
    return DGS_OK;
}

extern "C" dgs_status dgs_state_counts(dgs_ctx *ctx, const dgs_fwd_state *state, dgs_counts *out) {
    if (!ctx || !state || !out) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    if (!ctx->live_states.count(const_cast<dgs_fwd_state *>(state)))
        return set_error(DGS_ERR_NOT_FOUND, "unknown or released forward state");
    Workspace &ws = *state->ws;
    cudaStream_t st = ws.stream;
    dgs_status s = ctx->aux.ensure(64);
    if (s) return s;
    unsigned long long *c = (unsigned long long *)ctx->aux.p;
    CK(cudaStreamWaitEvent(st, ws.done, 0));
    CK(cudaMemsetAsync(c, 0, 32, st));
    launch_count_pairs((const ViewDesc *)ws.views.p, ws.V, ws.total_tiles, (const uint2 *)ws.ranges.p,
                       (const uint32_t *)ws.tval.p, (const float4 *)ws.rec.p, (const int *)ws.ndpix.p, c, st);
    CK(cudaGetLastError());
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, c, 32, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->pairs_blended = (int64_t)h[0];
    out->inbox_rendered = (int64_t)h[1];
    out->inbox_all = (int64_t)h[2];
    out->cells_blended = (int64_t)h[3];
    return DGS_OK;
}

extern "C" dgs_status dgs_profile_enable(dgs_ctx *ctx, int32_t on) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    ctx->prof.drain();
    for (int i = 0; i < 16; ++i) {
        ctx->prof.ms[i] = 0.0;
        ctx->prof.launches[i] = 0;
    }
    ctx->prof.on = on != 0;
    return DGS_OK;
}

extern "C" dgs_status dgs_profile_read(dgs_ctx *ctx, dgs_profile *out) {
    if (!ctx || !out) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    ctx->prof.drain();
    for (int i = 0; i < 16; ++i) {
        out->ms[i] = ctx->prof.ms[i];
        out->launches[i] = ctx->prof.launches[i];
    }
    return DGS_OK;
}

// ---------------------------------------------------------------- debugging and faults
extern "C" dgs_status dgs_debug_guards(int32_t on) {
    g_guards.store(on ? 1 : 0);
    return DGS_OK;
}

extern "C" dgs_status dgs_debug_check_guards(int64_t *n_checked) {
    int cur = 0;
    cudaGetDevice(&cur);
    std::lock_guard<std::mutex> lk(g_guard_mu);
    std::set<int> synced;
    std::vector<unsigned char> h(kGuardBytes);
    int64_t n = 0;
    std::string bad;
    cudaError_t e = cudaSuccess;
    for (const DevBuf *b : g_guarded) {
        e = cudaSetDevice(b->dev);
        if (e == cudaSuccess && synced.insert(b->dev).second) e = cudaDeviceSynchronize();
        const char *base = static_cast<const char *>(b->p);
        for (int side = 0; side < 2 && e == cudaSuccess; ++side) {
            const char *g = side == 0 ? base - kGuardBytes : base + b->cap;
            e = cudaMemcpy(h.data(), g, kGuardBytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess || !bad.empty()) continue;
            for (size_t i = 0; i < kGuardBytes; ++i) {
                if (h[i] == kGuardByte) continue;
                bad = "guard word changed next to a device buffer of " + std::to_string(b->cap) + " bytes (device " +
                      std::to_string(b->dev) + "): byte " +
                      (side == 0 ? std::to_string(kGuardBytes - i) + " before its start"
                                 : std::to_string(i) + " after its end");
                break;
            }
        }
        if (e != cudaSuccess) break;
        ++n;
    }
    cudaSetDevice(cur);
    if (n_checked) *n_checked = n;
    if (e != cudaSuccess) return cuda_error(e, "reading guard words");
    return bad.empty() ? DGS_OK : set_error(DGS_ERR_GUARD, bad);
}

extern "C" dgs_status dgs_debug_inject_fault(dgs_ctx *ctx, int32_t kind, int32_t count) {
    if (count < 0) return set_error(DGS_ERR_INVALID_ARG, "count must be >= 0");
    switch (kind) {
        case DGS_FAULT_ALLOC:
            g_fail_allocs.store(count);
            return DGS_OK;
        case DGS_FAULT_SORT_WAIT: {
            if (ctx) CK(cudaSetDevice(ctx->cfg.device));
            CK(set_sort_fault(count != 0));
            return DGS_OK;
        }
        case DGS_FAULT_TC_WAIT: {
            if (ctx) CK(cudaSetDevice(ctx->cfg.device));
            CK(set_tc_fault(count != 0));
            return DGS_OK;
        }
        case DGS_FAULT_SERVE_WORKER:
            return serve_inject_fault(ctx, count);
        case DGS_FAULT_GUARD:
            g_corrupt_next.store(count);
            return DGS_OK;
        default:
            return set_error(DGS_ERR_INVALID_ARG, "unknown fault kind");
    }
}
