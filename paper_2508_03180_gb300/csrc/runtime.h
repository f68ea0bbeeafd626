// Host-side runtime objects of the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dgs.h"
#include "internal.cuh"

namespace dgs {

constexpr int kMaxCamSlots = 4096;
// words of the per-workspace "small" device block (and its pinned mirror)
constexpr int kSmallTotal = 0;    // sort length L
constexpr int kSmallSortErr = 1;  // a radix-sort look-back wait gave up
constexpr int kSmallVisible = 2;  // (view, cell) pairs that survived culling
constexpr int kSmallPairs = 3;    // L clamped to the pair capacity (captured chains)
constexpr int kSmallOverflow = 4; // L exceeded the pair capacity (captured chains)
constexpr int kSmallWork = 5;     // work counter of the pulling blend (captured chains)
constexpr int kSmallTcErr = 6;    // a tensor-core product's completion wait gave up (decode)

dgs_status set_error(dgs_status code, const std::string &msg);
dgs_status cuda_error(cudaError_t e, const char *what);

// Returns the recorded error status from the enclosing ABI function when a
// CUDA call fails.
#define CK(x)                                                 \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_error(e_, #x);     \
    } while (0)

// Grow-only device allocation.  In debug mode (dgs_debug_guards) the
// allocation is padded by guard words on both sides (`guarded`, `dev`).
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    bool guarded = false;
    int dev = 0;
    dgs_status ensure(size_t bytes);
    void release();
    ~DevBuf() { release(); }
};

// A resident scene: parameters as structure-of-arrays planes in HBM.
struct Scene {
    int64_t N = 0, G = 0;
    int K = 1, deg = 0, C = 1;
    int vdeg = -1, Cv = 0;  // SH degree / coefficients of a view-dependent v_n (-1: scalar v_n)
    int F = 0, H = 0;       // neural cells: feature width, hidden width (0: explicit Gaussians)
    DevBuf cell, gauss, sh, vsh;
    DevBuf feat, goff, mlp; // neural cells: [F][N] features, [3][G] offsets, packed decoder weights
    SceneDev dev() const;
};

// One view of a launch chain, as requested.
struct ChainView {
    uint32_t scene_id;
    dgs_camera cam;
    float *out = nullptr;  // device destination of this view's image (NULL = chain buffer)
};

// Buffers of one launch chain (a render, or a serving batch).  A forward
// state owns its workspace until released; otherwise workspaces go back to
// a pool and are reused once their `done` event has fired.
struct Workspace {
    DevBuf views, scenes;
    DevBuf zkey, zval, rect, depth, count, cnt_sorted, offs;  // per (view, cell)
    DevBuf tkey, tval;                                       // per (tile, cell) pair
    DevBuf ranges;                                           // per tile
    DevBuf rec, g2d;                                         // per (view, Gaussian)
    DevBuf Dpix, ndpix, rgb;                                 // per pixel
    DevBuf gstage;                                           // backward staging
    DevBuf sort_k, sort_v, sort_hist, sort_status, sort_ctr, small, scan;
    DevBuf vview, gvview;         // per (view, cell): v_n as rendered, dL/dv_n
    DevBuf dec;                   // per (view, Gaussian) of neural scenes: decoded values
    DevBuf gdec;                  // and dL/d of them in the backward
    DevBuf wpack;                 // decoder weights repacked for the decode kernels
    DevBuf gscratch;              // sink of the decode adjoint's unrequested outputs
    DevBuf sizes;                 // ChainSizes of a captured chain
    uint32_t *h_small = nullptr;  // pinned mirror of `small`
    ChainSizes *h_sizes = nullptr;
    ViewDesc *h_views = nullptr;
    size_t h_views_cap = 0;
    SceneDev *h_scenes = nullptr;
    size_t h_scenes_cap = 0;
    cudaEvent_t done = nullptr;
    cudaStream_t stream = 0;
    // description of the last chain
    std::vector<ViewDesc> hviews;
    std::vector<uint32_t> scene_ids;  // slot -> scene id
    int V = 0, total_tiles = 0;
    long long total_px = 0, L = 0, n_entries = 0, n_records = 0;
    long long n_vis = 0;  // (view, cell) entries that survived culling: the first n_vis of zval after the depth sort
    bool bwd_done = false;
    // A device-sized chain (dgs_render without stats): the pair count L lives
    // on the device only (pair buffers sized L_cap), and L, n_vis and the
    // chain's flags are read from h_small once it has completed (observe_chain).
    bool async_pending = false;
    bool check_tc = false;  // the chain ran tensor-core kernels: observe their wait flag once it completes
    long long L_cap = 0;
    dgs_status init();
    std::vector<DevBuf *> all();
    ~Workspace();
};

dgs_status ensure_sort_scratch(Workspace &ws, long long n);
SortScratch sort_scratch_of(Workspace &ws);
BlendParams blend_params(const dgs_config &c);

// ---------------------------------------------------------------- serving
struct PendingReq {
    uint64_t ticket;
    dgs_request req;
    double t_submit;
    int64_t bytes;  // admission estimate
};

// Capacities of a serving chain slot.  Every buffer of the slot's workspace
// is sized for them, so its captured graphs stay valid until one grows.
struct ChainCaps {
    int V = 0, S = 0;
    long long E = 0, R = 0, T = 0, P = 0, L = 0;
    long long G = 0;  // Gaussians of the largest scene (sizes the projection grid)
    long long W = 0;  // decode scratch floats (neural scenes resident; 0: none)
};

// One stream's serving chain: a workspace sized for `caps` and one
// instantiated graph of the whole forward chain per Gaussians-per-cell class
// of the batch (K = 8, 10 or mixed pick the blend's specialisation).  Scenes,
// views and every size are read from device memory when the graph runs.
struct GraphSlot {
    std::unique_ptr<Workspace> ws;
    ChainCaps caps;
    long long view_tiles = 0, view_px = 0;  // largest view seen
    long long L_need = 0;                   // pairs of the last overflowing batch, with headroom
    uint64_t scene_epoch = 0;
    // per batch class: the K specialisation, then (slot, scene id) of each
    // neural scene (its decode launches are part of the graph)
    std::map<std::vector<uint32_t>, cudaGraphExec_t> graphs;
    void drop();
    ~GraphSlot() { drop(); }
};

struct InflightBatch {
    std::unique_ptr<Workspace> ws;  // non-graph chains only
    std::vector<PendingReq> reqs;
    int stream_idx = 0;
    double t_start = 0;
    int64_t bytes = 0;
    dgs_status status = DGS_OK;
    bool graph = false;             // ran as a replay of a captured chain
};

constexpr int kServeStreams = 2;  // launch chains in flight at once

struct ServeState {
    std::thread worker;
    bool stop = false;
    int max_batch = 8, queue_cap = 1024;
    std::mutex m;                           // guards everything below
    std::condition_variable cv_work, cv_done;
    std::deque<PendingReq> pending;
    std::unordered_map<uint64_t, dgs_result> finished;
    std::set<uint64_t> open;                // submitted and not yet consumed by poll
    std::set<uint64_t> cancelled;           // admitted requests cancelled while their batch ran
    uint64_t next_ticket = 1;
    int64_t reserved = 0;                   // admission estimates of batches in flight
    int64_t budget = 0;
    cudaStream_t streams[kServeStreams] = {};
    cudaEvent_t events[kServeStreams] = {};
    bool busy[kServeStreams] = {};
    bool use_graphs = true;
    bool gpu_signal = false;                // a chain completed since the worker last looked
    uint64_t submits = 0;                   // requests accepted so far
    GraphSlot gslot[kServeStreams];
    double pairs_per_tile = 128.0;          // running estimate that sizes the pair buffers
    int64_t graphs_captured = 0, batches = 0, overflow_retries = 0;
    InflightBatch slot[kServeStreams];      // the worker's batches in flight (worker thread only)
    int inject_fault = 0;                   // test-only: raise a host-side fault at the next admission
    bool dead = false;                      // the worker stopped after a host-side fault
    std::string dead_msg;
};

// Test-only: arm a host-side fault in ctx's serving worker (dgs_debug_inject_fault).
dgs_status serve_inject_fault(dgs_ctx *ctx, int count);

}  // namespace dgs

struct dgs_fwd_state {
    std::unique_ptr<dgs::Workspace> ws;
    uint32_t scene_id = 0;
};

namespace dgs {
// Per-stage event profiling (dgs_profile_enable / dgs_profile_read).
struct Profiler {
    bool on = false;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> spare;
    double ms[16] = {};
    int64_t launches[16] = {};
    cudaEvent_t take();
    void drain();
    ~Profiler();
};
// RAII bracket of one stage on stream st (no-op when profiling is off).
struct StageTimer {
    Profiler &p;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageTimer(Profiler &p_, int s, cudaStream_t st_);
    ~StageTimer();
};
}  // namespace dgs

struct dgs_ctx {
    dgs_config cfg;
    dgs::Profiler prof;
    std::mutex mu;  // serialises every ABI call (and the serving worker's launches)
    std::map<uint32_t, std::unique_ptr<dgs::Scene>> scenes;
    uint32_t next_scene = 1;
    std::vector<dgs_camera> cams;
    std::vector<uint8_t> cam_set;
    std::vector<std::unique_ptr<dgs::Workspace>> pool;
    std::set<dgs_fwd_state *> live_states;
    dgs::DevBuf aux, loss_partial;
    dgs::DevBuf align_tmp;  // dgs_cell_align: one view's decode and host staging
    std::unique_ptr<dgs::Workspace> sort_ws;
    std::unique_ptr<dgs::ServeState> serve;
    uint64_t scene_epoch = 0;  // bumped when a scene's buffers go away
    double pairs_per_tile = 0.0;         // largest (tile, cell) pairs per tile seen: sizes device-sized chains
    dgs_status pending_status = DGS_OK;  // error of a completed device-sized chain, for the next render / backward
    std::string pending_msg;
};

namespace dgs {
std::unique_ptr<Workspace> acquire_ws(dgs_ctx *ctx, cudaStream_t st, dgs_status *err);
// Forward launch chain over views of one or more resident scenes (caller
// holds ctx->mu).  Writes the images to out_img (device, [3][H][W] per view
// back to back) and, if keep_rgb, also to ws.rgb.  grad_buffers: allocate and
// zero the screen-space gradient accumulators for a later backward.
// device_sized: no host synchronisation; the (tile, cell) pair buffers are
// sized from ctx->pairs_per_tile and the kernels read the pair count from
// device memory (see observe_chain).
dgs_status chain_forward(dgs_ctx *ctx, Workspace &ws, const std::vector<ChainView> &views, float *out_img,
                         bool keep_rgb, bool grad_buffers, cudaStream_t st, bool device_sized = false);
// Read a device-sized chain's sizes and flags once it has completed (wait:
// block until then; otherwise look only if it has).  A pair overflow or a
// sort that gave up becomes ctx->pending_status.
dgs_status observe_chain(dgs_ctx *ctx, Workspace &ws, bool wait);
ViewDesc make_view(const dgs_camera &c, int tile_base, long long pix_base, int slot, const Scene &sc,
                   long long cell_base, long long rec_base);
}  // namespace dgs
