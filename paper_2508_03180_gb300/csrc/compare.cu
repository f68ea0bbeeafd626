// Comparator renderers (the two models Duplex-GS is measured against, Sec.
// III-A; the paper's Tab. VI compares sort lengths): per-Gaussian
// alpha-blending over a global depth order (Eq. 2-3, vanilla 3DGS) and
// sort-free weighted-sum rendering (Eq. 4) with the LC-WSR weight (Eq. 5-6).
// They share the Duplex path's per-Gaussian record, AABB skip, colour, binning
// and radix sort; only the unit that is sorted (every Gaussian instead of
// every cell) and the blending differ.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "runtime.h"

namespace dgs {

constexpr int CT = 32;    // threads per work unit (one warp per 16x4 sub-tile)
constexpr int CSUB = 4;   // sub-tiles per tile

__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int view_of_tile(const ViewDesc *views, int n_views, int tile) {
    int lo = 0, hi = n_views;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

// One warp per 16x4-pixel sub-tile, two vertically adjacent pixels per lane.
// The tile's Gaussians are taken 32 at a time: each lane fetches one record
// into shared memory, a ballot keeps those whose AABB reaches the sub-tile,
// and the warp walks them in list order (depth order for alpha-blending).
//   ALPHA: C += T alpha c, T *= 1 - alpha; a pixel stops before the entry at
//          which T < eps (the cell rule of the hybrid renderer at K = 1);
//          out = C + T bg, out_nd = entries processed.
//   !ALPHA (weighted sums): A += alpha w c, B += alpha w over every entry;
//          out = (bg w_bg + A) / (w_bg + B), background if that denominator
//          is not above d_min.
template <bool ALPHA>
__global__ void __launch_bounds__(CT) k_gauss_blend(const ViewDesc *__restrict__ views, int n_views,
                                                    const uint2 *__restrict__ ranges,
                                                    const uint32_t *__restrict__ list,
                                                    const float4 *__restrict__ rec, BlendParams bp, float w_bg,
                                                    float *__restrict__ out_rgb, int *__restrict__ out_nd) {
    __shared__ float4 s_rec[CT][kRecF4];
    const int lane = threadIdx.x;
    const int tile = blockIdx.x / CSUB, sub = blockIdx.x % CSUB;
    const ViewDesc &V = views[view_of_tile(views, n_views, tile)];
    const int local = tile - V.tile_base;
    const int tx = local % V.Tx, ty = local / V.Tx;
    const float bx0 = (float)(tx * kTile), by0 = (float)(ty * kTile + CSUB * sub);
    const int xi = tx * kTile + (lane & (kTile - 1));
    const int yi0 = ty * kTile + CSUB * sub + 2 * (lane >> 4), yi1 = yi0 + 1;
    const bool in0 = xi < V.W && yi0 < V.H, in1 = xi < V.W && yi1 < V.H;
    const float px = (float)xi + 0.5f, py0 = (float)yi0 + 0.5f, py1 = (float)yi1 + 0.5f;
    const float4 *vrec = rec + V.rec_base * kRecF4;
    const uint2 rg = ranges[tile];
    const float lx = bx0 + 0.5f, hx = bx0 + (float)kTile - 0.5f;
    const float ly = by0 + 0.5f, hy = by0 + (float)CSUB - 0.5f;

    float C00 = 0.f, C01 = 0.f, C02 = 0.f, X0 = 0.f;  // X: T (alpha) or B (weighted sums)
    float C10 = 0.f, C11 = 0.f, C12 = 0.f, X1 = 0.f;
    if (ALPHA) X0 = X1 = 1.0f;
    int n0 = (int)(rg.y - rg.x), n1 = n0;
    bool done0 = !in0, done1 = !in1;
    for (uint32_t base = rg.x; base < rg.y; base += CT) {
        if (ALPHA && __all_sync(0xffffffffu, done0 && done1)) break;
        const uint32_t e = base + lane;
        bool hit = false;
        if (e < rg.y) {
            const float4 *src = vrec + (long long)__ldg(list + e) * kRecF4;
            const float4 r0 = __ldg(src);
            hit = !(lx - r0.x > r0.z || r0.x - hx > r0.z || ly - r0.y > r0.w || r0.y - hy > r0.w);
            if (hit) {
                s_rec[lane][0] = r0;
                s_rec[lane][1] = __ldg(src + 1);
                s_rec[lane][2] = __ldg(src + 2);
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, hit);
        __syncwarp();
        for (; mask; mask &= mask - 1) {
            const int k = __ffs(mask) - 1;
            const float4 r0 = s_rec[k][0];
            const float dx = px - r0.x;
            if (!(fabsf(dx) <= r0.z)) continue;
            const float dy0 = py0 - r0.y, dy1 = py1 - r0.y;
            const bool h0 = !done0 && fabsf(dy0) <= r0.w;
            const bool h1 = !done1 && fabsf(dy1) <= r0.w;
            if (!(h0 || h1)) continue;
            const float4 r1 = s_rec[k][1];
            const float4 r2 = s_rec[k][2];
            const float pdx = r1.x * dx;
            if (h0) {
                const float s1 = fmaf(r1.y, dy0, pdx), s2 = r1.z * dy0;
                const float al = fminf(r1.w * ex2_fast(-fmaf(s1, s1, s2 * s2)), bp.alpha_max);
                if (ALPHA) {
                    const float wt = X0 * al;
                    C00 += wt * r2.x; C01 += wt * r2.y; C02 += wt * r2.z;
                    X0 -= wt;
                    if (X0 < bp.eps) { done0 = true; n0 = (int)(base + k + 1 - rg.x); }
                } else {
                    const float aw = al * r2.w;
                    C00 += aw * r2.x; C01 += aw * r2.y; C02 += aw * r2.z;
                    X0 += aw;
                }
            }
            if (h1) {
                const float s1 = fmaf(r1.y, dy1, pdx), s2 = r1.z * dy1;
                const float al = fminf(r1.w * ex2_fast(-fmaf(s1, s1, s2 * s2)), bp.alpha_max);
                if (ALPHA) {
                    const float wt = X1 * al;
                    C10 += wt * r2.x; C11 += wt * r2.y; C12 += wt * r2.z;
                    X1 -= wt;
                    if (X1 < bp.eps) { done1 = true; n1 = (int)(base + k + 1 - rg.x); }
                } else {
                    const float aw = al * r2.w;
                    C10 += aw * r2.x; C11 += aw * r2.y; C12 += aw * r2.z;
                    X1 += aw;
                }
            }
        }
        __syncwarp();
    }
    const long long HW = (long long)V.W * V.H;
    float *img = V.out ? V.out : out_rgb + 3 * V.pix_base;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q == 0 ? in0 : in1)) continue;
        const long long pin = (long long)(q == 0 ? yi0 : yi1) * V.W + xi;
        const float X = q == 0 ? X0 : X1;
        float c0 = q == 0 ? C00 : C10, c1 = q == 0 ? C01 : C11, c2 = q == 0 ? C02 : C12;
        if (ALPHA) {
            c0 += X * bp.bg0; c1 += X * bp.bg1; c2 += X * bp.bg2;
            if (out_nd) out_nd[V.pix_base + pin] = q == 0 ? n0 : n1;
        } else {
            const float den = w_bg + X;
            const bool hit = den > bp.d_min;
            c0 = hit ? (bp.bg0 * w_bg + c0) / den : bp.bg0;
            c1 = hit ? (bp.bg1 * w_bg + c1) / den : bp.bg1;
            c2 = hit ? (bp.bg2 * w_bg + c2) / den : bp.bg2;
        }
        img[pin] = c0;
        img[HW + pin] = c1;
        img[2 * HW + pin] = c2;
    }
}

}  // namespace dgs

using namespace dgs;


namespace {

// The comparator's launch chain over views of one scene (caller holds ctx->mu).
dgs_status compare_chain(dgs_ctx *ctx, Workspace &ws, const Scene &sc, const std::vector<dgs_camera> &cams,
                         const dgs_compare_config &cfg, float *out_img, int *out_nd, cudaStream_t st) {
    const bool wsr = cfg.mode == DGS_COMPARE_WSR;
    const int V = (int)cams.size();
    std::vector<ViewDesc> hv;
    int tiles = 0;
    long long px = 0;
    for (int v = 0; v < V; ++v) {
        ViewDesc d = make_view(cams[v], tiles, px, 0, sc, (long long)v * sc.G, (long long)v * sc.G);
        d.N = sc.G;  // entries of this view: one per Gaussian
        d.K = 1;
        hv.push_back(d);
        tiles += d.Tx * d.Ty;
        px += (long long)cams[v].W * cams[v].H;
    }
    const long long n = (long long)V * sc.G;
    if (n >= (1LL << 32) - 1) return set_error(DGS_ERR_CAPACITY, "views x Gaussians exceeds 2^32");
    ws.V = V;
    ws.total_tiles = tiles;
    ws.total_px = px;
    ws.n_entries = n;
    ws.n_records = n;
    const long long n1 = std::max(1LL, n);
    dgs_status s;
    if ((s = ws.views.ensure(sizeof(ViewDesc) * V)) || (s = ws.small.ensure(256)) || (s = ws.zkey.ensure(4 * n1)) ||
        (s = ws.zval.ensure(4 * n1)) || (s = ws.rect.ensure(8 * n1)) || (s = ws.count.ensure(4 * n1)) ||
        (s = ws.cnt_sorted.ensure(4 * n1)) || (s = ws.offs.ensure(4 * n1)) ||
        (s = ws.scan.ensure(4 * scan_scratch_words(n1))) || (s = ensure_sort_scratch(ws, n)) ||
        (s = ws.rec.ensure(sizeof(float4) * kRecF4 * n1)) || (s = ws.ranges.ensure(8 * (size_t)std::max(1, tiles))))
        return s;
    if (ws.h_views_cap < (size_t)V) {
        if (ws.h_views) cudaFreeHost(ws.h_views);
        ws.h_views = nullptr;
        ws.h_views_cap = 0;
        CK(cudaMallocHost(&ws.h_views, sizeof(ViewDesc) * V));
        ws.h_views_cap = V;
    }
    memcpy(ws.h_views, hv.data(), sizeof(ViewDesc) * V);
    CK(cudaMemcpyAsync(ws.views.p, ws.h_views, sizeof(ViewDesc) * V, cudaMemcpyHostToDevice, st));
    uint32_t *small = (uint32_t *)ws.small.p;
    CK(cudaMemsetAsync(small, 0, 256, st));
    const ViewDesc *dv = (const ViewDesc *)ws.views.p;
    const BlendParams bp = blend_params(ctx->cfg);
    const float tau = std::isfinite(cfg.tau) && cfg.tau > 0.f ? cfg.tau : 0.f;
    launch_gauss_bin(dv, V, sc.dev(), bp, wsr, tau, (float4 *)ws.rec.p, (uint32_t *)ws.zkey.p, (uint32_t *)ws.zval.p,
                     (short4 *)ws.rect.p, (uint32_t *)ws.count.p, small + kSmallVisible, st);
    const uint32_t *counts = (const uint32_t *)ws.count.p;
    if (!wsr) {  // global depth order over every (view, Gaussian) entry
        radix_sort_pairs((uint32_t *)ws.zkey.p, (uint32_t *)ws.zval.p, n, 32, sort_scratch_of(ws), st);
        launch_gather_counts((const uint32_t *)ws.zval.p, counts, n, (uint32_t *)ws.cnt_sorted.p, st);
        counts = (const uint32_t *)ws.cnt_sorted.p;
    }  // weighted sums: entries stay in index order (zval is the identity)
    exclusive_scan_u32(counts, (uint32_t *)ws.offs.p, n, small + kSmallTotal, (uint32_t *)ws.scan.p, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ws.h_small, small, 64, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ws.h_small[kSmallSortErr]) return set_error(DGS_ERR_TIMEOUT, "radix sort look-back wait gave up");
    const long long L = ws.h_small[kSmallTotal];
    ws.L = L;
    if ((s = ws.tkey.ensure(4 * std::max(1LL, L))) || (s = ws.tval.ensure(4 * std::max(1LL, L))) ||
        (s = ensure_sort_scratch(ws, L)))
        return s;
    launch_emit((const uint32_t *)ws.offs.p, (const uint32_t *)ws.zval.p, (const short4 *)ws.rect.p, dv, V, n, L,
                (uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, st);
    int bits = 1;
    while ((1LL << bits) < tiles) ++bits;
    radix_sort_pairs((uint32_t *)ws.tkey.p, (uint32_t *)ws.tval.p, L, bits, sort_scratch_of(ws), st);
    CK(cudaMemsetAsync(ws.ranges.p, 0, 8 * (size_t)std::max(1, tiles), st));
    launch_tile_ranges((const uint32_t *)ws.tkey.p, L, (uint2 *)ws.ranges.p, st);
    if (tiles > 0) {
        const unsigned grid = (unsigned)tiles * CSUB;
        if (wsr)
            k_gauss_blend<false><<<grid, CT, 0, st>>>(dv, V, (const uint2 *)ws.ranges.p, (const uint32_t *)ws.tval.p,
                                                      (const float4 *)ws.rec.p, bp, cfg.w_bg, out_img, nullptr);
        else
            k_gauss_blend<true><<<grid, CT, 0, st>>>(dv, V, (const uint2 *)ws.ranges.p, (const uint32_t *)ws.tval.p,
                                                     (const float4 *)ws.rec.p, bp, 0.f, out_img, out_nd);
    }
    CK(cudaGetLastError());
    return DGS_OK;
}

}  // namespace

extern "C" dgs_status dgs_render_compare(dgs_ctx *ctx, uint32_t scene_id, int32_t n_views, const uint32_t *cam_slots,
                                         const dgs_compare_config *cfg, float *out_rgb, int32_t *out_ndone,
                                         dgs_stream stream, dgs_stats *stats) {
    if (!ctx || !cfg) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    if (n_views <= 0 || !cam_slots || !out_rgb) return set_error(DGS_ERR_INVALID_ARG, "need n_views > 0, cams, output");
    if (cfg->mode != DGS_COMPARE_ALPHA && cfg->mode != DGS_COMPARE_WSR)
        return set_error(DGS_ERR_INVALID_ARG, "unknown comparator mode");
    if (!(cfg->w_bg >= 0.f)) return set_error(DGS_ERR_INVALID_ARG, "w_bg must be >= 0");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
    if (it->second->F > 0) return set_error(DGS_ERR_INVALID_ARG, "the comparators take explicit Gaussians");
    std::vector<dgs_camera> cams;
    for (int v = 0; v < n_views; ++v) {
        if (cam_slots[v] >= (uint32_t)kMaxCamSlots || !ctx->cam_set[cam_slots[v]])
            return set_error(DGS_ERR_NOT_FOUND, "camera slot not set");
        cams.push_back(ctx->cams[cam_slots[v]]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    dgs_status s;
    std::unique_ptr<Workspace> ws = acquire_ws(ctx, st, &s);
    if (!ws) return s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timing = stats && stats->timing;
    if (timing) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    s = compare_chain(ctx, *ws, *it->second, cams, *cfg, out_rgb, out_ndone, st);
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
    ctx->pool.push_back(std::move(ws));
    return s;
}
