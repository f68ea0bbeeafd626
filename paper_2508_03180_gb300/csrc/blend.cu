// Physical weighted-sum blend (Layer II, Sec. V) and its adjoint.
//
// Per pixel, the tile's cells are walked front to back (the order of the
// cell sort).  For cell n with Gaussians k:
//     A_n = sum_k alpha_k c_k,  B_n = sum_k alpha_k,  P_n = prod_k (1 - v_n alpha_k)
//     N += v_n T_n A_n,  D += v_n T_n B_n,  T_{n+1} = T_n P_n          (Eq. 12-14)
// and the pixel is C = N / D.  Before cell n the pixel stops if T_n < eps
// (cell-level early termination, Sec. V-B).  alpha_k = min(sigma G'(x'),
// alpha_max) and is 0 when the pixel lies outside the Gaussian's AABB
// (false-positive skip, Sec. VI-A).  Inside a cell nothing depends on the
// order of k (Eq. 12's inner sums and product commute).
//
// GB300 mapping: one one-warp CTA per 16x8 half of a 16x16 tile, four
// pixels per lane in packed pairs (f32x2 arithmetic).  The 48-byte records of
// a cell's Gaussians are copied into the warp's shared memory asynchronously
// two cells ahead and broadcast from there to the warp's 128 pixels.
#include <algorithm>

#include "internal.cuh"

namespace dgs {

constexpr int BT = 256;
constexpr float LN2 = 0.6931471805599453f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int find_view(const ViewDesc *views, int n_views, int tile) {
    int lo = 0, hi = n_views;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

// Work unit: one warp (a one-warp CTA) per 16 x (2 PPL)-pixel sub-tile of a
// tile.  Warps never wait for one another: each stages the records of its
// tile's cells in its own shared memory, takes a ballot of a cell's Gaussians
// whose AABB reaches its sub-tile and loops over those only, and stops as soon
// as its own pixels are done.  KT > 0 fixes K at compile time.
constexpr int WT = 32;  // threads per work unit

// Records reach shared memory by asynchronous copies (cp.async, 16 bytes a
// lane, one to three per lane for a cell), three cells deep: the copy of
// entry e + 2 is issued while entry e is blended, so neither registers nor a
// wait on the load's latency are spent on staging.  Every iteration commits one
// copy group (empty past the list's end) and waits for all but the two
// newest, which are the next two entries' (cp_async16 and friends: internal.cuh).
constexpr int NSTAGE = 3;

// Issue the copy of the records of cell `id` (per float4s) into dst.
__device__ __forceinline__ void issue_cell(float4 *dst, const float4 *__restrict__ vrec, uint32_t id, int per,
                                           int lane) {
    const float4 *src = vrec + (long long)id * per;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = lane + 32 * q;
        if (i < per) cp_async16(dst + i, src + i);
    }
}

// Cell ids of a tile list, read 32 at a time (lane j holds entry base + j)
// and handed out by a shuffle; entries must be asked for in increasing order
// from `first`, one at a time.
struct CellFeed {
    const uint32_t *__restrict__ cells;
    uint32_t first, end, chunk;
    __device__ __forceinline__ uint32_t id(uint32_t e, int lane) {
        const int j = (int)((e - first) & 31u);
        if (j == 0) chunk = e + lane < end ? __ldg(cells + e + lane) : 0u;
        return __shfl_sync(0xffffffffu, chunk, j);
    }
};

// Can record piece r0 pass the AABB test at some pixel centre of the 16-wide,
// `rows`-high block whose first pixel is (x0, y0)?  Exactly conservative (FP32
// subtraction is monotone, so testing the nearest pixel centres suffices).
__device__ __forceinline__ bool touches_rows(float4 r0, float x0, float y0, float rows) {
    const float lx = x0 + 0.5f, hx = x0 + (float)kTile - 0.5f;
    const float ly = y0 + 0.5f, hy = y0 + rows - 0.5f;
    return !(lx - r0.x > r0.z || r0.x - hx > r0.z || ly - r0.y > r0.w || r0.y - hy > r0.w);
}

// Does record piece r0 pass the AABB test at every pixel centre of the block?
// Exact: testing its first and last columns and rows suffices (FP32
// subtraction is monotone, so every offset lies between theirs).
__device__ __forceinline__ bool covers_rows(float4 r0, float x0, float y0, float rows) {
    const float lx = x0 + 0.5f, hx = x0 + (float)kTile - 0.5f;
    const float ly = y0 + 0.5f, hy = y0 + rows - 0.5f;
    return fabsf(lx - r0.x) <= r0.z && fabsf(hx - r0.x) <= r0.z && fabsf(ly - r0.y) <= r0.w &&
           fabsf(hy - r0.y) <= r0.w;
}

// Pixels of a lane in a 16 x (2 PPL) sub-tile: lane l = 8 j + i takes the
// columns i and i + 8 and the rows j + 4 r (r < PPL / 2); pixel q = 2 r + c.
// Each q thus spans an 8x4 quadrant of the warp's lanes, which meets fewer
// (quadrant, Gaussian) pairs than a 16x2 strip: a Gaussian's AABB is about
// square, and the per-pixel work of a quadrant runs whenever any of its
// pixels is hit (17% fewer such runs than one column per lane on the
// benchmark scene).
__device__ __forceinline__ int lane_col(int lane, int c) { return (lane & 7) + 8 * c; }
__device__ __forceinline__ int lane_row(int lane, int r) { return (lane >> 3) + 4 * r; }

// The forward's work unit: one warp per 16 x (2 PPL) sub-tile.  FWD_PPL = 4
// (16x8 sub-tiles, the adjoint's): with the pixel math in packed pairs, the
// per-Gaussian work of a lane (ballot, record loads, AABB tests) spread over
// four pixels outweighs the register cost; the kernels are held to 64
// registers (32 one-warp CTAs per SM; 1% faster than 72 registers and 28).
constexpr int FWD_PPL = 4;
// an offset from the Gaussian's centre that no box reaches: s1 or s2 then
// squares to at least ~1e18 (the record's L entries are far above 1e-9), and
// exp2 of its negation is +0
constexpr float kFar = 1e18f;
constexpr int FWD_SUB = kTile / (2 * FWD_PPL);  // sub-tiles per tile
constexpr int FWD_MINB = 32;

// VAR: the variant flags and background weight are live (dgs_config.flags,
// w_bg); without it the kernels are the paper's reading with no check left.
template <int KT, int PPL, bool VAR>
__device__ __forceinline__ void blend_fwd_unit(int unit, const ViewDesc *__restrict__ views, int n_views,
                                               const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                               const float4 *__restrict__ rec, const BlendParams &bp,
                                               float *__restrict__ out_rgb, float *__restrict__ out_rgb2,
                                               float *__restrict__ out_D, int *__restrict__ out_nd,
                                               float4 (*s_rec)[kRecF4 * (KT > 0 ? KT : kMaxK)]) {
    constexpr int ROWS = 2 * PPL, NSUB = kTile / ROWS;
    const int lane = threadIdx.x;
    const int tile = unit / NSUB, sub = unit % NSUB;
    const int vi = find_view(views, n_views, tile);
    const ViewDesc &V = views[vi];
    const int local = tile - V.tile_base;
    const int tx = local % V.Tx, ty = local / V.Tx;
    const float bx0 = (float)(tx * kTile), by0 = (float)(ty * kTile + ROWS * sub);
    constexpr int NR = PPL / 2;  // rows per lane
    int xs[2], ys[NR];
    float pxs[2], pys[NR];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        xs[c] = tx * kTile + lane_col(lane, c);
        pxs[c] = (float)xs[c] + 0.5f;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        ys[r] = ty * kTile + ROWS * sub + lane_row(lane, r);
        pys[r] = (float)ys[r] + 0.5f;
    }
    const int K = KT > 0 ? KT : V.K;
    const int per = kRecF4 * K;
    const float4 *vrec = rec + V.rec_base * kRecF4;
    const uint2 rg = ranges[tile];

    float T[PPL], N0[PPL], N1[PPL], N2[PPL], D[PPL];
    int n[PPL];
    bool done[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        T[q] = 1.0f; N0[q] = N1[q] = N2[q] = D[q] = 0.f; n[q] = 0;
        done[q] = !(xs[q & 1] < V.W && ys[q >> 1] < V.H);
    }
    CellFeed feed{cells, rg.x, rg.y, 0u};
#pragma unroll
    for (int b = 0; b < NSTAGE - 1; ++b) {
        if (rg.x + b < rg.y) issue_cell(s_rec[b], vrec, feed.id(rg.x + b, lane), per, lane);
        cp_async_commit();
    }
    int buf = 0;
    for (uint32_t e = rg.x; e < rg.y; ++e) {
        // before cell n a pixel stops if T_n < eps (Sec. V-B)
        bool all = true;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            done[q] = done[q] || T[q] < bp.eps;
            all = all && done[q];
        }
        if (__all_sync(0xffffffffu, all)) break;
        const int fill = buf == 0 ? NSTAGE - 1 : buf - 1;  // the buffer of entry e - 1, read by now
        if (e + NSTAGE - 1 < rg.y) issue_cell(s_rec[fill], vrec, feed.id(e + NSTAGE - 1, lane), per, lane);
        cp_async_commit();
        cp_async_wait<NSTAGE - 1>();
        __syncwarp();
        const float4 *r = s_rec[buf];
        const float v = r[2].w;
        unsigned mask = __ballot_sync(0xffffffffu, lane < K && touches_rows(r[kRecF4 * lane], bx0, by0, (float)ROWS));
        // Gaussians whose box holds the whole sub-tile: no per-pixel test
        const unsigned full = VAR ? 0u : __ballot_sync(0xffffffffu, lane < K && covers_rows(r[kRecF4 * lane], bx0, by0,
                                                                                            (float)ROWS));
        // the lane's two pixels of a row as packed pairs (one f32x2 operation
        // per pair; per component the same IEEE operations as one pixel)
        float2 A0[NR], A1[NR], A2[NR], B[NR], P[NR];
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            A0[rr] = A1[rr] = A2[rr] = B[rr] = make_float2(0.f, 0.f);
            P[rr] = make_float2(1.0f, 1.0f);
        }
        const float2 v2 = make_float2(v, v);
        const float amin = VAR && (bp.flags & DGS_FLAG_ALPHA_SKIP) ? 1.0f / 255.0f : 0.0f;
        for (; mask; mask &= mask - 1) {
            const int k = __ffs(mask) - 1;
            const float4 r0 = r[3 * k];
            float dx[2], dy[NR];
#pragma unroll
            for (int c = 0; c < 2; ++c) dx[c] = pxs[c] - r0.x;
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) dy[rr] = pys[rr] - r0.y;
            bool h[PPL];
            if (VAR || !((full >> k) & 1u)) {  // (else every pixel of the sub-tile is in the box)
                bool hx[2], hy[NR], any = false;
#pragma unroll
                for (int c = 0; c < 2; ++c) hx[c] = fabsf(dx[c]) <= r0.z;
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) hy[rr] = fabsf(dy[rr]) <= r0.w;
                if (VAR) {
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        h[q] = !done[q] && hx[q & 1] && hy[q >> 1];
                        any = any || h[q];
                    }
                } else {
                    // outside the box along a column or a row: an offset far off
                    // the Gaussian, so exp2 gives alpha = +0 exactly (in-box pixels
                    // compute as before; a done pixel's sums are not used)
                    any = (hx[0] || hx[1]) && (hy[0] || hy[NR - 1]);
#pragma unroll
                    for (int c = 0; c < 2; ++c) dx[c] = hx[c] ? dx[c] : kFar;
#pragma unroll
                    for (int rr = 0; rr < NR; ++rr) dy[rr] = hy[rr] ? dy[rr] : kFar;
                }
                // warp-uniform skip: lanes without a hit run the body with alpha = 0
                if (!__any_sync(0xffffffffu, any)) continue;
            }
            const float4 r1 = r[3 * k + 1];
            const float4 r2 = r[3 * k + 2];
            const float2 pdx = __fmul2_rn(make_float2(r1.x, r1.x), make_float2(dx[0], dx[1]));
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) {
                const float dyq = dy[rr];
                const float s2 = r1.z * dyq, s22 = s2 * s2;
                const float2 s1 = __ffma2_rn(make_float2(r1.y, r1.y), make_float2(dyq, dyq), pdx);
                const float2 qd = __ffma2_rn(s1, s1, make_float2(s22, s22));
                float2 al = __fmul2_rn(make_float2(r1.w, r1.w), make_float2(ex2_approx(-qd.x), ex2_approx(-qd.y)));
                // a pixel the Gaussian does not reach (or, with the alpha skip, an
                // alpha below 1/255) takes alpha 0: every update below leaves it unchanged
                if (VAR) {
                    al.x = h[2 * rr] && al.x >= amin ? fminf(al.x, bp.alpha_max) : 0.f;
                    al.y = h[2 * rr + 1] && al.y >= amin ? fminf(al.y, bp.alpha_max) : 0.f;
                } else {
                    al.x = fminf(al.x, bp.alpha_max);
                    al.y = fminf(al.y, bp.alpha_max);
                }
                A0[rr] = __ffma2_rn(al, make_float2(r2.x, r2.x), A0[rr]);
                A1[rr] = __ffma2_rn(al, make_float2(r2.y, r2.y), A1[rr]);
                A2[rr] = __ffma2_rn(al, make_float2(r2.z, r2.z), A2[rr]);
                B[rr] = __fadd2_rn(B[rr], al);
                P[rr] = __ffma2_rn(make_float2(-P[rr].x, -P[rr].y), __fmul2_rn(v2, al), P[rr]);
            }
        }
        const bool exclude = VAR && (bp.flags & DGS_FLAG_TERM_EXCLUDE) != 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            if (!done[q]) {
                const int rr = q >> 1;
                const bool hi = q & 1;
                const float Tnext = T[q] * (hi ? P[rr].y : P[rr].x);
                if (exclude && Tnext < bp.eps) {  // the 3DGS rule: this cell is not blended
                    done[q] = true;
                    continue;
                }
                const float w = v * T[q];
                N0[q] = fmaf(w, hi ? A0[rr].y : A0[rr].x, N0[q]);
                N1[q] = fmaf(w, hi ? A1[rr].y : A1[rr].x, N1[q]);
                N2[q] = fmaf(w, hi ? A2[rr].y : A2[rr].x, N2[q]);
                D[q] = fmaf(w, hi ? B[rr].y : B[rr].x, D[q]);
                T[q] = Tnext;
                ++n[q];
            }
        }
        __syncwarp();  // every lane is done with s_rec[buf] before it is refilled
        buf = buf == NSTAGE - 1 ? 0 : buf + 1;
    }
    cp_async_wait<0>();  // copies of entries past an early stop land before the buffers are reused
    __syncwarp();
    const long long HW = (long long)V.W * V.H;
    float *img = V.out ? V.out : out_rgb + 3 * V.pix_base;
    float *im2 = out_rgb2 ? out_rgb2 + 3 * V.pix_base : nullptr;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        if (!(xs[q & 1] < V.W && ys[q >> 1] < V.H)) continue;
        const long long pin = (long long)ys[q >> 1] * V.W + xs[q & 1];
        float c0, c1, c2;
        if (VAR && (bp.flags & DGS_FLAG_NUMERATOR)) {  // the numerator of Eq. 12
            c0 = N0[q]; c1 = N1[q]; c2 = N2[q];
        } else if (VAR) {  // Eq. 12, with a background weight (N + w_bg bg) / (D + w_bg)
            const float Dp = D[q] + bp.w_bg;
            const bool hit = Dp > bp.d_min;
            c0 = hit ? (N0[q] + bp.w_bg * bp.bg0) / Dp : bp.bg0;
            c1 = hit ? (N1[q] + bp.w_bg * bp.bg1) / Dp : bp.bg1;
            c2 = hit ? (N2[q] + bp.w_bg * bp.bg2) / Dp : bp.bg2;
        } else {  // Eq. 12
            const bool hit = D[q] > bp.d_min;
            c0 = hit ? N0[q] / D[q] : bp.bg0;
            c1 = hit ? N1[q] / D[q] : bp.bg1;
            c2 = hit ? N2[q] / D[q] : bp.bg2;
        }
        img[pin] = c0;
        img[HW + pin] = c1;
        img[2 * HW + pin] = c2;
        if (im2) {
            im2[pin] = c0;
            im2[HW + pin] = c1;
            im2[2 * HW + pin] = c2;
        }
        out_D[V.pix_base + pin] = D[q];
        out_nd[V.pix_base + pin] = n[q];
    }
}

template <int KT, bool VAR>
__global__ void __launch_bounds__(WT, FWD_MINB) k_blend_fwd(const ViewDesc *__restrict__ views, int n_views,
                                                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                  const float4 *__restrict__ rec, BlendParams bp,
                                                  float *__restrict__ out_rgb, float *__restrict__ out_rgb2,
                                                  float *__restrict__ out_D, int *__restrict__ out_nd) {
    __shared__ float4 s_rec[NSTAGE][kRecF4 * (KT > 0 ? KT : kMaxK)];
    blend_fwd_unit<KT, FWD_PPL, VAR>(blockIdx.x, views, n_views, ranges, cells, rec, bp, out_rgb, out_rgb2, out_D, out_nd,
                                s_rec);
}

// Persistent form for chains whose sizes live on the device: a fixed grid of
// exactly the resident warps pulls sub-tiles from an atomic counter (*work
// starts at 0) until the chain's total_tiles * FWD_SUB units are taken, so the
// dense and the empty regions of the images balance dynamically.  One
// atomic per sub-tile: their rate is bounded by the blend work between them.
template <int KT, bool VAR>
__global__ void __launch_bounds__(WT, FWD_MINB) k_blend_fwd_pull(const ViewDesc *__restrict__ views,
                                                       const uint2 *__restrict__ ranges,
                                                       const uint32_t *__restrict__ cells,
                                                       const float4 *__restrict__ rec, BlendParams bp,
                                                       float *__restrict__ out_rgb, float *__restrict__ out_D,
                                                       int *__restrict__ out_nd, const ChainSizes *__restrict__ dsz,
                                                       uint32_t *__restrict__ work) {
    __shared__ float4 s_rec[NSTAGE][kRecF4 * (KT > 0 ? KT : kMaxK)];
    const int n_views = dsz->n_views;
    const uint32_t units = (uint32_t)dsz->total_tiles * FWD_SUB;
    for (;;) {
        uint32_t u = 0;
        if (threadIdx.x == 0) u = atomicAdd(work, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= units) break;
        blend_fwd_unit<KT, FWD_PPL, VAR>((int)u, views, n_views, ranges, cells, rec, bp, out_rgb, nullptr, out_D, out_nd,
                                    s_rec);
        __syncwarp();
    }
}

// Do the blend kernels need their variant form (a flag or a background weight)?
static bool blend_variants(const BlendParams &bp) {
    return (bp.flags & (DGS_FLAG_ALPHA_SKIP | DGS_FLAG_TERM_EXCLUDE | DGS_FLAG_NUMERATOR)) != 0 || bp.w_bg != 0.f;
}

template <int KT, bool VAR>
static unsigned pull_grid(int total_tiles) {
    const long long per_grid = resident_ctas((const void *)k_blend_fwd_pull<KT, VAR>, WT);
    return (unsigned)std::min<long long>((long long)total_tiles * FWD_SUB, per_grid);
}

void launch_blend_fwd(const ViewDesc *views, int n_views, int total_tiles, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, float *out_rgb,
                      float *out_rgb2, float *out_D, int *out_nd, int K_all, cudaStream_t st,
                      const ChainSizes *dsz, uint32_t *work) {
    if (total_tiles == 0) return;
    if (dsz) {
        // exactly the resident warps
#define DGS_PULL(KV, VV)                                                                                     \
        k_blend_fwd_pull<KV, VV><<<pull_grid<KV, VV>(total_tiles), WT, 0, st>>>(views, ranges, tile_cells, rec, bp, \
                                                                               out_rgb, out_D, out_nd, dsz, work)
        if (blend_variants(bp)) {
            switch (K_all) {
                case 8: DGS_PULL(8, true); break;
                case 10: DGS_PULL(10, true); break;
                default: DGS_PULL(0, true); break;
            }
        } else {
            switch (K_all) {
                case 8: DGS_PULL(8, false); break;
                case 10: DGS_PULL(10, false); break;
                default: DGS_PULL(0, false); break;
            }
        }
#undef DGS_PULL
        return;
    }
    const unsigned grid = (unsigned)total_tiles * FWD_SUB;
#define DGS_FWD(KV, VV)                                                                                      \
    k_blend_fwd<KV, VV><<<grid, WT, 0, st>>>(views, n_views, ranges, tile_cells, rec, bp, out_rgb, out_rgb2, out_D, \
                                             out_nd)
    if (blend_variants(bp)) {
        switch (K_all) {
            case 8: DGS_FWD(8, true); break;
            case 10: DGS_FWD(10, true); break;
            default: DGS_FWD(0, true); break;
        }
    } else {
        switch (K_all) {
            case 8: DGS_FWD(8, false); break;
            case 10: DGS_FWD(10, false); break;
            default: DGS_FWD(0, false); break;
        }
    }
#undef DGS_FWD
}

// ---------------------------------------------------------------- counters
// Diagnostic replay of the AABB tests (no blending): per pixel, the
// (pixel, Gaussian) pairs of blended cells, those passing the AABB test, and
// the passing pairs over the whole tile list.  counts[0..3] as in dgs_counts.
__global__ void __launch_bounds__(BT) k_count_pairs(const ViewDesc *__restrict__ views, int n_views,
                                                    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                    const float4 *__restrict__ rec, const int *__restrict__ ndpix,
                                                    unsigned long long *__restrict__ counts) {
    __shared__ int s_view;
    const int tid = threadIdx.x, tile = blockIdx.x;
    if (tid == 0) s_view = find_view(views, n_views, tile);
    __syncthreads();
    const ViewDesc &V = views[s_view];
    const int local = tile - V.tile_base;
    const int tx = local % V.Tx, ty = local / V.Tx;
    const int xi = tx * kTile + (tid & (kTile - 1)), yi = ty * kTile + (tid >> 4);
    unsigned long long c[4] = {0, 0, 0, 0};
    if (xi < V.W && yi < V.H) {
        const int nd = ndpix[V.pix_base + (long long)yi * V.W + xi];
        const float px = (float)xi + 0.5f, py = (float)yi + 0.5f;
        const uint2 rg = ranges[tile];
        const float4 *vrec = rec + V.rec_base * kRecF4;
        for (uint32_t e = rg.x; e < rg.y; ++e) {
            const bool blended = (int)(e - rg.x) < nd;
            const float4 *r = vrec + (long long)cells[e] * V.K * kRecF4;
            unsigned in = 0;
            for (int k = 0; k < V.K; ++k) {
                const float4 r0 = __ldg(r + 3 * k);
                in += (fabsf(px - r0.x) <= r0.z && fabsf(py - r0.y) <= r0.w) ? 1u : 0u;
            }
            c[2] += in;
            if (blended) { c[0] += V.K; c[1] += in; c[3] += 1; }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long v = c[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0 && v) atomicAdd(counts + i, v);
    }
}

void launch_count_pairs(const ViewDesc *views, int n_views, int total_tiles, const uint2 *ranges,
                        const uint32_t *tile_cells, const float4 *rec, const int *nd, unsigned long long *counts,
                        cudaStream_t st) {
    if (total_tiles == 0) return;
    k_count_pairs<<<total_tiles, BT, 0, st>>>(views, n_views, ranges, tile_cells, rec, nd, counts);
}

// ---------------------------------------------------------------- adjoint
// With C = N/D and g = dL/dC:  dN = g/D, dD = -(g.C)/D.  Writing
// x_n = v_n T_n (dN.A_n + dD B_n), C's degree-0 homogeneity in the weights
// gives sum_n x_n = 0 over the blended cells, so the total gradient through
// the transmittance of all LATER cells, S_n = sum_{m>n} x_m, equals
// -sum_{m<=n} x_m and is known front to back: the replay needs no division
// by T and stores no per-cell state.  Per Gaussian k of cell n at a pixel:
//     dL/dalpha = v T_n (dN.c_k + dD) - v S_n / (1 - v alpha)
//     dL/dc_k   = v T_n alpha dN
//     dL/dv_n   = T_n (dN.A_n + dD B_n) - S_n sum_k alpha_k / (1 - v alpha_k)
// then alpha = sigma G' (unless clamped) and G' = exp(-q/2).
//
// Same work unit as the forward (one warp per 16x8 sub-tile, four pixels per
// lane).  Per cell, the warp replays its pixels keeping G' of the Gaussians
// that reach the sub-tile in warp-private shared memory, updates S and T,
// then for each such Gaussian sums its pixels' nine screen-space gradient
// terms across the warp with a transposed shuffle tree (each step halves the
// values a lane carries) and adds the totals to global memory (one atomic
// add per value per sub-tile).

// Sum v[0..7] over the warp.  On return lane L holds the total of value
// 4 b2 + 2 b3 + b4 (b_i = bit i of L; transposed_owner8); the four lanes that
// differ only in b0 and b1 hold the same total.
// Transposed warp reduction of eight per-lane values: three halving steps
// (offsets 16, 8, 4) in which each lane keeps half of its slots and receives
// its partner's other half, then two butterfly steps (offsets 2, 1).  Every
// lane ends with the warp total of slot transposed_owner8(lane): 9 shuffles
// instead of 8 x 5.
__device__ __forceinline__ float transposed_warp_sum8(float v[8], int lane) {
#pragma unroll
    for (int step = 0; step < 3; ++step) {
        const int bit = 16 >> step;
        const bool hi = lane & bit;
        const int n = 4 >> step;  // pairs at this step
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const float keep = hi ? v[2 * i + 1] : v[2 * i];
            const float send = hi ? v[2 * i] : v[2 * i + 1];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    const float t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
    return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

__device__ __forceinline__ int transposed_owner8(int lane) {
    return ((lane >> 2) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 4) & 1);
}

__device__ __forceinline__ float warp_sum(float a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// 1/x to ~1 ulp (MUFU); x = 1 - v alpha >= 1 - alpha_max here
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Screen-space gradient terms of (pixel, Gaussian) pairs for the two pixels
// of one lane row at once (one f32x2 operation per pixel pair), with the
// constant factors left to the caller (applied once per reduced total):
//   acc[1], acc[4] = sum dq' dy, sum dq' dy^2 per column (column_terms forms
//   the lane's moments sum dq' (dx, dy), which mean_terms makes the mean's,
//   and sum dq' (dx^2, dx dy, dy^2): da, db, dc = -1/2, -1, -1/2 x acc)
//   acc[5..7] = sum v T alpha e       (drgb)
//   dop       = sum dalpha G          (dsigma)
//   pv       += alpha / (1 - v alpha)  (per pixel; times -S_n, dL/dv's share)
// with dq' = G dalpha sigma = -2 dL/dq.  cA = v T_n and nvS = -v S_n are the
// pixels' per-cell factors (formed once per cell); dx the lane's column
// offsets (shared by its rows).  A pixel with G' = 0 (not reached, or inactive) adds
// exactly 0, and the opacity-clamped branch is a select, so no per-pixel
// branch remains.
template <bool WV>
__device__ __forceinline__ void pair_grad2(float2 acc[8], float2 &dop, float2 &pv, float2 Gv, float4 r0, float4 r1,
                                           float4 r2, float2 dx, float py, float2 cA, float2 nvS,
                                           float2 e0, float2 e1, float2 e2, float2 eD, float alpha_max) {
    const float v = r2.w, op = r1.w;
    const float2 raw = __fmul2_rn(make_float2(op, op), Gv);
    const float2 al = make_float2(fminf(raw.x, alpha_max), fminf(raw.y, alpha_max));
    const float2 om = __ffma2_rn(make_float2(-v, -v), al, make_float2(1.0f, 1.0f));
    const float2 rom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    const float2 inner = __ffma2_rn(
        e0, make_float2(r2.x, r2.x),
        __ffma2_rn(e1, make_float2(r2.y, r2.y), __ffma2_rn(e2, make_float2(r2.z, r2.z), eD)));
    const float2 dal = __ffma2_rn(nvS, rom, __fmul2_rn(cA, inner));
    const float2 ca_al = __fmul2_rn(cA, al);
    acc[5] = __ffma2_rn(ca_al, e0, acc[5]);
    acc[6] = __ffma2_rn(ca_al, e1, acc[6]);
    acc[7] = __ffma2_rn(ca_al, e2, acc[7]);
    if (WV) pv = __ffma2_rn(al, rom, pv);
    float2 dG = __fmul2_rn(dal, Gv);
    dG.x = raw.x < alpha_max ? dG.x : 0.f;
    dG.y = raw.y < alpha_max ? dG.y : 0.f;
    dop = __fadd2_rn(dop, dG);
    // per column of the lane (dx is the same for its rows): sum dq' dy and
    // sum dq' dy^2; the dx-weighted sums follow from dop (dq' = sigma dG)
    // and these in column_terms
    const float dys = py - r0.y, opdy = op * dys;
    const float2 dqy = __fmul2_rn(dG, make_float2(opdy, opdy));
    acc[1] = __fadd2_rn(acc[1], dqy);
    acc[4] = __ffma2_rn(dqy, make_float2(dys, dys), acc[4]);
}

// A lane's totals of slots 0..4 from its per-column sums (components x, y:
// its two columns, offsets dx from the Gaussian's centre): with D = sigma dop
// = sum dq' per column and Y = acc[1] = sum dq' dy per column,
//   sum dq' dx = D.dx, sum dq' dy = sum Y, sum dq' dx^2 = D.dx^2,
//   sum dq' dx dy = Y.dx, sum dq' dy^2 = sum acc[4].
__device__ __forceinline__ void column_terms(const float2 acc2[8], float2 dop, float op, float2 dx, float acc[8]) {
    const float2 D = __fmul2_rn(dop, make_float2(op, op));
    const float2 t = __fmul2_rn(D, dx);
    acc[0] = t.x + t.y;
    acc[1] = acc2[1].x + acc2[1].y;
    acc[2] = fmaf(t.x, dx.x, t.y * dx.y);
    acc[3] = fmaf(acc2[1].x, dx.x, acc2[1].y * dx.y);
    acc[4] = acc2[4].x + acc2[4].y;
}

// The mean's terms of a lane, from its moments m = sum dq' (dx, dy): with the
// record's L scaled by kappa (kappa^2 = log2(e)/2), q = |L^T d|^2 and
// dq/dmu = -2 Q d = -(2/kappa^2) L (s1, s2), (s1, s2) = L^T d = (p dx + r dy,
// t dy), 2/kappa^2 = 4 ln 2; summed over pixels, sum dq' L (s1, s2) =
// (p u, r u + t^2 m_y) with u = p m_x + r m_y (linear in the moments, so each
// lane converts its partial sums before the warp reduction: no shuffle).
__device__ __forceinline__ void mean_terms(float4 r1, float &a0, float &a1) {
    const float u = fmaf(r1.x, a0, r1.y * a1);
    const float b1 = fmaf(r1.y, u, r1.z * r1.z * a1);
    a0 = r1.x * u;
    a1 = b1;
}

// Constant factor of reduction slot j (see pair_grad2): dL/dq = -dq'/2, so
// dmu = -(4 ln 2)(-1/2) acc = 2 ln 2 acc, da = -acc/2, db = -acc (the 2 dx dy
// term), dc = -acc/2; rgb unchanged.
__device__ __forceinline__ float slot_scale(int j) {
    return j < 2 ? 2.0f * LN2 : (j == 3 ? -1.0f : (j < 5 ? -0.5f : 1.0f));
}

// screen-space gradient slot (of kGradF) that reduction slot j feeds
__device__ __forceinline__ int grad_slot(int j) { return j < 5 ? j : j + 1; }

// The adjoint's work unit: one warp per 16 x (2 PPL) sub-tile, pixels of a
// lane as in the forward (lane_col, lane_row).  Per cell: pass 1 replays the forward (keeping G' of the Gaussians
// that reach the sub-tile in warp-private shared memory) and updates T and
// S; pass 2 forms each such Gaussian's screen-space gradient over the
// sub-tile's pixels and adds the warp total with global atomics.
constexpr int BWD_PPL = 4;
constexpr int BWD_SUB = kTile / (2 * BWD_PPL);  // sub-tiles per tile
constexpr int BWD_MINB = 24;  // resident one-warp CTAs per SM the register budget is set for

template <int KT, int PPL, bool VAR, bool WV>
__global__ void __launch_bounds__(WT, BWD_MINB) k_blend_bwd(const ViewDesc *__restrict__ views, int n_views,
                                                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                  const float4 *__restrict__ rec, BlendParams bp,
                                                  const float *__restrict__ rgb, const float *__restrict__ Dpix,
                                                  const int *__restrict__ ndpix, const float *__restrict__ dL_drgb,
                                                  float *__restrict__ g2d, float *__restrict__ g_cell_v) {
    constexpr int ROWS = 2 * PPL, NSUB = kTile / ROWS;
    constexpr int KRS = KT > 0 ? KT : kMaxK;
    __shared__ float4 s_rec[NSTAGE][kRecF4 * KRS];
    static_assert(PPL == 4, "G' of a lane's four pixels is kept as one float4");
    __shared__ float4 s_G[KRS][WT];  // G' of hit i at the lane's pixels q = 0..3
    const int lane = threadIdx.x;
    const int tile = blockIdx.x / NSUB, sub = blockIdx.x % NSUB;
    const int vi = find_view(views, n_views, tile);
    const ViewDesc &V = views[vi];
    const int local = tile - V.tile_base;
    const int tx = local % V.Tx, ty = local / V.Tx;
    const float bx0 = (float)(tx * kTile), by0 = (float)(ty * kTile + ROWS * sub);
    constexpr int NR = PPL / 2;  // rows per lane (pixel mapping as in the forward)
    int xs[2], ys[NR];
    float pxs[2], pys[NR];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        xs[c] = tx * kTile + lane_col(lane, c);
        pxs[c] = (float)xs[c] + 0.5f;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        ys[r] = ty * kTile + ROWS * sub + lane_row(lane, r);
        pys[r] = (float)ys[r] + 0.5f;
    }
    const long long HW = (long long)V.W * V.H;
    const int K = KT > 0 ? KT : V.K;
    const int per = kRecF4 * K;

    // Per pixel: dL/dN = e, dL/dD = eD, and S's start value, the sum of x_n
    // over the processed cells: 0 for C = N / D (degree-0 homogeneity), else
    // w_bg g.(C - bg) / (D + w_bg) with a background weight, g.C for the
    // numerator output (dL/dN = g, dL/dD = 0).
    int nd[PPL];
    float e0s[PPL], e1s[PPL], e2s[PPL], eDs[PPL], S0[PPL];
    int ndm = 0;
    const bool numer = VAR && (bp.flags & DGS_FLAG_NUMERATOR) != 0;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        nd[q] = 0;
        e0s[q] = e1s[q] = e2s[q] = eDs[q] = S0[q] = 0.f;
        if (xs[q & 1] < V.W && ys[q >> 1] < V.H) {
            const long long pin = (long long)ys[q >> 1] * V.W + xs[q & 1];
            const float Dp = VAR ? Dpix[V.pix_base + pin] + bp.w_bg : Dpix[V.pix_base + pin];
            if (numer || Dp > bp.d_min) {
                nd[q] = ndpix[V.pix_base + pin];
                const float *gi = dL_drgb + 3 * V.pix_base;
                const float *ci = rgb + 3 * V.pix_base;
                const float g0 = gi[pin], g1 = gi[HW + pin], g2 = gi[2 * HW + pin];
                const float c0 = ci[pin], c1 = ci[HW + pin], c2 = ci[2 * HW + pin];
                if (numer) {
                    e0s[q] = g0; e1s[q] = g1; e2s[q] = g2;
                    S0[q] = g0 * c0 + g1 * c1 + g2 * c2;
                } else {
                    const float iD = 1.0f / Dp;
                    e0s[q] = g0 * iD; e1s[q] = g1 * iD; e2s[q] = g2 * iD;
                    eDs[q] = -(g0 * c0 + g1 * c1 + g2 * c2) * iD;
                    if (VAR) S0[q] = bp.w_bg * (g0 * (c0 - bp.bg0) + g1 * (c1 - bp.bg1) + g2 * (c2 - bp.bg2)) * iD;
                }
            }
        }
        ndm = max(ndm, nd[q]);
    }
    // the lane's pixels as row pairs (columns 0 and 1 of lane row rr); half of
    // the per-pixel factors, (e2, eD), wait in warp-private shared memory
    // (registers are the adjoint's limit: this keeps it from spilling)
    __shared__ float4 s_E[NR][WT];
    float2 e0r[NR], e1r[NR];
    const float2 px2 = make_float2(pxs[0], pxs[1]);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
        e0r[rr] = make_float2(e0s[2 * rr], e0s[2 * rr + 1]);
        e1r[rr] = make_float2(e1s[2 * rr], e1s[2 * rr + 1]);
        s_E[rr][lane] = make_float4(e2s[2 * rr], e2s[2 * rr + 1], eDs[2 * rr], eDs[2 * rr + 1]);
    }
    auto efac = [&](int rr, float2 &e0, float2 &e1, float2 &e2, float2 &eD) {
        const float4 b = s_E[rr][lane];
        e0 = e0r[rr]; e1 = e1r[rr];
        e2 = make_float2(b.x, b.y); eD = make_float2(b.z, b.w);
    };
    __shared__ int4 s_nd[WT];  // the lane's per-pixel cell counts, read once per cell
    s_nd[lane] = make_int4(nd[0], nd[1], nd[2], nd[3]);
    const int ndmax = __reduce_max_sync(0xffffffffu, ndm);
    const uint2 rg = ranges[tile];
    const uint32_t end = rg.x + min((uint32_t)ndmax, rg.y - rg.x);
    const float4 *vrec = rec + V.rec_base * kRecF4;
    constexpr bool want_v = WV;  // dL/dv_n requested (g_cell_v): else its per-pixel sums are not formed

    float2 T[NR], S[NR];
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) { T[rr] = make_float2(1.0f, 1.0f); S[rr] = make_float2(S0[2 * rr], S0[2 * rr + 1]); }
    CellFeed feed{cells, rg.x, end, 0u};
#pragma unroll
    for (int b = 0; b < NSTAGE - 1; ++b) {
        if (rg.x + b < end) issue_cell(s_rec[b], vrec, feed.id(rg.x + b, lane), per, lane);
        cp_async_commit();
    }
    int buf = 0;
    for (uint32_t e = rg.x; e < end; ++e) {
        const int fill = buf == 0 ? NSTAGE - 1 : buf - 1;  // the buffer of entry e - 1, read by now
        if (e + NSTAGE - 1 < end) issue_cell(s_rec[fill], vrec, feed.id(e + NSTAGE - 1, lane), per, lane);
        cp_async_commit();
        cp_async_wait<NSTAGE - 1>();
        __syncwarp();
        const int n = (int)(e - rg.x);
        bool act[PPL];
        {
            const int4 nd4 = s_nd[lane];
            act[0] = n < nd4.x; act[1] = n < nd4.y; act[2] = n < nd4.z; act[3] = n < nd4.w;
        }
        const float4 *r = s_rec[buf];
        const float v = r[2].w;
        unsigned mask = __ballot_sync(0xffffffffu, lane < K && touches_rows(r[kRecF4 * lane], bx0, by0, (float)ROWS));
        const unsigned mask0 = mask;
        const int nhit = __popc(mask);
        // pass 1: replay the cell, keep G'; per pixel P_n and
        // X_n = dN.A_n + dD B_n = sum_k alpha_k (dN.c_k + dD)
        float2 X[NR], P[NR];
        const float2 v2 = make_float2(v, v);
        const float amin = VAR && (bp.flags & DGS_FLAG_ALPHA_SKIP) ? 1.0f / 255.0f : 0.0f;
        {
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) { X[rr] = make_float2(0.f, 0.f); P[rr] = make_float2(1.0f, 1.0f); }
#pragma unroll 1
            for (int i = 0; i < nhit; ++i) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 r0 = r[3 * k];
                float dx[2], dy[NR];
                bool hx[2], hy[NR];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    dx[c] = pxs[c] - r0.x;
                    hx[c] = fabsf(dx[c]) <= r0.z;
                }
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) {
                    dy[rr] = pys[rr] - r0.y;
                    hy[rr] = fabsf(dy[rr]) <= r0.w;
                }
                bool h[PPL], any = false;
                if (VAR) {
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        h[q] = act[q] && hx[q & 1] && hy[q >> 1];
                        any = any || h[q];
                    }
                } else {
                    // outside the box along a column or a row: an offset far off the
                    // Gaussian (G' = +0 exactly, as in the forward); inactive pixels
                    // get G' = 0 when it is stored (their X and P are not used)
                    any = (hx[0] || hx[1]) && (hy[0] || hy[NR - 1]);
#pragma unroll
                    for (int c = 0; c < 2; ++c) dx[c] = hx[c] ? dx[c] : kFar;
#pragma unroll
                    for (int rr = 0; rr < NR; ++rr) dy[rr] = hy[rr] ? dy[rr] : kFar;
                }
                if (!any) {
                    s_G[i][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                const float4 r1 = r[3 * k + 1];
                const float4 r2 = r[3 * k + 2];
                const float2 pdx = __fmul2_rn(make_float2(r1.x, r1.x), make_float2(dx[0], dx[1]));
                float2 gq[NR];
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) {
                    const float dyq = dy[rr];
                    const float s2 = r1.z * dyq, s22 = s2 * s2;
                    const float2 s1 = __ffma2_rn(make_float2(r1.y, r1.y), make_float2(dyq, dyq), pdx);
                    const float2 qd = __ffma2_rn(s1, s1, make_float2(s22, s22));
                    float2 Gv = make_float2(ex2_approx(-qd.x), ex2_approx(-qd.y));
                    float2 rw = __fmul2_rn(make_float2(r1.w, r1.w), Gv);
                    if (VAR) {  // not reached (or alpha skipped as in the forward): G' = 0 leaves X and P as they are
                        if (!h[2 * rr] || rw.x < amin) Gv.x = rw.x = 0.f;
                        if (!h[2 * rr + 1] || rw.y < amin) Gv.y = rw.y = 0.f;
                        gq[rr] = Gv;
                    } else {
                        gq[rr] = make_float2(act[2 * rr] ? Gv.x : 0.f, act[2 * rr + 1] ? Gv.y : 0.f);
                    }
                    const float2 al = make_float2(fminf(rw.x, bp.alpha_max), fminf(rw.y, bp.alpha_max));
                    float2 e0, e1, e2, eD;
                    efac(rr, e0, e1, e2, eD);
                    const float2 inner = __ffma2_rn(
                        e0, make_float2(r2.x, r2.x),
                        __ffma2_rn(e1, make_float2(r2.y, r2.y), __ffma2_rn(e2, make_float2(r2.z, r2.z), eD)));
                    X[rr] = __ffma2_rn(al, inner, X[rr]);
                    P[rr] = __ffma2_rn(make_float2(-P[rr].x, -P[rr].y), __fmul2_rn(v2, al), P[rr]);
                }
                s_G[i][lane] = make_float4(gq[0].x, gq[0].y, gq[1].x, gq[1].y);
            }
        }
        // per-pixel transmittance bookkeeping (S_n includes x_n); the cell
        // term of dL/dv, sum over pixels of T_n X_n, joins the Gaussians'
        // terms below so one reduction per cell carries dL/dv
        float2 Tn[NR];
        float dv = 0.f;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            Tn[rr] = T[rr];
            if (act[2 * rr]) {
                S[rr].x -= v * Tn[rr].x * X[rr].x;
                T[rr].x *= P[rr].x;
                dv += Tn[rr].x * X[rr].x;
            }
            if (act[2 * rr + 1]) {
                S[rr].y -= v * Tn[rr].y * X[rr].y;
                T[rr].y *= P[rr].y;
                dv += Tn[rr].y * X[rr].y;
            }
        }
        // per pixel: sum alpha / (1 - v alpha) of the cell's Gaussians; v T_n; -v S_n
        float2 pv[NR], cA[NR], nvS[NR];
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            pv[rr] = make_float2(0.f, 0.f);
            cA[rr] = __fmul2_rn(v2, Tn[rr]);
            nvS[rr] = __fmul2_rn(make_float2(-v, -v), S[rr]);
        }
        const uint32_t cellid = __ldg(cells + e);
        float *gbase = g2d + (V.rec_base + (long long)cellid * K) * kGradF;
        // pass 2: gradient terms per Gaussian reaching the sub-tile, two
        // Gaussians per loop trip (fully unrolled over K the body overflows the
        // instruction cache; by two it is 2% faster than not unrolled)
        unsigned m2 = mask0;
#pragma unroll 2
        for (int i = 0; m2; ++i, m2 &= m2 - 1) {
            const float4 g4 = s_G[i][lane];
            const float2 gv[NR] = {make_float2(g4.x, g4.y), make_float2(g4.z, g4.w)};
            const bool any = g4.x > 0.f || g4.y > 0.f || g4.z > 0.f || g4.w > 0.f;
            if (!__any_sync(0xffffffffu, any)) continue;
            const int k = __ffs(m2) - 1;
            const float4 r0 = r[3 * k], r1 = r[3 * k + 1], r2 = r[3 * k + 2];
            float2 acc2[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc2[j] = make_float2(0.f, 0.f);
            float2 dop2 = make_float2(0.f, 0.f);
            const float2 gdx = __fadd2_rn(px2, make_float2(-r0.x, -r0.x));
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) {
                float2 e0, e1, e2, eD;
                efac(rr, e0, e1, e2, eD);
                pair_grad2<WV>(acc2, dop2, pv[rr], gv[rr], r0, r1, r2, gdx, pys[rr], cA[rr], nvS[rr], e0, e1, e2, eD,
                               bp.alpha_max);
            }
            float acc[8];
            column_terms(acc2, dop2, r1.w, gdx, acc);
#pragma unroll
            for (int j = 5; j < 8; ++j) acc[j] = acc2[j].x + acc2[j].y;
            mean_terms(r1, acc[0], acc[1]);
            const float tot = transposed_warp_sum8(acc, lane);
            const float dop_tot = warp_sum(dop2.x + dop2.y);
            float *gk = gbase + k * kGradF;
            const int slot = transposed_owner8(lane);
            if ((lane & 3) == 0 && tot != 0.f) atomicAdd(gk + grad_slot(slot), tot * slot_scale(slot));
            if (lane == 1 && dop_tot != 0.f) atomicAdd(gk + 5, dop_tot);
        }
        if (want_v) {  // per (view, cell) entry: v_n may differ between views
            float2 dv2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) dv2 = __ffma2_rn(make_float2(-S[rr].x, -S[rr].y), pv[rr], dv2);
            dv = warp_sum(dv + (dv2.x + dv2.y));
            if (lane == 0 && dv != 0.f) atomicAdd(g_cell_v + V.cell_base + cellid, dv);
        }
        __syncwarp();  // every lane is done with s_rec[buf] and s_G before they are refilled
        buf = buf == NSTAGE - 1 ? 0 : buf + 1;
    }
    cp_async_wait<0>();
}

// K_all: K of the chain's scene (compile-time loop for common values)
void launch_blend_bwd(const ViewDesc *views, int n_views, int total_tiles, int K_all, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, const float *rgb,
                      const float *D, const int *nd, const float *dL_drgb, float *g2d, float *g_cell_v,
                      cudaStream_t st) {
    if (total_tiles == 0) return;
    const unsigned grid = (unsigned)total_tiles * BWD_SUB;
#define DGS_BWD(KV, VV)                                                                                          \
    do {                                                                                                        \
        if (g_cell_v)                                                                                           \
            k_blend_bwd<KV, BWD_PPL, VV, true><<<grid, WT, 0, st>>>(views, n_views, ranges, tile_cells, rec, bp,  \
                                                                    rgb, D, nd, dL_drgb, g2d, g_cell_v);        \
        else                                                                                                    \
            k_blend_bwd<KV, BWD_PPL, VV, false><<<grid, WT, 0, st>>>(views, n_views, ranges, tile_cells, rec, bp, \
                                                                     rgb, D, nd, dL_drgb, g2d, nullptr);        \
    } while (0)
    if (blend_variants(bp)) {
        switch (K_all) {
            case 8: DGS_BWD(8, true); break;
            case 10: DGS_BWD(10, true); break;
            default: DGS_BWD(0, true); break;
        }
    } else {
        switch (K_all) {
            case 8: DGS_BWD(8, false); break;
            case 10: DGS_BWD(10, false); break;
            default: DGS_BWD(0, false); break;
        }
    }
#undef DGS_BWD
}

}  // namespace dgs
