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
// GB300 mapping: one 256-thread CTA per 16x16 tile, one pixel per thread.
// The 48-byte records of the Gaussians of a chunk of cells are fetched with
// one 16-byte load per thread into registers while the previous chunk is
// blended from shared memory (double buffer), so every record is read from
// L2/HBM once per tile and then broadcast from shared memory to 256 pixels.
// A block-wide count of finished pixels ends the tile early.
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

// One 16-byte piece of the records of chunk [start, start + CH) for thread tid.
__device__ __forceinline__ float4 fetch_rec(const float4 *__restrict__ vrec, const uint32_t *__restrict__ cells,
                                            uint32_t start, uint32_t end, int tid, int nload, int per, float4 keep) {
    if (tid < nload) {
        const int c = tid / per, j = tid - c * per;
        const uint32_t e = start + c;
        if (e < end) return __ldg(vrec + (long long)cells[e] * per + j);
    }
    return keep;
}

// Can Gaussian record piece r0 = (mu_x, mu_y, ext_x, ext_y) pass the per-pixel
// AABB test at any pixel centre of the tile whose first pixel is (x0, y0)?
// Exactly conservative: FP32 subtraction is monotone, so if the nearest pixel
// centre of the tile already fails |p - mu| <= ext, every pixel does.
__device__ __forceinline__ bool touches_tile(float4 r0, float x0, float y0) {
    const float lx = x0 + 0.5f, hx = x0 + (float)kTile - 0.5f;
    const float ly = y0 + 0.5f, hy = y0 + (float)kTile - 0.5f;
    return !(lx - r0.x > r0.z || r0.x - hx > r0.z || ly - r0.y > r0.w || r0.y - hy > r0.w);
}

// Rows of the tile (0..15) that can hold a pixel passing the AABB test of
// record piece r0, packed as yl | yh << 8 (a superset with a one-row margin
// over FP32 rounding; 0x00FF = no row, when the record misses the tile).
// Warp w blends tile rows 2w and 2w+1 and skips the record if both lie
// outside [yl, yh]: a warp-uniform branch that changes no pixel's result.
__device__ __forceinline__ int row_span(float4 r0, float x0, float y0) {
    if (!touches_tile(r0, x0, y0)) return 0x00FF;
    const int yl = (int)fmaxf(floorf(r0.y - r0.w - 0.5f - y0) - 1.0f, 0.0f);
    const int yh = (int)fminf(ceilf(r0.y + r0.w - 0.5f - y0) + 1.0f, (float)(kTile - 1));
    return yl | (yh << 8);
}

__device__ __forceinline__ bool rows_hit(int span, int warp) {
    return !(2 * warp + 1 < (span & 0xFF) || 2 * warp > (span >> 8));
}

__device__ __forceinline__ int find_view(const ViewDesc *views, int n_views, int tile) {
    int lo = 0, hi = n_views;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

// Work unit: one warp per 16x4-pixel sub-tile (a quarter of a 16x16 tile,
// a one-warp CTA), each lane blending the two vertically adjacent pixels
// (x, 2r) and (x, 2r+1).  Warps never wait for one another: each stages the
// 48-byte records of one cell at a time in its own shared memory (double
// buffered through registers), takes a ballot of the cell's Gaussians whose
// AABB reaches its sub-tile and loops over those only, and stops as soon as
// its own 64 pixels are done.  KT > 0 fixes K at compile time.
constexpr int WT = 32;       // threads per work unit
constexpr int WSUB = 4;      // sub-tiles per tile (rows 4s .. 4s+3)
constexpr int MAXPER = kRecF4 * kMaxK;  // float4s of one cell's records

// Can record piece r0 pass the AABB test at some pixel centre of the 16-wide,
// 4-high block whose first pixel is (x0, y0)?  Exactly conservative (FP32
// subtraction is monotone, so testing the nearest centres suffices).
__device__ __forceinline__ bool touches_block(float4 r0, float x0, float y0) {
    const float lx = x0 + 0.5f, hx = x0 + (float)kTile - 0.5f;
    const float ly = y0 + 0.5f, hy = y0 + (float)WSUB - 0.5f;
    return !(lx - r0.x > r0.z || r0.x - hx > r0.z || ly - r0.y > r0.w || r0.y - hy > r0.w);
}

// Stage the records of tile-list entry e (per float4s) into dst; one to three
// 16-byte loads per lane.
__device__ __forceinline__ void stage_cell(float4 *dst, const float4 *__restrict__ vrec,
                                           const uint32_t *__restrict__ cells, uint32_t e, int per, int lane,
                                           float4 pre[3]) {
    const float4 *src = vrec + (long long)__ldg(cells + e) * per;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = lane + 32 * q;
        if (i < per) pre[q] = __ldg(src + i);
    }
    (void)dst;
}

__device__ __forceinline__ void stash_cell(float4 *dst, int per, int lane, const float4 pre[3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = lane + 32 * q;
        if (i < per) dst[i] = pre[q];
    }
}

// Can record piece r0 pass the AABB test at some pixel centre of the 16-wide,
// `rows`-high block whose first pixel is (x0, y0)?  (As touches_block.)
__device__ __forceinline__ bool touches_rows(float4 r0, float x0, float y0, float rows) {
    const float lx = x0 + 0.5f, hx = x0 + (float)kTile - 0.5f;
    const float ly = y0 + 0.5f, hy = y0 + rows - 0.5f;
    return !(lx - r0.x > r0.z || r0.x - hx > r0.z || ly - r0.y > r0.w || r0.y - hy > r0.w);
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

// The forward's work unit: one warp per 16 x (2 PPL) sub-tile.  FWD_PPL = 2 (16x4 sub-tiles, 68 registers):
// 16x8 sub-tiles halve the (sub-tile, Gaussian) pairs on the benchmark scene
// but need ~95 registers (21 warps/SM) and measured no faster.
constexpr int FWD_PPL = 2;
constexpr int FWD_SUB = kTile / (2 * FWD_PPL);  // sub-tiles per tile

template <int KT, int PPL>
__device__ __forceinline__ void blend_fwd_unit(int unit, const ViewDesc *__restrict__ views, int n_views,
                                               const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                               const float4 *__restrict__ rec, const BlendParams &bp,
                                               float *__restrict__ out_rgb, float *__restrict__ out_rgb2,
                                               float *__restrict__ out_D, int *__restrict__ out_nd,
                                               float4 (*s_rec)[MAXPER]) {
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
    float4 pre[3];
    if (rg.x < rg.y) {
        stage_cell(s_rec[0], vrec, cells, rg.x, per, lane, pre);
        stash_cell(s_rec[0], per, lane, pre);
    }
    __syncwarp();
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
        if (e + 1 < rg.y) stage_cell(s_rec[buf ^ 1], vrec, cells, e + 1, per, lane, pre);
        const float4 *r = s_rec[buf];
        const float v = r[2].w;
        unsigned mask = __ballot_sync(0xffffffffu, lane < K && touches_rows(r[kRecF4 * lane], bx0, by0, (float)ROWS));
        float A0[PPL], A1[PPL], A2[PPL], B[PPL], P[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) { A0[q] = A1[q] = A2[q] = B[q] = 0.f; P[q] = 1.0f; }
        for (; mask; mask &= mask - 1) {
            const int k = __ffs(mask) - 1;
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
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                h[q] = !done[q] && hx[q & 1] && hy[q >> 1];
                any = any || h[q];
            }
            if (!any) continue;
            const float4 r1 = r[3 * k + 1];
            const float4 r2 = r[3 * k + 2];
            const float pdx[2] = {r1.x * dx[0], r1.x * dx[1]};
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                if (h[q]) {
                    const float dyq = dy[q >> 1];
                    const float s1 = fmaf(r1.y, dyq, pdx[q & 1]), s2 = r1.z * dyq;
                    const float al = fminf(r1.w * ex2_approx(-fmaf(s1, s1, s2 * s2)), bp.alpha_max);
                    A0[q] += al * r2.x; A1[q] += al * r2.y; A2[q] += al * r2.z;
                    B[q] += al;
                    P[q] -= P[q] * (v * al);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            if (!done[q]) {
                const float w = v * T[q];
                N0[q] += w * A0[q]; N1[q] += w * A1[q]; N2[q] += w * A2[q];
                D[q] += w * B[q];
                T[q] *= P[q];
                ++n[q];
            }
        }
        __syncwarp();
        if (e + 1 < rg.y) stash_cell(s_rec[buf ^ 1], per, lane, pre);
        __syncwarp();
        buf ^= 1;
    }
    const long long HW = (long long)V.W * V.H;
    float *img = V.out ? V.out : out_rgb + 3 * V.pix_base;
    float *im2 = out_rgb2 ? out_rgb2 + 3 * V.pix_base : nullptr;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        if (!(xs[q & 1] < V.W && ys[q >> 1] < V.H)) continue;
        const long long pin = (long long)ys[q >> 1] * V.W + xs[q & 1];
        const bool hit = D[q] > bp.d_min;
        const float c0 = hit ? N0[q] / D[q] : bp.bg0;
        const float c1 = hit ? N1[q] / D[q] : bp.bg1;
        const float c2 = hit ? N2[q] / D[q] : bp.bg2;
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

template <int KT>
__global__ void __launch_bounds__(WT) k_blend_fwd(const ViewDesc *__restrict__ views, int n_views,
                                                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                  const float4 *__restrict__ rec, BlendParams bp,
                                                  float *__restrict__ out_rgb, float *__restrict__ out_rgb2,
                                                  float *__restrict__ out_D, int *__restrict__ out_nd) {
    __shared__ float4 s_rec[2][MAXPER];
    blend_fwd_unit<KT, FWD_PPL>(blockIdx.x, views, n_views, ranges, cells, rec, bp, out_rgb, out_rgb2, out_D, out_nd,
                                s_rec);
}

// Persistent form for chains whose sizes live on the device: a fixed grid of
// exactly the resident warps pulls sub-tiles from an atomic counter (*work
// starts at 0) until the chain's total_tiles * FWD_SUB units are taken, so the
// dense and the empty regions of the images balance dynamically.  One
// atomic per sub-tile: their rate is bounded by the blend work between them.
template <int KT>
__global__ void __launch_bounds__(WT) k_blend_fwd_pull(const ViewDesc *__restrict__ views,
                                                       const uint2 *__restrict__ ranges,
                                                       const uint32_t *__restrict__ cells,
                                                       const float4 *__restrict__ rec, BlendParams bp,
                                                       float *__restrict__ out_rgb, float *__restrict__ out_D,
                                                       int *__restrict__ out_nd, const ChainSizes *__restrict__ dsz,
                                                       uint32_t *__restrict__ work) {
    __shared__ float4 s_rec[2][MAXPER];
    const int n_views = dsz->n_views;
    const uint32_t units = (uint32_t)dsz->total_tiles * FWD_SUB;
    for (;;) {
        uint32_t u = 0;
        if (threadIdx.x == 0) u = atomicAdd(work, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= units) break;
        blend_fwd_unit<KT, FWD_PPL>((int)u, views, n_views, ranges, cells, rec, bp, out_rgb, nullptr, out_D, out_nd,
                                    s_rec);
        __syncwarp();
    }
}

// min(units, SMs x resident CTAs of k_blend_fwd_pull<KT>), queried once.
template <int KT>
static unsigned pull_grid(int total_tiles) {
    static int per_grid = 0;
    if (!per_grid) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_fwd_pull<KT>, WT, 0);
        per_grid = std::max(1, sms * std::max(1, per_sm));
    }
    return (unsigned)std::min<long long>((long long)total_tiles * FWD_SUB, per_grid);
}

void launch_blend_fwd(const ViewDesc *views, int n_views, int total_tiles, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, float *out_rgb,
                      float *out_rgb2, float *out_D, int *out_nd, int K_all, cudaStream_t st,
                      const ChainSizes *dsz, uint32_t *work) {
    if (total_tiles == 0) return;
    if (dsz) {
        // exactly the resident warps
#define DGS_PULL(KV)                                                                                            \
        k_blend_fwd_pull<KV><<<pull_grid<KV>(total_tiles), WT, 0, st>>>(views, ranges, tile_cells, rec, bp, out_rgb, \
                                                                       out_D, out_nd, dsz, work)
        switch (K_all) {
            case 8: DGS_PULL(8); break;
            case 10: DGS_PULL(10); break;
            default: DGS_PULL(0); break;
        }
#undef DGS_PULL
        return;
    }
    const unsigned grid = (unsigned)total_tiles * FWD_SUB;
#define DGS_FWD(KV)                                                                                          \
    k_blend_fwd<KV><<<grid, WT, 0, st>>>(views, n_views, ranges, tile_cells, rec, bp, out_rgb, out_rgb2, out_D, \
                                         out_nd)
    switch (K_all) {
        case 8: DGS_FWD(8); break;
        case 10: DGS_FWD(10); break;
        default: DGS_FWD(0); break;
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
// Same work unit as the forward (one warp per 16x4 sub-tile, two pixels per
// lane, no inter-warp waits).  Per cell, the warp replays its pixels keeping
// G' of the Gaussians that reach the sub-tile in warp-private shared memory
// (registers capped at 64 so 32 warps fit per SM), updates S and T,
// then for each such Gaussian sums its pixels' nine screen-space gradient
// terms across the warp with a transposed shuffle tree (each step halves the
// values a lane carries) and adds the totals to global memory (one atomic
// add per value per sub-tile).

// Sum v[0..15] over the warp.  On return lane L holds the total of value
// 8 b1 + 4 b2 + 2 b3 + b4 (b_i = bit i of L); lanes with b0 = 1 duplicate it.
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

// Screen-space gradient terms of one (pixel, Gaussian) pair, with the
// constant factors left to the caller (applied once per reduced total):
//   acc[0..1] = sum L (s1, s2) dq'     (dmu = 2 ln 2 acc, see below)
//   acc[2..4] = sum dq' (dx^2, dx dy, dy^2)  (da, db, dc = -1/2, -1, -1/2 x acc)
//   acc[5..7] = sum v T alpha e       (drgb)
//   dop       = sum dalpha G          (dsigma)
//   dv       -= S alpha / (1 - v alpha)  (the pair's share of dL/dv, per cell)
// with dq' = G dalpha sigma = -2 dL/dq.  cA = v T_n and vS = v S_n are the
// pixel's per-cell factors.
__device__ __forceinline__ void pair_grad(float acc[8], float &dop, float &dv, float Gv, float4 r0, float4 r1,
                                          float4 r2, float px, float py, float cA, float Sn, float vS, float e0,
                                          float e1, float e2, float eD, float alpha_max) {
    const float v = r2.w, op = r1.w;
    const float raw = op * Gv;
    const float al = fminf(raw, alpha_max);
    const float rom = rcp_approx(1.0f - v * al);
    const float dal = cA * (e0 * r2.x + e1 * r2.y + e2 * r2.z + eD) - vS * rom;
    const float ca_al = cA * al;
    acc[5] += ca_al * e0;
    acc[6] += ca_al * e1;
    acc[7] += ca_al * e2;
    dv -= Sn * al * rom;
    if (raw < alpha_max) {
        const float dG = dal * Gv;
        dop += dG;
        const float dq = dG * op;
        const float dx = px - r0.x, dy = py - r0.y;
        // q = |L^T d|^2 with the record's L scaled by kappa (kappa^2 = log2(e)/2):
        // dq/dmu = -2 Q d = -(2/kappa^2) L (s1, s2), 2/kappa^2 = 4 ln 2
        const float s1 = fmaf(r1.y, dy, r1.x * dx), s2 = r1.z * dy;
        acc[0] += dq * (r1.x * s1);
        acc[1] += dq * fmaf(r1.y, s1, r1.z * s2);
        const float dqx = dq * dx;
        acc[2] += dqx * dx;
        acc[3] += dqx * dy;
        acc[4] += dq * dy * dy;
    }
}

// Constant factor of reduction slot j (see pair_grad): dL/dq = -dq'/2, so
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

template <int KT, int PPL>
__global__ void __launch_bounds__(WT, BWD_MINB) k_blend_bwd(const ViewDesc *__restrict__ views, int n_views,
                                                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                  const float4 *__restrict__ rec, BlendParams bp,
                                                  const float *__restrict__ rgb, const float *__restrict__ Dpix,
                                                  const int *__restrict__ ndpix, const float *__restrict__ dL_drgb,
                                                  float *__restrict__ g2d, float *__restrict__ g_cell_v) {
    constexpr int ROWS = 2 * PPL, NSUB = kTile / ROWS;
    __shared__ float4 s_rec[2][MAXPER];
    constexpr int KRS = KT > 0 ? KT : kMaxK;
    __shared__ float s_G[PPL][KRS][WT];
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

    int nd[PPL];
    float e0[PPL], e1[PPL], e2[PPL], eD[PPL];
    int ndm = 0;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        nd[q] = 0;
        e0[q] = e1[q] = e2[q] = eD[q] = 0.f;
        if (xs[q & 1] < V.W && ys[q >> 1] < V.H) {
            const long long pin = (long long)ys[q >> 1] * V.W + xs[q & 1];
            const float Dv = Dpix[V.pix_base + pin];
            if (Dv > bp.d_min) {
                nd[q] = ndpix[V.pix_base + pin];
                const float *gi = dL_drgb + 3 * V.pix_base;
                const float *ci = rgb + 3 * V.pix_base;
                const float g0 = gi[pin], g1 = gi[HW + pin], g2 = gi[2 * HW + pin];
                const float c0 = ci[pin], c1 = ci[HW + pin], c2 = ci[2 * HW + pin];
                const float iD = 1.0f / Dv;
                e0[q] = g0 * iD; e1[q] = g1 * iD; e2[q] = g2 * iD;
                eD[q] = -(g0 * c0 + g1 * c1 + g2 * c2) * iD;
            }
        }
        ndm = max(ndm, nd[q]);
    }
    const int ndmax = __reduce_max_sync(0xffffffffu, ndm);
    const uint2 rg = ranges[tile];
    const uint32_t end = rg.x + min((uint32_t)ndmax, rg.y - rg.x);
    const float4 *vrec = rec + V.rec_base * kRecF4;
    const bool want_v = g_cell_v != nullptr;

    float T[PPL], S[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) { T[q] = 1.0f; S[q] = 0.f; }
    float4 pre[3];
    if (rg.x < end) {
        stage_cell(s_rec[0], vrec, cells, rg.x, per, lane, pre);
        stash_cell(s_rec[0], per, lane, pre);
    }
    __syncwarp();
    int buf = 0;
    for (uint32_t e = rg.x; e < end; ++e) {
        if (e + 1 < end) stage_cell(s_rec[buf ^ 1], vrec, cells, e + 1, per, lane, pre);
        const int n = (int)(e - rg.x);
        bool act[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) act[q] = n < nd[q];
        const float4 *r = s_rec[buf];
        const float v = r[2].w;
        unsigned mask = __ballot_sync(0xffffffffu, lane < K && touches_rows(r[kRecF4 * lane], bx0, by0, (float)ROWS));
        const unsigned mask0 = mask;
        const int nhit = __popc(mask);
        // pass 1: replay the cell, keep G'; per pixel P_n and
        // X_n = dN.A_n + dD B_n = sum_k alpha_k (dN.c_k + dD)
        float X[PPL], P[PPL];
        {
#pragma unroll
            for (int q = 0; q < PPL; ++q) { X[q] = 0.f; P[q] = 1.0f; }
#pragma unroll 1
            for (int i = 0; i < nhit; ++i) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1;
#pragma unroll
                for (int q = 0; q < PPL; ++q) s_G[q][i][lane] = 0.f;
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
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    h[q] = act[q] && hx[q & 1] && hy[q >> 1];
                    any = any || h[q];
                }
                if (!any) continue;
                const float4 r1 = r[3 * k + 1];
                const float4 r2 = r[3 * k + 2];
                const float pdx[2] = {r1.x * dx[0], r1.x * dx[1]};
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    if (h[q]) {
                        const float dyq = dy[q >> 1];
                        const float s1 = fmaf(r1.y, dyq, pdx[q & 1]), s2 = r1.z * dyq;
                        const float Gv = ex2_approx(-fmaf(s1, s1, s2 * s2));
                        s_G[q][i][lane] = Gv;
                        const float al = fminf(r1.w * Gv, bp.alpha_max);
                        X[q] += al * fmaf(e0[q], r2.x, fmaf(e1[q], r2.y, fmaf(e2[q], r2.z, eD[q])));
                        P[q] -= P[q] * (v * al);
                    }
                }
            }
        }
        // per-pixel transmittance bookkeeping (S_n includes x_n); the cell
        // term of dL/dv, sum over pixels of T_n X_n, joins the Gaussians'
        // terms below so one reduction per cell carries dL/dv
        float Tn[PPL];
        float dv = 0.f;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            Tn[q] = T[q];
            if (act[q]) {
                S[q] -= v * Tn[q] * X[q];
                T[q] *= P[q];
                dv += Tn[q] * X[q];
            }
        }
        const uint32_t cellid = __ldg(cells + e);
        float *gbase = g2d + (V.rec_base + (long long)cellid * K) * kGradF;
        // pass 2: gradient terms per Gaussian reaching the sub-tile (not
        // unrolled: the body is large and the instruction cache is the limit)
        unsigned m2 = mask0;
#pragma unroll 1
        for (int i = 0; m2; ++i, m2 &= m2 - 1) {
            float gv[PPL];
            bool any = false;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                gv[q] = s_G[q][i][lane];
                any = any || gv[q] > 0.f;
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const int k = __ffs(m2) - 1;
            const float4 r0 = r[3 * k], r1 = r[3 * k + 1], r2 = r[3 * k + 2];
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = 0.f;
            float dop = 0.f;
#pragma unroll
            for (int q = 0; q < PPL; ++q)
                if (gv[q] > 0.f)
                    pair_grad(acc, dop, dv, gv[q], r0, r1, r2, pxs[q & 1], pys[q >> 1], v * Tn[q], S[q], v * S[q],
                              e0[q], e1[q],
                              e2[q], eD[q], bp.alpha_max);
            const float tot = transposed_warp_sum8(acc, lane);
            const float dop_tot = warp_sum(dop);
            float *gk = gbase + k * kGradF;
            const int slot = transposed_owner8(lane);
            if ((lane & 3) == 0 && tot != 0.f) atomicAdd(gk + grad_slot(slot), tot * slot_scale(slot));
            if (lane == 1 && dop_tot != 0.f) atomicAdd(gk + 5, dop_tot);
        }
        if (want_v) {  // per (view, cell) entry: v_n may differ between views
            dv = warp_sum(dv);
            if (lane == 0 && dv != 0.f) atomicAdd(g_cell_v + V.cell_base + cellid, dv);
        }
        __syncwarp();
        if (e + 1 < end) stash_cell(s_rec[buf ^ 1], per, lane, pre);
        __syncwarp();
        buf ^= 1;
    }
}

// K_all: K of the chain's scene (compile-time loop for common values)
void launch_blend_bwd(const ViewDesc *views, int n_views, int total_tiles, int K_all, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, const float *rgb,
                      const float *D, const int *nd, const float *dL_drgb, float *g2d, float *g_cell_v,
                      cudaStream_t st) {
    if (total_tiles == 0) return;
    const unsigned grid = (unsigned)total_tiles * BWD_SUB;
#define DGS_BWD(KV)                                                                                             \
    k_blend_bwd<KV, BWD_PPL><<<grid, WT, 0, st>>>(views, n_views, ranges, tile_cells, rec, bp, rgb, D, nd, dL_drgb, \
                                                  g2d, g_cell_v)
    switch (K_all) {
        case 8: DGS_BWD(8); break;
        case 10: DGS_BWD(10); break;
        default: DGS_BWD(0); break;
    }
#undef DGS_BWD
}

}  // namespace dgs
