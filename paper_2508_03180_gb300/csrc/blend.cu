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

// Forward: 128 threads per 16x16 tile, each thread blends the two
// vertically adjacent pixels (x, 2r) and (x, 2r+1), so a record fetched from
// shared memory, its tile-row test and the x half of its AABB test serve two
// pixels; warp w owns tile rows 4w..4w+3.  KT > 0 fixes K at compile time.
constexpr int FT = 128;

__device__ __forceinline__ bool rows_hit4(int span, int warp) {
    return !(4 * warp + 3 < (span & 0xFF) || 4 * warp > (span >> 8));
}

template <int KT>
__global__ void __launch_bounds__(FT) k_blend_fwd(const ViewDesc *__restrict__ views, int n_views,
                                                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                  const float4 *__restrict__ rec, BlendParams bp,
                                                  float *__restrict__ out_rgb, float *__restrict__ out_rgb2,
                                                  float *__restrict__ out_D, int *__restrict__ out_nd) {
    __shared__ float4 s_rec[2][FT];
    __shared__ int s_span[2][FT / kRecF4 + 1];  // row span of each record in this tile
    __shared__ int s_view;
    const int tid = threadIdx.x, tile = blockIdx.x, warp = tid >> 5;
    if (tid == 0) s_view = find_view(views, n_views, tile);
    __syncthreads();
    const ViewDesc &V = views[s_view];
    const int local = tile - V.tile_base;
    const int tx = local % V.Tx, ty = local / V.Tx;
    const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
    const int xi = tx * kTile + (tid & (kTile - 1));
    const int yi0 = ty * kTile + 2 * (tid >> 4), yi1 = yi0 + 1;
    const bool in0 = xi < V.W && yi0 < V.H, in1 = xi < V.W && yi1 < V.H;
    const float px = (float)xi + 0.5f, py0 = (float)yi0 + 0.5f, py1 = (float)yi1 + 0.5f;

    const int K = KT > 0 ? KT : V.K;
    const int per = kRecF4 * K;               // float4s per cell
    const int CH = max(1, FT / per);          // cells per chunk
    const int nload = CH * per;
    const float4 *vrec = rec + V.rec_base * kRecF4;
    const uint2 rg = ranges[tile];

    float T0 = 1.0f, N00 = 0.f, N01 = 0.f, N02 = 0.f, D0 = 0.f;
    float T1 = 1.0f, N10 = 0.f, N11 = 0.f, N12 = 0.f, D1 = 0.f;
    int n0 = 0, n1 = 0;
    bool done0 = !in0, done1 = !in1;
    float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t cur = rg.x;
    if (cur < rg.y) {
        pre = fetch_rec(vrec, cells, cur, rg.y, tid, nload, per, pre);
        s_rec[0][tid] = pre;
        if (tid < nload && tid % kRecF4 == 0) s_span[0][tid / kRecF4] = row_span(pre, tx0, ty0);
    }
    __syncthreads();
    int buf = 0;
    while (cur < rg.y) {
        const int nc = (int)min((uint32_t)CH, rg.y - cur);
        const uint32_t nxt = cur + nc;
        if (nxt < rg.y) pre = fetch_rec(vrec, cells, nxt, rg.y, tid, nload, per, pre);
        for (int c = 0; c < nc; ++c) {
            // before cell n a pixel stops if T_n < eps (Sec. V-B)
            done0 = done0 || T0 < bp.eps;
            done1 = done1 || T1 < bp.eps;
            if (done0 && done1) break;
            const float4 *r = &s_rec[buf][c * per];
            const int *sp = &s_span[buf][c * K];
            const float v = r[2].w;
            float A00 = 0.f, A01 = 0.f, A02 = 0.f, B0 = 0.f, P0 = 1.0f;
            float A10 = 0.f, A11 = 0.f, A12 = 0.f, B1 = 0.f, P1 = 1.0f;
#pragma unroll (KT > 0 ? KT : 1)
            for (int k = 0; k < K; ++k) {
                if (!rows_hit4(sp[k], warp)) continue;
                const float4 r0 = r[3 * k];
                const float dx = px - r0.x;
                if (!(fabsf(dx) <= r0.z)) continue;
                const float dy0 = py0 - r0.y, dy1 = py1 - r0.y;
                const bool h0 = !done0 && fabsf(dy0) <= r0.w;
                const bool h1 = !done1 && fabsf(dy1) <= r0.w;
                if (!(h0 || h1)) continue;
                const float4 r1 = r[3 * k + 1];
                const float4 r2 = r[3 * k + 2];
                const float qx = r1.x * dx * dx;
                const float bx = r1.y * dx;
                if (h0) {
                    const float al = fminf(r1.w * ex2_approx(qx + (bx + r1.z * dy0) * dy0), bp.alpha_max);
                    A00 += al * r2.x; A01 += al * r2.y; A02 += al * r2.z;
                    B0 += al;
                    P0 -= P0 * (v * al);
                }
                if (h1) {
                    const float al = fminf(r1.w * ex2_approx(qx + (bx + r1.z * dy1) * dy1), bp.alpha_max);
                    A10 += al * r2.x; A11 += al * r2.y; A12 += al * r2.z;
                    B1 += al;
                    P1 -= P1 * (v * al);
                }
            }
            if (!done0) {
                const float w = v * T0;
                N00 += w * A00; N01 += w * A01; N02 += w * A02;
                D0 += w * B0;
                T0 *= P0;
                ++n0;
            }
            if (!done1) {
                const float w = v * T1;
                N10 += w * A10; N11 += w * A11; N12 += w * A12;
                D1 += w * B1;
                T1 *= P1;
                ++n1;
            }
        }
        done0 = done0 || T0 < bp.eps;
        done1 = done1 || T1 < bp.eps;
        if (nxt < rg.y) {
            s_rec[buf ^ 1][tid] = pre;
            if (tid < nload && tid % kRecF4 == 0) s_span[buf ^ 1][tid / kRecF4] = row_span(pre, tx0, ty0);
        }
        if (__syncthreads_count(done0 && done1) == FT) break;
        buf ^= 1;
        cur = nxt;
    }
    const long long HW = (long long)V.W * V.H;
    float *img = V.out ? V.out : out_rgb + 3 * V.pix_base;
    float *im2 = out_rgb2 ? out_rgb2 + 3 * V.pix_base : nullptr;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q == 0 ? in0 : in1)) continue;
        const float D = q == 0 ? D0 : D1;
        const long long pin = (long long)(q == 0 ? yi0 : yi1) * V.W + xi;
        const bool hit = D > bp.d_min;
        const float c0 = hit ? (q == 0 ? N00 : N10) / D : bp.bg0;
        const float c1 = hit ? (q == 0 ? N01 : N11) / D : bp.bg1;
        const float c2 = hit ? (q == 0 ? N02 : N12) / D : bp.bg2;
        img[pin] = c0;
        img[HW + pin] = c1;
        img[2 * HW + pin] = c2;
        if (im2) {
            im2[pin] = c0;
            im2[HW + pin] = c1;
            im2[2 * HW + pin] = c2;
        }
        out_D[V.pix_base + pin] = D;
        out_nd[V.pix_base + pin] = q == 0 ? n0 : n1;
    }
}

// K of the chain's views when they all share one (compile-time loop), else 0
void launch_blend_fwd(const ViewDesc *views, int n_views, int total_tiles, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, float *out_rgb,
                      float *out_rgb2, float *out_D, int *out_nd, int K_all, cudaStream_t st) {
    if (total_tiles == 0) return;
#define DGS_FWD(KV)                                                                                              \
    k_blend_fwd<KV><<<total_tiles, FT, 0, st>>>(views, n_views, ranges, tile_cells, rec, bp, out_rgb, out_rgb2, \
                                                out_D, out_nd)
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
// Phase 1 (thread = pixel) replays a chunk of cells, writing G' per
// (Gaussian touching the tile, pixel) and T_n, S_n per (cell, pixel) to
// shared memory.  Phase 2 (warp = Gaussian) walks only the pixels of the
// Gaussian's AABB inside the tile, sums its nine screen-space gradients in
// registers, reduces them across the warp with a transposed shuffle tree
// (each step halves the values each lane carries) and issues one atomic add
// per value.  Gaussians whose AABB misses the tile cost one flag test.
constexpr int BW_G = 32;  // Gaussians per chunk (shared G' table = 32 x 256 floats)
constexpr int BW_CH = 8;  // cells per chunk at most

__host__ __device__ constexpr int bwd_cells_per_chunk(int K) {
    return BW_G / K < 1 ? 1 : (BW_G / K > BW_CH ? BW_CH : BW_G / K);
}

// Sum v[0..15] over the warp.  On return lane L holds the total of value
// 8 b1 + 4 b2 + 2 b3 + b4 (b_i = bit i of L); lanes with b0 = 1 duplicate it.
__device__ __forceinline__ float transposed_warp_sum16(float v[16], int lane) {
#pragma unroll
    for (int step = 0; step < 4; ++step) {
        const int bit = 16 >> step;
        const bool hi = lane & bit;
        const int n = 8 >> step;  // pairs at this step
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const float keep = hi ? v[2 * i + 1] : v[2 * i];
            const float send = hi ? v[2 * i] : v[2 * i + 1];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ int transposed_owner(int lane) {
    return ((lane >> 1) & 1) * 8 + ((lane >> 2) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 4) & 1);
}

__global__ void __launch_bounds__(BT, 4) k_blend_bwd(const ViewDesc *__restrict__ views, int n_views,
                                                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ cells,
                                                  const float4 *__restrict__ rec, BlendParams bp,
                                                  const float *__restrict__ rgb, const float *__restrict__ Dpix,
                                                  const int *__restrict__ ndpix, const float *__restrict__ dL_drgb,
                                                  float *__restrict__ g2d, float *__restrict__ g_cell_v) {
    extern __shared__ float4 smem_f4[];
    __shared__ int s_view, s_ndmax, s_task;
    __shared__ int s_flag[2][BW_G];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    if (tid == 0) { s_view = find_view(views, n_views, tile); s_ndmax = 0; }
    __syncthreads();
    const ViewDesc &V = views[s_view];
    const int K = V.K;
    const int per = kRecF4 * K;
    const int CH = bwd_cells_per_chunk(K);
    const int nrec = CH * per;                     // float4s per chunk (<= 3 * BW_G < BT)
    float4 *s_rec0 = smem_f4;                      // [2][nrec]
    float4 *sdN = smem_f4 + 2 * nrec;              // [BT]: dL/dN xyz, dL/dD per pixel
    float2 *sTS = reinterpret_cast<float2 *>(sdN + BT);  // [CH][BT]: T_n, S_n per (cell, pixel)
    float *sG = reinterpret_cast<float *>(sTS + CH * BT);  // [CH*K][BT]
    float *sTX = sG + CH * K * BT;                 // [CH][BT]: T_n X_n for dL/dv
    const int local = tile - V.tile_base;
    const int tx = local % V.Tx, ty = local / V.Tx;
    const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
    const int xi = tx * kTile + (tid & (kTile - 1)), yi = ty * kTile + (tid >> 4);
    const bool inside = xi < V.W && yi < V.H;
    const float px = (float)xi + 0.5f, py = (float)yi + 0.5f;
    const long long HW = (long long)V.W * V.H;
    const long long pin = (long long)yi * V.W + xi;

    int nd = 0;
    float dN0 = 0.f, dN1 = 0.f, dN2 = 0.f, dD = 0.f;
    if (inside) {
        const float Dv = Dpix[V.pix_base + pin];
        if (Dv > bp.d_min) {
            nd = ndpix[V.pix_base + pin];
            const float *gi = dL_drgb + 3 * V.pix_base;
            const float *ci = rgb + 3 * V.pix_base;
            const float g0 = gi[pin], g1 = gi[HW + pin], g2 = gi[2 * HW + pin];
            const float c0 = ci[pin], c1 = ci[HW + pin], c2 = ci[2 * HW + pin];
            const float iD = 1.0f / Dv;
            dN0 = g0 * iD; dN1 = g1 * iD; dN2 = g2 * iD;
            dD = -(g0 * c0 + g1 * c1 + g2 * c2) * iD;
        }
    }
    sdN[tid] = make_float4(dN0, dN1, dN2, dD);
    if (nd > 0) atomicMax(&s_ndmax, nd);
    __syncthreads();
    const uint2 rg = ranges[tile];
    const uint32_t end = rg.x + min((uint32_t)s_ndmax, rg.y - rg.x);
    const float4 *vrec = rec + V.rec_base * kRecF4;
    const bool want_v = g_cell_v != nullptr;

    float T = 1.0f, S = 0.0f;
    float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t cur = rg.x;
    if (cur < end) {
        pre = fetch_rec(vrec, cells, cur, end, tid, nrec, per, pre);
        if (tid < nrec) {
            s_rec0[tid] = pre;
            if (tid % kRecF4 == 0) s_flag[0][tid / kRecF4] = row_span(pre, tx0, ty0);
        }
    }
    __syncthreads();
    int buf = 0;
    while (cur < end) {
        const int nc = (int)min((uint32_t)CH, end - cur);
        const uint32_t nxt = cur + nc;
        if (nxt < end) pre = fetch_rec(vrec, cells, nxt, end, tid, nrec, per, pre);
        const float4 *sr = s_rec0 + buf * nrec;
        const int *fl = s_flag[buf];
        // ---- phase 1: replay per pixel
        if (tid == 0) s_task = 0;
        for (int c = 0; c < nc; ++c) {
            const int n = (int)(cur - rg.x) + c;
            const float4 *r = sr + c * per;
            if (n < nd) {
                const float v = r[2].w;
                float A0 = 0.f, A1 = 0.f, A2 = 0.f, B = 0.f, P = 1.0f;
                for (int k = 0; k < K; ++k) {
                    if (!rows_hit(fl[c * K + k], warp)) continue;
                    const float4 r0 = r[3 * k];
                    const float dx = px - r0.x, dy = py - r0.y;
                    float Gv = 0.f;
                    if (fabsf(dx) <= r0.z && fabsf(dy) <= r0.w) {
                        const float4 r1 = r[3 * k + 1];
                        const float4 r2 = r[3 * k + 2];
                        Gv = ex2_approx(r1.x * dx * dx + r1.y * dx * dy + r1.z * dy * dy);
                        const float al = fminf(r1.w * Gv, bp.alpha_max);
                        A0 += al * r2.x; A1 += al * r2.y; A2 += al * r2.z;
                        B += al;
                        P -= P * (v * al);
                    }
                    sG[(c * K + k) * BT + tid] = Gv;
                }
                const float X = dN0 * A0 + dN1 * A1 + dN2 * A2 + dD * B;
                S -= v * T * X;
                sTS[c * BT + tid] = make_float2(T, S);
                sTX[c * BT + tid] = T * X;
                T *= P;
            } else {
                for (int k = 0; k < K; ++k)
                    if (rows_hit(fl[c * K + k], warp)) sG[(c * K + k) * BT + tid] = 0.f;
                sTX[c * BT + tid] = 0.f;
            }
        }
        __syncthreads();
        // ---- phase 2: per Gaussian, over its AABB within the tile; warps take
        // the next task from a shared counter so uneven windows balance out
        const int n_tasks = nc * K + (want_v ? nc : 0);
        for (;;) {
            int j = 0;
            if (lane == 0) j = atomicAdd(&s_task, 1);
            j = __shfl_sync(0xffffffffu, j, 0);
            if (j >= n_tasks) break;
            if (j >= nc * K) {  // per-cell term of dL/dv: sum_p T_n X over the tile
                const int c = j - nc * K;
                float a = 0.f;
#pragma unroll
                for (int q = 0; q < BT / 32; ++q) a += sTX[c * BT + lane + 32 * q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0 && a != 0.f) atomicAdd(g_cell_v + cells[cur + c], a);
                continue;
            }
            const int span = fl[j];
            if ((span & 0xFF) > (span >> 8)) continue;  // misses the tile
            const int c = j / K, k = j - c * K;
            const float4 r0 = sr[c * per + 3 * k], r1 = sr[c * per + 3 * k + 1], r2 = sr[c * per + 3 * k + 2];
            const float v = r2.w, op = r1.w;
            const float ca = -2.0f * LN2 * r1.x, cb = -LN2 * r1.y, cc = -2.0f * LN2 * r1.z;  // real conic
            // columns of the tile that can lie in the AABB (a superset; sG decides);
            // rows [yl, yh] are exactly those whose warps wrote sG for this record
            const int xl = (int)fmaxf(floorf(r0.x - r0.z - 0.5f - tx0) - 1.0f, 0.0f);
            const int xh = (int)fminf(ceilf(r0.x + r0.z - 0.5f - tx0) + 1.0f, (float)(kTile - 1));
            const int yl = span & 0xFF, yh = span >> 8;
            const int w = xh - xl + 1;
            const int npx = w * (yh - yl + 1);
            const float inv_w = 1.0f / (float)w;
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.f;
            bool any = false;
            for (int i = lane; i < npx; i += 32) {
                const int row = (int)(((float)i + 0.5f) * inv_w);  // exact: i < 256, w <= 16
                const int xx = xl + i - row * w, yy = yl + row;
                const int p = yy * kTile + xx;
                const float Gv = sG[j * BT + p];
                if (Gv == 0.f) continue;
                any = true;
                const float2 ts = sTS[c * BT + p];
                const float4 e = sdN[p];
                const float raw = op * Gv;
                const float al = fminf(raw, bp.alpha_max);
                const float cA = v * ts.x;
                const float rom = __frcp_rn(1.0f - v * al);
                const float dal = cA * (e.x * r2.x + e.y * r2.y + e.z * r2.z + e.w) - v * ts.y * rom;
                const float ca_al = cA * al;
                acc[6] += ca_al * e.x;
                acc[7] += ca_al * e.y;
                acc[8] += ca_al * e.z;
                acc[9] -= ts.y * al * rom;
                if (raw < bp.alpha_max) {
                    acc[5] += dal * Gv;
                    const float dq = -0.5f * Gv * (dal * op);
                    const float dx = (tx0 + (float)xx + 0.5f) - r0.x;
                    const float dy = (ty0 + (float)yy + 0.5f) - r0.y;
                    acc[0] -= dq * 2.0f * (ca * dx + cb * dy);
                    acc[1] -= dq * 2.0f * (cb * dx + cc * dy);
                    acc[2] += dq * dx * dx;
                    acc[3] += dq * 2.0f * dx * dy;
                    acc[4] += dq * dy * dy;
                }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float tot = transposed_warp_sum16(acc, lane);
            const int idx = transposed_owner(lane);
            if ((lane & 1) == 0 && tot != 0.f) {
                const uint32_t cellid = cells[cur + c];
                if (idx < 9) atomicAdd(g2d + (V.rec_base + (long long)cellid * K + k) * kGradF + idx, tot);
                else if (idx == 9 && want_v) atomicAdd(g_cell_v + cellid, tot);
            }
        }
        if (nxt < end && tid < nrec) {
            s_rec0[(buf ^ 1) * nrec + tid] = pre;
            if (tid % kRecF4 == 0) s_flag[buf ^ 1][tid / kRecF4] = row_span(pre, tx0, ty0);
        }
        __syncthreads();
        buf ^= 1;
        cur = nxt;
    }
}

static size_t bwd_smem_bytes(int K) {
    const int per = kRecF4 * K;
    const int CH = bwd_cells_per_chunk(K);
    return sizeof(float4) * (2 * CH * per + BT) + sizeof(float2) * CH * BT + sizeof(float) * ((size_t)CH * K * BT + CH * BT);
}

// K: Gaussians per cell of the chain's scene (shared-memory sizing)
void launch_blend_bwd(const ViewDesc *views, int n_views, int total_tiles, int K, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, const float *rgb,
                      const float *D, const int *nd, const float *dL_drgb, float *g2d, float *g_cell_v,
                      cudaStream_t st) {
    if (total_tiles == 0) return;
    const size_t sm = bwd_smem_bytes(K);
    cudaFuncSetAttribute(k_blend_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_blend_bwd<<<total_tiles, BT, sm, st>>>(views, n_views, ranges, tile_cells, rec, bp, rgb, D, nd, dL_drgb, g2d,
                                             g_cell_v);
}

}  // namespace dgs
