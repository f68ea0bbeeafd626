// Decode of neural cells (the step before the path): the K Gaussians of a
// visible cell are predicted per view from the cell's latent feature f_n,
// the viewing distance delta_n and direction d_n by four MLPs with one ReLU
// hidden layer, F_sigma, F_c, F_s, F_q (Sec. III, Eq. 1-7; Sec. IV-A, Eq.
// 8-11).  Activations: opacity tanh (sigma <= 0 is not drawn), colour
// sigmoid, scale ratio sigmoid bounded by 1 - |O_pos| (Eq. 11) times the cell
// semi-axes S_n (Eq. 8), rotation normalised (a zero output is the identity
// rotation); centre x_n + R(Q_n)(O_pos * S_n) with O_pos moved into the unit
// ball (the centre stays inside the cell).
//
// The unit of work is a sample: one (view, cell) entry that survived culling
// (the first entries of the depth-sorted entry list).  A CTA takes M samples
// at a time (8 per warp: 64 with eight warps, fewer where the widths need
// more shared memory) and runs the four decoders as two dense products from
// shared memory:
//   layer 1  H[M x 4Hp] = relu(Z[M x I] W1^T + b1)   (the decoders side by side)
//   layer 2  O[M x Rp]  = H_D W2_D^T + b2 per decoder  (block diagonal)
// with I = F + 4 inputs, Hp = H rounded up (zero hidden units) and the
// decoders' output blocks rounded up to 4 (zero outputs), Rp in total.  A
// lane keeps 8 samples x 4 (or 8) outputs in registers; the inputs of a
// sample are broadcast to the warp, the weights are read as float4 rows.
// Sample-minor arrays keep one row per unit with the M samples contiguous
// (row stride M + 4 floats); decoder blocks are staggered by 8 floats so lanes
// of different decoders reading the same row index hit distinct banks.
#include <algorithm>

#include "project.cuh"
#include "tc.cuh"

namespace dgs {

constexpr int DINFO = 24;     // words of per-sample information (a record of k_decode_samples)
constexpr int kSmemMax = 227 * 1024;

struct MlpShape {
    int W, M, LD;                        // warps per CTA, samples per tile (8 per warp), sample-row stride
    int dbuf;                            // adjoint: two weight buffers (copies overlap the phase before)
    int F, H, K, I, Hp, HW, P;
    int nout[4], rb[5];                  // output widths; padded output block bases (rb[4] = Rp)
    int w1o[4], b1o[4], w2o[4], b2o[4];  // packed weight offsets per decoder
    // shared-memory layout (floats)
    int s_w, s_w2, s_b1, s_b2, s_z, s_h, s_o, s_dh, s_info, s_total;
    // backward rows per sample: Z [I], H [4Hp], dL/dh [4Hp], dL/do [Rp]
    int row_z, row_h, row_dh, row_do, row_all;
    // the weights in their shared-memory layouts, packed once per call in global memory:
    // W1^T [I][4Hp], b1 [4Hp], b2 [Rp], W2^T [Hp][Rp], W2 [Rp][Hp], W1 [4Hp][I]
    int g_w1t, g_b1, g_b2, g_w2t, g_w2, g_w1r, g_total;
};

static int up_to(int x, int m) { return (x + m - 1) / m * m; }

// Layout for W warps per CTA (W = 8, 4 or 2: the largest whose shared memory fits).
static MlpShape mlp_shape_w(int F, int H, int K, bool bwd, int W, bool dbuf) {
    MlpShape S{};
    S.W = W; S.M = 8 * W; S.LD = S.M + 4;
    S.dbuf = bwd && dbuf;
    const int DM = S.M, DLM = S.LD;
    S.F = F; S.H = H; S.K = K; S.I = F + 4;
    S.HW = 4 * up_to(H, 4) <= 128 ? 4 : 8;
    S.Hp = up_to(H, S.HW);
    const int outs[4] = {K, 3 * K, 3 * K, 4 * K};
    int o = 0;
    S.rb[0] = 0;
    for (int D = 0; D < 4; ++D) {
        S.nout[D] = outs[D];
        S.rb[D + 1] = S.rb[D] + up_to(outs[D], 4);
        S.w1o[D] = o; S.b1o[D] = o + H * S.I; S.w2o[D] = S.b1o[D] + H; S.b2o[D] = S.w2o[D] + outs[D] * H;
        o = S.b2o[D] + outs[D];
    }
    S.P = o;
    const int Rp = S.rb[4], H4 = 4 * S.Hp;
    int at = 0;
    auto take = [&](int n) { const int r = at; at += up_to(n, 4); return r; };
    S.s_w = take(std::max(S.I * H4, S.Hp * Rp));
    S.s_w2 = S.dbuf ? take(std::max(S.I * H4, S.Hp * Rp)) : S.s_w;  // the adjoint's second weight buffer
    S.s_b1 = take(H4);
    S.s_b2 = take(Rp);
    S.s_z = take(S.I * DLM);
    S.s_h = take(4 * (S.Hp * DLM + 8));
    S.s_o = take(Rp * DLM + 32);
    S.s_dh = bwd ? take(4 * (S.Hp * DLM + 8)) : 0;
    S.s_info = take(DM * DINFO);
    S.s_total = at;
    S.row_z = 0; S.row_h = S.I; S.row_dh = S.row_h + H4; S.row_do = S.row_dh + H4; S.row_all = S.row_do + Rp;
    at = 0;
    S.g_w1t = take(S.I * H4);
    S.g_b1 = take(H4);
    S.g_b2 = take(Rp);
    S.g_w2t = take(S.Hp * Rp);
    S.g_w2 = take(Rp * S.Hp);
    S.g_w1r = take(H4 * S.I);
    S.g_total = at;
    return S;
}

// The adjoint's weight gradients in registers (k_decode_bwd<4, true>): tiles
// of FW_M samples, thread t holding row t of dW1 (over all decoders) and of
// dW2, so 4Hp and Rp at most the CTA's threads, I <= FW_I, Hp <= FW_H.
constexpr int FW_I = 40, FW_H = 32, FW_M = 32;
static bool wgrad_fused(const MlpShape &S) {
    const int threads = 32 * S.W;
    return S.HW == 4 && S.M == FW_M && 4 * S.Hp <= threads && S.rb[4] <= threads && S.I <= FW_I && S.Hp <= FW_H;
}

// Two CTAs per SM where the shared memory allows (one CTA's barrier waits
// overlap the other's products), else the largest tile that fits; the
// adjoint prefers the fused weight gradients, then two weight buffers, then one.
static MlpShape mlp_shape(int F, int H, int K, bool bwd) {
    if (bwd)
        for (int db = 1; db >= 0; --db) {
            const MlpShape S = mlp_shape_w(F, H, K, true, FW_M / 8, db);
            if (wgrad_fused(S) && 2 * sizeof(float) * (size_t)S.s_total <= (size_t)kSmemMax) return S;
        }
    for (int db = bwd ? 1 : 0; db >= 0; --db) {
        for (int W = 8; W >= 2; W /= 2) {
            const MlpShape S = mlp_shape_w(F, H, K, bwd, W, db);
            if (2 * sizeof(float) * (size_t)S.s_total <= (size_t)kSmemMax) return S;
        }
        for (int W = 8; W >= 2; W /= 2) {
            const MlpShape S = mlp_shape_w(F, H, K, bwd, W, db);
            if (sizeof(float) * (size_t)S.s_total <= (size_t)kSmemMax) return S;
        }
    }
    return mlp_shape_w(F, H, K, bwd, 2, false);
}

// Logistic and tanh from the fast exponential and a fast divide (about 1e-6
// relative error; the decode and its adjoint use the same functions, so the
// adjoint sees the forward's values and decisions).
__device__ __forceinline__ float sigmoid_fast(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float tanh_fast(float x) { return 1.0f - __fdividef(2.0f, 1.0f + __expf(2.0f * x)); }
__device__ __forceinline__ int hrow(const MlpShape &S, int D, int j) { return D * (S.Hp * S.LD + 8) + j * S.LD; }
__device__ __forceinline__ int orow(const MlpShape &S, int D, int r) { return (S.rb[D] + r) * S.LD + 8 * D; }
__device__ __forceinline__ int out_block(const MlpShape &S, int rr) {
    return rr >= S.rb[3] ? 3 : (rr >= S.rb[2] ? 2 : (rr >= S.rb[1] ? 1 : 0));
}

// Per-sample information in shared memory.
struct SampleInfo {
    int n, valid;
    long long rec;   // first record (Gaussian k = 0) of this (view, cell)
    float x[3], S[3], R[9];
    float z4[4];     // distance and unit direction from the eye (the last four inputs)
    int v;           // the view
};
__device__ __forceinline__ void put_info(float *s_info, int s, const SampleInfo &a) {
    float *p = s_info + s * DINFO;
    p[0] = __int_as_float(a.n);
    p[1] = __int_as_float(a.valid);
    p[2] = __int_as_float((int)(a.rec & 0xffffffffLL));
    p[3] = __int_as_float((int)(a.rec >> 32));
#pragma unroll
    for (int i = 0; i < 3; ++i) { p[4 + i] = a.x[i]; p[7 + i] = a.S[i]; }
#pragma unroll
    for (int i = 0; i < 9; ++i) p[10 + i] = a.R[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[19 + i] = a.z4[i];
    p[23] = __int_as_float(a.v);
}
__device__ __forceinline__ SampleInfo get_info(const float *s_info, int s) {
    const float *p = s_info + s * DINFO;
    SampleInfo a;
    a.n = __float_as_int(p[0]);
    a.valid = __float_as_int(p[1]);
    a.rec = (long long)(unsigned)__float_as_int(p[2]) | ((long long)__float_as_int(p[3]) << 32);
#pragma unroll
    for (int i = 0; i < 3; ++i) { a.x[i] = p[4 + i]; a.S[i] = p[7 + i]; }
#pragma unroll
    for (int i = 0; i < 9; ++i) a.R[i] = p[10 + i];
#pragma unroll
    for (int i = 0; i < 4; ++i) a.z4[i] = p[19 + i];
    a.v = __float_as_int(p[23]);
    return a;
}

// One record per sample (DINFO words): the view holding entry e (binary
// search over the views' first entries), the cell, its first record, frame
// and the last four inputs; invalid for entries of another scene slot.
__global__ void __launch_bounds__(128) k_decode_samples(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                        SceneDev sc, const uint32_t *__restrict__ samples,
                                                        long long nsamp,
                                                        const uint32_t *__restrict__ d_n, float *__restrict__ srec) {
    if (d_n) nsamp = min(nsamp, (long long)*d_n);  // the count on the device (capacity nsamp)
    const long long N = sc.N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nsamp;
         q += (long long)gridDim.x * blockDim.x) {
        SampleInfo a{};
        a.valid = 0;
        const long long e = samples ? (long long)samples[q] : q;
        int lo = 0, hi = n_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (views[mid].cell_base <= e) lo = mid; else hi = mid - 1;
        }
        const ViewDesc &Vw = views[lo];
        const long long n = e - Vw.cell_base;
        if (Vw.scene_slot == slot && n >= 0 && n < N) {
            a.valid = 1;
            a.n = (int)n;
            a.v = lo;
            a.rec = Vw.rec_base + n * sc.K;
#pragma unroll
            for (int i = 0; i < 3; ++i) { a.x[i] = sc.cell[i * N + n]; a.S[i] = sc.cell[(3 + i) * N + n]; }
            const float qw = sc.cell[6 * N + n], qx = sc.cell[7 * N + n], qy = sc.cell[8 * N + n],
                        qz = sc.cell[9 * N + n];
            const float in = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            const float w = qw * in, x = qx * in, y = qy * in, z = qz * in;
            a.R[0] = 1.f - 2.f * (y * y + z * z); a.R[1] = 2.f * (x * y - w * z); a.R[2] = 2.f * (x * z + w * y);
            a.R[3] = 2.f * (x * y + w * z); a.R[4] = 1.f - 2.f * (x * x + z * z); a.R[5] = 2.f * (y * z - w * x);
            a.R[6] = 2.f * (x * z - w * y); a.R[7] = 2.f * (y * z + w * x); a.R[8] = 1.f - 2.f * (x * x + y * y);
            const float r0 = a.x[0] - Vw.eye[0], r1 = a.x[1] - Vw.eye[1], r2 = a.x[2] - Vw.eye[2];
            const float delta = sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
            a.z4[0] = delta; a.z4[1] = r0 / delta; a.z4[2] = r1 / delta; a.z4[3] = r2 / delta;
        }
        float rec[DINFO];
        put_info(rec, 0, a);
        float4 *dst = reinterpret_cast<float4 *>(srec + q * DINFO);
#pragma unroll
        for (int i = 0; i < DINFO / 4; ++i) dst[i] = make_float4(rec[4 * i], rec[4 * i + 1], rec[4 * i + 2], rec[4 * i + 3]);
    }
}

// Every Gaussian's centre x_n + R(Q_n)(O_pos S_n) and Eq. 11 bound 1 - |O_pos|
// (the same in every view), for the forward's epilogue.
__global__ void __launch_bounds__(128) k_decode_centres(SceneDev sc, float4 *__restrict__ gc) {
    const long long N = sc.N, G = sc.G;
    const int K = sc.K;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long n = g / K;
        const float qw = sc.cell[6 * N + n], qx = sc.cell[7 * N + n], qy = sc.cell[8 * N + n], qz = sc.cell[9 * N + n];
        const float in = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float w = qw * in, x = qx * in, y = qy * in, z = qz * in;
        float o0 = sc.goff[g], o1 = sc.goff[G + g], o2 = sc.goff[2 * G + g];
        const float on = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
        if (on > 1.0f) { o0 /= on; o1 /= on; o2 /= on; }
        const float l0 = o0 * sc.cell[3 * N + n], l1 = o1 * sc.cell[4 * N + n], l2 = o2 * sc.cell[5 * N + n];
        const float R0 = 1.f - 2.f * (y * y + z * z), R1 = 2.f * (x * y - w * z), R2 = 2.f * (x * z + w * y);
        const float R3 = 2.f * (x * y + w * z), R4 = 1.f - 2.f * (x * x + z * z), R5 = 2.f * (y * z - w * x);
        const float R6 = 2.f * (x * z - w * y), R7 = 2.f * (y * z + w * x), R8 = 1.f - 2.f * (x * x + y * y);
        gc[g] = make_float4(sc.cell[n] + R0 * l0 + R1 * l1 + R2 * l2, sc.cell[N + n] + R3 * l0 + R4 * l1 + R5 * l2,
                            sc.cell[2 * N + n] + R6 * l0 + R7 * l1 + R8 * l2, 1.0f - fminf(on, 1.0f));
    }
}

// Stage the samples [q0, q0 + S.M): their records (invalid past the end) and
// the input columns Z[i][s] (zero for invalid samples).
__device__ void stage_samples(const MlpShape &S, float *sm, const SceneDev &sc, const float *__restrict__ srec,
                              long long nsamp, long long q0) {
    const int t = threadIdx.x;
    float *Zt = sm + S.s_z, *info = sm + S.s_info;
    const int nv = (int)min((long long)S.M, nsamp - q0);
    {
        const float4 *s4 = reinterpret_cast<const float4 *>(srec + q0 * DINFO);
        float4 *d4 = reinterpret_cast<float4 *>(info);
#pragma unroll 2
        for (int i = t; i < S.M * (DINFO / 4); i += blockDim.x)
            d4[i] = i < nv * (DINFO / 4) ? __ldg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);  // valid = 0 past the end
    }
    __syncthreads();
    if (t < S.M) {
        const float *p = info + t * DINFO;
        const bool v = __float_as_int(p[1]) != 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) Zt[(S.F + i) * S.LD + t] = v ? p[19 + i] : 0.f;
    }
    // latent features: row n of the [N][F] feature matrix into column s; each
    // warp fetches the rows of its own 8 samples, all loads in flight at once
    // (lanes along the row, features lane and lane + 32)
    {
        const int w = t >> 5, l = t & 31;
        float fv[8][2];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float *p = info + (8 * w + u) * DINFO;
            const bool v = __float_as_int(p[1]) != 0;
            const float *row = sc.feat + (long long)__float_as_int(p[0]) * S.F;
            fv[u][0] = v && l < S.F ? __ldg(row + l) : 0.f;
            fv[u][1] = v && l + 32 < S.F ? __ldg(row + l + 32) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (l < S.F) Zt[l * S.LD + 8 * w + u] = fv[u][0];
            if (l + 32 < S.F) Zt[(l + 32) * S.LD + 8 * w + u] = fv[u][1];
        }
    }
}

// The packed weights in their shared-memory layouts (zero for padded hidden
// units and outputs); one thread per packed float.
__global__ void k_mlp_pack(const float *__restrict__ w, MlpShape S, float *__restrict__ pk) {
    const int H4 = 4 * S.Hp, Rp = S.rb[4];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S.g_total; idx += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (idx >= S.g_w1t && idx < S.g_w1t + S.I * H4) {              // W1^T [k][jj]
            const int e = idx - S.g_w1t, k = e / H4, jj = e - k * H4, D = jj / S.Hp, j = jj - D * S.Hp;
            if (j < S.H) v = w[S.w1o[D] + j * S.I + k];
        } else if (idx >= S.g_b1 && idx < S.g_b1 + H4) {               // b1 [jj]
            const int jj = idx - S.g_b1, D = jj / S.Hp, j = jj - D * S.Hp;
            if (j < S.H) v = w[S.b1o[D] + j];
        } else if (idx >= S.g_b2 && idx < S.g_b2 + Rp) {               // b2 [rr]
            const int rr = idx - S.g_b2, D = out_block(S, rr), r = rr - S.rb[D];
            if (r < S.nout[D]) v = w[S.b2o[D] + r];
        } else if (idx >= S.g_w2t && idx < S.g_w2t + S.Hp * Rp) {      // W2^T [k][rr]
            const int e = idx - S.g_w2t, k = e / Rp, rr = e - k * Rp, D = out_block(S, rr), r = rr - S.rb[D];
            if (r < S.nout[D] && k < S.H) v = w[S.w2o[D] + r * S.H + k];
        } else if (idx >= S.g_w2 && idx < S.g_w2 + Rp * S.Hp) {        // W2 [rr][j]
            const int e = idx - S.g_w2, rr = e / S.Hp, j = e - rr * S.Hp, D = out_block(S, rr), r = rr - S.rb[D];
            if (r < S.nout[D] && j < S.H) v = w[S.w2o[D] + r * S.H + j];
        } else if (idx >= S.g_w1r && idx < S.g_w1r + H4 * S.I) {       // W1 [jj][i]
            const int e = idx - S.g_w1r, jj = e / S.I, i = e - jj * S.I, D = jj / S.Hp, j = jj - D * S.Hp;
            if (j < S.H) v = w[S.w1o[D] + j * S.I + i];
        }
        pk[idx] = v;
    }
}

// n floats (a multiple of 4, both ends 16-byte aligned) from global to shared memory.
__device__ __forceinline__ void copy_f4(float *dst, const float *__restrict__ src, int n) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll 4
    for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) d4[i] = __ldg(s4 + i);
}

// The same as one commit group of asynchronous copies: complete after the
// issuing threads' cp_async_wait and a barrier.
__device__ __forceinline__ void copy_f4_async(float *dst, const float *__restrict__ src, int n) {
    for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
    cp_async_commit();
}

// Layer 1: H = relu(Z W1^T + b1) into the decoder-staggered rows of s_h (W: W1^T).
template <int HW>
__device__ __forceinline__ void layer1(const MlpShape &S, float *sm, const float *W) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, j0 = lane * HW;
    if (j0 >= 4 * S.Hp) return;
    const float *Zt = sm + S.s_z, *b1 = sm + S.s_b1;
    const int H4 = 4 * S.Hp;
    float acc[8][HW];
#pragma unroll
    for (int c = 0; c < HW; ++c) {
        const float b = b1[j0 + c];
#pragma unroll
        for (int s = 0; s < 8; ++s) acc[s][c] = b;
    }
#pragma unroll 2
    for (int k = 0; k < S.I; ++k) {
        const float4 za = *reinterpret_cast<const float4 *>(Zt + k * S.LD + 8 * warp);
        const float4 zb = *reinterpret_cast<const float4 *>(Zt + k * S.LD + 8 * warp + 4);
        const float z[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
        float wv[HW];
#pragma unroll
        for (int c = 0; c < HW; c += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(W + k * H4 + j0 + c);
            wv[c] = q.x; wv[c + 1] = q.y; wv[c + 2] = q.z; wv[c + 3] = q.w;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int c = 0; c < HW; ++c) acc[s][c] = fmaf(z[s], wv[c], acc[s][c]);
    }
    const int D = j0 / S.Hp, j = j0 - D * S.Hp;
    float *Ht = sm + S.s_h;
#pragma unroll
    for (int c = 0; c < HW; ++c) {
        float *dst = Ht + hrow(S, D, j + c) + 8 * warp;
        *reinterpret_cast<float4 *>(dst) = make_float4(fmaxf(acc[0][c], 0.f), fmaxf(acc[1][c], 0.f),
                                                       fmaxf(acc[2][c], 0.f), fmaxf(acc[3][c], 0.f));
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(fmaxf(acc[4][c], 0.f), fmaxf(acc[5][c], 0.f),
                                                           fmaxf(acc[6][c], 0.f), fmaxf(acc[7][c], 0.f));
    }
}

// Layer 2: O = H_D W2_D^T + b2 per decoder into the rows of s_o (W: W2^T).
__device__ __forceinline__ void layer2(const MlpShape &S, float *sm, const float *W) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, Rp = S.rb[4];
    const float *Ht = sm + S.s_h, *b2 = sm + S.s_b2;
    float *Ot = sm + S.s_o;
    for (int rr = 4 * lane; rr < Rp; rr += 128) {
        const int D = out_block(S, rr);
        float acc[8][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float b = b2[rr + c];
#pragma unroll
            for (int s = 0; s < 8; ++s) acc[s][c] = b;
        }
        const float *hb = Ht + hrow(S, D, 0) + 8 * warp;
#pragma unroll 2
        for (int k = 0; k < S.Hp; ++k) {
            const float4 ha = *reinterpret_cast<const float4 *>(hb + k * S.LD);
            const float4 hc = *reinterpret_cast<const float4 *>(hb + k * S.LD + 4);
            const float h[8] = {ha.x, ha.y, ha.z, ha.w, hc.x, hc.y, hc.z, hc.w};
            const float4 q = *reinterpret_cast<const float4 *>(W + k * Rp + rr);
            const float wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int s = 0; s < 8; ++s)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[s][c] = fmaf(h[s], wv[c], acc[s][c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float *dst = Ot + (rr + c) * S.LD + 8 * D + 8 * warp;
            *reinterpret_cast<float4 *>(dst) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
            *reinterpret_cast<float4 *>(dst + 4) = make_float4(acc[4][c], acc[5][c], acc[6][c], acc[7][c]);
        }
    }
}

// The offset of Gaussian g moved into the unit ball, and the Eq. 11 bound.
__device__ __forceinline__ void ball_offset(const SceneDev &sc, long long g, float Ob[3], float O[3], float &on) {
    const long long G = sc.G;
    O[0] = sc.goff[g]; O[1] = sc.goff[G + g]; O[2] = sc.goff[2 * G + g];
    on = sqrtf(O[0] * O[0] + O[1] * O[1] + O[2] * O[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) Ob[c] = on > 1.0f ? O[c] / on : O[c];
}

// The global inputs of Gaussian k's epilogue: its centre and Eq. 11 bound,
// and the cell's v_n in the sample's view (zero for an invalid sample, or
// without vview).
__device__ __forceinline__ void decode_inputs(const ViewDesc *__restrict__ views, const float *p, int k, int K,
                                              const float4 *__restrict__ gc, const float *__restrict__ vview,
                                              float4 &c4, float &vn) {
    if (__float_as_int(p[1]) == 0) {
        c4 = make_float4(0.f, 0.f, 0.f, 0.f);
        vn = 0.f;
        return;
    }
    const int n = __float_as_int(p[0]);
    c4 = __ldg(gc + (long long)n * K + k);
    vn = vview ? __ldg(vview + views[__float_as_int(p[23])].cell_base + n) : 0.f;  // (no records: no v_n)
}

// The forward's epilogue for Gaussian k of one sample (p: its information
// row): the activations, the centre and the Eq. 11 bound, the decoded values
// (kept for the adjoint) and the Gaussian's record for the blend (the
// projection fused into the decode).  out(D, r) is output r of decoder D for
// this sample, before its activation; c4 the Gaussian's centre and Eq. 11
// bound, vn the cell's v_n in this view (decode_inputs).
template <typename Out>
__device__ __forceinline__ void decode_gaussian(const ViewDesc *__restrict__ views, const float *p, int k,
                                                float4 c4, float vn, float *__restrict__ dec, const BlendParams &bp,
                                                float4 *__restrict__ rec, float *__restrict__ g2d_zero, Out out) {
    if (__float_as_int(p[1]) == 0) return;
    const long long rid = (long long)(unsigned)__float_as_int(p[2]) | ((long long)__float_as_int(p[3]) << 32);
    float o[kDecF];
    o[0] = c4.x; o[1] = c4.y; o[2] = c4.z;
#pragma unroll
    for (int c = 0; c < 3; ++c) o[3 + c] = fminf(sigmoid_fast(out(2, 3 * k + c)), c4.w) * p[7 + c];
    float qv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) qv[c] = out(3, 4 * k + c);
    const float qn2 = qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3];
    if (qn2 > 0.f) {
        const float iq = rsqrtf(qn2);
#pragma unroll
        for (int c = 0; c < 4; ++c) o[6 + c] = qv[c] * iq;
    } else {  // no direction to normalise: the identity rotation
        o[6] = 1.f; o[7] = 0.f; o[8] = 0.f; o[9] = 0.f;
    }
    o[10] = tanh_fast(out(0, k));
#pragma unroll
    for (int c = 0; c < 3; ++c) o[11 + c] = sigmoid_fast(out(1, 3 * k + c));
    float2 *dst = reinterpret_cast<float2 *>(dec + (rid + k) * kDecF);
#pragma unroll
    for (int i = 0; i < kDecF / 2; ++i) dst[i] = make_float2(o[2 * i], o[2 * i + 1]);
    if (rec) {  // the Gaussian's record for the blend (the projection fused into the decode)
        const ViewDesc &Vw = views[__float_as_int(p[23])];
        GaussIn gi;
#pragma unroll
        for (int i = 0; i < 3; ++i) { gi.mean[i] = o[i]; gi.scale[i] = o[3 + i]; }
#pragma unroll
        for (int i = 0; i < 4; ++i) gi.quat[i] = o[6 + i];
        gi.logit = 0.f;
        const float knone[16][3] = {};
        ProjCore c;
        float4 r0, r1, r2;
        gauss_record<true>(Vw, gi, knone, 0, o[10], vn, bp, c, r0, r1, r2, o + 11);
        if (!(o[10] > 0.f)) r0 = make_float4(0.f, 0.f, -1.f, -1.f);  // sigma <= 0: not drawn
        float4 *rp = rec + (rid + k) * kRecF4;
        rp[0] = r0; rp[1] = r1; rp[2] = r2;
        if (g2d_zero) {
            float4 *z = reinterpret_cast<float4 *>(g2d_zero + (rid + k) * kGradF);
            z[0] = z[1] = z[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

template <int HW>
__global__ void __launch_bounds__(256) k_decode(const ViewDesc *__restrict__ views, SceneDev sc, MlpShape S,
                                                const float *__restrict__ pk, const float *__restrict__ srec,
                                                const float4 *__restrict__ gc, long long nsamp,
                                                const uint32_t *__restrict__ d_n,
                                                float *__restrict__ dec, const float *__restrict__ vview,
                                                BlendParams bp, float4 *__restrict__ rec,
                                                float *__restrict__ g2d_zero) {
    if (d_n) nsamp = min(nsamp, (long long)*d_n);  // the count on the device (capacity nsamp)
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *Wb = sm + S.s_w;
    const int K = S.K;
    // W1^T of a CTA's next tile is copied while the tile's epilogue runs
    copy_f4_async(Wb, pk + S.g_w1t, S.I * 4 * S.Hp);
    for (long long q0 = (long long)blockIdx.x * S.M; q0 < nsamp; q0 += (long long)gridDim.x * S.M) {
        copy_f4(sm + S.s_b1, pk + S.g_b1, 4 * S.Hp);
        copy_f4(sm + S.s_b2, pk + S.g_b2, S.rb[4]);
        stage_samples(S, sm, sc, srec, nsamp, q0);
        cp_async_wait<0>();
        __syncthreads();
        layer1<HW>(S, sm, Wb);
        __syncthreads();
        copy_f4(Wb, pk + S.g_w2t, S.Hp * S.rb[4]);
        __syncthreads();
        layer2(S, sm, Wb);
        __syncthreads();
        if (q0 + (long long)gridDim.x * S.M < nsamp) copy_f4_async(Wb, pk + S.g_w1t, S.I * 4 * S.Hp);
        // activations and the centres, one (sample, Gaussian) per thread
        const float *Ot = sm + S.s_o, *info = sm + S.s_info;
        for (int idx = threadIdx.x; idx < S.M * K; idx += blockDim.x) {
            const int s = idx / K, k = idx - s * K;
            const float *p = info + s * DINFO;
            float4 c4;
            float vn;
            decode_inputs(views, p, k, K, gc, vview, c4, vn);
            decode_gaussian(views, p, k, c4, vn, dec, bp, rec, g2d_zero,
                            [&](int D, int r) { return Ot[orow(S, D, r) + s]; });
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- tensor cores
// The same two layers on the fifth-generation tensor cores (tcgen05, TF32
// products with FP32 accumulation in tensor memory) for the common widths:
// I = F + 4 <= 40 inputs, H <= 32 hidden units per decoder and output blocks
// that fit 128 columns when each is rounded up to 16 (K <= 10).  A tile is
// M = 128 samples, one row of the product per sample:
//   layer 1  D1[128 x 128] = Z[128 x IP] W1^T            (TMEM columns 0 .. 127)
//   layer 2  D2[128 x N_D] = H[:, 32D .. 32D+32] W2_D^T  (columns 128 + rb_D, per decoder)
// with IP = I rounded up to 8 (one product consumes K = 8) and every decoder's
// hidden units padded to 32.  Each factor is split as x = hi + lo with hi
// exact in TF32, and a product is the sum lo*hi + hi*lo + hi*hi accumulated
// in FP32 (the dropped lo*lo term is below 2^-21 relative), which keeps the
// decoded values at the CUDA-core kernels' FP32 accuracy.  One thread issues
// the products; they complete through an mbarrier (bounded wait).  Biases and
// the ReLU are applied as the accumulators leave tensor memory: layer 1's
// into the hi/lo operand tiles of layer 2, layer 2's into an output tile in
// shared memory, from which the epilogue (decode_gaussian) runs as in
// k_decode, one (sample, Gaussian) per thread.
constexpr int TC_M = 128;
constexpr int TC_THREADS = 768;  // 24 warps: the epilogue's latency is what they hide (72 registers)
constexpr int TC_CW = 32;        // accumulator columns a warp moves out of tensor memory (warps 0-15)
constexpr int TC_ITEMS = 2;      // (sample, Gaussian) items a thread decodes per tile: 128 K <= 2 x 768
constexpr int TC_LDO = TC_M + 1;  // output tile row stride (floats): (column, sample) reads spread over banks

struct TcShape {
    int F, H, K, I, IP;
    int nout[4], rb[5];                  // output widths; column bases, blocks rounded up to 16 (rb[4] <= 128)
    int w1o[4], b1o[4], w2o[4], b2o[4];  // offsets in the packed weights
    // the weight image (floats; its order is the shared-memory layout's):
    // W1 hi | W1 lo [128 x IP], W2 hi | W2 lo [128 x 32], b1 [128], b2 [128]
    int g_w1h, g_w1l, g_w2h, g_w2l, g_b1, g_b2, g_total;
    // dynamic shared memory (bytes): the image, then the operand/output union, then the sample records
    int s_u, s_info, s_total;
};

static TcShape tc_shape(int F, int H, int K) {
    TcShape T{};
    T.F = F; T.H = H; T.K = K; T.I = F + 4; T.IP = up_to(T.I, 8);
    const int outs[4] = {K, 3 * K, 3 * K, 4 * K};
    int o = 0;
    T.rb[0] = 0;
    for (int D = 0; D < 4; ++D) {
        T.nout[D] = outs[D];
        T.rb[D + 1] = T.rb[D] + up_to(outs[D], 16);
        T.w1o[D] = o; T.b1o[D] = o + H * T.I; T.w2o[D] = T.b1o[D] + H; T.b2o[D] = T.w2o[D] + outs[D] * H;
        o = T.b2o[D] + outs[D];
    }
    T.g_w1h = 0;
    T.g_w1l = T.g_w1h + TC_M * T.IP;
    T.g_w2h = T.g_w1l + TC_M * T.IP;
    T.g_w2l = T.g_w2h + TC_M * 32;
    T.g_b1 = T.g_w2l + TC_M * 32;
    T.g_b2 = T.g_b1 + TC_M;
    T.g_total = T.g_b2 + TC_M;
    T.s_u = 4 * T.g_total;
    // the union holds Z hi|lo, then H hi|lo, then the output tile
    const int u = std::max(std::max(2 * 4 * TC_M * T.IP, 2 * 4 * TC_M * TC_M), 4 * TC_M * TC_LDO);
    T.s_info = T.s_u + u;
    T.s_total = T.s_info + 4 * TC_M * DINFO;
    return T;
}

static bool tc_fits(int F, int H, int K) {
    if (F + 4 > 40 || H > 32 || H < 1 || F < 1 || K < 1 || TC_M * K > TC_ITEMS * TC_THREADS) return false;
    const TcShape T = tc_shape(F, H, K);
    return T.rb[4] <= TC_M && T.s_total <= kSmemMax;
}

// The weight image: element e of a region holds the operand entry at its
// core-matrix position (the inverse of tc::cm_off), hi or lo part.
__global__ void k_mlp_pack_tc(const float *__restrict__ w, TcShape T, float *__restrict__ img) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < T.g_total; idx += gridDim.x * blockDim.x) {
        float v = 0.f;
        bool lo = false;
        if (idx < T.g_w2h) {  // W1 [hidden jj][input k], KK = IP
            lo = idx >= T.g_w1l;
            const int o = 4 * (idx - (lo ? T.g_w1l : T.g_w1h)), sbo = T.IP * 32;
            const int rem = o % sbo, jj = 8 * (o / sbo) + (rem % 128) / 16, k = 4 * (rem / 128) + (rem % 16) / 4;
            const int D = jj / 32, j = jj % 32;
            if (j < T.H && k < T.I) v = w[T.w1o[D] + j * T.I + k];
        } else if (idx < T.g_b1) {  // W2 [padded output column cc][hidden j], KK = 32
            lo = idx >= T.g_w2l;
            const int o = 4 * (idx - (lo ? T.g_w2l : T.g_w2h));
            const int rem = o % 1024, cc = 8 * (o / 1024) + (rem % 128) / 16, j = 4 * (rem / 128) + (rem % 16) / 4;
            int D = 0;
            while (D < 3 && cc >= T.rb[D + 1]) ++D;
            const int r = cc - T.rb[D];
            if (cc < T.rb[4] && r < T.nout[D] && j < T.H) v = w[T.w2o[D] + r * T.H + j];
        } else if (idx < T.g_b2) {
            const int jj = idx - T.g_b1, D = jj / 32, j = jj % 32;
            if (j < T.H) v = w[T.b1o[D] + j];
        } else {
            const int cc = idx - T.g_b2;
            int D = 0;
            while (D < 3 && cc >= T.rb[D + 1]) ++D;
            const int r = cc - T.rb[D];
            if (cc < T.rb[4] && r < T.nout[D]) v = w[T.b2o[D] + r];
        }
        if (idx < T.g_b1) {
            float hi, l;
            tc::split_tf32(v, hi, l);
            v = lo ? l : hi;
        }
        img[idx] = v;
    }
}

// Fault injection (dgs_debug_inject_fault, DGS_FAULT_TC_WAIT): while set, the
// tensor-core decode issues no products for its first tile and waits about
// 2^24 clocks, so its completion wait runs out with nothing in flight.
__device__ int g_tc_fault = 0;

cudaError_t set_tc_fault(bool on) {
    const int v = on ? 1 : 0;
    return cudaMemcpyToSymbol(g_tc_fault, &v, sizeof(int));
}

// Stage samples [q0, q0 + 128): records (invalid past the end) and Z as the
// hi and lo operand tiles (zero for invalid samples and padded inputs).
__device__ __forceinline__ void tc_stage(const TcShape &T, unsigned char *sm, const SceneDev &sc,
                                         const float *__restrict__ srec, long long nsamp, long long q0) {
    float *info = reinterpret_cast<float *>(sm + T.s_info);
    const int nv = (int)min((long long)TC_M, nsamp - q0);
    {
        const float4 *s4 = reinterpret_cast<const float4 *>(srec + q0 * DINFO);
        float4 *d4 = reinterpret_cast<float4 *>(info);
        for (int i = threadIdx.x; i < TC_M * (DINFO / 4); i += blockDim.x)
            d4[i] = i < nv * (DINFO / 4) ? __ldg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    unsigned char *zh = sm + T.s_u, *zl = zh + 4 * TC_M * T.IP;
    // one 16-byte chunk (4 inputs) of one sample per item; consecutive threads
    // walk a sample's feature row (16-byte loads where the row allows)
    const int nc = T.IP / 4;
    const bool vec = (T.F & 3) == 0;
    for (int it = threadIdx.x; it < TC_M * nc; it += blockDim.x) {
        const int s = it / nc, c = it - s * nc;
        const float *p = info + s * DINFO;
        const bool valid = __float_as_int(p[1]) != 0;
        const float *row = sc.feat + (long long)__float_as_int(p[0]) * T.F;
        float z[4];
        if (valid && vec && 4 * c + 3 < T.F) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(row) + c);
            z[0] = f.x; z[1] = f.y; z[2] = f.z; z[3] = f.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = 4 * c + u;
                z[u] = !valid || i >= T.I ? 0.f : (i < T.F ? __ldg(row + i) : p[19 + i - T.F]);
            }
        }
        float4 h, l;
        tc::split_tf32(z[0], h.x, l.x);
        tc::split_tf32(z[1], h.y, l.y);
        tc::split_tf32(z[2], h.z, l.z);
        tc::split_tf32(z[3], h.w, l.w);
        const uint32_t off = tc::cm_off(s, 4 * c, T.IP);
        *reinterpret_cast<float4 *>(zh + off) = h;
        *reinterpret_cast<float4 *>(zl + off) = l;
    }
}

// Products of one layer: D (+)= A B^T as lo*hi + hi*lo + hi*hi over ksteps
// steps of 8.  a/b: byte addresses of the hi tiles; the lo tiles follow at
// a_lo / b_lo bytes; sbo_a, sbo_b: their 8-row group strides.
__device__ __forceinline__ void tc_layer(uint32_t d, uint32_t a, uint32_t a_lo, uint32_t sbo_a, uint32_t b,
                                         uint32_t b_lo, uint32_t sbo_b, int ksteps, uint32_t idesc) {
    const uint32_t as[3] = {a + a_lo, a, a}, bs[3] = {b, b + b_lo, b};
    bool acc = false;
#pragma unroll
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < ksteps; ++k) {
            tc::mma_tf32(d, tc::desc(as[t] + 256 * k, sbo_a), tc::desc(bs[t] + 256 * k, sbo_b), idesc, acc);
            acc = true;
        }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_decode_tc(const ViewDesc *__restrict__ views, SceneDev sc,
                                                               TcShape T, const float *__restrict__ img,
                                                               const float *__restrict__ srec,
                                                               const float4 *__restrict__ gc, long long nsamp,
                                                               const uint32_t *__restrict__ d_n,
                                                               float *__restrict__ dec, const float *__restrict__ vview,
                                                               BlendParams bp, float4 *__restrict__ rec,
                                                               float *__restrict__ g2d_zero, uint32_t *err) {
    if (d_n) nsamp = min(nsamp, (long long)*d_n);  // the count on the device (capacity nsamp)
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int K = T.K;
    // the weight image once per CTA (its layout is the shared-memory layout)
    {
        const float4 *s4 = reinterpret_cast<const float4 *>(img);
        float4 *d4 = reinterpret_cast<float4 *>(sm);
        for (int i = t; i < T.g_total / 4; i += blockDim.x) d4[i] = __ldg(s4 + i);
    }
    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        abort_flag = 0;
    }
    if (warp == 0) tc::tmem_alloc<256>(&tslot);
    tc::sync_threads();
    const uint32_t tm = tslot;
    const uint32_t base = tc::smem_u32(sm);
    const uint32_t w1 = base + 4 * T.g_w1h, w1_lo = 4 * (T.g_w1l - T.g_w1h);
    const uint32_t w2 = base + 4 * T.g_w2h, w2_lo = 4 * (T.g_w2l - T.g_w2h);
    const uint32_t u = base + T.s_u;
    const float *b1 = reinterpret_cast<const float *>(sm) + T.g_b1;
    const float *b2 = reinterpret_cast<const float *>(sm) + T.g_b2;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
    const int s = 32 * (warp & 3) + lane;                         // its sample (TMEM lane)
    const int cbase = warp < 16 ? TC_CW * (warp >> 2) : 0;       // its TC_CW of the 128 columns
    const int cend = warp < 16 ? cbase + TC_CW : 0;               // (warps 16.. move none)
    uint32_t phase = 0;
    const bool fault = g_tc_fault != 0;
    const long long wait_clocks = fault ? (1LL << 24) : (1LL << 31);
    for (long long q0 = (long long)blockIdx.x * TC_M; q0 < nsamp; q0 += (long long)gridDim.x * TC_M) {
        tc_stage(T, sm, sc, srec, nsamp, q0);
        const float *info = reinterpret_cast<const float *>(sm + T.s_info);
        tc::fence_async_smem();
        tc::sync_threads();
        if (t == 0 && !fault) {
            tc_layer(tm, u, 4 * TC_M * T.IP, T.IP * 32, w1, w1_lo, T.IP * 32, T.IP / 8, tc::idesc_tf32(TC_M, TC_M));
            tc::commit(&mbar);
        }
        if (!tc::mbar_wait(&mbar, phase, wait_clocks)) abort_flag = 1;
        phase ^= 1;
        tc::fence_after();
        __syncthreads();
        if (abort_flag) break;
        // layer 1 leaves tensor memory: + b1, ReLU, split into the H operand tiles (over Z, now read)
        {
            unsigned char *hh = sm + T.s_u, *hl = hh + 4 * TC_M * TC_M;
#pragma unroll 1
            for (int c0 = cbase; c0 < cend; c0 += 16) {
                float v[16];
                tc::ld16(tm + lane_base + (uint32_t)c0, v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 h, l;
                    float x[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) x[j] = fmaxf(v[4 * q + j] + b1[c0 + 4 * q + j], 0.f);
                    tc::split_tf32(x[0], h.x, l.x);
                    tc::split_tf32(x[1], h.y, l.y);
                    tc::split_tf32(x[2], h.z, l.z);
                    tc::split_tf32(x[3], h.w, l.w);
                    const uint32_t off = tc::cm_off(s, c0 + 4 * q, TC_M);
                    *reinterpret_cast<float4 *>(hh + off) = h;
                    *reinterpret_cast<float4 *>(hl + off) = l;
                }
            }
        }
        tc::fence_async_smem();
        tc::sync_threads();
        if (t == 0) {
            for (int D = 0; D < 4; ++D) {
                const int n = T.rb[D + 1] - T.rb[D];
                tc_layer(tm + 128 + (uint32_t)T.rb[D], u + 32 * D * 32, 4 * TC_M * TC_M, TC_M * 32,
                         w2 + (uint32_t)(T.rb[D] / 8) * 1024, w2_lo, 1024, 4, tc::idesc_tf32(TC_M, n));
            }
            tc::commit(&mbar);
        }
        if (!tc::mbar_wait(&mbar, phase, wait_clocks)) abort_flag = 1;
        phase ^= 1;
        tc::fence_after();
        __syncthreads();
        if (abort_flag) break;
        // layer 2 leaves tensor memory: + b2 into the output tile (over H, now read)
        float *Ot = reinterpret_cast<float *>(sm + T.s_u);
        for (int c0 = cbase; c0 < cend; c0 += 16) {
            if (c0 >= T.rb[4]) break;
            float v[16];
            tc::ld16(tm + lane_base + 128u + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) Ot[(c0 + j) * TC_LDO + s] = v[j] + b2[c0 + j];
        }
        tc::sync_threads();
#pragma unroll
        for (int j = 0; j < TC_ITEMS; ++j) {
            const int idx = t + j * TC_THREADS;
            if (idx >= TC_M * K) break;
            const int si = idx / K, k = idx - si * K;
            float4 c4;
            float vn;
            decode_inputs(views, info + si * DINFO, k, K, gc, vview, c4, vn);
            decode_gaussian(views, info + si * DINFO, k, c4, vn, dec, bp, rec, g2d_zero,
                            [&](int D, int r) { return Ot[(T.rb[D] + r) * TC_LDO + si]; });
        }
        tc::sync_threads();  // the tiles are read before the next stage overwrites them
    }
    if (abort_flag && t == 0) atomicOr(err, 1u);
    tc::sync_threads();
    if (warp == 0) tc::tmem_free<256>(tm);
}

// ---------------------------------------------------------------- adjoint
// Per tile of samples: the forward again (layers 1 and 2), then
//   dL/do (in place of O) from gdec through the activations, the offsets'
//     gradients (atomic adds to g_offset: mu = x + R(Q)(O_pos S) and the
//     Eq. 11 bound);
//   dL/dh = relu'(h) (dL/do_D W2_D) per decoder;
//   dL/df = sum over decoders of dL/dh_D W1_D[:, :F]  (atomic adds to g_feat);
// and the weight gradients.  With cg: the cell's centre, semi-axes and
// rotation through mu = x_n + R(Q_n)(O_pos S_n) and s = ratio S_n (atomic adds
// per Gaussian), and the centre through the decoder inputs delta_n = |r|,
// d_n = r / |r| (r = x_n - eye; columns F .. F+3 of W1, atomic adds per sample):
//   dL/dx_n += dL/ddelta d_n + (I - d_n d_n^T) dL/dd_n / delta_n.  FUSE (the common widths, wgrad_fused: a tile of
// 32 samples, 4Hp and the padded outputs Rp at most the CTA's threads,
// I <= FW_I, Hp <= FW_H): thread t keeps row t of dW1 | db1 (over all decoders) and row
// t of dW2 | db2 in registers, adds each tile's products from shared memory
// and flushes them to g_mlp once, with atomic adds, at the end.  Otherwise
// the rows Z, H, dL/dh, dL/do of every sample go to `rows` for k_mlp_wgrad,
// stored per tile of M samples as unit rows of M values (the tile's
// shared-memory layout, so they leave as float4 copies).  Decisions held
// fixed: the ReLU masks, the side of the Eq. 11 minimum, sigma <= 0 (gdec is
// zero there).  CELL: some cell gradient is requested (without, the cell
// terms are compiled out).
template <int HW, bool FUSE, bool CELL>
__global__ void __launch_bounds__(256) k_decode_bwd(SceneDev sc, MlpShape S, const float *__restrict__ pk,
                                                    const float *__restrict__ srec, long long nsamp,
                                                    const uint32_t *__restrict__ d_n,
                                                    const float *__restrict__ gdec,
                                                        float *__restrict__ g_feat, float *__restrict__ g_offset,
                                                        float *__restrict__ rows, float *__restrict__ g_mlp,
                                                        CellGrads cg) {
    if (d_n) nsamp = min(nsamp, (long long)*d_n);  // the count on the device (capacity nsamp)
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int K = S.K, F = S.F, Hp = S.Hp, H4 = 4 * S.Hp, Rp = S.rb[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // With two weight buffers (S.dbuf) each phase's weights are copied
    // asynchronously while the phase before it computes (A: W1^T, then W2;
    // B: W2^T, then W1); with one (WA == WB) each is copied between barriers.
    float *WA = sm + S.s_w, *WB = sm + S.s_w2;
    auto prefetch = [&](float *dst, const float *src, int n) {
        if (S.dbuf) copy_f4_async(dst, src, n);
    };
    auto ready = [&](float *dst, const float *src, int n) {
        if (S.dbuf) {
            cp_async_wait<0>();
            __syncthreads();
        } else {
            __syncthreads();
            copy_f4(dst, src, n);
            __syncthreads();
        }
    };
    copy_f4(sm + S.s_b1, pk + S.g_b1, H4);
    copy_f4(sm + S.s_b2, pk + S.g_b2, Rp);
    prefetch(WA, pk + S.g_w1t, S.I * H4);
    float aw1[FUSE ? FW_I : 1], aw2[FUSE ? FW_H : 1], ab1 = 0.f, ab2 = 0.f;  // FUSE: this thread's rows of dW1, dW2
#pragma unroll
    for (int b = 0; b < (FUSE ? FW_I : 1); ++b) aw1[b] = 0.f;
#pragma unroll
    for (int b = 0; b < (FUSE ? FW_H : 1); ++b) aw2[b] = 0.f;
    for (long long q0 = (long long)blockIdx.x * S.M; q0 < nsamp; q0 += (long long)gridDim.x * S.M) {
        stage_samples(S, sm, sc, srec, nsamp, q0);
        ready(WA, pk + S.g_w1t, S.I * H4);
        prefetch(WB, pk + S.g_w2t, Hp * Rp);
        layer1<HW>(S, sm, WA);
        ready(WB, pk + S.g_w2t, Hp * Rp);
        prefetch(WA, pk + S.g_w2, Rp * Hp);
        layer2(S, sm, WB);
        __syncthreads();
        float *Ot = sm + S.s_o;
        const float *info = sm + S.s_info;
        // dL/do through the activations, in place; offsets' gradients
        for (int idx = threadIdx.x; idx < S.M * K; idx += blockDim.x) {
            const int s = idx / K, k = idx - s * K;
            const SampleInfo a = get_info(info, s);
            float *po = Ot + orow(S, 0, k) + s;
            float *pc[3], *ps[3], *pq[4];
#pragma unroll
            for (int c = 0; c < 3; ++c) { pc[c] = Ot + orow(S, 1, 3 * k + c) + s; ps[c] = Ot + orow(S, 2, 3 * k + c) + s; }
#pragma unroll
            for (int c = 0; c < 4; ++c) pq[c] = Ot + orow(S, 3, 4 * k + c) + s;
            if (!a.valid) {
                *po = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) { *pc[c] = 0.f; *ps[c] = 0.f; }
#pragma unroll
                for (int c = 0; c < 4; ++c) *pq[c] = 0.f;
                continue;
            }
            const long long g = (long long)a.n * K + k;
            float gk[kDecF];
            {
                const float2 *src = reinterpret_cast<const float2 *>(gdec + (a.rec + k) * kDecF);
#pragma unroll
                for (int i = 0; i < kDecF / 2; ++i) { const float2 v = src[i]; gk[2 * i] = v.x; gk[2 * i + 1] = v.y; }
            }
            // opacity
            {
                const float sg = tanh_fast(*po);
                *po = gk[10] * (1.0f - sg * sg);
            }
            // colour
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float cc = sigmoid_fast(*pc[c]);
                *pc[c] = gk[11 + c] * cc * (1.0f - cc);
            }
            // scale and the Eq. 11 bound; then the offset
            float Ob[3], O[3], on;
            ball_offset(sc, g, Ob, O, on);
            const float lim = 1.0f - fminf(on, 1.0f);
            float dlim = 0.f, ratio[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float sg = sigmoid_fast(*ps[c]);
                if (sg < lim) {
                    *ps[c] = gk[3 + c] * a.S[c] * sg * (1.0f - sg);
                    ratio[c] = sg;
                } else {
                    *ps[c] = 0.f;
                    dlim += gk[3 + c] * a.S[c];
                    ratio[c] = lim;
                }
            }
            float dOb[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dOb[c] = a.S[c] * (a.R[c] * gk[0] + a.R[3 + c] * gk[1] + a.R[6 + c] * gk[2]);
            float dO[3];
            if (on > 1.0f) {  // O_pos = O / |O| has unit length: lim = 0 does not move
                const float io = 1.0f / on;
                const float pr = (dOb[0] * O[0] + dOb[1] * O[1] + dOb[2] * O[2]) * io * io;
#pragma unroll
                for (int c = 0; c < 3; ++c) dO[c] = (dOb[c] - pr * O[c]) * io;
            } else {
                const float io = on > 0.f ? dlim / on : 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) dO[c] = dOb[c] - io * O[c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (dO[c] != 0.f) atomicAdd(g_offset + 3 * g + c, dO[c]);
            // the cell's own parameters: mu = x + R (Ob S), s = ratio S
            if (CELL && cg.center) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (gk[c] != 0.f) atomicAdd(cg.center + 3LL * a.n + c, gk[c]);
            }
            if (CELL && cg.axes) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float rt = a.R[c] * gk[0] + a.R[3 + c] * gk[1] + a.R[6 + c] * gk[2];
                    const float v = Ob[c] * rt + gk[3 + c] * ratio[c];
                    if (v != 0.f) atomicAdd(cg.axes + 3LL * a.n + c, v);
                }
            }
            if (CELL && cg.quat) {
                const long long N = sc.N;
                const float cq[4] = {sc.cell[6 * N + a.n], sc.cell[7 * N + a.n], sc.cell[8 * N + a.n],
                                     sc.cell[9 * N + a.n]};
                float gR[9], gq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) gR[3 * i + j] = gk[i] * Ob[j] * a.S[j];
                rot_quat_adjoint(cq, gR, gq);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (gq[c] != 0.f) atomicAdd(cg.quat + 4LL * a.n + c, gq[c]);
            }
            // rotation (a zero output decodes to a constant)
            float qv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) qv[c] = *pq[c];
            const float qn2 = qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3];
            if (qn2 > 0.f) {
                const float iq = rsqrtf(qn2);
                float pr = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) pr += gk[6 + c] * qv[c] * iq;
#pragma unroll
                for (int c = 0; c < 4; ++c) *pq[c] = (gk[6 + c] - pr * qv[c] * iq) * iq;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) *pq[c] = 0.f;
            }
        }
        ready(WA, pk + S.g_w2, Rp * Hp);
        prefetch(WB, pk + S.g_w1r, H4 * S.I);
        // dL/dh = relu'(h) * (dL/do_D W2_D)
        const int j0 = lane * HW;
        float *DHt = sm + S.s_dh;
        const float *Ht = sm + S.s_h;
        if (j0 < H4) {
            const int D = j0 / Hp, j = j0 - D * Hp;
            const float *W = WA;
            float acc[8][HW];
#pragma unroll
            for (int s = 0; s < 8; ++s)
#pragma unroll
                for (int c = 0; c < HW; ++c) acc[s][c] = 0.f;
            const float *db = Ot + orow(S, D, 0) + 8 * warp;
#pragma unroll 2
            for (int r = 0; r < S.nout[D]; ++r) {
                const float4 da = *reinterpret_cast<const float4 *>(db + r * S.LD);
                const float4 dc = *reinterpret_cast<const float4 *>(db + r * S.LD + 4);
                const float d[8] = {da.x, da.y, da.z, da.w, dc.x, dc.y, dc.z, dc.w};
                float wv[HW];
#pragma unroll
                for (int c = 0; c < HW; c += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(W + (S.rb[D] + r) * Hp + j + c);
                    wv[c] = q.x; wv[c + 1] = q.y; wv[c + 2] = q.z; wv[c + 3] = q.w;
                }
#pragma unroll
                for (int s = 0; s < 8; ++s)
#pragma unroll
                    for (int c = 0; c < HW; ++c) acc[s][c] = fmaf(d[s], wv[c], acc[s][c]);
            }
#pragma unroll
            for (int c = 0; c < HW; ++c) {
                const int hr = hrow(S, D, j + c) + 8 * warp;
                const float4 ha = *reinterpret_cast<const float4 *>(Ht + hr);
                const float4 hc = *reinterpret_cast<const float4 *>(Ht + hr + 4);
                *reinterpret_cast<float4 *>(DHt + hr) =
                    make_float4(ha.x > 0.f ? acc[0][c] : 0.f, ha.y > 0.f ? acc[1][c] : 0.f,
                                ha.z > 0.f ? acc[2][c] : 0.f, ha.w > 0.f ? acc[3][c] : 0.f);
                *reinterpret_cast<float4 *>(DHt + hr + 4) =
                    make_float4(hc.x > 0.f ? acc[4][c] : 0.f, hc.y > 0.f ? acc[5][c] : 0.f,
                                hc.z > 0.f ? acc[6][c] : 0.f, hc.w > 0.f ? acc[7][c] : 0.f);
            }
        }
        ready(WB, pk + S.g_w1r, H4 * S.I);
        if (q0 + (long long)gridDim.x * S.M < nsamp) prefetch(WA, pk + S.g_w1t, S.I * H4);
        // dL/df = sum_jj dL/dh[jj] W1[jj][:F]; lanes take features cb + lane and
        // cb + lane + 32 per group of 64 columns (and the view inputs F .. F+3
        // when the cell centre's gradient is wanted)
        const bool zin = CELL && cg.center != nullptr;  // the view inputs' columns too
        for (int cb = 0; cb < (zin ? S.I : 1); cb += 64) {
            const float *W = WB;
            const int ncol = zin ? S.I : F;
            const int i0 = cb + lane, i1 = cb + lane + 32;
            const bool u1 = i1 < ncol;
            if (i0 < ncol) {
                float acc[8][2];
#pragma unroll
                for (int s = 0; s < 8; ++s) acc[s][0] = acc[s][1] = 0.f;
                for (int D = 0; D < 4; ++D) {
                    const float *dh = DHt + hrow(S, D, 0) + 8 * warp;
                    const float *wd = W + D * Hp * S.I;
                    if (ncol - cb > 32) {  // (uniform) two columns per lane
#pragma unroll 2
                        for (int j = 0; j < Hp; ++j) {
                            const float4 da = *reinterpret_cast<const float4 *>(dh + j * S.LD);
                            const float4 dc = *reinterpret_cast<const float4 *>(dh + j * S.LD + 4);
                            const float d[8] = {da.x, da.y, da.z, da.w, dc.x, dc.y, dc.z, dc.w};
                            const float w0 = wd[j * S.I + i0], w1 = u1 ? wd[j * S.I + i1] : 0.f;
#pragma unroll
                            for (int s = 0; s < 8; ++s) {
                                acc[s][0] = fmaf(d[s], w0, acc[s][0]);
                                acc[s][1] = fmaf(d[s], w1, acc[s][1]);
                            }
                        }
                    } else {
#pragma unroll 4
                        for (int j = 0; j < Hp; ++j) {
                            const float4 da = *reinterpret_cast<const float4 *>(dh + j * S.LD);
                            const float4 dc = *reinterpret_cast<const float4 *>(dh + j * S.LD + 4);
                            const float d[8] = {da.x, da.y, da.z, da.w, dc.x, dc.y, dc.z, dc.w};
                            const float w0 = wd[j * S.I + i0];
#pragma unroll
                            for (int s = 0; s < 8; ++s) acc[s][0] = fmaf(d[s], w0, acc[s][0]);
                        }
                    }
                }
                // column i >= F: dL/d of the view input i - F (delta, then d) -> the centre
                auto to_centre = [&](const float *p, long long n, int m, float gz) {
                    const float delta = p[19], d[3] = {p[20], p[21], p[22]};
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float v = m == 0 ? gz * d[j] : gz * ((j == m - 1 ? 1.0f : 0.0f) - d[j] * d[m - 1]) / delta;
                        if (v != 0.f) atomicAdd(cg.center + 3 * n + j, v);
                    }
                };
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const float *p = info + (8 * warp + s) * DINFO;
                    if (__float_as_int(p[1]) == 0) continue;
                    const long long n = __float_as_int(p[0]);
                    if (i0 < F) {
                        if (acc[s][0] != 0.f) atomicAdd(g_feat + n * F + i0, acc[s][0]);
                    } else {
                        to_centre(p, n, i0 - F, acc[s][0]);
                    }
                    if (u1) {
                        if (i1 < F) {
                            if (acc[s][1] != 0.f) atomicAdd(g_feat + n * F + i1, acc[s][1]);
                        } else {
                            to_centre(p, n, i1 - F, acc[s][1]);
                        }
                    }
                }
            }
        }
        if (FUSE) {
            // dW1 | db1 row t: sum over the tile's samples of dL/dh[t] [z | 1];
            // dW2 | db2 row t (padded output t of decoder D): dL/do[t] [h_D | 1]
            const int t = threadIdx.x;
            const float *Zt = sm + S.s_z;
            auto row_dot = [&](const float *a, const float *rowsrc, int n_rows, float *acc, int nmax, float &bias) {
                float d[FW_M];
#pragma unroll
                for (int q = 0; q < FW_M / 4; ++q) {
                    const float4 v = reinterpret_cast<const float4 *>(a)[q];
                    d[4 * q] = v.x; d[4 * q + 1] = v.y; d[4 * q + 2] = v.z; d[4 * q + 3] = v.w;
                }
                float bs = 0.f;
#pragma unroll
                for (int q = 0; q < FW_M; ++q) bs += d[q];
                bias += bs;
#pragma unroll
                for (int b = 0; b < nmax; ++b) {
                    if (b < n_rows) {
                        const float4 *z4 = reinterpret_cast<const float4 *>(rowsrc + b * S.LD);
                        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;  // four chains: latency, not issue
#pragma unroll
                        for (int q = 0; q < FW_M / 4; ++q) {
                            const float4 z = z4[q];
                            s0 = fmaf(d[4 * q], z.x, s0);
                            s1 = fmaf(d[4 * q + 1], z.y, s1);
                            s2 = fmaf(d[4 * q + 2], z.z, s2);
                            s3 = fmaf(d[4 * q + 3], z.w, s3);
                        }
                        acc[b] += (s0 + s1) + (s2 + s3);
                    }
                }
            };
            if (t < H4) {
                const int D = t / Hp, j = t - D * Hp;
                row_dot(DHt + hrow(S, D, j), Zt, S.I, aw1, FUSE ? FW_I : 1, ab1);
            }
            if (t < Rp) {
                const int D = out_block(S, t);
                row_dot(Ot + orow(S, D, t - S.rb[D]), Ht + hrow(S, D, 0), Hp, aw2, FUSE ? FW_H : 1, ab2);
            }
        } else {
        // this tile's rows for the weight gradients, in the tile's own layout
        // (unit rows of M samples: Z, H, dL/dh, dL/do), as float4 copies
            float *blk = rows + (q0 / S.M) * (long long)S.row_all * S.M;
            const int M4 = S.M >> 2;
            const float *Zt = sm + S.s_z;
            auto put = [&](int unit, const float *src, int n_rows, int src_stride) {
                for (int idx = threadIdx.x; idx < n_rows * M4; idx += blockDim.x) {
                    const int u = idx / M4, c = idx - u * M4;
                    reinterpret_cast<float4 *>(blk + (long long)(unit + u) * S.M)[c] =
                        reinterpret_cast<const float4 *>(src + u * src_stride)[c];
                }
            };
            put(S.row_z, Zt, S.I, S.LD);
            for (int D = 0; D < 4; ++D) {
                put(S.row_h + D * Hp, Ht + hrow(S, D, 0), Hp, S.LD);
                put(S.row_dh + D * Hp, DHt + hrow(S, D, 0), Hp, S.LD);
                put(S.row_do + S.rb[D], Ot + orow(S, D, 0), S.rb[D + 1] - S.rb[D], S.LD);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    if (FUSE) {  // this CTA's sums into the packed weight gradient (padded rows and columns dropped)
        const int t = threadIdx.x;
        if (t < H4) {
            const int D = t / Hp, j = t - D * Hp;
            if (j < S.H) {
#pragma unroll
                for (int b = 0; b < (FUSE ? FW_I : 1); ++b)
                    if (b < S.I && aw1[b] != 0.f) atomicAdd(g_mlp + S.w1o[D] + j * S.I + b, aw1[b]);
                if (ab1 != 0.f) atomicAdd(g_mlp + S.b1o[D] + j, ab1);
            }
        }
        if (t < Rp) {
            const int D = out_block(S, t), r = t - S.rb[D];
            if (r < S.nout[D]) {
#pragma unroll
                for (int b = 0; b < (FUSE ? FW_H : 1); ++b)
                    if (b < S.H && aw2[b] != 0.f) atomicAdd(g_mlp + S.w2o[D] + r * S.H + b, aw2[b]);
                if (ab2 != 0.f) atomicAdd(g_mlp + S.b2o[D] + r, ab2);
            }
        }
    }
}

// Weight gradients from the per-sample rows:
//   dW1 | db1 of all decoders at once: C[jj][b] = sum_s dh_s[jj] [z_s | 1][b]  (jj over 4Hp)
//   dW2_D | db2_D per decoder:       C[r][b]  = sum_s do_s[rb_D + r] [h_D,s | 1][b]
// (the ones column gives the biases).  A CTA takes one 32 x 48 tile of one
// product over a chunk of samples: slabs of 32 samples pass through shared
// memory (double-buffered; the next slab is loaded into registers while the
// current one is multiplied), 4 x 4 outputs per thread, and the tile goes to
// g_mlp with one atomic add per output at the end.
constexpr int WT_A = 32, WT_B = 48, WT_S = 32, WT_T = 96;
constexpr int WT_LA = (WT_S * WT_A + WT_T - 1) / WT_T, WT_LB = WT_S * WT_B / WT_T;
struct WgProblem {
    int a_col, na, b_col, nb;  // first column of A and of B in a row, their widths
    int kind;                  // -1: W1 of all decoders; D >= 0: W2 of decoder D
};
struct WgProblems { WgProblem p[5]; };

__global__ void __launch_bounds__(WT_T) k_mlp_wgrad(const float *__restrict__ rows, MlpShape S, long long nsamp,
                                                    const uint32_t *__restrict__ d_n,
                                                    int chunk, WgProblems probs, float *__restrict__ g_mlp) {
    if (d_n) nsamp = min(nsamp, (long long)*d_n);  // the count on the device (capacity nsamp)
    __shared__ __align__(16) float sA[2][WT_S][WT_A + 4];
    __shared__ __align__(16) float sB[2][WT_S][WT_B + 4];
    const WgProblem P = probs.p[blockIdx.z];
    const int a0 = WT_A * (blockIdx.y >> 1), b0 = WT_B * (blockIdx.y & 1);
    if (a0 >= P.na || b0 > P.nb) return;
    const long long s0 = (long long)blockIdx.x * chunk, s1 = min(nsamp, s0 + chunk);
    if (s0 >= s1) return;
    const int t = threadIdx.x, ga = t / 12, gb = t - 12 * ga;
    float ra[WT_LA], rb[WT_LB];
    // element (sample s, column col) of the rows, stored per tile of S.M samples as unit rows
    const int lgM = __ffs(S.M) - 1;
    auto at = [&](long long s, int col) -> float {
        return rows[((s >> lgM) * S.row_all + col) * S.M + (s & (S.M - 1))];
    };
    auto load = [&](long long sb) {
    // consecutive threads take consecutive samples of one column (contiguous in the rows' layout)
#pragma unroll
        for (int u = 0; u < WT_LA; ++u) {
            const int idx = t + WT_T * u, r = idx & 31, c = idx >> 5;
            const long long s = sb + r;
            ra[u] = (idx < WT_S * WT_A && s < s1 && a0 + c < P.na) ? at(s, P.a_col + a0 + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < WT_LB; ++u) {
            const int idx = t + WT_T * u, r = idx & 31, c = idx >> 5, b = b0 + c;
            const long long s = sb + r;
            rb[u] = s < s1 ? (b < P.nb ? at(s, P.b_col + b) : (b == P.nb ? 1.0f : 0.f)) : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < WT_LA; ++u) {
            const int idx = t + WT_T * u;
            if (idx < WT_S * WT_A) sA[buf][idx & 31][idx >> 5] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < WT_LB; ++u) {
            const int idx = t + WT_T * u;
            sB[buf][idx & 31][idx >> 5] = rb[u];
        }
    };
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    load(s0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (long long sb = s0; sb < s1; sb += WT_S) {
        const bool more = sb + WT_S < s1;
        if (more) load(sb + WT_S);
#pragma unroll 8
        for (int r = 0; r < WT_S; ++r) {
            const float4 av = *reinterpret_cast<const float4 *>(&sA[buf][r][4 * ga]);
            const float4 bv = *reinterpret_cast<const float4 *>(&sB[buf][r][4 * gb]);
            const float x[4] = {av.x, av.y, av.z, av.w}, y[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(x[i], y[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + 4 * ga + i;
        if (a >= P.na) continue;
        int wrow, brow;  // packed offsets of row a's weights and of its bias
        if (P.kind < 0) {
            const int D = a / S.Hp, j = a - D * S.Hp;
            if (j >= S.H) continue;
            wrow = S.w1o[D] + j * S.I;
            brow = S.b1o[D] + j;
        } else {
            wrow = S.w2o[P.kind] + a * S.H;
            brow = S.b2o[P.kind] + a;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + 4 * gb + j;
            if (b <= P.nb && acc[i][j] != 0.f) atomicAdd(g_mlp + (b < P.nb ? wrow + b : brow), acc[i][j]);
        }
    }
}

// ---------------------------------------------------------------- launchers

template <typename Kern>
static int persistent_grid(Kern k, int threads, size_t smem, long long tiles) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long cap = (long long)std::max(1, per_sm) * std::max(1, sms);
    return (int)std::max(1LL, std::min(tiles, cap));
}

// Scratch of one decode call: [packed weights][sample records][forward: centres
// and bounds per Gaussian | adjoint: per-sample rows, unless fused].
long long decode_scratch_floats(int F, int H, int K, long long nsamp, long long G, bool bwd) {
    const MlpShape S = mlp_shape(F, H, K, bwd);
    const long long n = std::max(1LL, nsamp);
    const long long tiles = (n + S.M - 1) / S.M;
    const int img = tc_fits(F, H, K) ? std::max(S.g_total, tc_shape(F, H, K).g_total) : S.g_total;
    return up_to(img, 4) + n * DINFO +
           (bwd ? (wgrad_fused(S) ? 0LL : (long long)S.row_all * S.M * tiles) : 4 * std::max(1LL, G));
}

static void decode_prep(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const MlpShape &S,
                        const uint32_t *samples, long long nsamp, const uint32_t *d_n, float *pk, float *srec,
                        cudaStream_t st) {
    k_mlp_pack<<<(S.g_total + 255) / 256, 256, 0, st>>>(sc.mlp, S, pk);
    const long long b = std::min((nsamp + 127) / 128, 152LL * 16);
    k_decode_samples<<<(unsigned)std::max(1LL, b), 128, 0, st>>>(views, n_views, slot, sc, samples, nsamp, d_n, srec);
}

void launch_decode(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *samples,
                   long long nsamp, const uint32_t *d_nsamp, float *dec, float *scratch, const float *vview,
                   const BlendParams &bp, float4 *rec, float *g2d_zero, uint32_t *err, cudaStream_t st) {
    if (nsamp <= 0 || !sc.feat) return;
    if (tc_fits(sc.F, sc.H, sc.K)) {
        const TcShape T = tc_shape(sc.F, sc.H, sc.K);
        float *img = scratch, *srec = scratch + up_to(T.g_total, 4);
        float4 *gc = reinterpret_cast<float4 *>(srec + nsamp * DINFO);
        k_mlp_pack_tc<<<(T.g_total + 255) / 256, 256, 0, st>>>(sc.mlp, T, img);
        const long long b = std::min((nsamp + 127) / 128, 152LL * 16);
        k_decode_samples<<<(unsigned)std::max(1LL, b), 128, 0, st>>>(views, n_views, slot, sc, samples, nsamp, d_nsamp,
                                                                     srec);
        const long long bg = std::min((sc.G + 127) / 128, 152LL * 16);
        k_decode_centres<<<(unsigned)std::max(1LL, bg), 128, 0, st>>>(sc, gc);
        const long long tiles = (nsamp + TC_M - 1) / TC_M;
        const int grid = persistent_grid(k_decode_tc, TC_THREADS, (size_t)T.s_total, tiles);
        k_decode_tc<<<grid, TC_THREADS, (size_t)T.s_total, st>>>(views, sc, T, img, srec, gc, nsamp, d_nsamp, dec,
                                                               vview, bp, rec, g2d_zero, err);
        return;
    }
    const MlpShape S = mlp_shape(sc.F, sc.H, sc.K, false);
    float *pk = scratch, *srec = scratch + up_to(S.g_total, 4);
    float4 *gc = reinterpret_cast<float4 *>(srec + nsamp * DINFO);
    decode_prep(views, n_views, slot, sc, S, samples, nsamp, d_nsamp, pk, srec, st);
    const long long bg = std::min((sc.G + 127) / 128, 152LL * 16);
    k_decode_centres<<<(unsigned)std::max(1LL, bg), 128, 0, st>>>(sc, gc);
    const size_t smem = sizeof(float) * (size_t)S.s_total;
    const long long tiles = (nsamp + S.M - 1) / S.M;
    if (S.HW == 4) {
        const int b = persistent_grid(k_decode<4>, 32 * S.W, smem, tiles);
        k_decode<4><<<b, 32 * S.W, smem, st>>>(views, sc, S, pk, srec, gc, nsamp, d_nsamp, dec, vview, bp, rec,
                                               g2d_zero);
    } else {
        const int b = persistent_grid(k_decode<8>, 32 * S.W, smem, tiles);
        k_decode<8><<<b, 32 * S.W, smem, st>>>(views, sc, S, pk, srec, gc, nsamp, d_nsamp, dec, vview, bp, rec,
                                               g2d_zero);
    }
}

void launch_decode_bwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *samples,
                       long long nsamp, const uint32_t *d_nsamp, const float *gdec, float *g_mlp, float *g_feat,
                       float *g_offset, CellGrads cg, float *scratch, cudaStream_t st) {
    if (nsamp <= 0 || !sc.feat) return;
    const MlpShape S = mlp_shape(sc.F, sc.H, sc.K, true);
    float *pk = scratch, *srec = scratch + up_to(S.g_total, 4), *rows = srec + nsamp * DINFO;
    decode_prep(views, n_views, slot, sc, S, samples, nsamp, d_nsamp, pk, srec, st);
    const size_t smem = sizeof(float) * (size_t)S.s_total;
    const long long tiles = (nsamp + S.M - 1) / S.M;
    const bool cell = cg.center || cg.axes || cg.quat;
#define DGS_DBWD(HWV, FUSEV, CELLV, ROWS)                                                                      \
    do {                                                                                                      \
        const int b = persistent_grid(k_decode_bwd<HWV, FUSEV, CELLV>, 32 * S.W, smem, tiles);                \
        k_decode_bwd<HWV, FUSEV, CELLV><<<b, 32 * S.W, smem, st>>>(sc, S, pk, srec, nsamp, d_nsamp, gdec,     \
                                                                   g_feat, g_offset, ROWS, g_mlp, cg);        \
    } while (0)
    if (wgrad_fused(S)) {
        if (cell) DGS_DBWD(4, true, true, nullptr); else DGS_DBWD(4, true, false, nullptr);
        return;
    }
    if (S.HW == 4) {
        if (cell) DGS_DBWD(4, false, true, rows); else DGS_DBWD(4, false, false, rows);
    } else {
        if (cell) DGS_DBWD(8, false, true, rows); else DGS_DBWD(8, false, false, rows);
    }
#undef DGS_DBWD
    WgProblems pr{};
    pr.p[0] = WgProblem{S.row_dh, 4 * S.Hp, S.row_z, S.I, -1};
    for (int D = 0; D < 4; ++D) pr.p[1 + D] = WgProblem{S.row_do + S.rb[D], S.nout[D], S.row_h + D * S.Hp, S.H, D};
    const int chunk = 4096;
    const dim3 grid((unsigned)((nsamp + chunk - 1) / chunk), 16, 5);
    k_mlp_wgrad<<<grid, WT_T, 0, st>>>(rows, S, nsamp, d_nsamp, chunk, pr, g_mlp);
}

}  // namespace dgs
