// Decode of neural cells (the step before the path): the K Gaussians of a
// visible cell are predicted per view from the cell's latent feature f_n,
// the viewing distance delta_n and direction d_n by four MLPs with one ReLU
// hidden layer, F_sigma, F_c, F_s, F_q (Sec. III, Eq. 1-7; Sec. IV-A, Eq.
// 8-11).  Activations: opacity tanh (sigma <= 0 is not drawn), colour
// sigmoid, scale ratio sigmoid bounded by 1 - |O_pos| (Eq. 11) times the cell
// semi-axes S_n (Eq. 8), rotation normalised (a zero output is the identity
// rotation); centre x_n + R(Q_n)(O_pos * S_n)
// with O_pos moved into the unit ball (the centre stays inside the cell).
#include <algorithm>

#include "internal.cuh"

namespace dgs {

constexpr int DEC_THREADS = 64;
constexpr int DEC_MAXW = 64;  // maximum feature / hidden width

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// One thread per cell of scene `slot`, looping over the views in which the
// cell survived culling.  The thread's input vector z and hidden vector h
// live in shared memory columns (z[i] at s_z[i][tid]); the weights are read
// from global memory, where all threads of a warp read the same address.
__global__ void __launch_bounds__(DEC_THREADS) k_decode(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                        SceneDev sc, const uint32_t *__restrict__ count,
                                                        float *__restrict__ dec) {
    __shared__ float s_z[DEC_MAXW + 4][DEC_THREADS];
    __shared__ float s_h[DEC_MAXW][DEC_THREADS];
    const int t = threadIdx.x;
    const long long N = sc.N, G = sc.G;
    const int K = sc.K, F = sc.F, H = sc.H;
    const int outs[4] = {K, 3 * K, 3 * K, 4 * K};
    for (long long n = blockIdx.x * (long long)blockDim.x + t; n < N; n += (long long)gridDim.x * blockDim.x) {
        const float x0 = sc.cell[n], x1 = sc.cell[N + n], x2 = sc.cell[2 * N + n];
        const float S[3] = {sc.cell[3 * N + n], sc.cell[4 * N + n], sc.cell[5 * N + n]};
        float Rq[9];
        {
            const float qw = sc.cell[6 * N + n], qx = sc.cell[7 * N + n], qy = sc.cell[8 * N + n],
                        qz = sc.cell[9 * N + n];
            const float in = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            const float w = qw * in, x = qx * in, y = qy * in, z = qz * in;
            Rq[0] = 1.f - 2.f * (y * y + z * z); Rq[1] = 2.f * (x * y - w * z); Rq[2] = 2.f * (x * z + w * y);
            Rq[3] = 2.f * (x * y + w * z); Rq[4] = 1.f - 2.f * (x * x + z * z); Rq[5] = 2.f * (y * z - w * x);
            Rq[6] = 2.f * (x * z - w * y); Rq[7] = 2.f * (y * z + w * x); Rq[8] = 1.f - 2.f * (x * x + y * y);
        }
        for (int i = 0; i < F; ++i) s_z[i][t] = sc.feat[(long long)i * N + n];
        for (int v = 0; v < n_views; ++v) {
            const ViewDesc &Vw = views[v];
            if (Vw.scene_slot != slot || count[Vw.cell_base + n] == 0u) continue;
            const float r0 = x0 - Vw.eye[0], r1 = x1 - Vw.eye[1], r2 = x2 - Vw.eye[2];
            const float delta = sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
            s_z[F][t] = delta;
            s_z[F + 1][t] = r0 / delta;
            s_z[F + 2][t] = r1 / delta;
            s_z[F + 3][t] = r2 / delta;
            float *out = dec + (Vw.rec_base + n * K) * kDecF;
            // centres (no MLP) and the offsets' Eq. 11 bound
            for (int k = 0; k < K; ++k) {
                const long long g = n * K + k;
                float o0 = sc.goff[g], o1 = sc.goff[G + g], o2 = sc.goff[2 * G + g];
                const float on = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
                if (on > 1.0f) { o0 /= on; o1 /= on; o2 /= on; }
                const float l0 = o0 * S[0], l1 = o1 * S[1], l2 = o2 * S[2];
                float *o = out + k * kDecF;
                o[0] = x0 + Rq[0] * l0 + Rq[1] * l1 + Rq[2] * l2;
                o[1] = x1 + Rq[3] * l0 + Rq[4] * l1 + Rq[5] * l2;
                o[2] = x2 + Rq[6] * l0 + Rq[7] * l1 + Rq[8] * l2;
                o[3] = 1.0f - fminf(on, 1.0f);  // the ratio bound, consumed by the scale decoder below
            }
            const float *w = sc.mlp;
            for (int D = 0; D < 4; ++D) {
                const float *W1 = w, *b1 = w + H * (F + 4), *W2 = b1 + H, *b2 = W2 + outs[D] * H;
                for (int j = 0; j < H; ++j) {
                    float a = b1[j];
                    for (int i = 0; i < F + 4; ++i) a = fmaf(W1[j * (F + 4) + i], s_z[i][t], a);
                    s_h[j][t] = fmaxf(a, 0.0f);
                }
                for (int k = 0; k < K; ++k) {
                    float *o = out + k * kDecF;
                    const int nv = D == 0 ? 1 : (D == 3 ? 4 : 3);
                    float val[4];
                    for (int c = 0; c < nv; ++c) {
                        const int r = k * nv + c;
                        float a = b2[r];
                        for (int j = 0; j < H; ++j) a = fmaf(W2[r * H + j], s_h[j][t], a);
                        val[c] = a;
                    }
                    if (D == 0) {
                        o[10] = tanhf(val[0]);
                    } else if (D == 1) {
                        o[11] = sigmoidf_(val[0]); o[12] = sigmoidf_(val[1]); o[13] = sigmoidf_(val[2]);
                    } else if (D == 2) {
                        const float lim = o[3];
                        o[3] = fminf(sigmoidf_(val[0]), lim) * S[0];
                        o[4] = fminf(sigmoidf_(val[1]), lim) * S[1];
                        o[5] = fminf(sigmoidf_(val[2]), lim) * S[2];
                    } else {
                        const float qn2 = val[0] * val[0] + val[1] * val[1] + val[2] * val[2] + val[3] * val[3];
                        if (qn2 > 0.f) {
                            const float qn = rsqrtf(qn2);
                            o[6] = val[0] * qn; o[7] = val[1] * qn; o[8] = val[2] * qn; o[9] = val[3] * qn;
                        } else {  // no direction to normalise: the identity rotation
                            o[6] = 1.f; o[7] = 0.f; o[8] = 0.f; o[9] = 0.f;
                        }
                    }
                }
                w = b2 + outs[D];
            }
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Gradients through the decode, summed over the views in which each cell was
// decoded, from gdec (dL/d of the decoded values, layout of dec).  One thread
// per cell recomputes its decoders' hidden layers and outputs; the block
// keeps, in shared memory, the columns of its cells' inputs z, hidden values
// h, dL/dh (pre-activation) and dL/do of the decoder at hand, and the
// block's partial sums of every weight gradient (the packed layout).  Per
// decoder and view the block adds sum over its cells of dh z^T (W1, b1) and
// do h^T (W2, b2) to those sums, one weight per thread at a time; at the end
// they go to g_mlp with one atomic add per weight and block.  Columns are
// blockDim.x + 1 floats apart, so lanes reading consecutive rows at the same
// cell hit distinct banks.  Decisions held fixed: the ReLU masks, the Eq. 11
// bound (which of sigmoid and 1 - |O_pos| is smaller), sigma <= 0.
struct DecBwdSmem {
    int T, LD, F, H, K, P;
    __host__ __device__ int z_off() const { return 0; }
    __host__ __device__ int h_off() const { return (F + 4) * LD; }
    __host__ __device__ int dh_off() const { return h_off() + H * LD; }
    __host__ __device__ int do_off() const { return dh_off() + H * LD; }
    __host__ __device__ int gf_off() const { return do_off() + 4 * K * LD; }
    __host__ __device__ int acc_off() const { return gf_off() + F * LD; }
    __host__ __device__ int floats() const { return acc_off() + P; }
};

__host__ __device__ inline int dec_packed_size(int F, int H, int K) {
    return 4 * (H * (F + 4) + H) + (K + 3 * K + 3 * K + 4 * K) * (H + 1);
}

__global__ void __launch_bounds__(64) k_decode_bwd(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                   SceneDev sc, const uint32_t *__restrict__ count,
                                                   const float *__restrict__ gdec, float *__restrict__ g_mlp,
                                                   float *__restrict__ g_feat, float *__restrict__ g_offset) {
    extern __shared__ float smem[];
    const int T = blockDim.x, t = threadIdx.x;
    const long long N = sc.N, G = sc.G;
    const int K = sc.K, F = sc.F, H = sc.H;
    const DecBwdSmem L{T, T + 1, F, H, K, dec_packed_size(F, H, K)};
    float *s_z = smem + L.z_off(), *s_h = smem + L.h_off(), *s_dh = smem + L.dh_off(), *s_do = smem + L.do_off(),
          *s_gf = smem + L.gf_off(), *s_acc = smem + L.acc_off();
    const int LD = L.LD;
    const int outs[4] = {K, 3 * K, 3 * K, 4 * K};
    for (int i = t; i < L.P; i += T) s_acc[i] = 0.f;
    for (long long base = (long long)blockIdx.x * T; base < N; base += (long long)gridDim.x * T) {
        const long long n = base + t;
        const bool live = n < N;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, S[3] = {0.f, 0.f, 0.f}, Rq[9];
        if (live) {
            x0 = sc.cell[n]; x1 = sc.cell[N + n]; x2 = sc.cell[2 * N + n];
            S[0] = sc.cell[3 * N + n]; S[1] = sc.cell[4 * N + n]; S[2] = sc.cell[5 * N + n];
        }
        {
            const float qw = live ? sc.cell[6 * N + n] : 1.f, qx = live ? sc.cell[7 * N + n] : 0.f,
                        qy = live ? sc.cell[8 * N + n] : 0.f, qz = live ? sc.cell[9 * N + n] : 0.f;
            const float in = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            const float w = qw * in, x = qx * in, y = qy * in, z = qz * in;
            Rq[0] = 1.f - 2.f * (y * y + z * z); Rq[1] = 2.f * (x * y - w * z); Rq[2] = 2.f * (x * z + w * y);
            Rq[3] = 2.f * (x * y + w * z); Rq[4] = 1.f - 2.f * (x * x + z * z); Rq[5] = 2.f * (y * z - w * x);
            Rq[6] = 2.f * (x * z - w * y); Rq[7] = 2.f * (y * z + w * x); Rq[8] = 1.f - 2.f * (x * x + y * y);
        }
        for (int i = 0; i < F; ++i) {
            s_z[i * LD + t] = live ? sc.feat[(long long)i * N + n] : 0.f;
            s_gf[i * LD + t] = 0.f;
        }
        for (int i = F; i < F + 4; ++i) s_z[i * LD + t] = 0.f;
        if (live)
            for (int k = 0; k < K; ++k) {
                const long long g = n * K + k;
                g_offset[3 * g] = 0.f; g_offset[3 * g + 1] = 0.f; g_offset[3 * g + 2] = 0.f;
            }
        for (int v = 0; v < n_views; ++v) {
            const ViewDesc &Vw = views[v];
            if (Vw.scene_slot != slot) continue;  // uniform over the block
            const bool act = live && count[Vw.cell_base + n] != 0u;
            if (!__syncthreads_or(act)) continue;
            if (act) {
                const float r0 = x0 - Vw.eye[0], r1 = x1 - Vw.eye[1], r2 = x2 - Vw.eye[2];
                const float delta = sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
                s_z[F * LD + t] = delta;
                s_z[(F + 1) * LD + t] = r0 / delta;
                s_z[(F + 2) * LD + t] = r1 / delta;
                s_z[(F + 3) * LD + t] = r2 / delta;
            }
            const float *gd = gdec + (Vw.rec_base + (live ? n : 0) * K) * kDecF;
            const float *w = sc.mlp;
            int off = 0;  // packed offset of decoder D
            for (int D = 0; D < 4; ++D) {
                const int nout = outs[D], I = F + 4;
                const float *W1 = w, *b1 = w + H * I, *W2 = b1 + H, *b2 = W2 + nout * H;
                // hidden layer
                for (int j = 0; j < H; ++j) {
                    float a = 0.f;
                    if (act) {
                        a = b1[j];
                        for (int i = 0; i < I; ++i) a = fmaf(W1[j * I + i], s_z[i * LD + t], a);
                        a = fmaxf(a, 0.0f);
                    }
                    s_h[j * LD + t] = a;
                }
                // outputs and dL/do through the activation
                const int nv = D == 0 ? 1 : (D == 3 ? 4 : 3);
                for (int k = 0; k < K; ++k) {
                    float val[4] = {0.f, 0.f, 0.f, 0.f}, dov[4] = {0.f, 0.f, 0.f, 0.f};
                    if (act) {
                        for (int c = 0; c < nv; ++c) {
                            const int r = k * nv + c;
                            float a = b2[r];
                            for (int j = 0; j < H; ++j) a = fmaf(W2[r * H + j], s_h[j * LD + t], a);
                            val[c] = a;
                        }
                        const float *gk = gd + k * kDecF;
                        if (D == 0) {
                            const float sg = tanhf(val[0]);
                            dov[0] = gk[10] * (1.0f - sg * sg);
                        } else if (D == 1) {
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float cc = sigmoidf_(val[c]);
                                dov[c] = gk[11 + c] * cc * (1.0f - cc);
                            }
                        } else if (D == 2) {
                            const long long g = n * K + k;
                            const float O[3] = {sc.goff[g], sc.goff[G + g], sc.goff[2 * G + g]};
                            const float on = sqrtf(O[0] * O[0] + O[1] * O[1] + O[2] * O[2]);
                            const float lim = 1.0f - fminf(on, 1.0f);
                            float dlim = 0.f;
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float sg = sigmoidf_(val[c]);
                                if (sg < lim) dov[c] = gk[3 + c] * S[c] * sg * (1.0f - sg);
                                else dlim += gk[3 + c] * S[c];
                            }
                            // offset: mu = x + R(Q) (O_pos * S), lim = 1 - |O_pos|
                            float dOb[3];
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                dOb[c] = S[c] * (Rq[c] * gk[0] + Rq[3 + c] * gk[1] + Rq[6 + c] * gk[2]);
                            float dO[3];
                            if (on > 1.0f) {  // O_pos = O / |O| (unit length, so lim = 0 is constant)
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
                            for (int c = 0; c < 3; ++c) g_offset[3 * g + c] += dO[c];
                        } else {
                            const float qn2 = val[0] * val[0] + val[1] * val[1] + val[2] * val[2] + val[3] * val[3];
                            if (qn2 > 0.f) {  // a zero output decodes to the constant identity
                                const float iq = rsqrtf(qn2);
                                float pr = 0.f;
#pragma unroll
                                for (int c = 0; c < 4; ++c) pr += gk[6 + c] * val[c] * iq;
#pragma unroll
                                for (int c = 0; c < 4; ++c) dov[c] = (gk[6 + c] - pr * val[c] * iq) * iq;
                            }
                        }
                    }
                    for (int c = 0; c < nv; ++c) s_do[(k * nv + c) * LD + t] = dov[c];
                }
                // dL/dh (pre-activation) and the feature part of dL/dz
                for (int j = 0; j < H; ++j) {
                    float a = 0.f;
                    if (act && s_h[j * LD + t] > 0.f)
                        for (int r = 0; r < nout; ++r) a = fmaf(W2[r * H + j], s_do[r * LD + t], a);
                    s_dh[j * LD + t] = a;
                }
                if (act)
                    for (int i = 0; i < F; ++i) {
                        float a = s_gf[i * LD + t];
                        for (int j = 0; j < H; ++j) a = fmaf(W1[j * I + i], s_dh[j * LD + t], a);
                        s_gf[i * LD + t] = a;
                    }
                __syncthreads();
                // the block's weight gradients: W1 | b1 = sum dh [z | 1]^T, W2 | b2 = sum do [h | 1]^T
                {
                    const int n1 = H * (I + 1);
                    for (int idx = t; idx < n1; idx += T) {
                        const int j = idx / (I + 1), i = idx - j * (I + 1);
                        const float *a = s_dh + j * LD;
                        float acc = 0.f;
                        if (i < I) {
                            const float *b = s_z + i * LD;
                            for (int c = 0; c < T; ++c) acc = fmaf(a[c], b[c], acc);
                            s_acc[off + j * I + i] += acc;
                        } else {
                            for (int c = 0; c < T; ++c) acc += a[c];
                            s_acc[off + H * I + j] += acc;
                        }
                    }
                    const int o2 = off + H * I + H, n2 = nout * (H + 1);
                    for (int idx = t; idx < n2; idx += T) {
                        const int r = idx / (H + 1), j = idx - r * (H + 1);
                        const float *a = s_do + r * LD;
                        float acc = 0.f;
                        if (j < H) {
                            const float *b = s_h + j * LD;
                            for (int c = 0; c < T; ++c) acc = fmaf(a[c], b[c], acc);
                            s_acc[o2 + r * H + j] += acc;
                        } else {
                            for (int c = 0; c < T; ++c) acc += a[c];
                            s_acc[o2 + nout * H + r] += acc;
                        }
                    }
                }
                __syncthreads();
                off += H * I + H + nout * H + nout;
                w = b2 + nout;
            }
        }
        if (live)
            for (int i = 0; i < F; ++i) g_feat[n * F + i] = s_gf[i * LD + t];
    }
    __syncthreads();
    for (int i = t; i < L.P; i += T)
        if (s_acc[i] != 0.f) atomicAdd(g_mlp + i, s_acc[i]);
}

void launch_decode_bwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                       const float *gdec, float *g_mlp, float *g_feat, float *g_offset, cudaStream_t st) {
    if (sc.N == 0 || !sc.feat) return;
    // 64 cells per block while the shared memory fits, else 32
    int T = 64;
    DecBwdSmem L{T, T + 1, sc.F, sc.H, sc.K, dec_packed_size(sc.F, sc.H, sc.K)};
    if (L.floats() * 4 > 227 * 1024) {
        T = 32;
        L = DecBwdSmem{T, T + 1, sc.F, sc.H, sc.K, dec_packed_size(sc.F, sc.H, sc.K)};
    }
    const size_t bytes = sizeof(float) * (size_t)L.floats();
    cudaFuncSetAttribute(k_decode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decode_bwd, T, bytes);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long b = (sc.N + T - 1) / T;
    const long long cap = (long long)std::max(1, per_sm) * std::max(1, sms);
    if (b > cap) b = cap;
    k_decode_bwd<<<(unsigned)b, T, bytes, st>>>(views, n_views, slot, sc, count, gdec, g_mlp, g_feat, g_offset);
}

void launch_decode(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count, float *dec,
                   cudaStream_t st) {
    if (sc.N == 0 || n_views == 0 || !sc.feat) return;
    long long b = (sc.N + DEC_THREADS - 1) / DEC_THREADS;
    if (b > 152LL * 16) b = 152LL * 16;
    k_decode<<<(unsigned)b, DEC_THREADS, 0, st>>>(views, n_views, slot, sc, count, dec);
}

}  // namespace dgs
