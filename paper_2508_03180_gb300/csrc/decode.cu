// Decode of neural cells (the step before the path): the K Gaussians of a
// visible cell are predicted per view from the cell's latent feature f_n,
// the viewing distance delta_n and direction d_n by four MLPs with one ReLU
// hidden layer, F_sigma, F_c, F_s, F_q (Sec. III, Eq. 1-7; Sec. IV-A, Eq.
// 8-11).  Activations: opacity tanh (sigma <= 0 is not drawn), colour
// sigmoid, scale ratio sigmoid bounded by 1 - |O_pos| (Eq. 11) times the cell
// semi-axes S_n (Eq. 8), rotation normalised; centre x_n + R(Q_n)(O_pos * S_n)
// with O_pos moved into the unit ball (the centre stays inside the cell).
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
                        const float qn = rsqrtf(val[0] * val[0] + val[1] * val[1] + val[2] * val[2] + val[3] * val[3]);
                        o[6] = val[0] * qn; o[7] = val[1] * qn; o[8] = val[2] * qn; o[9] = val[3] * qn;
                    }
                }
                w = b2 + outs[D];
            }
        }
    }
}

void launch_decode(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count, float *dec,
                   cudaStream_t st) {
    if (sc.N == 0 || n_views == 0 || !sc.feat) return;
    long long b = (sc.N + DEC_THREADS - 1) / DEC_THREADS;
    if (b > 152LL * 16) b = 152LL * 16;
    k_decode<<<(unsigned)b, DEC_THREADS, 0, st>>>(views, n_views, slot, sc, count, dec);
}

}  // namespace dgs
