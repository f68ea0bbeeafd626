// Cell alignment (Sec. IV-B): every cell's rotation becomes the normalised
// opacity-weighted sum of its Gaussians' unit quaternions (Eq. 10) and its
// centre the mean of their centres, both from the values before the call.
// Explicit Gaussians: sigma = sigmoid(logit), q = g_quat / |g_quat|, mu = the
// stored mean.  Neural cells: sigma and q as decoded for one view (sigma <= 0,
// not drawn, weighs 0), mu = x_n + R(Q_n)(O_pos * S_n) (view-independent).
// A cell whose weighted sum is the zero vector keeps its rotation.
#include <cstring>

#include "runtime.h"

namespace dgs {

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

__global__ void __launch_bounds__(128) k_cell_align(SceneDev sc, float *__restrict__ cell, const float *__restrict__ dec,
                                                    int what, float *__restrict__ out_center,
                                                    float *__restrict__ out_quat) {
    const long long N = sc.N, G = sc.G;
    const int K = sc.K;
    const bool neural = sc.feat != nullptr;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        float x[3], Q[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = cell[i * N + n];
#pragma unroll
        for (int i = 0; i < 4; ++i) Q[i] = cell[(6 + i) * N + n];
        float nx[3] = {x[0], x[1], x[2]}, nq[4] = {Q[0], Q[1], Q[2], Q[3]};
        if (what & DGS_ALIGN_CENTER) {
            float s[3] = {0.f, 0.f, 0.f};
            if (!neural) {
                for (int k = 0; k < K; ++k) {
                    const long long g = n * K + k;
#pragma unroll
                    for (int i = 0; i < 3; ++i) s[i] += sc.gauss[i * G + g];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) nx[i] = s[i] / (float)K;
            } else {  // mean of x + R(Q)(O_pos * S) = x + R(Q)(S * mean O_pos)
                for (int k = 0; k < K; ++k) {
                    const long long g = n * K + k;
                    float o0 = sc.goff[g], o1 = sc.goff[G + g], o2 = sc.goff[2 * G + g];
                    const float on = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
                    if (on > 1.0f) { o0 /= on; o1 /= on; o2 /= on; }
                    s[0] += o0; s[1] += o1; s[2] += o2;
                }
                const float l0 = s[0] / (float)K * cell[3 * N + n], l1 = s[1] / (float)K * cell[4 * N + n],
                            l2 = s[2] / (float)K * cell[5 * N + n];
                const float in = rsqrtf(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]);
                const float w = Q[0] * in, a = Q[1] * in, b = Q[2] * in, c = Q[3] * in;
                nx[0] = x[0] + (1.f - 2.f * (b * b + c * c)) * l0 + 2.f * (a * b - w * c) * l1 + 2.f * (a * c + w * b) * l2;
                nx[1] = x[1] + 2.f * (a * b + w * c) * l0 + (1.f - 2.f * (a * a + c * c)) * l1 + 2.f * (b * c - w * a) * l2;
                nx[2] = x[2] + 2.f * (a * c - w * b) * l0 + 2.f * (b * c + w * a) * l1 + (1.f - 2.f * (a * a + b * b)) * l2;
            }
        }
        if (what & DGS_ALIGN_QUAT) {
            float s[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < K; ++k) {
                const long long g = n * K + k;
                float q[4], sg;
                if (!neural) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) q[i] = sc.gauss[(6 + i) * G + g];
                    const float iq = 1.0f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) q[i] *= iq;
                    sg = 1.0f / (1.0f + expf(-sc.gauss[10 * G + g]));
                } else {
                    const float *d = dec + g * kDecF;
#pragma unroll
                    for (int i = 0; i < 4; ++i) q[i] = d[6 + i];
                    sg = fmaxf(d[10], 0.0f);
                }
                // rounded products, then sums: q and -q of equal weight cancel exactly
                // (a fused multiply-add would leave the product's rounding error)
#pragma unroll
                for (int i = 0; i < 4; ++i) s[i] = __fadd_rn(s[i], __fmul_rn(sg, q[i]));
            }
            const float n2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3];
            if (n2 > 0.f) {
                const float nn = sqrtf(n2);
#pragma unroll
                for (int i = 0; i < 4; ++i) nq[i] = s[i] / nn;
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) cell[i * N + n] = nx[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) cell[(6 + i) * N + n] = nq[i];
        if (out_center) {
#pragma unroll
            for (int i = 0; i < 3; ++i) out_center[3 * n + i] = nx[i];
        }
        if (out_quat) {
#pragma unroll
            for (int i = 0; i < 4; ++i) out_quat[4 * n + i] = nq[i];
        }
    }
}

void launch_cell_align(const SceneDev &sc, float *cell, const float *dec, int what, float *out_center, float *out_quat,
                       cudaStream_t st) {
    if (sc.N == 0) return;
    k_cell_align<<<grid_for(sc.N, 128), 128, 0, st>>>(sc, cell, dec, what, out_center, out_quat);
}

}  // namespace dgs

using namespace dgs;

extern "C" dgs_status dgs_cell_align(dgs_ctx *ctx, uint32_t scene_id, int32_t what, int32_t cam_slot,
                                     float *out_center, float *out_quat, int32_t out_location, dgs_stream stream) {
    if (!ctx) return set_error(DGS_ERR_INVALID_ARG, "NULL ctx");
    if (what < 1 || what > (DGS_ALIGN_QUAT | DGS_ALIGN_CENTER))
        return set_error(DGS_ERR_INVALID_ARG, "what must be DGS_ALIGN_QUAT, DGS_ALIGN_CENTER or both");
    if (out_location != DGS_HOST && out_location != DGS_DEVICE) return set_error(DGS_ERR_INVALID_ARG, "bad location");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return set_error(DGS_ERR_NOT_FOUND, "unknown scene id");
    Scene &sc = *it->second;
    const bool neural = sc.F > 0, decode = neural && (what & DGS_ALIGN_QUAT);
    if (decode && (cam_slot < 0 || cam_slot >= kMaxCamSlots || !ctx->cam_set[cam_slot]))
        return set_error(DGS_ERR_INVALID_ARG, "a neural scene's Eq. 10 needs a set camera slot (sigma, q depend on the view)");
    const long long N = sc.N, G = sc.G;
    if (N == 0) return DGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // scratch: [view][packed weights][decoded G][host staging 7 N], each 256-byte aligned
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_pk = up(sizeof(ViewDesc)),
                 o_dec = o_pk + up(decode ? sizeof(float) * decode_scratch_floats(sc.F, sc.H, sc.K, N, G, false) : 0),
                 o_stg = o_dec + up(decode ? sizeof(float) * kDecF * G : 0),
                 o_err = o_stg + up(out_location == DGS_HOST ? sizeof(float) * 7 * N : 0),
                 total = o_err + 256;
    dgs_status s;
    if ((s = ctx->align_tmp.ensure(total))) return s;
    char *base = (char *)ctx->align_tmp.p;
    float *dec = nullptr;
    const SceneDev sd = sc.dev();
    if (decode) {
        const ViewDesc v = make_view(ctx->cams[cam_slot], 0, 0, 0, sc, 0, 0);
        CK(cudaMemcpyAsync(base, &v, sizeof(v), cudaMemcpyHostToDevice, st));  // pageable: staged before return
        dec = (float *)(base + o_dec);
        CK(cudaMemsetAsync(base + o_err, 0, 4, st));
        launch_decode((const ViewDesc *)base, 1, 0, sd, nullptr, N, nullptr, dec, (float *)(base + o_pk), nullptr,
                      BlendParams{}, nullptr, nullptr, (uint32_t *)(base + o_err), st);  // every cell of the one view; no records
    }
    float *oc = out_center, *oq = out_quat;
    if (out_location == DGS_HOST) {
        float *stg = (float *)(base + o_stg);
        oc = out_center ? stg : nullptr;
        oq = out_quat ? stg + 3 * N : nullptr;
    }
    launch_cell_align(sd, (float *)sc.cell.p, dec, what, oc, oq, st);
    CK(cudaGetLastError());
    if (out_location == DGS_HOST) {
        if (out_center) CK(cudaMemcpyAsync(out_center, oc, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, st));
        if (out_quat) CK(cudaMemcpyAsync(out_quat, oq, sizeof(float) * 4 * N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (decode) {  // the decode's tensor-core completion waits (synchronises the stream)
        uint32_t e = 0;
        CK(cudaStreamSynchronize(st));
        CK(cudaMemcpy(&e, base + o_err, 4, cudaMemcpyDeviceToHost));
        if (e) return set_error(DGS_ERR_TIMEOUT, "the decode's tensor-core completion wait gave up");
    }
    return DGS_OK;
}
