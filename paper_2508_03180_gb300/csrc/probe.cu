// Throughput probes for the roofline of the blend kernels, which are bound by
// FP32 and SFU instruction issue rather than by memory: the FP32 FMA rate and
// the rate of ex2.approx (the blend's exponential) measured on the running
// GPU with CUDA events.
#include "runtime.h"

namespace dgs {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_UNROLL = 16;

// 8 independent FMA chains per thread: a <- a b + c (b, c chosen so values stay finite).
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(float *out, int iters, float seed) {
    float a0 = seed + threadIdx.x * 1e-3f, a1 = a0 + 0.1f, a2 = a0 + 0.2f, a3 = a0 + 0.3f;
    float a4 = a0 + 0.4f, a5 = a0 + 0.5f, a6 = a0 + 0.6f, a7 = a0 + 0.7f;
    const float b = 0.9999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
            a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
            a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == -1.0f) out[blockIdx.x] = s;  // never true: keeps the chains alive
}

__device__ __forceinline__ float probe_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 8 independent chains a <- 2^-a (stays in [0.5, 1]).
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ex2(float *out, int iters, float seed) {
    float a0 = seed + threadIdx.x * 1e-4f, a1 = a0 + 0.01f, a2 = a0 + 0.02f, a3 = a0 + 0.03f;
    float a4 = a0 + 0.04f, a5 = a0 + 0.05f, a6 = a0 + 0.06f, a7 = a0 + 0.07f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
            a0 = probe_ex2(-a0); a1 = probe_ex2(-a1); a2 = probe_ex2(-a2); a3 = probe_ex2(-a3);
            a4 = probe_ex2(-a4); a5 = probe_ex2(-a5); a6 = probe_ex2(-a6); a7 = probe_ex2(-a7);
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == -1.0f) out[blockIdx.x] = s;
}

}  // namespace dgs

using namespace dgs;


namespace {

// Device time (ms) of `launch` after one untimed launch.
template <typename F>
dgs_status time_ms(F launch, float *ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    launch();
    CK(cudaGetLastError());
    CK(cudaEventRecord(a, 0));
    launch();
    CK(cudaEventRecord(b, 0));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return DGS_OK;
}

}  // namespace

extern "C" dgs_status dgs_probe_alu(dgs_ctx *ctx, dgs_alu_peaks *out) {
    if (!ctx || !out) return set_error(DGS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->cfg.device));
    int sms = 0, per_fma = 0, per_ex2 = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->cfg.device));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_fma, k_probe_fma, PROBE_THREADS, 0));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_ex2, k_probe_ex2, PROBE_THREADS, 0));
    dgs_status s;
    if ((s = ctx->aux.ensure(sizeof(float) * 65536))) return s;
    float *sink = (float *)ctx->aux.p;
    const int gf = sms * per_fma, ge = sms * per_ex2;
    const int it_f = 4096, it_e = 512;
    float ms_f = 0.f, ms_e = 0.f;
    if ((s = time_ms([&] { k_probe_fma<<<gf, PROBE_THREADS>>>(sink, it_f, 0.5f); }, &ms_f))) return s;
    if ((s = time_ms([&] { k_probe_ex2<<<ge, PROBE_THREADS>>>(sink, it_e, 0.5f); }, &ms_e))) return s;
    const double fma = (double)gf * PROBE_THREADS * it_f * PROBE_UNROLL * 8;
    const double ex2 = (double)ge * PROBE_THREADS * it_e * PROBE_UNROLL * 8;
    out->fp32_tflops = 2.0 * fma / (ms_f * 1e-3) / 1e12;
    out->ex2_per_s = ex2 / (ms_e * 1e-3);
    out->ms_fma = ms_f;
    out->ms_ex2 = ms_e;
    out->sm_count = sms;
    out->reserved = 0;
    return DGS_OK;
}
