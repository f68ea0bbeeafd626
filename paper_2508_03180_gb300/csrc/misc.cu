// Layout conversion between the ABI's per-parameter row-major arrays and the
// library's structure-of-arrays planes, and the L1 photometric loss.
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"

namespace dgs {

// src [rows][cols] -> dst plane j at dst + j * dst_stride (column j of src).
// A block moves 32 rows at a time through shared memory: the rows are read
// as one contiguous run and every plane receives 32 consecutive floats.
constexpr int TR_ROWS = 32, TR_MAXC = 64;
__global__ void __launch_bounds__(256) k_aos_to_soa(const float *__restrict__ src, int64_t rows, int cols,
                                                    float *__restrict__ dst, int64_t dst_stride) {
    __shared__ float t[TR_ROWS][TR_MAXC + 1];
    for (int64_t r0 = blockIdx.x * (int64_t)TR_ROWS; r0 < rows; r0 += (int64_t)gridDim.x * TR_ROWS) {
        const int nr = (int)min((int64_t)TR_ROWS, rows - r0);
        const float *s = src + r0 * cols;
        for (int i = threadIdx.x; i < nr * cols; i += blockDim.x) t[i / cols][i % cols] = s[i];
        __syncthreads();
        for (int i = threadIdx.x; i < cols * TR_ROWS; i += blockDim.x) {
            const int c = i / TR_ROWS, r = i % TR_ROWS;
            if (r < nr) dst[c * dst_stride + r0 + r] = t[r][c];
        }
        __syncthreads();
    }
}

// Fallback for more than TR_MAXC columns: one element per thread.
__global__ void k_aos_to_soa_wide(const float *__restrict__ src, int64_t rows, int cols, float *__restrict__ dst,
                                  int64_t dst_stride) {
    const int64_t total = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols;
        const int c = (int)(i - r * cols);
        dst[c * dst_stride + r] = src[i];
    }
}

__global__ void k_soa_to_aos(const float *__restrict__ src, int64_t rows, int cols, int64_t src_stride,
                             float *__restrict__ dst) {
    const int64_t total = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols;
        const int c = (int)(i - r * cols);
        dst[i] = src[c * src_stride + r];
    }
}

__global__ void k_fill(float *__restrict__ dst, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = v;
}

long long resident_ctas(const void *kernel, int threads) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, long long> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, kernel);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    const long long n = (long long)std::max(1, sms) * std::max(1, per_sm);
    cache[key] = n;
    return n;
}

static int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

void launch_aos_to_soa(const float *src, int64_t rows, int cols, float *dst, int64_t dst_stride, cudaStream_t st) {
    if (rows * cols == 0) return;
    if (cols > TR_MAXC) {
        k_aos_to_soa_wide<<<grid_for(rows * cols), 256, 0, st>>>(src, rows, cols, dst, dst_stride);
        return;
    }
    int64_t b = (rows + TR_ROWS - 1) / TR_ROWS;
    if (b > 152 * 8) b = 152 * 8;
    k_aos_to_soa<<<(int)b, 256, 0, st>>>(src, rows, cols, dst, dst_stride);
}

void launch_soa_to_aos(const float *src, int64_t rows, int cols, int64_t src_stride, float *dst, cudaStream_t st) {
    if (rows * cols == 0) return;
    k_soa_to_aos<<<grid_for(rows * cols), 256, 0, st>>>(src, rows, cols, src_stride, dst);
}

void launch_fill_f32(float *dst, int64_t n, float v, cudaStream_t st) {
    if (n == 0) return;
    k_fill<<<grid_for(n), 256, 0, st>>>(dst, n, v);
}

// L1 loss: dL/drgb = sign(rgb - target) / n; per-block partial sums of
// |rgb - target| then a single-block sum in fixed order (deterministic).
constexpr int LOSS_T = 256;

int loss_l1_blocks(int64_t n) {
    int64_t b = (n + LOSS_T * 8 - 1) / (LOSS_T * 8);
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ float block_sum(float v, float *s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < LOSS_T / 32; ++w) t += s[w];
    return t;
}

__global__ void __launch_bounds__(LOSS_T) k_loss_l1(const float *__restrict__ rgb, const float *__restrict__ target,
                                                    int64_t n, float inv_n, float *__restrict__ dL,
                                                    float *__restrict__ partial) {
    __shared__ float s[LOSS_T / 32];
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)LOSS_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * LOSS_T) {
        const float d = rgb[i] - target[i];
        acc += fabsf(d);
        dL[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    }
    const float t = block_sum(acc, s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(LOSS_T) k_loss_final(const float *__restrict__ partial, int nb, float inv_n,
                                                       float *__restrict__ loss) {
    __shared__ float s[LOSS_T / 32];
    float acc = 0.f;
    for (int i = threadIdx.x; i < nb; i += LOSS_T) acc += partial[i];
    const float t = block_sum(acc, s);
    if (threadIdx.x == 0) *loss = t * inv_n;
}

void launch_loss_l1(const float *rgb, const float *target, int64_t n, float *dL, float *partial, int nblocks,
                    float *loss, cudaStream_t st) {
    const float inv_n = n > 0 ? 1.0f / (float)n : 0.f;
    k_loss_l1<<<nblocks, LOSS_T, 0, st>>>(rgb, target, n, inv_n, dL, partial);
    k_loss_final<<<1, LOSS_T, 0, st>>>(partial, nblocks, inv_n, loss);
}

}  // namespace dgs
