// dgs_sort_pairs_noalloc: the library's stable radix sort for callers that
// must not allocate device memory -- for example a process whose caching
// allocator has already reserved the device's free memory for its own pool,
// or a real-time loop that forbids allocation after start-up because
// cudaMalloc/cudaFree can block and synchronise the whole device.  Its scratch
// (alternate key/value buffers, digit histograms, look-back status words,
// partition counters, error flag) is one file-scope device array below, so
// the call itself allocates nothing; the array is part of this file's module,
// which the CUDA runtime loads into a device's context on first use (with
// lazy loading, the default, at the first call on that device), and every
// GPU that has loaded it holds it until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "internal.cuh"
#include "runtime.h"

namespace {

constexpr long long kMaxItems = 1LL << 20;                // 1,048,576 pairs per call at most
constexpr long long kMaxParts = (kMaxItems + dgs::kSortPartition - 1) / dgs::kSortPartition;  // sort partitions
// layout of the scratch array, in 32-bit words
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + kMaxItems;
constexpr size_t kOffHist = kOffVals + kMaxItems;          // 4 passes x 256 digits
constexpr size_t kOffStatus = kOffHist + 4 * 256;          // 2 x kMaxParts x 256 look-back words
constexpr size_t kOffCounters = kOffStatus + 2 * kMaxParts * 256;
constexpr size_t kOffErr = kOffCounters + 4;
constexpr size_t kWords = kOffErr + 60;                    // about 9.1 MB in total

// Device-side scratch.  In host code this name is only a stand-in: its
// device address in the current context comes from cudaGetSymbolAddress.
static __device__ __align__(256) uint32_t g_sort_scratch[kWords];

// Device address of the scratch array in the current device's context.  It is
// looked up on every call (a host-side lookup, no allocation once the module
// is loaded), so a context that was reset and created again gets the array's
// new address.  The first lookup in a context loads this file's module -- the
// CUDA driver then allocates the array's device memory -- which is why the
// first call on a device belongs to the caller's set-up.
dgs_status scratch_address(uint32_t **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return dgs::cuda_error(e, "cudaGetSymbolAddress of the sort scratch");
    *out = static_cast<uint32_t *>(p);
    return DGS_OK;
}

}  // namespace

extern "C" dgs_status dgs_sort_pairs_noalloc(uint32_t *keys, uint32_t *vals, int64_t n, int32_t bits,
                                            dgs_stream stream) {
    if (n < 0 || bits < 0 || bits > 32 || (n > 0 && (!keys || !vals)))
        return dgs::set_error(DGS_ERR_INVALID_ARG, "dgs_sort_pairs_noalloc: bad argument");
    if (n > kMaxItems)
        return dgs::set_error(DGS_ERR_CAPACITY, "dgs_sort_pairs_noalloc: n = " + std::to_string(n) +
                                                    " exceeds the fixed maximum of 1048576 pairs");
    if (n <= 1 || bits == 0) return DGS_OK;
    uint32_t *base = nullptr;
    dgs_status s = scratch_address(&base);
    if (s) return s;
    cudaError_t e;
    dgs::SortScratch sc;
    sc.keys_alt = base + kOffKeys;
    sc.vals_alt = base + kOffVals;
    sc.hist = base + kOffHist;
    sc.status = base + kOffStatus;
    sc.counters = base + kOffCounters;
    sc.err = base + kOffErr;
    sc.cap_items = kMaxItems;
    sc.cap_parts = kMaxParts;
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the error flag starts at
    // zero here; histograms, counters and look-back words are cleared by the
    // sort itself before each use
    if ((e = cudaMemsetAsync(sc.err, 0, sizeof(uint32_t), st)) != cudaSuccess)
        return dgs::cuda_error(e, "clearing the sort error flag");
    dgs::radix_sort_pairs(keys, vals, n, bits, sc, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return dgs::cuda_error(e, "radix sort launch");
    uint32_t flag = 0;
    if ((e = cudaMemcpyAsync(&flag, sc.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return dgs::cuda_error(e, "dgs_sort_pairs_noalloc");
    if (flag) return dgs::set_error(DGS_ERR_TIMEOUT, "radix sort look-back wait gave up");
    return DGS_OK;
}
