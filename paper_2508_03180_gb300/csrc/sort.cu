// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits,
// one "onesweep" pass per digit: every CTA ranks a 3072-item partition
// locally, then learns the global offset of each digit from its predecessors
// through decoupled look-back (Merrill & Garland single-pass prefix scan,
// applied per digit as in Adinets & Merrill's Onesweep), and writes the
// partition out through shared memory in digit order (coalesced runs).  The digit
// histograms of all passes come from one upfront read of the keys.
//
// Sec. IV-B sorts the cell sequence with a radix sort; its cost grows with
// the sequence length, which is why the sort runs over cells, not Gaussians
// (Sec. VII-D, Tab. VI).
//
// Every wait on another CTA is bounded: after kSpinLimit polls the CTA sets
// *err, treats the missing count as 0 and carries on, so the kernel always
// finishes; the host turns a set flag into an error.
#include <algorithm>

#include "internal.cuh"

namespace dgs {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 12;                       // per thread
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;      // 3072 items per partition
static_assert(RS_TILE == kSortPartition, "the partition size is shared with the fixed scratch of sort_noalloc.cu");
constexpr int RS_WARP_ITEMS = 32 * RS_ITEMS;        // 384 contiguous items per warp
constexpr uint32_t FLAG_AGG = 1u << 30;             // partition's own count published
constexpr uint32_t FLAG_INC = 2u << 30;             // inclusive prefix published
constexpr uint32_t COUNT_MASK = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;

// Fault injection for the failure-detection tests (dgs_debug_inject_fault,
// DGS_FAULT_SORT_WAIT): while set, partition 0 never publishes its digit
// counts and a wait gives up after kFaultSpinLimit polls, so the look-back
// waits of the other partitions run out -- each one still bounded.  A wait
// that gave up counts the missing partition as 0, so every destination stays
// below the digit's true end: the kernels write inside the arrays.
__device__ int g_rs_fault = 0;
constexpr int kFaultSpinLimit = 1024;

cudaError_t set_sort_fault(bool on) {
    const int v = on ? 1 : 0;
    return cudaMemcpyToSymbol(g_rs_fault, &v, sizeof(int));
}

long long sort_parts_for(long long n) { return (n + RS_TILE - 1) / RS_TILE; }

// Histograms of every digit of every pass in one read of the keys.
// Also clears the look-back words of the first pass (status0).
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *__restrict__ keys, long long n,
                                                        const uint32_t *__restrict__ d_n, int passes,
                                                        uint32_t *__restrict__ hist, uint32_t *__restrict__ status0) {
    if (d_n) n = *d_n;
    const long long words = 256LL * ((n + RS_TILE - 1) / RS_TILE);
    for (long long i = blockIdx.x * (long long)RS_THREADS + threadIdx.x; i < words; i += (long long)gridDim.x * RS_THREADS)
        status0[i] = 0u;
    __shared__ uint32_t sh[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += RS_THREADS) (&sh[0][0])[i] = 0;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)RS_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * RS_THREADS) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += RS_THREADS) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Exclusive scan of each pass's 256 counts (one warp-free block per pass).
__global__ void k_rs_hist_scan(uint32_t *hist) {
    __shared__ uint32_t s[256];
    const int p = blockIdx.x, t = threadIdx.x;
    s[t] = hist[p * 256 + t];
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const uint32_t v = t >= off ? s[t - off] : 0u;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    hist[p * 256 + t] = t == 0 ? 0u : s[t - 1];
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) { return *(const volatile uint32_t *)p; }

// Pass `pass` of the sort.  The data ping-pongs between (k0, v0) and
// (k1, v1).  With skip_trivial, a pass whose digit is 0 for every key (the
// histogram says so) is the identity permutation and does nothing; every pass
// then takes its input from the buffer the previous non-trivial pass wrote,
// and the look-back arrays alternate over non-trivial passes.
__device__ __forceinline__ bool rs_trivial(const uint32_t *hist, int q, long long n) {
    return (long long)hist[256 * q + 1] == n;  // scanned base of digit 1 = count of digit 0
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_pass(uint32_t *__restrict__ k0, uint32_t *__restrict__ v0,
                                                        uint32_t *__restrict__ k1, uint32_t *__restrict__ v1,
                                                        long long n, const uint32_t *__restrict__ d_n, int pass,
                                                        const uint32_t *__restrict__ hist, bool skip_trivial,
                                                        uint32_t *__restrict__ status0, uint32_t *__restrict__ status1,
                                                        uint32_t *__restrict__ counter,
                                                        uint32_t *__restrict__ err) {
    __shared__ uint32_t s_warp[RS_WARPS][256];   // per-warp digit counts, then per-warp offsets
    __shared__ uint32_t s_base[256];             // global destination of the partition's first item per digit
    __shared__ uint32_t s_local[256];            // partition-local start of each digit
    __shared__ uint32_t s_wsum[RS_WARPS];
    __shared__ uint32_t s_key[RS_TILE], s_val[RS_TILE];  // the partition in digit order
    __shared__ uint32_t s_part;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (d_n) n = *d_n;
    int ord = pass;  // non-trivial passes before this one
    if (skip_trivial) {
        if (rs_trivial(hist, pass, n)) return;
        ord = 0;
        for (int q = 0; q < pass; ++q) ord += rs_trivial(hist, q, n) ? 0 : 1;
    }
    const int shift = 8 * pass;
    const uint32_t *__restrict__ digit_base = hist + 256 * pass;
    const uint32_t *__restrict__ kin = (ord & 1) ? k1 : k0;
    const uint32_t *__restrict__ vin = (ord & 1) ? v1 : v0;
    uint32_t *__restrict__ kout = (ord & 1) ? k0 : k1;
    uint32_t *__restrict__ vout = (ord & 1) ? v0 : v1;
    uint32_t *__restrict__ status = (ord & 1) ? status1 : status0;
    uint32_t *__restrict__ status_next = (ord & 1) ? status0 : status1;
    const long long n_parts = (n + RS_TILE - 1) / RS_TILE;
    if (blockIdx.x >= n_parts) return;  // the first min(grid, n_parts) CTAs take every partition
    // Persistent CTAs claim partitions in increasing order: a partition only
    // waits for earlier ones, which CTAs that are already running own.
    for (;;) {
        __syncthreads();
        if (tid == 0) s_part = atomicAdd(counter, 1u);
        __syncthreads();
        const long long part = s_part;
        if (part >= n_parts) break;
        for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&s_warp[0][0])[i] = 0;
        // the next pass's look-back words of this partition: that array was
        // last used by the previous pass, which has finished
        status_next[part * 256 + tid] = 0u;
        __syncthreads();
        const long long base = part * RS_TILE + (long long)warp * RS_WARP_ITEMS;

        uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const long long idx = base + it * 32 + lane;
            const bool ok = idx < n;
            key[it] = ok ? kin[idx] : 0u;
            val[it] = ok ? vin[idx] : 0u;
        }
        const unsigned lt_mask = (1u << lane) - 1u;
        // rank inside the warp, in item order (it, lane): stable
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const long long idx = base + it * 32 + lane;
            const bool ok = idx < n;
            const unsigned active = __ballot_sync(0xffffffffu, ok);
            rank[it] = 0;
            if (ok) {
                const uint32_t d = (key[it] >> shift) & 255u;
                const unsigned peers = __match_any_sync(active, d);
                const uint32_t before = s_warp[warp][d];
                rank[it] = before + __popc(peers & lt_mask);
                __syncwarp(active);
                if (lane == __ffs(peers) - 1) s_warp[warp][d] = before + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        // thread t owns digit t: partition total and per-warp exclusive offsets
        const int d = tid;
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = s_warp[w][d];
            s_warp[w][d] = total;
            total += c;
        }
        {  // partition-local digit starts: exclusive scan of the totals over the 256 digits
            uint32_t x = total;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wsum[warp] = x;
            __syncthreads();
            uint32_t wb = 0;
            for (int w = 0; w < warp; ++w) wb += s_wsum[w];
            s_local[d] = wb + x - total;
        }
        uint32_t *my = status + part * 256 + d;
        const bool fault = g_rs_fault != 0;
        if (part == 0) {
            if (!fault) atomicExch(my, FLAG_INC | total);
            s_base[d] = digit_base[d];
        } else {
            const int limit = fault ? kFaultSpinLimit : kSpinLimit;
            atomicExch(my, FLAG_AGG | total);
            uint32_t excl = 0;
            for (long long p = part - 1; p >= 0; --p) {
                const uint32_t *q = status + p * 256 + d;
                uint32_t s = ld_volatile(q);
                int spins = 0;
                while ((s & (FLAG_AGG | FLAG_INC)) == 0u) {
                    if (++spins > limit) { atomicOr(err, 1u); s = FLAG_INC; break; }
                    __nanosleep(64);
                    s = ld_volatile(q);
                }
                excl += s & COUNT_MASK;
                if (s & FLAG_INC) break;
            }
            atomicExch(my, FLAG_INC | (excl + total));
            s_base[d] = digit_base[d] + excl;
        }
        __syncthreads();
        // the partition in digit order in shared memory, then out with
        // consecutive threads on consecutive destinations within each digit
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const long long idx = base + it * 32 + lane;
            if (idx < n) {
                const uint32_t dg = (key[it] >> shift) & 255u;
                const uint32_t lp = s_local[dg] + s_warp[warp][dg] + rank[it];
                s_key[lp] = key[it];
                s_val[lp] = val[it];
            }
        }
        __syncthreads();
        const int cnt = (int)min((long long)RS_TILE, n - part * RS_TILE);
        for (int i = tid; i < cnt; i += RS_THREADS) {
            const uint32_t k = s_key[i], dg = (k >> shift) & 255u;
            const uint32_t dst = s_base[dg] + ((uint32_t)i - s_local[dg]);
            kout[dst] = k;
            vout[dst] = s_val[i];
        }
    }
}

// Copy the result back to (kd, vd) if an odd number of non-trivial passes
// left it in (ks, vs).
__global__ void k_copy_pairs(const uint32_t *__restrict__ ks, const uint32_t *__restrict__ vs, uint32_t *__restrict__ kd,
                             uint32_t *__restrict__ vd, long long n, const uint32_t *__restrict__ d_n,
                             const uint32_t *__restrict__ hist, int passes) {
    if (d_n) n = *d_n;
    int ord = 0;
    for (int q = 0; q < passes; ++q) ord += rs_trivial(hist, q, n) ? 0 : 1;
    if (!(ord & 1)) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
    }
}

// Persistent grid: the CTAs of k_rs_pass every SM of the current device holds at once.
static long long rs_max_ctas() { return resident_ctas((const void *)k_rs_pass, RS_THREADS); }

int radix_sort_pairs(uint32_t *keys, uint32_t *vals, long long n, int bits, const SortScratch &s, cudaStream_t st,
                     const uint32_t *d_n) {
    // n: the item count, or (d_n != NULL) the capacity, the count being read
    // from device memory when the kernels run (graph-capturable)
    if ((!d_n && n <= 1) || n <= 0 || bits <= 0) return 0;
    const int passes = (bits + 7) / 8;
    cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * 4 * 256, st);
    cudaMemsetAsync(s.counters, 0, sizeof(uint32_t) * 4, st);
    const long long parts = sort_parts_for(n);
    // look-back words: two arrays of `parts` x 256, used by alternate passes;
    // the histogram kernel clears the first, every pass clears the other
    uint32_t *status[2] = {s.status, s.status + 256 * parts};
    int hb = (int)((n + RS_THREADS * 8 - 1) / (RS_THREADS * 8));
    if (hb > 152 * 8) hb = 152 * 8;
    k_rs_hist<<<hb, RS_THREADS, 0, st>>>(keys, n, d_n, passes, s.hist, status[0]);
    k_rs_hist_scan<<<passes, 256, 0, st>>>(s.hist);
    const unsigned grid = (unsigned)std::min(parts, rs_max_ctas());
    const bool skip = d_n != nullptr;  // device-sized: key ranges unknown on the host
    for (int p = 0; p < passes; ++p)
        k_rs_pass<<<grid, RS_THREADS, 0, st>>>(keys, vals, s.keys_alt, s.vals_alt, n, d_n, p, s.hist, skip,
                                               status[0], status[1], s.counters + p, s.err);
    if (skip) {
        k_copy_pairs<<<152 * 8, 256, 0, st>>>(s.keys_alt, s.vals_alt, keys, vals, n, d_n, s.hist, passes);
    } else if (passes & 1) {  // result sits in the alternate buffers
        cudaMemcpyAsync(keys, s.keys_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, s.vals_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    }
    return passes;
}

// ---------------------------------------------------------------- exclusive scan (reduce, scan partials, downsweep)
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 16;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

long long scan_scratch_words(long long n) { return (n + SC_TILE - 1) / SC_TILE + 1; }

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SC_THREADS / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SC_THREADS / 32) s_warp[lane] = w;  // inclusive per warp
    }
    __syncthreads();
    const uint32_t warp_excl = warp == 0 ? 0u : s_warp[warp - 1];
    *total = s_warp[SC_THREADS / 32 - 1];
    __syncthreads();
    return warp_excl + x - v;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const uint32_t *__restrict__ in, long long n,
                                                            const uint32_t *__restrict__ d_n,
                                                            uint32_t *__restrict__ partial) {
    __shared__ uint32_t s_warp[SC_THREADS / 32];
    if (d_n) n = *d_n;
    if (blockIdx.x * (long long)SC_TILE >= n && blockIdx.x > 0) return;
    const long long base = blockIdx.x * (long long)SC_TILE;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        const long long idx = base + i * SC_THREADS + threadIdx.x;
        if (idx < n) sum += in[idx];
    }
    uint32_t tot;
    block_excl_scan(sum, s_warp, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_partials(uint32_t *partial, long long nb,
                                                              const uint32_t *__restrict__ d_n, uint32_t *total) {
    __shared__ uint32_t s_warp[SC_THREADS / 32];
    if (d_n) nb = (*d_n + SC_TILE - 1) / SC_TILE;
    uint32_t carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += SC_THREADS) {
        const long long b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? partial[b] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(v, s_warp, &tot);
        if (b < nb) partial[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down(const uint32_t *__restrict__ in, long long n,
                                                          const uint32_t *__restrict__ d_n,
                                                          const uint32_t *__restrict__ partial, uint32_t *__restrict__ out) {
    __shared__ uint32_t s_warp[SC_THREADS / 32];
    if (d_n) n = *d_n;
    if (blockIdx.x * (long long)SC_TILE >= n) return;
    const long long base = blockIdx.x * (long long)SC_TILE + (long long)threadIdx.x * SC_ITEMS;  // blocked per thread
    uint32_t v[SC_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        const long long idx = base + i;
        v[i] = idx < n ? in[idx] : 0u;
        sum += v[i];
    }
    uint32_t tot;
    uint32_t run = partial[blockIdx.x] + block_excl_scan(sum, s_warp, &tot);
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        const long long idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, long long n, uint32_t *total, uint32_t *scratch,
                        cudaStream_t st, const uint32_t *d_n) {
    // n: the count, or (d_n != NULL) the capacity with the count in device memory
    if (n == 0) {
        cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return;
    }
    const long long nb = (n + SC_TILE - 1) / SC_TILE;
    k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, d_n, scratch);
    k_scan_partials<<<1, SC_THREADS, 0, st>>>(scratch, nb, d_n, total);
    k_scan_down<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, d_n, scratch, out);
}

}  // namespace dgs
