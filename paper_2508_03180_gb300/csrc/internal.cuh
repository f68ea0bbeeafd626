// Internal declarations shared by the kernel translation units of the
// sm_103a Duplex-GS renderer.  Not part of the public ABI (include/dgs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dgs.h"

namespace dgs {

constexpr int kTile = 16;          // tile edge in pixels (Sec. IV-B tile-based paradigm)
constexpr int kSortPartition = 3072;  // items per radix-sort partition (sort.cu; sizes the look-back words)
constexpr int kTilePix = kTile * kTile;
constexpr int kMaxK = 32;          // Gaussians per cell supported
constexpr int kRecF4 = 3;          // float4s per projected-Gaussian record (48 B)
constexpr int kGradF = 12;         // floats per screen-space gradient record (48 B)

// One view of a batched launch chain.  Tiles of all views are numbered
// view-major (tile_base), pixels too (pix_base); (view, cell) entries start
// at cell_base and the view's projected records at rec_base.  Views of one
// chain may belong to different resident scenes (scene_slot).
struct ViewDesc {
    int W, H, Tx, Ty;
    int tile_base;
    int scene_slot;        // index into the chain's scene table
    long long pix_base;    // first pixel of this view in per-pixel buffers
    long long cell_base;   // first (view, cell) entry of this view
    long long rec_base;    // first projected record of this view
    long long N;           // cells of the view's scene
    float *out;            // device image [3][H][W] of this view, or NULL (chain buffer)
    int K;                 // Gaussians per cell of the view's scene
    int pad0;
    float fx, fy, cx, cy, znear, pad1;
    float R[9], t[3], eye[3];
    float pad2[3];
};

// Device-side view of one resident scene (structure of arrays).
struct SceneDev {
    const float *cell;     // [11][N]: centre xyz, axes xyz, quat wxyz, v
    const float *gauss;    // [11][G]: mean xyz, scale xyz, quat wxyz, logit
    const float *sh;       // [C*3][G]: coefficient c, channel ch at plane c*3+ch
    const float *vsh;      // [Cv][N]: SH coefficients of a view-dependent v_n, or NULL (scalar v_n)
    const float *feat;     // neural cells: [N][F] latent features (rows), or NULL (explicit Gaussians)
    const float *goff;     // neural cells: [3][G] position offsets O_pos
    const float *mlp;      // neural cells: packed decoder weights
    long long N, G;
    int K, sh_degree;
    int v_sh_degree;       // -1 without vsh
    int F, H;              // neural cells: feature and hidden widths
    int pad;
};

constexpr int kDecF = 14;  // floats per decoded Gaussian: mean 3, scale 3, quat 4, opacity, rgb 3

// Sizes of one launch chain kept in device memory.  A captured CUDA graph
// replays over batches of other sizes: kernels handed a non-NULL pointer read
// their sizes here when they run, and their host arguments are then only the
// capacities that sized the grids and buffers.
struct ChainSizes {
    uint32_t n_entries;    // (view, cell) entries, <= capacity
    int32_t n_views;
    int32_t total_tiles;
    uint32_t L_cap;        // capacity of the (tile, cell) pair buffers
    int32_t n_scenes;      // entries of the chain's device scene table
    int32_t pad[3];
};

struct BlendParams {
    float eps, alpha_max, d_min, bg0, bg1, bg2, dilation, ksigma;
    float w_bg;  // background weight in the hybrid's normalisation
    int flags;   // DGS_FLAG_* variants of the readings
};

// ---------------------------------------------------------------- FP32 with one prescribed rounding order
// Every binning decision (cell culling and tile rectangle, the per-Gaussian
// AABB inputs) is computed with these: each is exactly one IEEE operation
// that the compiler may not fuse, so results are bit-identical to any other
// implementation that performs the same sequence of float operations.
__device__ __forceinline__ float fmul_s(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd_s(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub_s(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv_s(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt_s(float a) { return __fsqrt_rn(a); }

// Rotation matrix of quaternion (w,x,y,z) after normalisation, row-major.
__device__ __forceinline__ void rot_from_quat_s(float w, float x, float y, float z, float R[9]) {
    const float n = fsqrt_s(fadd_s(fadd_s(fadd_s(fmul_s(w, w), fmul_s(x, x)), fmul_s(y, y)), fmul_s(z, z)));
    w = fdiv_s(w, n); x = fdiv_s(x, n); y = fdiv_s(y, n); z = fdiv_s(z, n);
    const float xx = fmul_s(x, x), yy = fmul_s(y, y), zz = fmul_s(z, z);
    const float xy = fmul_s(x, y), xz = fmul_s(x, z), yz = fmul_s(y, z);
    const float wx = fmul_s(w, x), wy = fmul_s(w, y), wz = fmul_s(w, z);
    R[0] = fsub_s(1.0f, fmul_s(2.0f, fadd_s(yy, zz)));
    R[1] = fmul_s(2.0f, fsub_s(xy, wz));
    R[2] = fmul_s(2.0f, fadd_s(xz, wy));
    R[3] = fmul_s(2.0f, fadd_s(xy, wz));
    R[4] = fsub_s(1.0f, fmul_s(2.0f, fadd_s(xx, zz)));
    R[5] = fmul_s(2.0f, fsub_s(yz, wx));
    R[6] = fmul_s(2.0f, fsub_s(xz, wy));
    R[7] = fmul_s(2.0f, fadd_s(yz, wx));
    R[8] = fsub_s(1.0f, fmul_s(2.0f, fadd_s(xx, yy)));
}

// v = R p + t, rows summed left to right.
__device__ __forceinline__ void xform_s(const float R[9], const float t[3], float p0, float p1, float p2,
                                        float v[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
        v[i] = fadd_s(fadd_s(fadd_s(fmul_s(R[3 * i], p0), fmul_s(R[3 * i + 1], p1)), fmul_s(R[3 * i + 2], p2)), t[i]);
}

// ---------------------------------------------------------------- launchers
// binning.cu
// Every launcher taking `dsz` (nullable) reads the sizes from it at run time;
// `d_L` likewise points at the device-side pair count.
// vview[entry]: v_n as rendered in that view (the scalar, or the clamped SH
// value of a view-dependent v_n).
// flags: dgs_config.flags (DGS_FLAG_NEAR_FULL changes the footprint of cells at the near plane).
void launch_cell_project(const ViewDesc *views, int n_views, const SceneDev *scenes, long long n_entries,
                         uint32_t *zkey, uint32_t *zval, short4 *rect, float *depth, uint32_t *count,
                         uint32_t *visible, float *vview, int flags, cudaStream_t st,
                         const ChainSizes *dsz = nullptr);
void launch_gather_counts(const uint32_t *zval_sorted, const uint32_t *count, long long n, uint32_t *out,
                          cudaStream_t st, const uint32_t *d_n = nullptr);
void launch_emit(const uint32_t *offs, const uint32_t *zval_sorted, const short4 *rect, const ViewDesc *views,
                 int n_views, long long n_entries, long long L, uint32_t *tkey, uint32_t *tval, cudaStream_t st,
                 const ChainSizes *dsz = nullptr, const uint32_t *d_L = nullptr);
void launch_tile_ranges(const uint32_t *tkey_sorted, long long L, uint2 *ranges, cudaStream_t st,
                        const uint32_t *d_L = nullptr);
// small[total] = pairs needed; writes small[clamped] = min(total, L_cap) and
// small[overflow] = (total > L_cap), for chains whose pair buffers are
// sized in advance.
void launch_clamp_pairs(uint32_t *small, int total, int clamped, int overflow, const ChainSizes *dsz,
                        cudaStream_t st);

// sort.cu
struct SortScratch {
    uint32_t *keys_alt, *vals_alt;   // n each
    uint32_t *hist;                  // 4 * 256
    uint32_t *status;                // 2 * parts * 256 (alternate passes)
    uint32_t *counters;              // 4 (one per pass)
    uint32_t *err;                   // 1
    long long cap_items, cap_parts;
};
long long sort_parts_for(long long n);
// Stable LSD radix sort of (key, val) by the low `bits` bits.  Results end in
// keys/vals.  Returns the number of passes.
int radix_sort_pairs(uint32_t *keys, uint32_t *vals, long long n, int bits, const SortScratch &s,
                     cudaStream_t st, const uint32_t *d_n = nullptr);
// Exclusive scan; total written to *total (device).  scratch >= scan_scratch_words(n).
long long scan_scratch_words(long long n);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, long long n, uint32_t *total, uint32_t *scratch,
                        cudaStream_t st, const uint32_t *d_n = nullptr);

// project.cu  (one launch per distinct scene of the chain: views whose
// scene_slot differs from `slot` are skipped)
void launch_project_fwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                        const float *vview, const BlendParams &bp, float4 *rec, float *g2d_zero, cudaStream_t st);
// dL/dv per cell from the per-(view, cell) values gv of views [0, n_views)
// (all of scene sc): g_cell_v[n] = sum over views (nullable), and for a
// view-dependent v_n g_vsh[n][lm] = sum over views of gv Y_lm(d) where the
// clamp was inactive (nullable); both overwritten.  g_center [N][3]
// (nullable, accumulated): the cell centres' gradient through d.
void launch_cell_v_grad(const ViewDesc *views, int n_views, const SceneDev &sc, const float *gv, float *g_cell_v,
                        float *g_vsh, float *g_center, cudaStream_t st);
// Gradients of the cell proxies' parameters ([N][3], [N][3], [N][4];
// nullable, accumulated).
struct CellGrads {
    float *center, *axes, *quat;
};
// Comparator binning: one entry per (view, Gaussian), entry e = cell_base + g
// (views with N = G, K = 1 entries); wsr selects the LC-WSR weight in r2.w.
void launch_gauss_bin(const ViewDesc *views, int n_views, const SceneDev &sc, const BlendParams &bp, bool wsr,
                      float tau, float4 *rec, uint32_t *zkey, uint32_t *zval, short4 *rect, uint32_t *count,
                      uint32_t *visible, cudaStream_t st);
// Neural scenes: decode the Gaussians of the (view, cell) entries
// samples[0 .. nsamp) (entry e = cell_base of its view + cell; NULL: entry q
// for sample q) of scene `slot` into dec [rec_base + g][kDecF] and, with rec
// non-NULL, write their records (colour and opacity as decoded, sigma <= 0
// not drawn; v_n from vview) and zero their g2d rows (g2d_zero non-NULL).
// Features are rows [N][F].  d_nsamp (nullable): the sample count on the
// device, at most nsamp (then the capacity the scratch is sized for).  At the
// common widths the products run on the tensor cores; *err (a device word) is
// set to 1 if one of their completion waits gives up (the results are then
// not valid).
void launch_decode(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *samples,
                   long long nsamp, const uint32_t *d_nsamp, float *dec, float *scratch, const float *vview,
                   const BlendParams &bp, float4 *rec, float *g2d_zero, uint32_t *err, cudaStream_t st);
// Floats of scratch (16-byte aligned) that one launch_decode (bwd = false)
// or launch_decode_bwd (bwd = true) call needs.
long long decode_scratch_floats(int F, int H, int K, long long nsamp, long long G, bool bwd);
// Adjoints of a neural scene: the records' gradients with respect to the
// decoded values of every decoded (view, Gaussian) (gdec, layout of dec),
// then through the decode of the same samples to the packed weights g_mlp,
// the features g_feat [N][F] and the raw offsets g_offset [G][3], summed
// over views; all three are accumulated (zero them first).
void launch_project_bwd_neural(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                               const BlendParams &bp, const float *dec, const float *g2d, float *gdec,
                               cudaStream_t st);
// Cell alignment (Sec. IV-B, Eq. 10 and the centre update) of every cell,
// in place in `cell` (the scene's writable cell planes); dec: decoded values
// of one view for every Gaussian (neural scenes with DGS_ALIGN_QUAT).
void launch_cell_align(const SceneDev &sc, float *cell, const float *dec, int what, float *out_center, float *out_quat,
                       cudaStream_t st);
// cg: the cell gradients through the decode (centre: the decoder inputs and
// the Gaussian centres; axes: the centres and scales; rotation: the centres).
void launch_decode_bwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *samples,
                       long long nsamp, const uint32_t *d_nsamp, const float *gdec, float *g_mlp, float *g_feat,
                       float *g_offset, CellGrads cg, float *scratch, cudaStream_t st);
// One launch for every scene of the device scene table (dsz->n_scenes
// entries, Gaussian counts <= G_cap, which sizes the grid).
void launch_project_fwd_table(const ViewDesc *views, const SceneDev *scenes, long long G_cap, const uint32_t *count,
                              const float *vview, const BlendParams &bp, float4 *rec, cudaStream_t st,
                              const ChainSizes *dsz);
void launch_project_bwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                        const BlendParams &bp, const float *g2d, float *g_mean, float *g_scale,
                        float *g_log_scale, float *g_quat, float *g_logit, float *g_sh, cudaStream_t st);

// blend.cu
void launch_blend_fwd(const ViewDesc *views, int n_views, int total_tiles, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, float *out_rgb,
                      float *out_rgb2, float *out_D, int *out_nd, int K_all, cudaStream_t st,
                      const ChainSizes *dsz = nullptr, uint32_t *work = nullptr);
// g_v_entry (nullable): dL/dv_n accumulated per (view, cell) entry [cell_base + cell].
void launch_blend_bwd(const ViewDesc *views, int n_views, int total_tiles, int K, const uint2 *ranges,
                      const uint32_t *tile_cells, const float4 *rec, const BlendParams &bp, const float *rgb,
                      const float *D, const int *nd, const float *dL_drgb, float *g2d, float *g_v_entry,
                      cudaStream_t st);

void launch_count_pairs(const ViewDesc *views, int n_views, int total_tiles, const uint2 *ranges,
                        const uint32_t *tile_cells, const float4 *rec, const int *nd, unsigned long long *counts,
                        cudaStream_t st);

// misc.cu
void launch_aos_to_soa(const float *src, int64_t rows, int cols, float *dst, int64_t dst_stride,
                       cudaStream_t st);
void launch_soa_to_aos(const float *src, int64_t rows, int cols, int64_t src_stride, float *dst,
                       cudaStream_t st);
void launch_fill_f32(float *dst, int64_t n, float v, cudaStream_t st);
void launch_loss_l1(const float *rgb, const float *target, int64_t n, float *dL, float *partial,
                    int nblocks, float *loss, cudaStream_t st);
int loss_l1_blocks(int64_t n);

// CTAs of `kernel` that all SMs of the current device hold at once with
// `threads` threads and no dynamic shared memory (SMs x resident CTAs per SM,
// at least 1); computed once per (device, kernel) and cached under a lock, so
// threads and devices may call it concurrently.
long long resident_ctas(const void *kernel, int threads);

// Test-only: make the radix sort's look-back waits run out (see sort.cu).
cudaError_t set_sort_fault(bool on);
cudaError_t set_tc_fault(bool on);  // the tensor-core decode's completion wait runs out (DGS_FAULT_TC_WAIT)

// Asynchronous 16-byte global-to-shared copies (cp.async, cached in L2
// only): both addresses 16-byte aligned.  A copy is complete for the issuing
// thread after a cp_async_wait that covers its commit group, and visible to
// the other threads of the CTA (or warp) after a barrier that follows it.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace dgs
