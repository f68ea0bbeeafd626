/*
 * dgs.h -- C ABI of the GB300 (sm_103a) Duplex-GS hybrid renderer hot path.
 *
 * The operation (Duplex-GS, arXiv 2508.03180):
 *   * A scene is a set of ellipsoidal cell proxies (centre x_n, semi-axes
 *     S_n, rotation Q_n, calibration scalar v_n), each emitting K Gaussians
 *     (Sec. IV-A, Eq. 1).
 *   * Per view, cells are projected to the screen, culled to the frustum and
 *     assigned to 16x16 tiles; a radix sort orders (tile, cell depth) keys
 *     over cells only, never over Gaussians (Sec. IV-B).
 *   * Per pixel, the tile's cells are walked front to back.  Inside a cell
 *     the K Gaussians are summed order-independently (weighted-sum
 *     rendering); across cells the weights w_n = v_n T_n^cell follow
 *     alpha-blending style transmittance, and blending halts once T^cell
 *     drops below eps (Sec. V, Eq. 12-14).  A Gaussian is skipped at a pixel
 *     outside its screen AABB (Sec. VI-A).
 *   * render_backward is the adjoint of that image with respect to every
 *     Gaussian parameter (the paper trains through this renderer, Sec. VI).
 *
 * Conventions for every call:
 *   * Return value: DGS_OK (0) or a negative dgs_status; no call aborts the
 *     process.  dgs_last_error() gives a message for the calling thread.
 *   * Pointers are plain host or device addresses; a `location` field says
 *     which.  Inputs are read during the call (host inputs are copied before
 *     the call returns); the caller keeps ownership of everything it passes.
 *   * Device work is enqueued on the given stream (a cudaStream_t, NULL =
 *     legacy default stream) and is asynchronous unless stated otherwise.
 *     Host outputs are complete when the call returns.
 *   * Layouts are row-major, float32, structure-of-arrays per parameter.
 */
#ifndef DGS_H
#define DGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dgs_status;
enum {
    DGS_OK = 0,
    DGS_ERR_INVALID_ARG = -1, /* bad pointer, size, id or option */
    DGS_ERR_OOM = -2,         /* device allocation failed (or the HBM budget is exhausted) */
    DGS_ERR_NOT_FOUND = -3,   /* unknown scene / camera slot / ticket / state */
    DGS_ERR_CUDA = -4,        /* a CUDA call or a kernel failed; see dgs_last_error */
    DGS_ERR_TIMEOUT = -5,     /* poll timed out, or a bounded device wait gave up */
    DGS_ERR_BUSY = -6,        /* request queue full; retry later */
    DGS_ERR_CAPACITY = -7,    /* a size exceeds a fixed maximum of the call */
    DGS_ERR_GUARD = -8,       /* debug mode: a guard word next to a device buffer was overwritten */
    DGS_ERR_WORKER = -9,      /* the serving worker stopped after a host-side fault; restart serving */
    DGS_ERR_CANCELLED = -10   /* a serving request cancelled by dgs_cancel */
};

/* Where an argument array lives.  DGS_HOST arrays may be pageable or
 * page-locked (cudaHostAlloc / cudaMallocHost / cudaHostRegister).
 * Page-locked host arrays are read or written by the library's kernels
 * directly over the host link (no device staging copy; the transfer runs
 * while the kernel computes); pageable ones are staged through device
 * memory.  Either way a call that takes a DGS_HOST array returns only after
 * the transfer is complete, and the array is then the caller's again. */
enum { DGS_HOST = 0, DGS_DEVICE = 1 };

typedef struct dgs_ctx dgs_ctx;
typedef struct dgs_fwd_state dgs_fwd_state;
typedef void *dgs_stream; /* cudaStream_t */

/* Renderer settings.  dgs_config_default() fills the defaults below. */
typedef struct {
    float eps;        /* 1e-4: halt when T^cell < eps (Sec. V-B; the 3DGS threshold, Sec. VII-D) */
    float alpha_max;  /* 0.99: alpha = min(sigma G', alpha_max); alpha in [0,1] (Sec. V-A) */
    float d_min;      /* 1e-10: a pixel with sum_n w_n sum_k alpha <= d_min shows the background */
    float bg[3];      /* background colour (0,0,0) */
    float dilation;   /* 0.3 px^2 added to the EWA screen covariance */
    float ksigma;     /* 3: AABB half extent in standard deviations (Sec. VI-A) */
    int32_t device;   /* CUDA device ordinal (0) */
    int32_t flags;    /* 0: variants of the hybrid renderer's readings, DGS_FLAG_* below */
    int64_t hbm_budget_bytes; /* serving admission budget; 0 = 90% of free memory at create */
    float w_bg;       /* 0: background weight in the normalisation, C = (N + w_bg bg) / (D + w_bg)
                       * (Eq. 4's background term applied to Eq. 12); the background where
                       * D + w_bg <= d_min */
    int32_t reserved;
} dgs_config;

/* dgs_config.flags (the defaults are the paper's reading; each flag is an
 * alternative the paper leaves open):
 *   DGS_FLAG_ALPHA_SKIP    alpha < 1/255 contributes nothing (the 3DGS skip)
 *   DGS_FLAG_TERM_EXCLUDE  a cell whose blending would take the cell
 *                          transmittance below eps is not blended and ends the
 *                          pixel (the 3DGS rule; by default that cell is still
 *                          blended, Sec. V-B)
 *   DGS_FLAG_AABB_SQUARE   the per-Gaussian box is the square of radius
 *                          ceil(ksigma sqrt(lambda_max(Sigma'))) (the 3DGS box)
 *                          instead of ksigma sqrt(Sigma'_xx) by ksigma sqrt(Sigma'_yy)
 *   DGS_FLAG_NUMERATOR     the image is the numerator N of Eq. 12 (no
 *                          normalisation; with one Gaussian per cell and v = 1
 *                          this is alpha-blending, Eq. 2-3)
 *   DGS_FLAG_NEAR_FULL     a cell whose ellipsoid reaches the near plane
 *                          (c_z - sqrt(S_zz) <= znear) without lying wholly
 *                          behind it (c_z + sqrt(S_zz) > znear) covers every
 *                          tile of the image, sorted at depth max(c_z, 0),
 *                          instead of being culled (a conservative footprint;
 *                          its Gaussians are still culled one by one at znear)
 * ALPHA_SKIP, TERM_EXCLUDE, NUMERATOR, NEAR_FULL and w_bg apply to the hybrid
 * renderer (dgs_render, serving); AABB_SQUARE also to the comparators (it
 * changes the per-Gaussian records they share).  The adjoint follows every
 * flag. */
#define DGS_FLAG_ALPHA_SKIP 1
#define DGS_FLAG_TERM_EXCLUDE 2
#define DGS_FLAG_AABB_SQUARE 4
#define DGS_FLAG_NUMERATOR 8
#define DGS_FLAG_NEAR_FULL 16

void dgs_config_default(dgs_config *cfg);

/* Create a context on cfg->device (NULL = defaults).  The context owns every
 * device buffer it allocates; destroy frees them.  Thread-safe per call. */
dgs_status dgs_create(const dgs_config *cfg, dgs_ctx **out);
void dgs_destroy(dgs_ctx *ctx);
const char *dgs_last_error(dgs_ctx *ctx);

/* ---------------------------------------------------------------- scenes */

/* A scene: N cells, each emitting K Gaussians (Gaussian g belongs to cell
 * g / K; G = N K).  All arrays float32, in `location` memory:
 *   cell_center [N][3], cell_axes [N][3] (semi-axes S_n), cell_quat [N][4]
 *   (w,x,y,z; normalised by the renderer), cell_v [N] (v_n in [0,1]; NULL = 1)
 *   g_mean [G][3], g_scale [G][3] (linear standard deviations),
 *   g_quat [G][4] (w,x,y,z), g_logit [G] (opacity = sigmoid(logit)),
 *   g_sh [G][(sh_degree+1)^2][3] real spherical-harmonic colour
 *   coefficients (colour = max(0, 0.5 + sum_lm k_lm Y_lm(view dir))).
 * The data are copied into context memory.  K in [1, 32], sh_degree in 0..3,
 * N >= 0 (an empty scene renders the background).
 *
 * View-dependent v_n (Sec. V-A: v is parameterised by spherical harmonics
 * because cell occlusion depends on the view): with cell_v_sh
 * [N][(v_sh_degree+1)^2] (v_sh_degree in 0..3) the renderer uses, per view,
 *   v_n = clamp(sum_lm k_lm Y_lm(d), 0, 1),  d = (c_n - eye) / |c_n - eye|,
 * (the colour's real SH basis; c_n the cell centre); cell_v is then used
 * only by the comparators (dgs_render_compare).  cell_v_sh = NULL: the
 * scalar cell_v. */
/* Neural cells (the decode step before the path, Sec. III Eq. 1-7 and Sec.
 * IV-A Eq. 8-11): the K Gaussians of every visible cell are decoded per view
 * from the cell's latent feature f_n, the viewing distance delta_n = |x_n - eye|
 * and direction d_n = (x_n - eye) / delta_n by four MLPs with one ReLU hidden
 * layer of width `hidden` on z = [f_n, delta_n, d_n]:
 *   opacity  sigma_{n,k} = tanh(o_sigma[k])        (sigma <= 0: not drawn)
 *   colour   c_{n,k} = sigmoid(o_c[3k .. 3k+2])     (used directly, no SH)
 *   scale    s_{n,k} = min(sigmoid(o_s[3k .. 3k+2]), 1 - |O_pos|) * S_n
 *   rotation q_{n,k} = o_q[4k .. 4k+3] normalised
 *   centre   mu_{n,k} = x_n + R(Q_n) (O_pos * S_n), O_pos moved into the unit ball
 * Arrays (float32, in the scene's location memory): cell_feat [N][feat_dim],
 * g_offset [G][3] (O_pos), mlp: decoder after decoder (opacity, colour,
 * scale, rotation; output widths K, 3K, 3K, 4K): W1 [hidden][feat_dim+4]
 * row-major, b1 [hidden], W2 [out][hidden] row-major, b2 [out].
 * 1 <= feat_dim <= 64, 1 <= hidden <= 64.  Neural scenes render through
 * dgs_render and the serving loop, and dgs_render_backward gives the
 * gradients to the packed decoder weights, the cell features and the
 * offsets (g_mlp, g_feat, g_offset); the comparators take explicit scenes
 * only (INVALID_ARG for a neural one).  At feat_dim + 4 <= 40, hidden <= 32
 * and K <= 10 the decode's products run on the tensor cores (TF32 in three
 * split products, FP32 accumulation: FP32-level values). */
typedef struct {
    int32_t feat_dim;
    int32_t hidden;
    const float *cell_feat;
    const float *g_offset;
    const float *mlp;
} dgs_neural_desc;

typedef struct {
    int64_t num_cells;
    int32_t K;
    int32_t sh_degree;
    int32_t location; /* DGS_HOST or DGS_DEVICE */
    int32_t reserved;
    const float *cell_center, *cell_axes, *cell_quat, *cell_v;
    const float *g_mean, *g_scale, *g_quat, *g_logit, *g_sh;  /* ignored for neural scenes */
    const float *cell_v_sh;
    int32_t v_sh_degree;
    int32_t reserved2;
    const dgs_neural_desc *neural; /* NULL: explicit Gaussians */
} dgs_scene_desc;

dgs_status dgs_scene_upload(dgs_ctx *ctx, const dgs_scene_desc *desc, uint32_t *scene_id);
/* Overwrite the Gaussian parameters (and v, or its SH coefficients) of an
 * existing scene in place, same N, K and degrees (a training step's update).  Asynchronous on stream
 * for device inputs; host inputs synchronise the stream before return. */
dgs_status dgs_scene_update(dgs_ctx *ctx, uint32_t scene_id, const dgs_scene_desc *desc, dgs_stream stream);
dgs_status dgs_scene_release(dgs_ctx *ctx, uint32_t scene_id);

/* Scene files (the one persisted state of the renderer).  Little-endian: a
 * 40-byte header -- char magic[4] = "DGS1", uint32 version = 1, int64
 * num_cells, int32 K, sh_degree, v_sh_degree (-1: scalar v_n), feat_dim and
 * hidden (0: explicit Gaussians), uint32 reserved -- then the scene's float32
 * arrays in the layouts of dgs_scene_desc, in this order: cell_center,
 * cell_axes, cell_quat, cell_v; explicit Gaussians: g_mean, g_scale,
 * g_quat, g_logit, g_sh; neural cells: cell_feat, g_offset, mlp; then
 * cell_v_sh if v_sh_degree >= 0.
 * dgs_scene_save writes scene_id's current parameters to `path`; it reads them
 * on the legacy default stream and returns when the file is closed, so work on
 * non-blocking streams that writes the scene must be synchronised first.
 * dgs_scene_load reads such a file and uploads it as a new scene, as
 * dgs_scene_upload would: NOT_FOUND if the file cannot be opened,
 * INVALID_ARG if it is not a version-1 scene file of consistent size. */
dgs_status dgs_scene_save(dgs_ctx *ctx, uint32_t scene_id, const char *path);
dgs_status dgs_scene_load(dgs_ctx *ctx, const char *path, uint32_t *scene_id);

/* ---------------------------------------------------------------- cameras */

/* Pinhole camera.  R, t map world to view space (x right, y down, +z
 * forward; row-major R).  eye is the camera centre in world space (used for
 * the colour's view direction).  Pixel (i,j) is sampled at (i+0.5, j+0.5).
 * Gaussians and cells must lie beyond znear to be drawn. */
typedef struct {
    int32_t W, H;
    float fx, fy, cx, cy, znear;
    float R[9], t[3], eye[3];
} dgs_camera;

/* Store a camera in slot `slot` (0 .. 4095). */
dgs_status dgs_camera_set(dgs_ctx *ctx, uint32_t slot, const dgs_camera *cam);

/* ---------------------------------------------------------------- render */

typedef struct {
    int64_t sort_length;   /* L: (tile, cell) pairs sorted, summed over views */
    int64_t visible_cells; /* (view, cell) pairs that survived culling */
    int64_t num_tiles;     /* tiles over all views */
    float ms_total;        /* device time of the call, only if timing was requested */
    int32_t timing;        /* in: nonzero = record CUDA events and synchronise */
    int32_t reserved;
} dgs_stats;

/* Render n_views views of one scene in one batched launch chain.
 * cam_slots[v] selects each view's camera.  out_rgb receives the images
 * back to back, view v as [3][H_v][W_v] planar float32 (offset = sum of
 * 3 H W of the views before it), in out_location memory.
 * state (nullable): if non-NULL, *state receives a handle that keeps this
 * render's intermediate buffers for dgs_render_backward; it stays owned by
 * the context until dgs_state_release.  stats (nullable): filled on return.
 *
 * Synchronisation.  With device output and no stats the call is asynchronous
 * on `stream`: it enqueues the whole chain and returns.  The number L of
 * (tile, cell) pairs is then known on the device only; the pair buffers hold
 * 1.5 x the largest pairs-per-tile seen in this context (at least 65,536)
 * and the kernels stop at that capacity.  A render whose L exceeded it
 * leaves an incomplete image and state; this is found once its chain has
 * completed (when its buffers are reused, or by dgs_render_backward on its
 * state if it has completed by then), the capacity grows to fit, and the next
 * dgs_render or dgs_render_backward on the context returns DGS_ERR_CAPACITY
 * (a radix sort or a tensor-core wait of the decode that gave up:
 * DGS_ERR_TIMEOUT) once; render it again.  Neural scenes are asynchronous
 * too (the decode reads the visible-cell count on the device).  The call
 * synchronises the stream once after binning, and sizes the pairs exactly,
 * when stats are requested and on the context's first render (to learn its
 * pairs per tile); host output synchronises at the end. */
dgs_status dgs_render(dgs_ctx *ctx, uint32_t scene_id, int32_t n_views, const uint32_t *cam_slots,
                      float *out_rgb, int32_t out_location, dgs_fwd_state **state, dgs_stream stream,
                      dgs_stats *stats);

/* Gradients of a scalar loss with respect to the scene parameters, given
 * dL/d(image) in the layout of out_rgb.  Every non-NULL output is
 * OVERWRITTEN (not accumulated), same layout as the scene arrays:
 *   g_mean [G][3], g_scale [G][3] (dL/dscale), g_log_scale [G][3]
 *   (= scale * dL/dscale), g_quat [G][4], g_logit [G], g_sh [G][C][3],
 *   g_cell_v [N] (dL/dv_n summed over the views, v_n as rendered in each),
 *   g_cell_v_sh [N][(v_sh_degree+1)^2] (scenes with view-dependent v only:
 *   sum over views of dL/dv_n Y_lm(d), zero where the clamp was active).
 * Neural scenes (Sec. III, Eq. 1-7; Sec. IV-A, Eq. 8-11) take the gradients
 * through the per-view decode instead of the explicit Gaussian outputs,
 * which must then be NULL (and these NULL for explicit scenes):
 *   g_mlp [packed weight count] in the layout of dgs_neural_desc.mlp,
 *   g_feat [N][feat_dim], g_offset [G][3] (dL/d of the raw offsets),
 * each summed over the views in which the cell was decoded.  The decode's
 * own decisions (the ReLU masks, the Eq. 11 bound, sigma <= 0 not drawn)
 * are held fixed with the others.
 * The cell proxies' own parameters (Sec. IV-A: centre x_n, semi-axes S_n,
 * rotation Q_n; Sec. V-A: v_n), any scene:
 *   g_cell_center [N][3]: through the direction d = (x_n - eye)/|x_n - eye|
 *     of a view-dependent v_n, and for neural cells through the decoder
 *     inputs delta_n, d_n and the centres mu = x_n + R(Q_n)(O_pos * S_n);
 *   g_cell_axes [N][3]: neural cells, through the centres and the scales
 *     s = min(sigmoid, 1 - |O_pos|) * S_n (Eq. 8, 11);
 *   g_cell_quat [N][4]: neural cells, through R(Q_n) of the centres (Q_n as
 *     stored, normalised by the renderer);
 * each summed over the views.  The cells' footprints (culling, tile lists,
 * depth order) are held fixed, so an explicit scene with a scalar v_n has
 * zero gradients here.
 * Discrete choices of the forward (culling, tile lists, AABB skips, alpha
 * clamp, the per-pixel number of blended cells) are held fixed. */
typedef struct {
    int32_t location;
    int32_t reserved;
    float *g_mean, *g_scale, *g_log_scale, *g_quat, *g_logit, *g_sh, *g_cell_v;
    float *g_cell_v_sh;
    float *g_mlp, *g_feat, *g_offset;
    float *g_cell_center, *g_cell_axes, *g_cell_quat;
} dgs_grads;

/* Asynchronous on stream when dL_drgb and the outputs are device memory;
 * with host dL_drgb or host outputs (dgs_grads.location) the call
 * synchronises the stream before return. */
dgs_status dgs_render_backward(dgs_ctx *ctx, dgs_fwd_state *state, const float *dL_drgb, int32_t location,
                               const dgs_grads *out, dgs_stream stream);
dgs_status dgs_state_release(dgs_ctx *ctx, dgs_fwd_state *state);

/* L1 photometric loss mean|rgb - target| over n floats (device pointers),
 * writing dL/drgb = sign(rgb - target) / n and the loss value (device
 * float).  Deterministic. */
dgs_status dgs_loss_l1(dgs_ctx *ctx, const float *rgb, const float *target, int64_t n, float *dL_drgb,
                       float *loss, dgs_stream stream);

/* Copy one intermediate buffer of a forward state to host memory (tests
 * and diagnostics).  `what`:
 *   DGS_BUF_CELL_RECT   int32 [V][N][4]  tx0 ty0 tx1 ty1 (tx0 = -1: culled)
 *   DGS_BUF_CELL_DEPTH  float [V][N]     view depth of the cell centre
 *   DGS_BUF_TILE_CELLS  uint32 [L]       cell ids, ordered by (global tile, depth, cell)
 *   DGS_BUF_TILE_RANGES uint32 [T][2]    [start,end) per global tile (view-major tiles)
 *   DGS_BUF_GAUSS_REC   float [V][G][12] mu_x mu_y ext_x ext_y | k p, k r, k t, opacity | r g b v
 *                       where the conic Sigma'^-1 = L L^T, L = [[p, 0], [r, t]], k = sqrt(log2(e)/2)
 *   DGS_BUF_PIX_D       float [P]        per-pixel weight sum D (P = all views' pixels)
 *   DGS_BUF_PIX_NDONE   int32 [P]        per-pixel number of blended cells
 *   DGS_BUF_GRAD2D      float [V][G][12] after backward: dmu_x dmu_y da db dc dsigma dr dg db 0 0 0
 *   DGS_BUF_CELL_V      float [V][N]     v_n as rendered in each view
 *   DGS_BUF_DECODED     float [V][G][14] neural scenes: decoded mean(3) scale(3) quat(4) opacity
 *                       rgb(3) of the Gaussians of visible cells (others unspecified)
 * *needed receives the byte size; nothing is copied if bytes < needed.
 * Synchronises the stream the state was rendered on. */
enum {
    DGS_BUF_CELL_RECT = 1,
    DGS_BUF_CELL_DEPTH = 2,
    DGS_BUF_TILE_CELLS = 3,
    DGS_BUF_TILE_RANGES = 4,
    DGS_BUF_GAUSS_REC = 5,
    DGS_BUF_PIX_D = 6,
    DGS_BUF_PIX_NDONE = 7,
    DGS_BUF_GRAD2D = 8,
    DGS_BUF_CELL_V = 9,
    DGS_BUF_DECODED = 10
};
dgs_status dgs_state_read(dgs_ctx *ctx, const dgs_fwd_state *state, int32_t what, void *host_dst, int64_t bytes,
                          int64_t *needed);

/* Stable radix sort of (uint32 key, uint32 value) pairs by the low `bits`
 * bits of the key (the sort used for binning, exposed for tests).  All
 * pointers device; keys/vals are overwritten with the sorted sequence.
 * Uses context scratch memory. */
dgs_status dgs_sort_pairs(dgs_ctx *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int32_t bits, dgs_stream stream);

/* ---------------------------------------------------------------- diagnostics */

/* Work counters of a forward state, over all its views (Sec. VII-E defines
 * the termination ratio r_ET = 1 - N_rendered / N_val):
 *   pairs_blended   (pixel, Gaussian) pairs of the cells each pixel blended
 *   inbox_rendered  of those, pairs that passed the AABB test (N_rendered)
 *   inbox_all       pairs passing the AABB test over ALL cells of the pixel's
 *                   tile list, i.e. without early termination (N_val)
 *   cells_blended   (pixel, cell) pairs blended
 * Runs a counting kernel on the state's stream and synchronises it. */
typedef struct {
    int64_t pairs_blended, inbox_rendered, inbox_all, cells_blended;
} dgs_counts;
dgs_status dgs_state_counts(dgs_ctx *ctx, const dgs_fwd_state *state, dgs_counts *out);

/* Per-stage device time.  While enabled, every stage of render and
 * render_backward is bracketed by CUDA events on the stream it runs on (no
 * synchronisation); dgs_profile_read waits for the recorded events and
 * returns the accumulated milliseconds and launch counts per stage since
 * the last enable.  Stages: */
enum {
    DGS_STAGE_CELL_PROJECT = 0, /* a1: cull + footprint of every (view, cell) */
    DGS_STAGE_DEPTH_SORT = 1,   /* a4: radix sort of cells by depth */
    DGS_STAGE_COUNT_SCAN = 2,   /* a2: tile counts in depth order + exclusive scan */
    DGS_STAGE_EMIT = 3,         /* a3: (tile, cell) pairs */
    DGS_STAGE_TILE_SORT = 4,    /* a4: stable radix sort of the pairs by tile */
    DGS_STAGE_TILE_RANGES = 5,  /* a5 */
    DGS_STAGE_PROJECT_FWD = 6,  /* a6: Gaussian projection */
    DGS_STAGE_BLEND_FWD = 7,    /* a7 */
    DGS_STAGE_BLEND_BWD = 8,    /* a8 */
    DGS_STAGE_PROJECT_BWD = 9,  /* a9 */
    DGS_STAGE_DECODE = 10,      /* neural scenes: per-view decode of the visible cells' Gaussians */
    DGS_STAGE_DECODE_BWD = 11,  /* neural scenes: gradients through the decode */
    DGS_STAGE_COUNT = 12
};
typedef struct {
    double ms[16];
    int64_t launches[16];
} dgs_profile;
dgs_status dgs_profile_enable(dgs_ctx *ctx, int32_t on);
dgs_status dgs_profile_read(dgs_ctx *ctx, dgs_profile *out);

/* The radix sort above for callers that cannot allocate device memory: for
 * example a process whose caching allocator already holds the device's free
 * memory for its own pool, or a real-time loop that forbids allocation after
 * start-up because cudaMalloc/cudaFree can block and synchronise the device.
 * The paper has no counterpart; it is a service of this library.
 * Same contract as dgs_sort_pairs (stable, low `bits` bits of the uint32 key,
 * keys/vals device pointers sorted in place, no context needed), except:
 *   * n is at most 1,048,576; a larger n returns DGS_ERR_CAPACITY before any
 *     work is enqueued.
 *   * Scratch is a fixed file-scope device array (about 9.1 MB) that every
 *     GPU loading this library holds until the process exits; this call
 *     calls no cudaMalloc, cudaFree or other allocating routine.
 *   * The first call on a device is part of the caller's set-up: the CUDA
 *     runtime loads the array and the sort's kernels into that device's
 *     context on first use (lazy module loading, CUDA's default), and the
 *     driver allocates their device memory then.  Make one call (n >= 2,
 *     bits >= 1) before reserving the device's free memory or forbidding
 *     allocation; later calls allocate nothing.  Each call looks the array's
 *     address up again (cudaGetSymbolAddress), so a device reset followed by
 *     a new context needs only that set-up call again.
 *   * All calls share the array: calls whose work overlaps on the GPU (other
 *     streams, other threads) race and corrupt each other's results.
 *   * Uses the current CUDA device, enqueues on `stream` and synchronises it
 *     once at the end (to read the sort's error flag), so the call returns
 *     with the sort finished. */
dgs_status dgs_sort_pairs_noalloc(uint32_t *keys, uint32_t *vals, int64_t n, int32_t bits, dgs_stream stream);

/* ------------------------------------------------------------- comparators */

/* The two rendering models Duplex-GS is set against (Sec. III-A), on the same
 * resident scenes and per-Gaussian projection (record, AABB skip, colour,
 * alpha = min(sigma G', alpha_max)) as dgs_render, for the sort-length and
 * speed comparison of Tab. VI:
 *
 *   DGS_COMPARE_ALPHA  vanilla per-Gaussian alpha-blending, Eq. 2-3: every
 *                      (view, Gaussian) is binned to the tiles its AABB box
 *                      reaches and sorted by view depth (ties by index);
 *                      C = sum_i T_i alpha_i c_i + T_final bg with
 *                      T_i = prod_{j<i} (1 - alpha_j); a pixel stops before the
 *                      entry at which T < eps (config eps).
 *   DGS_COMPARE_WSR    sort-free weighted-sum rendering, Eq. 4, with the
 *                      LC-WSR weight of Eq. 5-6, w_i = max(0, 1 - d_i / tau) v_i
 *                      (d_i the view depth of the mean, v_i the v_n of its
 *                      cell; tau <= 0 or non-finite: w_i = v_i):
 *                      C = (bg w_bg + sum_i c_i alpha_i w_i) / (w_bg + sum_i alpha_i w_i),
 *                      the background where that denominator is not above d_min.
 *                      No depth sort, no termination.
 *
 * out_rgb: device, the images back to back as for dgs_render.  out_ndone
 * (nullable, device, int32 [H][W] per view back to back; ALPHA only): the
 * number of tile-list entries each pixel processed.  stats (nullable):
 * sort_length = (tile, Gaussian) pairs, visible_cells = (view, Gaussian)
 * entries kept.  Synchronises the stream once (to size the pair sort).
 * Errors: INVALID_ARG (mode, w_bg < 0, NULL), NOT_FOUND (scene, camera),
 * OOM, CAPACITY (views x Gaussians >= 2^32), TIMEOUT (sort wait gave up). */
#define DGS_COMPARE_ALPHA 1
#define DGS_COMPARE_WSR 2
typedef struct {
    int32_t mode;
    float tau;
    float w_bg;
    int32_t reserved;
} dgs_compare_config;
dgs_status dgs_render_compare(dgs_ctx *ctx, uint32_t scene_id, int32_t n_views, const uint32_t *cam_slots,
                              const dgs_compare_config *cfg, float *out_rgb, int32_t *out_ndone,
                              dgs_stream stream, dgs_stats *stats);

/* -------------------------------------------------------- cell alignment */

/* Cell alignment (Sec. IV-B), in place on the device: for every cell n,
 *   DGS_ALIGN_QUAT    Q_n = norm( sum_k sigma_{n,k} q_{n,k} )          (Eq. 10)
 *   DGS_ALIGN_CENTER  x_n = (1/K) sum_k mu_{n,k}
 * (what = either or both), computed from the values before the call.
 * q_{n,k} is the Gaussian's unit quaternion; quaternions are summed as
 * stored (no hemisphere alignment), and a cell whose weighted sum is the
 * zero vector keeps its Q_n.  Explicit scenes: sigma = sigmoid(logit),
 * mu = the Gaussian's mean; their Gaussians do not move.  Neural scenes:
 * mu = x_n + R(Q_n)(O_pos S_n) (view-independent); sigma and q are decoded
 * for the eye of camera slot cam_slot (required with DGS_ALIGN_QUAT,
 * ignored otherwise), sigma <= 0 weighing 0; their Gaussians move with the
 * cell (the offsets are in the cell's frame).
 * out_center [N][3], out_quat [N][4] (nullable): the new values, in
 * out_location memory (host outputs synchronise the stream, and so does a
 * neural DGS_ALIGN_QUAT, whose decode is checked).  Runs on
 * `stream`; renders of the scene on other streams must be ordered against
 * it by the caller (as for dgs_scene_update).
 * Errors: INVALID_ARG (what, location, camera slot unset for a neural
 * DGS_ALIGN_QUAT), NOT_FOUND (scene), OOM, TIMEOUT (a tensor-core
 * completion wait of the decode gave up). */
#define DGS_ALIGN_QUAT 1
#define DGS_ALIGN_CENTER 2
dgs_status dgs_cell_align(dgs_ctx *ctx, uint32_t scene_id, int32_t what, int32_t cam_slot, float *out_center,
                          float *out_quat, int32_t out_location, dgs_stream stream);

/* ------------------------------------------------------------------ probes */

/* Measured issue rates for the blend kernels' roofline (they are bound by
 * FP32 and SFU instruction issue, not by memory): fp32_tflops from eight
 * independent FMA chains per thread on a full-occupancy grid (2 FLOP per
 * FMA), ex2_per_s from eight independent ex2.approx.f32 chains; ms_* are
 * the timed launches' device times.  Runs on the context's device,
 * synchronises it, takes about 100 ms.  Errors: INVALID_ARG, CUDA, OOM. */
typedef struct {
    double fp32_tflops;
    double ex2_per_s;
    float ms_fma, ms_ex2;
    int32_t sm_count;
    int32_t reserved;
} dgs_alu_peaks;
dgs_status dgs_probe_alu(dgs_ctx *ctx, dgs_alu_peaks *out);

/* ---------------------------------------------------------------- serving */

/* Continuous-batching request loop (not in the paper; serving workload).
 * A request renders one view of a resident scene into out_rgb ([3][H][W],
 * device or host memory per out_location).  Requests that arrive while
 * others run are admitted into the next batch as slots and HBM allow; each
 * batch is one launch chain over views of mixed scenes and resolutions. */
typedef struct {
    uint32_t scene_id;
    int32_t out_location;
    dgs_camera camera;
    float *out_rgb;
} dgs_request;

typedef struct {
    dgs_status status;
    int32_t batch_size;   /* views in the batch this request ran in */
    double t_submit_ms, t_start_ms, t_done_ms; /* host monotonic clock */
} dgs_result;

/* Start the serving worker (max_batch views per launch chain, queue_cap
 * pending requests).  Idempotent.
 *
 * By default every batch is one replay of a captured CUDA graph of the whole
 * forward chain: each of the worker's streams keeps buffers sized for the
 * largest batch seen so far (plus headroom) and one graph per set of scenes
 * in a batch; the batch's views and sizes are copied to the device by the
 * graph's first nodes and every kernel reads its sizes there, so no host
 * synchronisation separates binning from blending.  If the (tile, cell)
 * pairs of a batch exceed the buffers, the kernels stop at the capacity, the
 * worker sees the overflow flag when the batch finishes, grows the buffers,
 * captures again and re-runs the batch before reporting it.  Scenes with
 * neural cells are served like explicit ones (their decode is part of the
 * chain; each composition of neural scenes in a batch has its own graph).
 * flags: DGS_SERVE_NO_GRAPHS runs every batch as a plain launch chain that
 * reads the sort length back to the host midway (for comparison). */
#define DGS_SERVE_NO_GRAPHS 1
dgs_status dgs_serve_start(dgs_ctx *ctx, int32_t max_batch, int32_t queue_cap, int32_t flags);
dgs_status dgs_serve_stop(dgs_ctx *ctx);
dgs_status dgs_submit(dgs_ctx *ctx, const dgs_request *req, uint64_t *ticket);
/* Wait up to timeout_us (0 = just check, <0 = forever) for a ticket.
 * DGS_ERR_TIMEOUT if not done yet; the ticket stays valid.  A finished
 * ticket is consumed by a successful poll; its result's status is the
 * request's own (DGS_OK, or the error of its batch).  If the serving worker
 * stopped after a host-side fault, every request it had not finished is
 * completed with status DGS_ERR_WORKER, so polls return at once (even with
 * timeout_us < 0) and dgs_submit returns DGS_ERR_WORKER until serving is
 * stopped and started again. */
dgs_status dgs_poll(dgs_ctx *ctx, uint64_t ticket, int64_t timeout_us, dgs_result *out);

/* Cancel a submitted request.  Still queued: it leaves the queue and its
 * result (status DGS_ERR_CANCELLED) is ready at once.  Admitted into a batch
 * that is on the GPU: the batch runs on (the request's output may be written),
 * the other requests of the batch are not affected, and the request completes
 * with status DGS_ERR_CANCELLED.  Already finished: nothing changes (the
 * result keeps its own status).  NOT_FOUND for an unknown or consumed ticket;
 * the ticket stays valid until polled. */
dgs_status dgs_cancel(dgs_ctx *ctx, uint64_t ticket);

/* Counters of the serving worker since dgs_serve_start: batches launched
 * (re-runs included), graphs captured, re-runs after a pair-buffer overflow,
 * and the current (tile, cell) pairs-per-tile estimate that sizes the
 * buffers.  INVALID_ARG if serving is not started. */
typedef struct {
    int64_t batches;
    int64_t graphs_captured;
    int64_t overflow_retries;
    double pairs_per_tile;
} dgs_serve_stats;
dgs_status dgs_serve_read_stats(dgs_ctx *ctx, dgs_serve_stats *out);

/* ---------------------------------------------------- debugging and faults */
/* The paper has no counterpart: these calls serve the library's own
 * failure-detection and bounds tests. */

/* Guard words around device buffers (a bounds check that needs no sanitizer).
 * With guards on, every device buffer the library allocates from then on is
 * padded by 256 bytes on each side, filled with the byte 0xA5 (the fill
 * synchronises the device).  dgs_debug_check_guards synchronises every
 * device holding a padded buffer, reads back the guards of every live padded
 * buffer of every context and returns DGS_ERR_GUARD, naming the buffer's
 * size and the first changed offset, if any kernel wrote next to its
 * buffer; *n_checked (nullable) receives the number of buffers checked.
 * Process-wide.  Off by default, unless the environment variable DGS_DEBUG
 * is "1" when the library allocates its first buffer; buffers allocated
 * while guards were off stay unpadded. */
dgs_status dgs_debug_guards(int32_t on);
dgs_status dgs_debug_check_guards(int64_t *n_checked);

/* Fault injection for failure-detection tests.  Nothing here faults, traps
 * or hangs a GPU: a fault is made on the host, or a bounded device wait is
 * made to run out.
 *   DGS_FAULT_ALLOC         the next `count` device allocations of the
 *                           library (any context) fail as if cudaMalloc had
 *                           run out of memory, without calling it: the call
 *                           returns DGS_ERR_OOM and the context stays usable.
 *   DGS_FAULT_SORT_WAIT     while count != 0, radix sorts launched on the
 *                           current device run with their first partition
 *                           withholding its digit counts and a poll limit of
 *                           1024, so the other partitions' look-back waits
 *                           run out: the kernels finish (every write stays
 *                           inside the sorted arrays), the order is
 *                           unspecified and dgs_sort_pairs /
 *                           dgs_sort_pairs_noalloc return DGS_ERR_TIMEOUT.
 *                           count = 0 switches it off.  Meanwhile call only
 *                           those two: a render would consume the order.
 *   DGS_FAULT_SERVE_WORKER  ctx's serving worker raises a host-side exception
 *                           the next time it admits requests; it catches it
 *                           at its top level, waits for its streams,
 *                           completes every open request with DGS_ERR_WORKER
 *                           and exits (see dgs_poll).
 *   DGS_FAULT_GUARD         the next padded device buffer gets one byte of
 *                           its trailing guard overwritten (a host-side
 *                           cudaMemset inside the allocation), so a later
 *                           dgs_debug_check_guards reports it.
 *   DGS_FAULT_TC_WAIT       while count != 0, the tensor-core decode of
 *                           neural cells launched on the current device
 *                           issues no products for its first tile and waits
 *                           about 2^24 clocks for them, so its completion
 *                           wait runs out with nothing in flight: the kernel
 *                           frees its tensor memory and returns, the decode
 *                           results are not valid, and the render's chain
 *                           reports DGS_ERR_TIMEOUT (returned, once it is
 *                           seen complete, by the next call on the context,
 *                           as for a render whose sort gave up).
 * ctx may be NULL except for DGS_FAULT_SERVE_WORKER (serving started). */
enum { DGS_FAULT_ALLOC = 1, DGS_FAULT_SORT_WAIT = 2, DGS_FAULT_SERVE_WORKER = 3, DGS_FAULT_GUARD = 4,
       DGS_FAULT_TC_WAIT = 5 };
dgs_status dgs_debug_inject_fault(dgs_ctx *ctx, int32_t kind, int32_t count);

#ifdef __cplusplus
}
#endif
#endif /* DGS_H */
