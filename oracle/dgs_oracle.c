/*
 * CPU oracle for the Duplex-GS hybrid renderer -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline leg use this
 * file.  It shares no code with the CUDA path.  It is written to be checked
 * by eye against the paper, not to be fast:
 *
 *   or_cell_rects      cell-proxy projection and tile footprint (Sec. IV-B)
 *   or_tile_lists      tile binning + ordering of (tile, cell depth) keys by a
 *                      comparison sort (Sec. IV-B; the radix sort's result)
 *   or_gauss_decisions FP32 inputs of the per-Gaussian AABB skip (Sec. VI-A)
 *   or_blend           hybrid renderer, Eq. 12-14, cell-level early
 *                      termination (Sec. V-B), AABB false-positive skip
 *   or_blend_grad      adjoint of or_blend (plain reverse mode), FP64
 *   or_gauss_rects     per-Gaussian tile footprint and depth (comparators)
 *   or_alpha_blend     per-Gaussian depth-ordered alpha-blending, Eq. 2-3
 *   or_wsr             weighted-sum rendering, Eq. 4 with the LC-WSR weight
 *                      of Eq. 5-6 supplied per Gaussian
 *
 * Discrete decisions (cull, tile rectangle, per-Gaussian AABB test) are taken
 * in FP32 with one prescribed operation order (no FMA contraction: build with
 * -ffp-contract=off), because the CUDA path takes them in FP32 too and the
 * same rounding must give the same integer result.  Everything that is a
 * value (alpha, colour, transmittance, sums, gradients) is FP64.
 *
 * Camera array (float[22]): W H fx fy cx cy znear R[9] (world->view,
 * row-major) t[3] eye[3].  View space: x right, y down, +z forward.
 * Pixel (i,j) is sampled at (i+0.5, j+0.5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* FP32 with one prescribed order: every operation below is a single IEEE   */
/* rounding in float (the file is compiled without contraction).            */

static void f32_rot_from_quat(const float q[4], float R[9]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float n = sqrtf(((w * w + x * x) + y * y) + z * z);
    w = w / n; x = x / n; y = y / n; z = z / n;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
}

/* v = R p + t, each row summed left to right */
static void f32_xform(const float R[9], const float t[3], const float p[3], float v[3]) {
    for (int i = 0; i < 3; ++i)
        v[i] = ((R[3 * i] * p[0] + R[3 * i + 1] * p[1]) + R[3 * i + 2] * p[2]) + t[i];
}

/*
 * Screen footprint of one ellipsoidal cell {c + R_Q diag(S) u : |u| <= 1}
 * (Sec. IV-A: "each cell defines a bounded visible region"; Sec. IV-B: only
 * cells intersecting the frustum are kept and assigned to tiles).
 *
 * The paper does not say how the region is bounded on screen.  Reading: the
 * exact bounding box of the perspective image of the ellipsoid.  With the
 * view-space centre c and Sigma = M M^T, M = R_view R_Q diag(S), a plane
 * X - t Z = 0 touches the ellipsoid where
 *     (c_z^2 - S_zz) t^2 - 2 (c_x c_z - S_xz) t + (c_x^2 - S_xx) = 0 ,
 * so t = (b -+ sqrt(disc)) / a with a = c_z^2 - S_zz, b = c_x c_z - S_xz and
 * disc = b^2 - a (c_x^2 - S_xx) expanded so the c_x^2 c_z^2 terms cancel
 * exactly:  disc = c_z^2 S_xx - 2 c_x c_z S_xz + c_x^2 S_zz - (S_xx S_zz - S_xz^2).
 * Pixel bound u = fx t + cx; the same for y.  A cell whose ellipsoid reaches
 * the near plane (c_z - sqrt(S_zz) <= znear) or whose box misses the image
 * is culled.  Tiles [floor(lo/tile), floor(hi/tile)] clamped to the grid.
 * Variant (flags & 16, the renderer's DGS_FLAG_NEAR_FULL): a cell that
 * reaches the near plane without lying wholly behind it (c_z + sqrt(S_zz) >
 * znear) is kept with every tile of the image, sort depth max(c_z, 0).
 *
 * rect[4n..4n+3] = tx0 ty0 tx1 ty1 (inclusive), tx0 = -1 when culled.
 * depth[n] = view-space z of the cell centre (the sort depth).
 * bounds (nullable) = lo_x hi_x lo_y hi_y in pixels, NaN when culled by the
 * near plane.
 */
void or_cell_rects(int64_t N, const float *center, const float *axes, const float *quat,
                   const float *cam, int tile, int flags, int32_t *rect, float *depth, float *bounds) {
    const int W = (int)cam[0], H = (int)cam[1];
    const float fx = cam[2], fy = cam[3], ppx = cam[4], ppy = cam[5], znear = cam[6];
    const float *Rv = cam + 7, *tv = cam + 16;
    const int Tx = (W + tile - 1) / tile, Ty = (H + tile - 1) / tile;
    const float ftile = (float)tile;
    for (int64_t n = 0; n < N; ++n) {
        float c[3], Rq[9], RR[9], M[9];
        f32_xform(Rv, tv, center + 3 * n, c);
        f32_rot_from_quat(quat + 4 * n, Rq);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                RR[3 * i + j] = (Rv[3 * i] * Rq[j] + Rv[3 * i + 1] * Rq[3 + j]) + Rv[3 * i + 2] * Rq[6 + j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[3 * i + j] = RR[3 * i + j] * axes[3 * n + j];
#define SIG(a, b) ((M[3 * (a)] * M[3 * (b)] + M[3 * (a) + 1] * M[3 * (b) + 1]) + M[3 * (a) + 2] * M[3 * (b) + 2])
        const float sxx = SIG(0, 0), syy = SIG(1, 1), szz = SIG(2, 2), sxz = SIG(0, 2), syz = SIG(1, 2);
#undef SIG
        depth[n] = c[2];
        rect[4 * n] = rect[4 * n + 1] = rect[4 * n + 2] = rect[4 * n + 3] = -1;
        if (bounds) bounds[4 * n] = bounds[4 * n + 1] = bounds[4 * n + 2] = bounds[4 * n + 3] = NAN;
        if (!((c[2] - sqrtf(szz)) > znear)) {
            if ((flags & 16) && (c[2] + sqrtf(szz)) > znear) {  /* straddles the near plane: every tile */
                depth[n] = c[2] > 0.0f ? c[2] : 0.0f;
                rect[4 * n] = 0; rect[4 * n + 1] = 0; rect[4 * n + 2] = Tx - 1; rect[4 * n + 3] = Ty - 1;
            }
            continue;
        }
        const float czz = c[2] * c[2];
        const float a = czz - szz;
        float lo[2], hi[2];
        for (int ax = 0; ax < 2; ++ax) {
            const float cu = c[ax];
            const float suu = ax == 0 ? sxx : syy, suz = ax == 0 ? sxz : syz;
            const float f = ax == 0 ? fx : fy, pp = ax == 0 ? ppx : ppy;
            const float cuz = cu * c[2], cuu = cu * cu;
            const float b = cuz - suz;
            float disc = ((czz * suu - (2.0f * cuz) * suz) + cuu * szz) - (suu * szz - suz * suz);
            disc = fmaxf(disc, 0.0f);
            const float sq = sqrtf(disc);
            lo[ax] = f * ((b - sq) / a) + pp;
            hi[ax] = f * ((b + sq) / a) + pp;
            if (bounds) { bounds[4 * n + 2 * ax] = lo[ax]; bounds[4 * n + 2 * ax + 1] = hi[ax]; }
        }
        if (!(hi[0] >= 0.0f && lo[0] < (float)W && hi[1] >= 0.0f && lo[1] < (float)H)) continue;
        int tx0 = (int)floorf(fmaxf(lo[0], 0.0f) / ftile);
        int ty0 = (int)floorf(fmaxf(lo[1], 0.0f) / ftile);
        int tx1 = (int)floorf(fminf(hi[0], (float)W) / ftile);
        int ty1 = (int)floorf(fminf(hi[1], (float)H) / ftile);
        if (tx1 > Tx - 1) tx1 = Tx - 1;
        if (ty1 > Ty - 1) ty1 = Ty - 1;
        rect[4 * n] = tx0; rect[4 * n + 1] = ty0; rect[4 * n + 2] = tx1; rect[4 * n + 3] = ty1;
    }
}

/* ------------------------------------------------------------------------ */
/* Tile binning by definition: every (tile, cell) pair whose rectangle      */
/* covers the tile, ordered by (tile, depth, cell index) with a comparison  */
/* sort.  The cell index as last key is the tie rule (equal depths keep     */
/* cell order), which is what a stable radix sort of cell-major emission    */
/* gives.  Sec. IV-B: the radix sort runs over the cell sequence only.      */

typedef struct { int32_t tile; float depth; int32_t cell; } or_entry;

static int or_entry_cmp(const void *pa, const void *pb) {
    const or_entry *a = (const or_entry *)pa, *b = (const or_entry *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    return 0;
}

/* Returns L (number of entries).  If L > cap nothing is written and -L is
 * returned.  range[2t], range[2t+1] = [start, end) of tile t in out_cell. */
int64_t or_tile_lists(int64_t N, const int32_t *rect, const float *depth, int Tx, int Ty,
                      int32_t *out_cell, int64_t cap, int64_t *range) {
    int64_t L = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (rect[4 * n] < 0) continue;
        L += (int64_t)(rect[4 * n + 2] - rect[4 * n] + 1) * (rect[4 * n + 3] - rect[4 * n + 1] + 1);
    }
    if (L > cap) return -L;
    or_entry *e = (or_entry *)malloc(sizeof(or_entry) * (size_t)(L > 0 ? L : 1));
    int64_t i = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (rect[4 * n] < 0) continue;
        for (int ty = rect[4 * n + 1]; ty <= rect[4 * n + 3]; ++ty)
            for (int tx = rect[4 * n]; tx <= rect[4 * n + 2]; ++tx) {
                e[i].tile = ty * Tx + tx; e[i].depth = depth[n]; e[i].cell = (int32_t)n; ++i;
            }
    }
    qsort(e, (size_t)L, sizeof(or_entry), or_entry_cmp);
    for (int64_t t = 0; t < (int64_t)Tx * Ty; ++t) { range[2 * t] = 0; range[2 * t + 1] = 0; }
    for (int64_t j = 0; j < L; ++j) {
        out_cell[j] = e[j].cell;
        const int32_t t = e[j].tile;
        if (j == 0 || e[j - 1].tile != t) range[2 * t] = j;
        range[2 * t + 1] = j + 1;
    }
    free(e);
    return L;
}

/*
 * FP32 inputs of the per-pixel AABB test (Sec. VI-A "pixel-level radius
 * based culling ... AABB check").  The paper gives no radius; reading: a
 * per-axis box of k standard deviations of the projected 2D Gaussian,
 * |x' - mu_x| <= k sqrt(S'_xx) and |y' - mu_y| <= k sqrt(S'_yy), with
 * S' = J W Sigma W^T J^T + dilation I the EWA screen covariance and
 * Sigma = R(q) diag(s)^2 R(q)^T.  J is evaluated at the view-space mean with
 * x/z and y/z clamped to +-1.3 tan(half FOV).  A Gaussian whose mean is not
 * in front of the near plane is invalid (never drawn).
 *
 * Outputs (per Gaussian): mu2[2g..], ext[2g..] (half extents), valid[g].
 */
void or_gauss_decisions(int64_t G, const float *mean, const float *scale, const float *quat,
                        const float *cam, float dilation, float ksigma, int square,
                        float *mu2, float *ext, uint8_t *valid) {
    const float W = cam[0], H = cam[1];
    const float fx = cam[2], fy = cam[3], ppx = cam[4], ppy = cam[5], znear = cam[6];
    const float *Rv = cam + 7, *tv = cam + 16;
    const float limx = 1.3f * ((0.5f * W) / fx);
    const float limy = 1.3f * ((0.5f * H) / fy);
    for (int64_t g = 0; g < G; ++g) {
        float t[3];
        f32_xform(Rv, tv, mean + 3 * g, t);
        if (!(t[2] > znear)) {
            valid[g] = 0; mu2[2 * g] = mu2[2 * g + 1] = 0.0f; ext[2 * g] = ext[2 * g + 1] = -1.0f;
            continue;
        }
        valid[g] = 1;
        const float x = t[0] / t[2], y = t[1] / t[2];
        mu2[2 * g] = fx * x + ppx;
        mu2[2 * g + 1] = fy * y + ppy;
        float Rg[9], M[9], S[9];
        f32_rot_from_quat(quat + 4 * g, Rg);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[3 * i + j] = Rg[3 * i + j] * scale[3 * g + j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                S[3 * i + j] = (M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1]) + M[3 * i + 2] * M[3 * j + 2];
        const float xc = fminf(fmaxf(x, -limx), limx);
        const float yc = fminf(fmaxf(y, -limy), limy);
        const float j00 = fx / t[2], j02 = -((fx * xc) / t[2]);
        const float j11 = fy / t[2], j12 = -((fy * yc) / t[2]);
        float T[6], V[6];
        for (int j = 0; j < 3; ++j) {
            T[j] = j00 * Rv[j] + j02 * Rv[6 + j];
            T[3 + j] = j11 * Rv[3 + j] + j12 * Rv[6 + j];
        }
        for (int a = 0; a < 2; ++a)
            for (int j = 0; j < 3; ++j)
                V[3 * a + j] = (T[3 * a] * S[j] + T[3 * a + 1] * S[3 + j]) + T[3 * a + 2] * S[6 + j];
        const float sxx = ((V[0] * T[0] + V[1] * T[1]) + V[2] * T[2]) + dilation;
        const float syy = ((V[3] * T[3] + V[4] * T[4]) + V[5] * T[5]) + dilation;
        if (square) {
            /* the 3DGS square box: radius ceil(k sqrt(lambda_max)) of Sigma' in both axes,
             * lambda_max = (sxx + syy)/2 + sqrt(((sxx - syy)/2)^2 + sxy^2) */
            const float sxy = (V[0] * T[3] + V[1] * T[4]) + V[2] * T[5];
            const float mid = 0.5f * (sxx + syy), hd = 0.5f * (sxx - syy);
            const float lam = mid + sqrtf(hd * hd + sxy * sxy);
            const float r = ceilf(ksigma * sqrtf(lam));
            ext[2 * g] = r;
            ext[2 * g + 1] = r;
        } else {
            ext[2 * g] = ksigma * sqrtf(sxx);
            ext[2 * g + 1] = ksigma * sqrtf(syy);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Hybrid renderer (Eq. 12-14) in FP64.                                     */

typedef struct {
    int W, H, tile, K;
    const int64_t *range;     /* 2 per tile */
    const int32_t *cells;     /* sorted cell list */
    const double *mu2;        /* 2G  FP64 projected means */
    const double *conic;      /* 3G  inverse screen covariance (a, b, c): q = a dx^2 + 2 b dx dy + c dy^2 */
    const double *opac;       /* G   sigma in [0,1] */
    const double *rgb;        /* 3G  colour */
    const float *mu2f;        /* 2G  FP32 decision inputs */
    const float *extf;        /* 2G */
    const uint8_t *valid;     /* G */
    const double *cell_v;     /* N   calibration scalar v_n */
    double eps, alpha_max, d_min, bg[3], delta;
    double w_bg;              /* background weight of Eq. 4 in the hybrid's normalisation (0: none) */
    int alpha_skip;           /* alpha < 1/255 contributes nothing (the 3DGS skip) */
    int term_exclude;         /* a cell that would take T below eps is not blended (3DGS rule) */
    int out_numerator;        /* output the numerator N of Eq. 12, not N / D */
} or_scene_view;

/* option bits of opts[8] (the same values as the renderer's config flags) */
enum { OR_ALPHA_SKIP = 1, OR_TERM_EXCLUDE = 2, OR_AABB_SQUARE = 4, OR_NUMERATOR = 8 };

static void or_unpack(or_scene_view *s, int W, int H, int tile, int K, const int64_t *range,
                      const int32_t *cells, const double *mu2, const double *conic, const double *opac,
                      const double *rgb, const float *mu2f, const float *extf, const uint8_t *valid,
                      const double *cell_v, const double *opts) {
    s->W = W; s->H = H; s->tile = tile; s->K = K; s->range = range; s->cells = cells;
    s->mu2 = mu2; s->conic = conic; s->opac = opac; s->rgb = rgb; s->mu2f = mu2f; s->extf = extf;
    s->valid = valid; s->cell_v = cell_v;
    s->eps = opts[0]; s->alpha_max = opts[1]; s->d_min = opts[2];
    s->bg[0] = opts[3]; s->bg[1] = opts[4]; s->bg[2] = opts[5]; s->delta = opts[6];
    s->w_bg = opts[7];
    const int flags = (int)opts[8];
    s->alpha_skip = (flags & OR_ALPHA_SKIP) != 0;
    s->term_exclude = (flags & OR_TERM_EXCLUDE) != 0;
    s->out_numerator = (flags & OR_NUMERATOR) != 0;
}

/* The comparators take the hybrid renderer's shared settings only: its
 * blending options (alpha skip, termination variant, background weight,
 * numerator output) are the hybrid's own. */
static void or_comparator_opts(or_scene_view *s) {
    s->alpha_skip = 0; s->term_exclude = 0; s->out_numerator = 0; s->w_bg = 0.0;
}

/* alpha of Gaussian g at pixel centre (px, py); 0 when the AABB test fails
 * (Sec. VI-A).  alpha = min(sigma G'(x'), alpha_max) (Eq. 2 with the paper's
 * alpha in [0,1], Sec. V-A).  Also returns G' and whether the clamp was active. */
static double or_alpha(const or_scene_view *s, int64_t g, float pxf, float pyf, double *Gout, int *clamped,
                       double *dxo, double *dyo) {
    *Gout = 0.0; *clamped = 0; *dxo = 0.0; *dyo = 0.0;
    if (!s->valid[g]) return 0.0;
    if (fabsf(pxf - s->mu2f[2 * g]) > s->extf[2 * g]) return 0.0;
    if (fabsf(pyf - s->mu2f[2 * g + 1]) > s->extf[2 * g + 1]) return 0.0;
    const double dx = (double)pxf - s->mu2[2 * g], dy = (double)pyf - s->mu2[2 * g + 1];
    const double a = s->conic[3 * g], b = s->conic[3 * g + 1], c = s->conic[3 * g + 2];
    const double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
    const double G = exp(-0.5 * q);
    double al = s->opac[g] * G;
    if (s->alpha_skip && al < 1.0 / 255.0) return 0.0; /* skipped like a failed AABB test */
    *Gout = G; *dxo = dx; *dyo = dy;
    if (al >= s->alpha_max) { al = s->alpha_max; *clamped = 1; }
    return al;
}

/* A, B and P of cell entry n at pixel centre (pxf, pyf) (Eq. 12-14). */
static void or_cell(const or_scene_view *s, int64_t beg, int n, float pxf, float pyf, double A[3], double *B,
                    double *P) {
    const int32_t cell = s->cells[beg + n];
    const double v = s->cell_v[cell];
    A[0] = A[1] = A[2] = 0.0; *B = 0.0; *P = 1.0;
    for (int k = 0; k < s->K; ++k) {
        const int64_t g = (int64_t)cell * s->K + k;
        double G, dx, dy; int cl;
        const double al = or_alpha(s, g, pxf, pyf, &G, &cl, &dx, &dy);
        A[0] += al * s->rgb[3 * g]; A[1] += al * s->rgb[3 * g + 1]; A[2] += al * s->rgb[3 * g + 2];
        *B += al;
        *P *= (1.0 - v * al);
    }
}

/* One pixel, Eq. 12-14.  Walk the tile's cells front to back.  With
 * count < 0 the paper's rule decides where to stop: before cell n, stop if
 * T_n < eps (Sec. V-B: blending halts once T^cell falls below eps, so the
 * cell that took T below eps is still blended); with term_exclude, a cell
 * whose blending would take T below eps is not blended and ends the pixel
 * (the 3DGS rule).  With count >= 0 exactly min(count, len) cells are
 * processed instead (used to check a given choice).  Returns the number of
 * cells processed; fills N (3), D, T (after the last processed cell), Tlast
 * (T_n before the last processed cell, 1 if none) and Tpeek (T times the P of
 * the first unprocessed cell; T if none). */
static int or_pixel(const or_scene_view *s, int64_t beg, int64_t end, int x, int y, int count,
                    double N[3], double *Dout, double *Tout, double *Tlast, double *Tpeek) {
    const float pxf = (float)x + 0.5f, pyf = (float)y + 0.5f;
    const int len = (int)(end - beg);
    double T = 1.0, D = 0.0;
    N[0] = N[1] = N[2] = 0.0;
    *Tlast = 1.0;
    *Tpeek = 1.0;
    int n = 0;
    for (; n < len; ++n) {
        if (count < 0 && T < s->eps) break;
        if (count >= 0 && n >= count) break;
        double A[3], B, P;
        or_cell(s, beg, n, pxf, pyf, A, &B, &P);
        if (count < 0 && s->term_exclude && T * P < s->eps) break;
        const double v = s->cell_v[s->cells[beg + n]];
        /* w_n = v_n T_n (Eq. 13); numerator and denominator of Eq. 12 */
        N[0] += v * T * A[0]; N[1] += v * T * A[1]; N[2] += v * T * A[2];
        D += v * T * B;
        *Tlast = T;
        T *= P; /* Eq. 14 */
    }
    *Tpeek = T;
    if (n < len) {
        double A[3], B, P;
        or_cell(s, beg, n, pxf, pyf, A, &B, &P);
        *Tpeek = T * P;
    }
    *Dout = D; *Tout = T;
    return n;
}

/* Is processing exactly `count` cells a valid outcome of the stopping rule
 * when transmittance is only known to relative accuracy delta?  The paper's
 * rule: every processed cell had T_n >= eps (1 - delta), and unless the list
 * ran out, the next T is < eps (1 + delta).  With term_exclude: T after every
 * processed cell is >= eps (1 - delta), and unless the list ran out, blending
 * the next cell would take T below eps (1 + delta). */
static int or_count_ok(const or_scene_view *s, int len, int count, double Tlast, double Tafter, double Tpeek) {
    if (count < 0 || count > len) return 0;
    if (s->term_exclude) {
        if (count > 0 && Tafter < s->eps * (1.0 - s->delta)) return 0;
        if (count < len && !(Tpeek < s->eps * (1.0 + s->delta))) return 0;
        return 1;
    }
    if (count > 0 && Tlast < s->eps * (1.0 - s->delta)) return 0;
    if (count < len && !(Tafter < s->eps * (1.0 + s->delta))) return 0;
    return 1;
}

/* Output colour of a pixel from N and D: N / D (Eq. 12); with a background
 * weight, (N + w_bg bg) / (D + w_bg) (Eq. 4's background term); the
 * background where that denominator is not above d_min; N itself with
 * out_numerator.  Returns the denominator used (0 with out_numerator). */
static double or_colour(const or_scene_view *s, const double N[3], double D, double C[3]) {
    if (s->out_numerator) {
        C[0] = N[0]; C[1] = N[1]; C[2] = N[2];
        return 0.0;
    }
    const double Dp = D + s->w_bg;
    for (int c = 0; c < 3; ++c) C[c] = Dp > s->d_min ? (N[c] + s->w_bg * s->bg[c]) / Dp : s->bg[c];
    return Dp;
}

/*
 * Render tile rows [ty0, ty1) of one view.  Outputs are [3][H][W] planar
 * (out_C, out_N) and [H][W] (out_D, out_T, out_ndone); pixels outside the
 * window are left untouched.  C = N / D if D > d_min else background
 * (Eq. 12 has no background term; a pixel that no Gaussian reaches keeps
 * the background colour).  forced_ndone (nullable): render with those
 * counts instead of the oracle's own and count the invalid ones (returned).
 * opts: eps alpha_max d_min bg_r bg_g bg_b delta w_bg flags.
 */
int64_t or_blend(int W, int H, int tile, int K, const int64_t *range, const int32_t *cells,
                 const double *mu2, const double *conic, const double *opac, const double *rgb,
                 const float *mu2f, const float *extf, const uint8_t *valid, const double *cell_v,
                 const double *opts, const int32_t *forced_ndone, int ty0, int ty1,
                 double *out_C, double *out_N, double *out_D, double *out_T, int32_t *out_ndone) {
    or_scene_view s;
    or_unpack(&s, W, H, tile, K, range, cells, mu2, conic, opac, rgb, mu2f, extf, valid, cell_v, opts);
    const int Tx = (W + tile - 1) / tile;
    const int64_t HW = (int64_t)H * W;
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int64_t tid = (int64_t)ty0 * Tx; tid < (int64_t)ty1 * Tx; ++tid) {
        const int tx = (int)(tid % Tx), ty = (int)(tid / Tx);
        const int64_t beg = range[2 * tid], end = range[2 * tid + 1];
        for (int y = ty * tile; y < (ty + 1) * tile && y < H; ++y)
            for (int x = tx * tile; x < (tx + 1) * tile && x < W; ++x) {
                const int64_t p = (int64_t)y * W + x;
                double N[3], D, T, Tl, Tp, C[3];
                const int own = or_pixel(&s, beg, end, x, y, -1, N, &D, &T, &Tl, &Tp);
                if (forced_ndone) {
                    const int cnt = forced_ndone[p];
                    or_pixel(&s, beg, end, x, y, cnt < 0 ? 0 : cnt, N, &D, &T, &Tl, &Tp);
                    if (!or_count_ok(&s, (int)(end - beg), cnt, Tl, T, Tp)) bad += 1;
                }
                or_colour(&s, N, D, C);
                for (int c = 0; c < 3; ++c) {
                    out_C[c * HW + p] = C[c];
                    if (out_N) out_N[c * HW + p] = N[c];
                }
                out_D[p] = D; out_T[p] = T; out_ndone[p] = own;
            }
    }
    return bad;
}

/*
 * Adjoint of or_blend, plain reverse mode per pixel, FP64.  Given dL/dC
 * ([3][H][W]) it accumulates, per Gaussian, dL/d(mu2) (2), dL/d(conic a,b,c)
 * (3), dL/d(sigma) (1), dL/d(rgb) (3), and per cell dL/dv_n.  Decisions (AABB
 * skip, alpha clamp, termination) are held fixed.  ndone (nullable) fixes the
 * processed-cell count per pixel, else the oracle's own is used.
 *
 * With C = N/D:  dL/dN = g/D,  dL/dD = -(g.C)/D (with a background weight
 * D + w_bg in place of D; with out_numerator dL/dN = g, dL/dD = 0).  For cell n with
 * A_n = sum_k alpha c, B_n = sum_k alpha, P_n = prod_k (1 - v alpha):
 *   direct        dL/dT_n  = v_n (dN.A_n + dD B_n)
 *   T_m = prod_{i<m} P_i, so for i < m   dT_m/dalpha_{ik} = -v_i T_m / (1 - v_i alpha_{ik})
 *   dL/dalpha_{ik} = v_i T_i (dN.c_{ik} + dD) - v_i R_i / (1 - v_i alpha_{ik}),
 *                    R_i = sum_{m>i} dL/dT_m T_m   (suffix sum over processed cells)
 *   dL/dc_{ik}     = v_i T_i alpha_{ik} dN
 *   dL/dv_i        = T_i (dN.A_i + dD B_i) - R_i sum_k alpha_{ik} / (1 - v_i alpha_{ik})
 * then alpha = sigma G (unclamped) and G = exp(-q/2) chain to sigma, mu2, conic.
 */
void or_blend_grad(int W, int H, int tile, int K, const int64_t *range, const int32_t *cells,
                   const double *mu2, const double *conic, const double *opac, const double *rgb,
                   const float *mu2f, const float *extf, const uint8_t *valid, const double *cell_v,
                   const double *opts, const int32_t *ndone, const double *dL_dC, int ty0, int ty1,
                   double *g_mu2, double *g_conic, double *g_opac, double *g_rgb, double *g_v) {
    or_scene_view s;
    or_unpack(&s, W, H, tile, K, range, cells, mu2, conic, opac, rgb, mu2f, extf, valid, cell_v, opts);
    const int Tx = (W + tile - 1) / tile;
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t tid = (int64_t)ty0 * Tx; tid < (int64_t)ty1 * Tx; ++tid) {
        const int tx = (int)(tid % Tx), ty = (int)(tid / Tx);
        const int64_t beg = range[2 * tid], end = range[2 * tid + 1];
        const int len = (int)(end - beg);
        double *Tn = (double *)malloc(sizeof(double) * (size_t)(len + 1));
        double *An = (double *)malloc(sizeof(double) * 3 * (size_t)(len + 1));
        double *Bn = (double *)malloc(sizeof(double) * (size_t)(len + 1));
        double *dTn = (double *)malloc(sizeof(double) * (size_t)(len + 1));
        for (int y = ty * tile; y < (ty + 1) * tile && y < H; ++y)
            for (int x = tx * tile; x < (tx + 1) * tile && x < W; ++x) {
                const int64_t p = (int64_t)y * W + x;
                const float pxf = (float)x + 0.5f, pyf = (float)y + 0.5f;
                double Nv[3], D, Tfin, Tl, Tp, C[3];
                const int nd = or_pixel(&s, beg, end, x, y, ndone ? (ndone[p] < 0 ? 0 : ndone[p]) : -1,
                                        Nv, &D, &Tfin, &Tl, &Tp);
                const double Dp = or_colour(&s, Nv, D, C);
                if (!s.out_numerator && !(Dp > s.d_min)) continue; /* background: constant output */
                const double g[3] = {dL_dC[p], dL_dC[HW + p], dL_dC[2 * HW + p]};
                const double iD = s.out_numerator ? 1.0 : 1.0 / Dp;
                const double dN[3] = {g[0] * iD, g[1] * iD, g[2] * iD};
                const double dD = s.out_numerator ? 0.0 : -(g[0] * C[0] + g[1] * C[1] + g[2] * C[2]) * iD;
                /* forward again, storing the per-cell quantities */
                double T = 1.0;
                for (int n = 0; n < nd; ++n) {
                    const int32_t cell = s.cells[beg + n];
                    const double v = s.cell_v[cell];
                    double A[3] = {0, 0, 0}, B = 0.0, P = 1.0;
                    for (int k = 0; k < K; ++k) {
                        const int64_t gi = (int64_t)cell * K + k;
                        double G, dx, dy; int cl;
                        const double al = or_alpha(&s, gi, pxf, pyf, &G, &cl, &dx, &dy);
                        A[0] += al * s.rgb[3 * gi]; A[1] += al * s.rgb[3 * gi + 1]; A[2] += al * s.rgb[3 * gi + 2];
                        B += al;
                        P *= (1.0 - v * al);
                    }
                    Tn[n] = T; An[3 * n] = A[0]; An[3 * n + 1] = A[1]; An[3 * n + 2] = A[2]; Bn[n] = B;
                    dTn[n] = v * (dN[0] * A[0] + dN[1] * A[1] + dN[2] * A[2] + dD * B);
                    T *= P;
                }
                /* suffix sums R_i = sum_{m>i} dL/dT_m T_m, walked back to front */
                double R = 0.0;
                for (int n = nd - 1; n >= 0; --n) {
                    const int32_t cell = s.cells[beg + n];
                    const double v = s.cell_v[cell];
                    double gv = Tn[n] * (dN[0] * An[3 * n] + dN[1] * An[3 * n + 1] + dN[2] * An[3 * n + 2] + dD * Bn[n]);
                    for (int k = 0; k < K; ++k) {
                        const int64_t gi = (int64_t)cell * K + k;
                        double G, dx, dy; int cl;
                        const double al = or_alpha(&s, gi, pxf, pyf, &G, &cl, &dx, &dy);
                        if (G == 0.0 && al == 0.0) continue; /* skipped by the AABB test */
                        const double dcdot = dN[0] * s.rgb[3 * gi] + dN[1] * s.rgb[3 * gi + 1] + dN[2] * s.rgb[3 * gi + 2];
                        const double om = 1.0 - v * al;
                        const double dal = v * Tn[n] * (dcdot + dD) - v * R / om;
                        /* dL/dv through P_n: dP_n/dv = sum_k -alpha_k prod_{k' != k}(...) */
                        gv += -R * al / om;
                        for (int c = 0; c < 3; ++c) {
#pragma omp atomic
                            g_rgb[3 * gi + c] += v * Tn[n] * al * dN[c];
                        }
                        if (!cl) {
                            const double dG = dal * s.opac[gi];
#pragma omp atomic
                            g_opac[gi] += dal * G;
                            const double dq = -0.5 * G * dG;
                            const double a = s.conic[3 * gi], b = s.conic[3 * gi + 1], cc = s.conic[3 * gi + 2];
#pragma omp atomic
                            g_mu2[2 * gi] += dq * (-(2.0 * a * dx + 2.0 * b * dy));
#pragma omp atomic
                            g_mu2[2 * gi + 1] += dq * (-(2.0 * b * dx + 2.0 * cc * dy));
#pragma omp atomic
                            g_conic[3 * gi] += dq * dx * dx;
#pragma omp atomic
                            g_conic[3 * gi + 1] += dq * 2.0 * dx * dy;
#pragma omp atomic
                            g_conic[3 * gi + 2] += dq * dy * dy;
                        }
                    }
                    if (g_v) {
#pragma omp atomic
                        g_v[cell] += gv;
                    }
                    R += dTn[n] * Tn[n];
                }
            }
        free(Tn); free(An); free(Bn); free(dTn);
    }
}

/* ------------------------------------------------------------------------ */
/* Comparators.  The two rendering models the paper sets Duplex-GS against  */
/* (Sec. III-A): vanilla per-Gaussian alpha-blending over a global depth    */
/* sort (Eq. 2-3), and sort-free weighted-sum rendering (Eq. 4) with the    */
/* LC-WSR weight w_i = max(0, 1 - d_i / tau) v_i (Eq. 5-6).  Both use the   */
/* same per-Gaussian alpha = min(sigma G', alpha_max), AABB skip and colour */
/* as the hybrid renderer above; only the blending differs.                 */

/*
 * Per Gaussian of one view: the tiles its FP32 AABB box reaches and its
 * depth.  lo = mu - ext, hi = mu + ext per axis (FP32), culled (rect = -1)
 * when the Gaussian is invalid or the box misses the image; otherwise tiles
 * [floor(max(lo, 0) / tile), floor(min(hi, size) / tile)] clamped to the
 * grid.  depth = FP32 view-space z of the mean (the sort key of Eq. 3's
 * order, and d_i of Eq. 6).
 */
void or_gauss_rects(int64_t G, const float *mean, const float *mu2f, const float *extf, const uint8_t *valid,
                    const float *cam, int tile, int32_t *rect, float *depth) {
    const int W = (int)cam[0], H = (int)cam[1];
    const float *Rv = cam + 7, *tv = cam + 16;
    const int Tx = (W + tile - 1) / tile, Ty = (H + tile - 1) / tile;
    const float ftile = (float)tile;
    for (int64_t g = 0; g < G; ++g) {
        float t[3];
        f32_xform(Rv, tv, mean + 3 * g, t);
        depth[g] = t[2];
        rect[4 * g] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = -1;
        if (!valid[g]) continue;
        const float lox = mu2f[2 * g] - extf[2 * g], hix = mu2f[2 * g] + extf[2 * g];
        const float loy = mu2f[2 * g + 1] - extf[2 * g + 1], hiy = mu2f[2 * g + 1] + extf[2 * g + 1];
        if (!(hix >= 0.0f && lox < (float)W && hiy >= 0.0f && loy < (float)H)) continue;
        int tx0 = (int)floorf(fmaxf(lox, 0.0f) / ftile);
        int ty0 = (int)floorf(fmaxf(loy, 0.0f) / ftile);
        int tx1 = (int)floorf(fminf(hix, (float)W) / ftile);
        int ty1 = (int)floorf(fminf(hiy, (float)H) / ftile);
        if (tx1 > Tx - 1) tx1 = Tx - 1;
        if (ty1 > Ty - 1) ty1 = Ty - 1;
        rect[4 * g] = tx0; rect[4 * g + 1] = ty0; rect[4 * g + 2] = tx1; rect[4 * g + 3] = ty1;
    }
}

/* One pixel of Eq. 2-3: walk the tile's Gaussians front to back,
 * C += T alpha c, T *= (1 - alpha).  Stopping rule as in the hybrid renderer
 * at K = 1 (before entry i, stop if T_i < eps); count >= 0 forces the number
 * of processed entries.  Returns the count; fills C, T (after), Tlast. */
static int or_alpha_pixel(const or_scene_view *s, int64_t beg, int64_t end, int x, int y, int count,
                          double C[3], double *Tout, double *Tlast) {
    const float pxf = (float)x + 0.5f, pyf = (float)y + 0.5f;
    const int len = (int)(end - beg);
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    *Tlast = 1.0;
    int n = 0;
    for (; n < len; ++n) {
        if (count < 0 && T < s->eps) break;
        if (count >= 0 && n >= count) break;
        const int64_t g = s->cells[beg + n];
        double G, dx, dy; int cl;
        const double al = or_alpha(s, g, pxf, pyf, &G, &cl, &dx, &dy);
        C[0] += T * al * s->rgb[3 * g]; C[1] += T * al * s->rgb[3 * g + 1]; C[2] += T * al * s->rgb[3 * g + 2];
        *Tlast = T;
        T *= (1.0 - al);
    }
    *Tout = T;
    return n;
}

/*
 * Per-Gaussian alpha-blending of tile rows [ty0, ty1) of one view; `list`
 * and `range` are the tile lists of Gaussians ordered by (tile, depth,
 * index).  out_C [3][H][W] = sum_i T_i alpha_i c_i + T_final bg (the 3DGS
 * background convention); out_T, out_ndone [H][W].  forced_ndone as in
 * or_blend (returns the number of invalid forced counts).
 * opts: as for or_blend (the hybrid-only options are ignored).
 */
int64_t or_alpha_blend(int W, int H, int tile, const int64_t *range, const int32_t *list,
                       const double *mu2, const double *conic, const double *opac, const double *rgb,
                       const float *mu2f, const float *extf, const uint8_t *valid, const double *opts,
                       const int32_t *forced_ndone, int ty0, int ty1, double *out_C, double *out_T,
                       int32_t *out_ndone) {
    or_scene_view s;
    or_unpack(&s, W, H, tile, 1, range, list, mu2, conic, opac, rgb, mu2f, extf, valid, NULL, opts);
    or_comparator_opts(&s);
    const int Tx = (W + tile - 1) / tile;
    const int64_t HW = (int64_t)H * W;
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int64_t tid = (int64_t)ty0 * Tx; tid < (int64_t)ty1 * Tx; ++tid) {
        const int tx = (int)(tid % Tx), ty = (int)(tid / Tx);
        const int64_t beg = range[2 * tid], end = range[2 * tid + 1];
        for (int y = ty * tile; y < (ty + 1) * tile && y < H; ++y)
            for (int x = tx * tile; x < (tx + 1) * tile && x < W; ++x) {
                const int64_t p = (int64_t)y * W + x;
                double C[3], T, Tl;
                const int own = or_alpha_pixel(&s, beg, end, x, y, -1, C, &T, &Tl);
                if (forced_ndone) {
                    const int cnt = forced_ndone[p];
                    or_alpha_pixel(&s, beg, end, x, y, cnt < 0 ? 0 : cnt, C, &T, &Tl);
                    if (!or_count_ok(&s, (int)(end - beg), cnt, Tl, T, T)) bad += 1;
                }
                for (int c = 0; c < 3; ++c) out_C[c * HW + p] = C[c] + T * s.bg[c];
                out_T[p] = T; out_ndone[p] = own;
            }
    }
    return bad;
}

/*
 * Weighted-sum rendering (Eq. 4) of tile rows [ty0, ty1) of one view over
 * the Gaussians of each tile's list (any order: the sums commute):
 *   C = (c_B w_B + sum_i c_i alpha_i w_i) / (w_B + sum_i alpha_i w_i),
 * with w_i given per Gaussian (Eq. 5-6: max(0, 1 - d_i / tau) v_i) and the
 * background weight w_bg; a pixel whose denominator is not above d_min
 * shows the background.  No transmittance, no termination.
 */
void or_wsr(int W, int H, int tile, const int64_t *range, const int32_t *list, const double *mu2,
            const double *conic, const double *opac, const double *rgb, const float *mu2f, const float *extf,
            const uint8_t *valid, const double *w, double w_bg, const double *opts, int ty0, int ty1,
            double *out_C) {
    or_scene_view s;
    or_unpack(&s, W, H, tile, 1, range, list, mu2, conic, opac, rgb, mu2f, extf, valid, NULL, opts);
    or_comparator_opts(&s);
    const int Tx = (W + tile - 1) / tile;
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t tid = (int64_t)ty0 * Tx; tid < (int64_t)ty1 * Tx; ++tid) {
        const int tx = (int)(tid % Tx), ty = (int)(tid / Tx);
        const int64_t beg = range[2 * tid], end = range[2 * tid + 1];
        for (int y = ty * tile; y < (ty + 1) * tile && y < H; ++y)
            for (int x = tx * tile; x < (tx + 1) * tile && x < W; ++x) {
                const int64_t p = (int64_t)y * W + x;
                const float pxf = (float)x + 0.5f, pyf = (float)y + 0.5f;
                double A[3] = {0, 0, 0}, B = 0.0;
                for (int64_t e = beg; e < end; ++e) {
                    const int64_t g = list[e];
                    double G, dx, dy; int cl;
                    const double aw = or_alpha(&s, g, pxf, pyf, &G, &cl, &dx, &dy) * w[g];
                    A[0] += aw * rgb[3 * g]; A[1] += aw * rgb[3 * g + 1]; A[2] += aw * rgb[3 * g + 2];
                    B += aw;
                }
                const double den = w_bg + B;
                for (int c = 0; c < 3; ++c)
                    out_C[c * HW + p] = den > s.d_min ? (s.bg[c] * w_bg + A[c]) / den : s.bg[c];
            }
    }
}
