// Per-Gaussian projection (the "projected 2D gaussian kernel" G' of Eq. 2)
// for every view of a batch, and its adjoint.
//
// Forward, per Gaussian of a cell that survived culling in that view:
//   t = R mu + t_cam, mu2 = (fx t_x/t_z + cx, fy t_y/t_z + cy)
//   Sigma = R(q) diag(s)^2 R(q)^T, Sigma' = J R Sigma R^T J^T + dilation I
//   (J the pinhole Jacobian at t, t_x/t_z and t_y/t_z clamped to
//   +-1.3 tan(half FOV)), conic = Sigma'^-1, opacity = sigmoid(logit),
//   colour = max(0, 0.5 + sum_lm k_lm Y_lm((mu - eye)/|mu - eye|)).
// mu2 and the AABB half extents k sqrt(Sigma'_xx), k sqrt(Sigma'_yy) are the
// inputs of the per-pixel skip test (Sec. VI-A): they are computed with the
// fixed-order FP32 helpers so the skip decision is reproducible.
//
// One thread per Gaussian reads its parameters once (SoA planes, coalesced)
// and writes one 48-byte record per view, so a batch of views costs one pass
// over the 236 B/Gaussian of parameters.
#include "project.cuh"

namespace dgs {

__device__ __forceinline__ void load_sh(const SceneDev &sc, long long g, float (&k)[16][3]) {
    const int C = (sc.sh_degree + 1) * (sc.sh_degree + 1);
#pragma unroll
    for (int c = 0; c < 16; ++c)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) k[c][ch] = c < C ? sc.sh[(c * 3 + ch) * sc.G + g] : 0.f;
}

// Records of every Gaussian of scene `slot` (grid-stride over its G) for each
// view of that scene in which its cell survived culling.
__device__ __forceinline__ void project_scene(const ViewDesc *__restrict__ views, int n_views, int slot,
                                              const SceneDev &sc, const uint32_t *__restrict__ count,
                                              const float *__restrict__ vview, const BlendParams &bp,
                                              float4 *__restrict__ rec, float *__restrict__ g2d_zero) {
    const long long G = sc.G;
    const int K = sc.K;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long cell = g / K;
        bool any = false;
        for (int v = 0; v < n_views; ++v)
            any |= views[v].scene_slot == slot && count[views[v].cell_base + cell] != 0u;
        if (!any) continue;  // cell culled in every view: nothing reads this Gaussian
        const GaussIn p = load_gauss(sc.gauss, G, g);
        float k[16][3];
        load_sh(sc, g, k);
        const float opac = 1.0f / (1.0f + expf(-p.logit));
        for (int v = 0; v < n_views; ++v) {
            const ViewDesc &Vw = views[v];
            if (Vw.scene_slot != slot || count[Vw.cell_base + cell] == 0u) continue;
            ProjCore c;
            float4 r0, r1, r2;
            gauss_record(Vw, p, k, sc.sh_degree, opac, vview[Vw.cell_base + cell], bp, c, r0, r1, r2);
            float4 *o = rec + (Vw.rec_base + g) * kRecF4;
            o[0] = r0; o[1] = r1; o[2] = r2;
            if (g2d_zero) {
                float4 *z = reinterpret_cast<float4 *>(g2d_zero + (Vw.rec_base + g) * kGradF);
                z[0] = z[1] = z[2] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
}

// Comparator binning (per-Gaussian alpha-blending, Eq. 2-3, and weighted-sum
// rendering, Eq. 4-6): every Gaussian of every view is an entry of its own.
// Per entry e = cell_base + g of view v: the record (r2.w = the weight w_i:
// v_n for alpha-blending, max(0, 1 - z / tau) v_n for LC-WSR, tau <= 0 meaning
// no depth decay), the tiles its FP32 AABB box reaches, its depth key (FP32
// view z; 0xFFFFFFFF when culled) and tile count.  Culled: invalid, box off
// the image, or (weighted sums) w = 0.
__global__ void __launch_bounds__(128) k_gauss_bin(const ViewDesc *__restrict__ views, int n_views, SceneDev sc,
                                                   BlendParams bp, bool wsr, float tau, float4 *__restrict__ rec,
                                                   uint32_t *__restrict__ zkey, uint32_t *__restrict__ zval,
                                                   short4 *__restrict__ rect, uint32_t *__restrict__ count,
                                                   uint32_t *__restrict__ visible) {
    const long long G = sc.G, N = sc.N;
    const int K = sc.K;
    uint32_t nvis = 0;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const GaussIn p = load_gauss(sc.gauss, G, g);
        float k[16][3];
        load_sh(sc, g, k);
        const float opac = 1.0f / (1.0f + expf(-p.logit));
        const float cv = sc.cell[10 * N + g / K];
        for (int v = 0; v < n_views; ++v) {
            const ViewDesc &Vw = views[v];
            ProjCore c;
            float4 r0, r1, r2;
            bool vis = gauss_record(Vw, p, k, sc.sh_degree, opac, cv, bp, c, r0, r1, r2);
            if (wsr) {
                r2.w = tau > 0.f ? fmaxf(0.f, 1.f - c.t[2] / tau) * cv : cv;
                vis = vis && r2.w > 0.f;
            }
            short4 r = make_short4(-1, -1, -1, -1);
            if (vis) {
                const float lox = fsub_s(r0.x, r0.z), hix = fadd_s(r0.x, r0.z);
                const float loy = fsub_s(r0.y, r0.w), hiy = fadd_s(r0.y, r0.w);
                const float fW = (float)Vw.W, fH = (float)Vw.H, ft = (float)kTile;
                vis = hix >= 0.0f && lox < fW && hiy >= 0.0f && loy < fH;
                if (vis) {
                    const int tx0 = (int)floorf(fdiv_s(fmaxf(lox, 0.0f), ft));
                    const int ty0 = (int)floorf(fdiv_s(fmaxf(loy, 0.0f), ft));
                    const int tx1 = min((int)floorf(fdiv_s(fminf(hix, fW), ft)), Vw.Tx - 1);
                    const int ty1 = min((int)floorf(fdiv_s(fminf(hiy, fH), ft)), Vw.Ty - 1);
                    r = make_short4((short)tx0, (short)ty0, (short)tx1, (short)ty1);
                }
            }
            const long long e = Vw.cell_base + g;
            float4 *o = rec + (Vw.rec_base + g) * kRecF4;
            o[0] = r0; o[1] = r1; o[2] = r2;
            rect[e] = r;
            zkey[e] = vis ? __float_as_uint(c.t[2]) : 0xFFFFFFFFu;
            zval[e] = (uint32_t)e;
            count[e] = vis ? (uint32_t)((r.z - r.x + 1) * (r.w - r.y + 1)) : 0u;
            nvis += vis ? 1u : 0u;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nvis += __shfl_xor_sync(0xffffffffu, nvis, o);
    if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(visible, nvis);
}

__global__ void __launch_bounds__(128) k_project_fwd(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                     SceneDev sc, const uint32_t *__restrict__ count,
                                                     const float *__restrict__ vview, BlendParams bp,
                                                     float4 *__restrict__ rec, float *__restrict__ g2d_zero) {
    project_scene(views, n_views, slot, sc, count, vview, bp, rec, g2d_zero);
}

// Every scene of a device scene table in one launch (sizes read at run time).
__global__ void __launch_bounds__(128) k_project_fwd_table(const ViewDesc *__restrict__ views,
                                                           const SceneDev *__restrict__ scenes,
                                                           const uint32_t *__restrict__ count,
                                                           const float *__restrict__ vview, BlendParams bp,
                                                           float4 *__restrict__ rec,
                                                           const ChainSizes *__restrict__ dsz) {
    const int n_views = dsz->n_views, n_scenes = dsz->n_scenes;
    for (int s = 0; s < n_scenes; ++s) {
        const SceneDev sc = scenes[s];
        if (sc.feat) continue;  // neural cells: the decode writes their records
        project_scene(views, n_views, s, sc, count, vview, bp, rec, nullptr);
    }
}

// One thread per cell: sums the views' dL/dv_n and chains it to the SH
// coefficients of a view-dependent v_n (d, Y and the clamp recomputed as in
// the cell projection).
//
// g_center (nullable, accumulated): the cell centre's gradient through the
// direction d = (x_n - eye)/|x_n - eye| of a view-dependent v_n,
//   dL/dx_n += dL/dv_n (I - d d^T) grad_d(sum_lm k_lm Y_lm)(d) / |x_n - eye|.
__global__ void k_cell_v_grad(const ViewDesc *__restrict__ views, int n_views, SceneDev sc,
                              const float *__restrict__ gv, float *__restrict__ g_cell_v, float *__restrict__ g_vsh,
                              float *__restrict__ g_center) {
    const long long N = sc.N;
    const int Cv = sc.vsh ? (sc.v_sh_degree + 1) * (sc.v_sh_degree + 1) : 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        float tot = 0.f, acc[16], gx[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.f;
        for (int v = 0; v < n_views; ++v) {
            const ViewDesc &Vw = views[v];
            const float g = gv[Vw.cell_base + n];
            tot += g;
            if (Cv == 0 || g == 0.f) continue;
            float d0 = sc.cell[n] - Vw.eye[0], d1 = sc.cell[N + n] - Vw.eye[1], d2 = sc.cell[2 * N + n] - Vw.eye[2];
            const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            d0 *= il; d1 *= il; d2 *= il;
            float Y[16];
            sh_eval(d0, d1, d2, sc.v_sh_degree, Y);
            float raw = 0.f;
            for (int c = 0; c < Cv; ++c) raw += sc.vsh[c * N + n] * Y[c];
            if (!(raw > 0.f && raw < 1.f)) continue;  // clamped: no gradient
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] += g * Y[c];
            if (g_center) {
                float k[16], gd[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int c = 0; c < 16; ++c) k[c] = c < Cv ? sc.vsh[c * N + n] : 0.f;
                sh_grad_dot(d0, d1, d2, sc.v_sh_degree, k, gd);
                const float dd = gd[0] * d0 + gd[1] * d1 + gd[2] * d2, s = g * il;
                gx[0] += s * (gd[0] - dd * d0);
                gx[1] += s * (gd[1] - dd * d1);
                gx[2] += s * (gd[2] - dd * d2);
            }
        }
        if (g_cell_v) g_cell_v[n] = tot;
        if (g_vsh)
            for (int c = 0; c < Cv; ++c) g_vsh[n * Cv + c] = acc[c];
        if (g_center)
            for (int j = 0; j < 3; ++j) g_center[3 * n + j] += gx[j];
    }
}

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

void launch_project_fwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                        const float *vview, const BlendParams &bp, float4 *rec, float *g2d_zero, cudaStream_t st) {
    if (sc.G == 0 || n_views == 0) return;
    k_project_fwd<<<grid_for(sc.G, 128), 128, 0, st>>>(views, n_views, slot, sc, count, vview, bp, rec, g2d_zero);
}

void launch_cell_v_grad(const ViewDesc *views, int n_views, const SceneDev &sc, const float *gv, float *g_cell_v,
                        float *g_vsh, float *g_center, cudaStream_t st) {
    if (sc.N == 0 || (!g_cell_v && !g_vsh && !g_center)) return;
    k_cell_v_grad<<<grid_for(sc.N, 128), 128, 0, st>>>(views, n_views, sc, gv, g_cell_v, g_vsh, g_center);
}

void launch_gauss_bin(const ViewDesc *views, int n_views, const SceneDev &sc, const BlendParams &bp, bool wsr,
                      float tau, float4 *rec, uint32_t *zkey, uint32_t *zval, short4 *rect, uint32_t *count,
                      uint32_t *visible, cudaStream_t st) {
    if (sc.G == 0 || n_views == 0) return;
    k_gauss_bin<<<grid_for(sc.G, 128), 128, 0, st>>>(views, n_views, sc, bp, wsr, tau, rec, zkey, zval, rect, count,
                                                     visible);
}

void launch_project_fwd_table(const ViewDesc *views, const SceneDev *scenes, long long G_cap, const uint32_t *count,
                              const float *vview, const BlendParams &bp, float4 *rec, cudaStream_t st,
                              const ChainSizes *dsz) {
    if (G_cap == 0) return;
    k_project_fwd_table<<<grid_for(G_cap, 128), 128, 0, st>>>(views, scenes, count, vview, bp, rec, dsz);
}

// a*b - c*d to about one rounding (Kahan's compensated form)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float cd = c * d;
    const float err = fmaf(-c, d, cd);
    return fmaf(a, b, -cd) + err;
}

// dL/dU (2x3, rows u, w) of a loss depending on Q = (U U^T + d I)^-1 through
// G_Q = dL/dQ = [[ga, gb/2], [gb/2, gc]] (see the comment at the call).
__device__ __forceinline__ void adjoint_U(const float u[3], const float w[3], float d, float ga, float gb, float gc,
                                          float gU[6]) {
    const float x0 = diff_of_products(u[1], w[2], u[2], w[1]);
    const float x1 = diff_of_products(u[2], w[0], u[0], w[2]);
    const float x2 = diff_of_products(u[0], w[1], u[1], w[0]);
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const float uw = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
    const float xx = x0 * x0 + x1 * x1 + x2 * x2;
    const float hd = 0.5f * (uu - ww);
    const float s1sq = 0.5f * (uu + ww) + sqrtf(hd * hd + uw * uw);
    if (!(s1sq > 0.f)) {  // U = 0: dL/dU = -2 Q G_Q Q U = 0
#pragma unroll
        for (int i = 0; i < 6; ++i) gU[i] = 0.f;
        return;
    }
    const float s2sq = xx / s1sq;
    // major eigenvector of [[uu, uw], [uw, ww]]: (s1^2 - ww, uw) or (uw, s1^2 - uu),
    // whichever does not cancel; any unit vector when the eigenvalues coincide
    float p1x, p1y;
    if (uu >= ww) { p1x = s1sq - ww; p1y = uw; } else { p1x = uw; p1y = s1sq - uu; }
    const float pn = p1x * p1x + p1y * p1y;
    if (pn > 0.f) {
        const float ip = rsqrtf(pn);
        p1x *= ip; p1y *= ip;
    } else {
        p1x = 1.f; p1y = 0.f;
    }
    const float p2x = -p1y, p2y = p1x;
    float r1[3], r2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) r1[i] = p1x * u[i] + p1y * w[i];
    const float is1 = 1.0f / s1sq;
    r2[0] = (x1 * r1[2] - x2 * r1[1]) * is1;
    r2[1] = (x2 * r1[0] - x0 * r1[2]) * is1;
    r2[2] = (x0 * r1[1] - x1 * r1[0]) * is1;
    const float g00 = fmaf(ga * p1x, p1x, fmaf(gb * p1x, p1y, gc * p1y * p1y));
    const float g11 = fmaf(ga * p2x, p2x, fmaf(gb * p2x, p2y, gc * p2y * p2y));
    const float g01 = fmaf(ga * p1x, p2x, fmaf(0.5f * gb, fmaf(p1x, p2y, p1y * p2x), gc * p1y * p2y));
    const float il1 = 1.0f / (s1sq + d), il2 = 1.0f / (s2sq + d);
    const float n00 = g00 * il1 * il1, n01 = g01 * il1 * il2, n11 = g11 * il2 * il2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float y0 = fmaf(n00, r1[i], n01 * r2[i]);
        const float y1 = fmaf(n01, r1[i], n11 * r2[i]);
        gU[i] = -2.0f * fmaf(p1x, y0, p2x * y1);
        gU[3 + i] = -2.0f * fmaf(p1y, y0, p2y * y1);
    }
}

// ---------------------------------------------------------------- adjoint
// Input per (view, Gaussian): dL/d(mu2 x, y), dL/d(conic a, b, c) with
// q = a dx^2 + 2 b dx dy + c dy^2, dL/d(opacity), dL/d(rgb).  Chain rule
// through the forward above (clamp masks as in the forward), summed over
// views; outputs are written, not accumulated.
// Geometry adjoint of one (view, Gaussian): from dL/d(mu2) (gmx, gmy) and
// dL/d(conic a, b, c) to dL/d(mean, linear scale, quaternion), accumulated
// into gm, gs, gq.  False if the Gaussian's mean is not in front of the near
// plane (never drawn).
__device__ __forceinline__ bool view_geom_adjoint(const ViewDesc &Vw, const GaussIn &p, const BlendParams &bp,
                                                  float gmx, float gmy, float gca, float gcb, float gcc, float gm[3],
                                                  float gs[3], float gq[4]) {
    ProjCore c;
    proj_core(Vw, p, bp.dilation, c);
    if (!c.valid) return false;
    // conic -> Sigma' -> U:  dL/dU = 2 H U with H = -Q G_Q Q,
    // G_Q = [[ga, gb/2], [gb/2, gc]], Q = Sigma'^-1, Sigma' = U U^T + d I.
    // Needle-like Gaussians make U nearly rank one, so Q is nearly
    // singular and Q G_Q Q U cancels heavily in the pixel frame.  In
    // the eigenframe P of U U^T (eigenvalues s1^2 >= s2^2) it does
    // not: with R = P^T U (rows r1 = p1^T U and r2 = x × r1 / s1^2,
    // x = u × w, an exact identity free of cancellation) and
    // lambda_i = s_i^2 + d,  dL/dU = -2 P N R,  N_ij = (P^T G_Q P)_ij / (lambda_i lambda_j).
    const ScreenCov sc2 = screen_cov(c, bp.dilation);
    float gU[6];
    adjoint_U(sc2.u, sc2.w, bp.dilation, gca, gcb, gcc, gU);
    // Sigma' = U U^T + d I, U = T M:  dL/dT = dL/dU M^T,  dL/dM = T^T dL/dU
    float gT[6];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            gT[3 * a + j] = gU[3 * a] * c.M[3 * j] + gU[3 * a + 1] * c.M[3 * j + 1] + gU[3 * a + 2] * c.M[3 * j + 2];
    float gMm[9];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) gMm[3 * j + k] = c.T[j] * gU[k] + c.T[3 + j] * gU[3 + k];
    // T = J R_view
    const float gJ00 = gT[0] * Vw.R[0] + gT[1] * Vw.R[1] + gT[2] * Vw.R[2];
    const float gJ02 = gT[0] * Vw.R[6] + gT[1] * Vw.R[7] + gT[2] * Vw.R[8];
    const float gJ11 = gT[3] * Vw.R[3] + gT[4] * Vw.R[4] + gT[5] * Vw.R[5];
    const float gJ12 = gT[3] * Vw.R[6] + gT[4] * Vw.R[7] + gT[5] * Vw.R[8];
    const float tz = c.t[2], itz = 1.0f / tz, itz2 = itz * itz;
    float gt[3] = {0.f, 0.f, 0.f};
    gt[2] += -gJ00 * Vw.fx * itz2 - gJ11 * Vw.fy * itz2;
    const float limx = 1.3f * (0.5f * (float)Vw.W / Vw.fx), limy = 1.3f * (0.5f * (float)Vw.H / Vw.fy);
    if (c.x >= -limx && c.x <= limx) {  // J02 = -fx t_x / t_z^2
        gt[0] += -gJ02 * Vw.fx * itz2;
        gt[2] += gJ02 * 2.0f * Vw.fx * c.t[0] * itz2 * itz;
    } else {                              // J02 = -fx xc / t_z
        gt[2] += gJ02 * Vw.fx * c.xc * itz2;
    }
    if (c.y >= -limy && c.y <= limy) {
        gt[1] += -gJ12 * Vw.fy * itz2;
        gt[2] += gJ12 * 2.0f * Vw.fy * c.t[1] * itz2 * itz;
    } else {
        gt[2] += gJ12 * Vw.fy * c.yc * itz2;
    }
    // projected mean
    gt[0] += gmx * Vw.fx * itz;
    gt[1] += gmy * Vw.fy * itz;
    gt[2] += -(gmx * Vw.fx * c.t[0] + gmy * Vw.fy * c.t[1]) * itz2;
    // t = R mu + t_cam
#pragma unroll
    for (int j = 0; j < 3; ++j) gm[j] += Vw.R[j] * gt[0] + Vw.R[3 + j] * gt[1] + Vw.R[6 + j] * gt[2];
    // M = R(q) diag(s)
    float gR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gs[j] += gMm[3 * i + j] * c.Rg[3 * i + j];
            gR[3 * i + j] = gMm[3 * i + j] * p.scale[j];
        }
    // R(q_hat), then q_hat = q / |q|
    rot_quat_adjoint(p.quat, gR, gq);
    return true;
}

// The views among [v0, v0 + 32) of the chain (bit u: view v0 + u) in which
// cell `cell` of scene `slot` survived culling.  The counts of all of them are
// requested before any is used.
__device__ __forceinline__ unsigned visible_views(const ViewDesc *__restrict__ views, int n_views, int v0, int slot,
                                                  const uint32_t *__restrict__ count, long long cell) {
    unsigned m = 0u;
    const int n = min(32, n_views - v0);
#pragma unroll 8
    for (int u = 0; u < n; ++u) {
        const ViewDesc &Vw = views[v0 + u];
        if (Vw.scene_slot == slot && count[Vw.cell_base + cell] != 0u) m |= 1u << u;
    }
    return m;
}

__global__ void __launch_bounds__(128) k_project_bwd_geom(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                     SceneDev sc, const uint32_t *__restrict__ count, BlendParams bp,
                                                     const float *__restrict__ g2d, float *__restrict__ g_mean,
                                                     float *__restrict__ g_scale,
                                                     float *__restrict__ g_log_scale, float *__restrict__ g_quat,
                                                     float *__restrict__ g_logit) {
    const long long G = sc.G;
    const int K = sc.K;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long cell = g / K;
        float gm[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f};
        float gq[4] = {0.f, 0.f, 0.f, 0.f}, glog = 0.f;
        GaussIn p;
        float opac = 0.f;
        bool loaded = false;
        for (int v0 = 0; v0 < n_views; v0 += 32) {
            unsigned m = visible_views(views, n_views, v0, slot, count, cell);
            if (!m) continue;
            if (!loaded) {
                p = load_gauss(sc.gauss, G, g);
                opac = 1.0f / (1.0f + expf(-p.logit));
                loaded = true;
            }
            // the next visible view's screen-space gradient is requested
            // before the current one is processed
            auto fetch = [&](int v, float4 &a0, float4 &a1) {
                const float4 *gr = reinterpret_cast<const float4 *>(g2d + (views[v].rec_base + g) * kGradF);
                a0 = gr[0];
                a1 = gr[1];
            };
            int v = v0 + __ffs(m) - 1;
            m &= m - 1;
            float4 a0, a1;
            fetch(v, a0, a1);
            for (;;) {
                const int vn = m ? v0 + __ffs(m) - 1 : -1;
                float4 b0 = a0, b1 = a1;
                if (vn >= 0) {
                    m &= m - 1;
                    fetch(vn, b0, b1);
                }
                const float gmx = a0.x, gmy = a0.y, gca = a0.z, gcb = a0.w, gcc = a1.x, gop = a1.y;
                if (gmx != 0.f || gmy != 0.f || gca != 0.f || gcb != 0.f || gcc != 0.f || gop != 0.f) {
                    const ViewDesc &Vw = views[v];
                    ProjCore c;
                    proj_core(Vw, p, bp.dilation, c);
                    if (c.valid) {
                        glog += gop * opac * (1.0f - opac);  // opacity
                        view_geom_adjoint(Vw, p, bp, gmx, gmy, gca, gcb, gcc, gm, gs, gq);
                    }
                }
                if (vn < 0) break;
                v = vn;
                a0 = b0;
                a1 = b1;
            }
        }
        if (loaded) {
            // d/d log s = s d/ds
#pragma unroll
            for (int j = 0; j < 3; ++j) gls[j] = gs[j] * p.scale[j];
        }
        if (g_mean) { g_mean[3 * g] = gm[0]; g_mean[3 * g + 1] = gm[1]; g_mean[3 * g + 2] = gm[2]; }
        if (g_scale) { g_scale[3 * g] = gs[0]; g_scale[3 * g + 1] = gs[1]; g_scale[3 * g + 2] = gs[2]; }
        if (g_log_scale) { g_log_scale[3 * g] = gls[0]; g_log_scale[3 * g + 1] = gls[1]; g_log_scale[3 * g + 2] = gls[2]; }
        if (g_quat) {
#pragma unroll
            for (int i = 0; i < 4; ++i) g_quat[4 * g + i] = gq[i];
        }
        if (g_logit) g_logit[g] = glog;
    }
}

// Adjoint of a neural scene's records with respect to the decoded values
// of every (view, Gaussian) whose cell was decoded in that view: gdec rows
// in the layout of dec (mean 3, scale 3, quaternion 4, opacity 1, rgb 3).
// The colour enters the record as decoded, so its gradient passes through;
// a Gaussian with sigma <= 0 was not drawn and gets zeros.
__global__ void __launch_bounds__(128) k_project_bwd_neural(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                            SceneDev sc, const uint32_t *__restrict__ count,
                                                            BlendParams bp, const float *__restrict__ dec,
                                                            const float *__restrict__ g2d, float *__restrict__ gdec) {
    const long long G = sc.G;
    const int K = sc.K;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long cell = g / K;
        for (int v = 0; v < n_views; ++v) {
            const ViewDesc &Vw = views[v];
            if (Vw.scene_slot != slot || count[Vw.cell_base + cell] == 0u) continue;
            const long long row = Vw.rec_base + g;
            const float *d = dec + row * kDecF;
            const float4 *gr = reinterpret_cast<const float4 *>(g2d + row * kGradF);
            const float4 a0 = gr[0], a1 = gr[1], a2 = gr[2];
            float o[kDecF];
#pragma unroll
            for (int i = 0; i < kDecF; ++i) o[i] = 0.f;
            if (d[10] > 0.f && (a0.x != 0.f || a0.y != 0.f || a0.z != 0.f || a0.w != 0.f || a1.x != 0.f ||
                                a1.y != 0.f || a1.z != 0.f || a1.w != 0.f || a2.x != 0.f)) {
                GaussIn p;
#pragma unroll
                for (int i = 0; i < 3; ++i) { p.mean[i] = d[i]; p.scale[i] = d[3 + i]; }
#pragma unroll
                for (int i = 0; i < 4; ++i) p.quat[i] = d[6 + i];
                p.logit = 0.f;
                if (view_geom_adjoint(Vw, p, bp, a0.x, a0.y, a0.z, a0.w, a1.x, o, o + 3, o + 6)) {
                    o[10] = a1.y;
                    o[11] = a1.z; o[12] = a1.w; o[13] = a2.x;
                }
            }
            float2 *dst = reinterpret_cast<float2 *>(gdec + row * kDecF);
#pragma unroll
            for (int i = 0; i < kDecF / 2; ++i) dst[i] = make_float2(o[2 * i], o[2 * i + 1]);
        }
    }
}

// Colour adjoint: colour_ch = max(0, 0.5 + sum_c k_c,ch Y_c(d)),
// d = (mu - eye)/|mu - eye|: dL/dk and the view direction's share of
// dL/dmu (added to g_mean, which the geometry kernel wrote).  Views outer:
// per view one SH basis Y(d) and, the direction gradient being linear in the
// weights, one sh_grad_dot with w_c = sum over unclamped channels of
// dL/dcolour_ch k_c,ch.  The 48 coefficients stay in registers; dL/dk
// accumulates in shared memory, transposed (column t of the block's thread t,
// stride 129: conflict-free both when accumulating and when the rows leave
// coalesced).  Gaussians that no view rendered (and invalid ones) have zero
// screen-space gradients.
constexpr int COL_T = 128, COL_LD = COL_T + 1;
__global__ void __launch_bounds__(COL_T) k_project_bwd_colour(const ViewDesc *__restrict__ views, int n_views, int slot,
                                                              SceneDev sc, const uint32_t *__restrict__ count,
                                                              const float *__restrict__ g2d, float *__restrict__ g_mean,
                                                              float *__restrict__ g_sh) {
    __shared__ float s_acc[48 * COL_LD];  // dL/dk[c * 3 + ch] of thread t at [c * 3 + ch][t]
    const long long G = sc.G;
    const int K = sc.K, C = (sc.sh_degree + 1) * (sc.sh_degree + 1), row = 3 * C;
    const int t = threadIdx.x;
    for (long long g0 = (long long)blockIdx.x * COL_T; g0 < G; g0 += (long long)gridDim.x * COL_T) {
        const long long g = g0 + t;
        const bool live = g < G;
        const long long cell = live ? g / K : 0;
        for (int j = 0; j < row; ++j) s_acc[j * COL_LD + t] = 0.f;
        float k[16][3];
#pragma unroll
        for (int c = 0; c < 16; ++c)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) k[c][ch] = live && c < C ? sc.sh[(c * 3 + ch) * G + g] : 0.f;
        const float m0 = live ? sc.gauss[g] : 0.f, m1 = live ? sc.gauss[G + g] : 0.f,
                    m2 = live ? sc.gauss[2 * G + g] : 0.f;
        float gdm[3] = {0.f, 0.f, 0.f};
        // visible views in order, the next one's colour gradient requested
        // before the current one is processed
        int v0 = 0;
        unsigned m = 0u;
        auto next_view = [&]() -> int {
            while (live && !m && v0 < n_views) {
                m = visible_views(views, n_views, v0, slot, count, cell);
                if (!m) v0 += 32;
            }
            if (!m) return -1;
            const int v = v0 + __ffs(m) - 1;
            m &= m - 1;
            if (!m) v0 += 32;
            return v;
        };
        auto fetch = [&](int v, float gc[3]) {
            const float *gr = g2d + (views[v].rec_base + g) * kGradF + 6;
            gc[0] = gr[0];
            gc[1] = gr[1];
            gc[2] = gr[2];
        };
        float gn[3] = {0.f, 0.f, 0.f};
        int vn = next_view();
        if (vn >= 0) fetch(vn, gn);
        while (vn >= 0) {
            const int v = vn;
            const float gc[3] = {gn[0], gn[1], gn[2]};
            vn = next_view();
            if (vn >= 0) fetch(vn, gn);
            const ViewDesc &Vw = views[v];
            if (gc[0] == 0.f && gc[1] == 0.f && gc[2] == 0.f) continue;
            const float u0 = m0 - Vw.eye[0], u1 = m1 - Vw.eye[1], u2 = m2 - Vw.eye[2];
            const float il = rsqrtf(u0 * u0 + u1 * u1 + u2 * u2);
            const float d0 = u0 * il, d1 = u1 * il, d2 = u2 * il;
            float Y[16];
            sh_eval(d0, d1, d2, sc.sh_degree, Y);
            float w[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) w[c] = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float sv = 0.5f;
#pragma unroll
                for (int c = 0; c < 16; ++c) sv += k[c][ch] * Y[c];
                if (sv <= 0.0f || gc[ch] == 0.f) continue;  // clamped at 0, or no gradient
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (c < C) s_acc[(c * 3 + ch) * COL_LD + t] += gc[ch] * Y[c];
                    w[c] += gc[ch] * k[c][ch];
                }
            }
            if (g_mean) {
                float gd[3] = {0.f, 0.f, 0.f};
                sh_grad_dot(d0, d1, d2, sc.sh_degree, w, gd);
                const float dd = gd[0] * d0 + gd[1] * d1 + gd[2] * d2;
                gdm[0] += (gd[0] - dd * d0) * il;
                gdm[1] += (gd[1] - dd * d1) * il;
                gdm[2] += (gd[2] - dd * d2) * il;
            }
        }
        __syncthreads();
        if (g_sh) {
            const long long nb = min((long long)COL_T, G - g0) * row;
            float *dst = g_sh + g0 * row;
            for (int i = t; i < nb; i += COL_T) {
                const int gl = i / row, j = i - gl * row;
                dst[i] = s_acc[j * COL_LD + gl];
            }
        }
        __syncthreads();
        if (live && g_mean) {
            g_mean[3 * g] += gdm[0];
            g_mean[3 * g + 1] += gdm[1];
            g_mean[3 * g + 2] += gdm[2];
        }
    }
}

void launch_project_bwd_neural(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                               const BlendParams &bp, const float *dec, const float *g2d, float *gdec,
                               cudaStream_t st) {
    if (sc.G == 0) return;
    k_project_bwd_neural<<<grid_for(sc.G, 128), 128, 0, st>>>(views, n_views, slot, sc, count, bp, dec, g2d, gdec);
}

void launch_project_bwd(const ViewDesc *views, int n_views, int slot, const SceneDev &sc, const uint32_t *count,
                        const BlendParams &bp, const float *g2d, float *g_mean, float *g_scale, float *g_log_scale,
                        float *g_quat, float *g_logit, float *g_sh, cudaStream_t st) {
    if (sc.G == 0) return;
    k_project_bwd_geom<<<grid_for(sc.G, 128), 128, 0, st>>>(views, n_views, slot, sc, count, bp, g2d, g_mean,
                                                            g_scale, g_log_scale, g_quat, g_logit);
    if (g_mean || g_sh)
        k_project_bwd_colour<<<grid_for(sc.G, 128), 128, 0, st>>>(views, n_views, slot, sc, count, g2d, g_mean, g_sh);
}

}  // namespace dgs
