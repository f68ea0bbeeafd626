// Per-Gaussian projection helpers shared by the projection kernels and the
// neural-cell decode (which forms the records of the Gaussians it decodes):
// the Gaussian's parameters, the fixed-order FP32 projection core (view-space
// mean, pinhole Jacobian, 3D and screen covariance) and the 48-byte record.
#pragma once
#include "internal.cuh"
#include "sh.cuh"

namespace dgs {

constexpr float KAPPA = 0.8493218002880191f;  // sqrt(log2(e) / 2), log2(e) = 1/ln 2



struct GaussIn {
    float mean[3], scale[3], quat[4], logit;
};

__device__ __forceinline__ GaussIn load_gauss(const float *__restrict__ gp, long long G, long long g) {
    GaussIn p;
#pragma unroll
    for (int i = 0; i < 3; ++i) p.mean[i] = gp[i * G + g];
#pragma unroll
    for (int i = 0; i < 3; ++i) p.scale[i] = gp[(3 + i) * G + g];
#pragma unroll
    for (int i = 0; i < 4; ++i) p.quat[i] = gp[(6 + i) * G + g];
    p.logit = gp[10 * G + g];
    return p;
}

// Fixed-order FP32 part shared by forward and backward: view-space mean,
// J, T = J R_view, 3D covariance, and the diagonal of Sigma'.
struct ProjCore {
    float t[3], x, y, xc, yc, J00, J02, J11, J12, T[6], Rg[9], M[9], S[9], V[6], sxx, syy;
    bool valid;
};

// Screen covariance without cancellation: with U = T M (2x3, rows u and w),
// Sigma' = U U^T + dilation I, so s_xx = |u|^2 + d, s_yy = |w|^2 + d, s_xy = u.w
// and det = |u x w|^2 + d (|u|^2 + |w|^2) + d^2 (Lagrange's identity), a sum of
// non-negative terms.  (The fixed-order s_xx, s_yy of ProjCore serve only the
// AABB extents.)
struct ScreenCov {
    float u[3], w[3], sxx, syy, sxy, det;
};

__device__ __forceinline__ ScreenCov screen_cov(const ProjCore &c, float dilation) {
    ScreenCov q;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        q.u[j] = c.T[0] * c.M[j] + c.T[1] * c.M[3 + j] + c.T[2] * c.M[6 + j];
        q.w[j] = c.T[3] * c.M[j] + c.T[4] * c.M[3 + j] + c.T[5] * c.M[6 + j];
    }
    const float uu = q.u[0] * q.u[0] + q.u[1] * q.u[1] + q.u[2] * q.u[2];
    const float ww = q.w[0] * q.w[0] + q.w[1] * q.w[1] + q.w[2] * q.w[2];
    q.sxy = q.u[0] * q.w[0] + q.u[1] * q.w[1] + q.u[2] * q.w[2];
    const float x0 = q.u[1] * q.w[2] - q.u[2] * q.w[1];
    const float x1 = q.u[2] * q.w[0] - q.u[0] * q.w[2];
    const float x2 = q.u[0] * q.w[1] - q.u[1] * q.w[0];
    q.sxx = uu + dilation;
    q.syy = ww + dilation;
    q.det = (x0 * x0 + x1 * x1 + x2 * x2) + dilation * (uu + ww) + dilation * dilation;
    return q;
}

__device__ __forceinline__ void proj_core(const ViewDesc &Vw, const GaussIn &p, float dilation, ProjCore &c) {
    xform_s(Vw.R, Vw.t, p.mean[0], p.mean[1], p.mean[2], c.t);
    c.valid = c.t[2] > Vw.znear;
    if (!c.valid) return;
    c.x = fdiv_s(c.t[0], c.t[2]);
    c.y = fdiv_s(c.t[1], c.t[2]);
    rot_from_quat_s(p.quat[0], p.quat[1], p.quat[2], p.quat[3], c.Rg);
    float *M = c.M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = fmul_s(c.Rg[3 * i + j], p.scale[j]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.S[3 * i + j] = fadd_s(fadd_s(fmul_s(M[3 * i], M[3 * j]), fmul_s(M[3 * i + 1], M[3 * j + 1])),
                                    fmul_s(M[3 * i + 2], M[3 * j + 2]));
    const float limx = fmul_s(1.3f, fdiv_s(fmul_s(0.5f, (float)Vw.W), Vw.fx));
    const float limy = fmul_s(1.3f, fdiv_s(fmul_s(0.5f, (float)Vw.H), Vw.fy));
    c.xc = fminf(fmaxf(c.x, -limx), limx);
    c.yc = fminf(fmaxf(c.y, -limy), limy);
    c.J00 = fdiv_s(Vw.fx, c.t[2]);
    c.J02 = -fdiv_s(fmul_s(Vw.fx, c.xc), c.t[2]);
    c.J11 = fdiv_s(Vw.fy, c.t[2]);
    c.J12 = -fdiv_s(fmul_s(Vw.fy, c.yc), c.t[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        c.T[j] = fadd_s(fmul_s(c.J00, Vw.R[j]), fmul_s(c.J02, Vw.R[6 + j]));
        c.T[3 + j] = fadd_s(fmul_s(c.J11, Vw.R[3 + j]), fmul_s(c.J12, Vw.R[6 + j]));
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.V[3 * a + j] = fadd_s(fadd_s(fmul_s(c.T[3 * a], c.S[j]), fmul_s(c.T[3 * a + 1], c.S[3 + j])),
                                    fmul_s(c.T[3 * a + 2], c.S[6 + j]));
    c.sxx = fadd_s(fadd_s(fadd_s(fmul_s(c.V[0], c.T[0]), fmul_s(c.V[1], c.T[1])), fmul_s(c.V[2], c.T[2])), dilation);
    c.syy = fadd_s(fadd_s(fadd_s(fmul_s(c.V[3], c.T[3]), fmul_s(c.V[4], c.T[4])), fmul_s(c.V[5], c.T[5])), dilation);
}

// The 48-byte record of Gaussian p in view Vw (an invalid Gaussian, mean not
// in front of the near plane, gets ext = -1 so no AABB test passes).  k: SH
// coefficients, cv: the cell's v_n.  Returns c.valid; c keeps the view-space mean.
template <bool DIRECT_RGB = false>
__device__ __forceinline__ bool gauss_record(const ViewDesc &Vw, const GaussIn &p, const float (&k)[16][3],
                                             int sh_degree, float opac, float cv, const BlendParams &bp,
                                             ProjCore &c, float4 &r0, float4 &r1, float4 &r2,
                                             const float *rgb = nullptr) {
    proj_core(Vw, p, bp.dilation, c);
    if (!c.valid) {
        r0 = make_float4(0.f, 0.f, -1.f, -1.f);
        r1 = make_float4(0.f, 0.f, 0.f, 0.f);
        r2 = make_float4(0.f, 0.f, 0.f, cv);
        return false;
    }
    const float mx = fadd_s(fmul_s(Vw.fx, c.x), Vw.cx);
    const float my = fadd_s(fmul_s(Vw.fy, c.y), Vw.cy);
    float ex, ey;
    if (bp.flags & DGS_FLAG_AABB_SQUARE) {
        // the square of radius ceil(k sqrt(lambda_max(Sigma'))),
        // lambda_max = (sxx + syy)/2 + sqrt(((sxx - syy)/2)^2 + sxy^2), fixed order
        const float sxy = fadd_s(fadd_s(fmul_s(c.V[0], c.T[3]), fmul_s(c.V[1], c.T[4])), fmul_s(c.V[2], c.T[5]));
        const float mid = fmul_s(0.5f, fadd_s(c.sxx, c.syy)), hd = fmul_s(0.5f, fadd_s(c.sxx, -c.syy));
        const float lam = fadd_s(mid, fsqrt_s(fadd_s(fmul_s(hd, hd), fmul_s(sxy, sxy))));
        ex = ey = ceilf(fmul_s(bp.ksigma, fsqrt_s(lam)));
    } else {
        ex = fmul_s(bp.ksigma, fsqrt_s(c.sxx));
        ey = fmul_s(bp.ksigma, fsqrt_s(c.syy));
    }
    // conic Q = Sigma'^-1 = L L^T, L = [[p, 0], [r, t]]:
    // p = sqrt(s_yy/det), r = -s_xy/sqrt(s_yy det), t = 1/sqrt(s_yy),
    // so q(d) = (p dx + r dy)^2 + (t dy)^2 is a sum of squares
    const ScreenCov sc2 = screen_cov(c, bp.dilation);
    const float ip = rsqrtf(sc2.syy * sc2.det);
    const float fp = sc2.syy * ip, fr = -sc2.sxy * ip, ft = rsqrtf(sc2.syy);
    float col[3];
    if (DIRECT_RGB) {
        col[0] = rgb[0]; col[1] = rgb[1]; col[2] = rgb[2];
    } else {
        float d0 = p.mean[0] - Vw.eye[0], d1 = p.mean[1] - Vw.eye[1], d2 = p.mean[2] - Vw.eye[2];
        const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        d0 *= il; d1 *= il; d2 *= il;
        float Y[16];
        sh_eval(d0, d1, d2, sh_degree, Y);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int cidx = 0; cidx < 16; ++cidx) s += k[cidx][ch] * Y[cidx];
            col[ch] = fmaxf(s, 0.0f);
        }
    }
    r0 = make_float4(mx, my, ex, ey);
    // L scaled by kappa = sqrt(log2(e)/2): G' = exp2(-(s1^2 + s2^2)),
    // s1 = r1.x dx + r1.y dy, s2 = r1.z dy
    r1 = make_float4(KAPPA * fp, KAPPA * fr, KAPPA * ft, opac);
    r2 = make_float4(col[0], col[1], col[2], cv);
    return true;
}

// dL/dq of a loss that depends on R(q / |q|) (q = (w, x, y, z) as stored)
// through gR = dL/dR (row-major 3x3), added to gq: the derivative of each
// entry of the rotation matrix in the unit quaternion, then the projection
// of the normalisation, (I - q^ q^T) / |q|.
__device__ __forceinline__ void rot_quat_adjoint(const float q[4], const float gR[9], float gq[4]) {
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    float gh[4];
    gh[0] = 2.0f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gh[1] = 2.0f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.0f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] - 2.0f * x * gR[8]);
    gh[2] = 2.0f * (-2.0f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] - 2.0f * y * gR[8]);
    gh[3] = 2.0f * (-2.0f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.0f * z * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
    const float hq = (gh[0] * w + gh[1] * x + gh[2] * y + gh[3] * z);
    gq[0] += (gh[0] - hq * w) / qn;
    gq[1] += (gh[1] - hq * x) / qn;
    gq[2] += (gh[2] - hq * y) / qn;
    gq[3] += (gh[3] - hq * z) / qn;
}

}  // namespace dgs
