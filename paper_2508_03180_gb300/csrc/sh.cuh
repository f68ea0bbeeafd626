// Real spherical harmonics of degree <= 3 (colour, Sec. III; view-dependent
// v_n, Sec. V-A) shared by the CUDA kernels.  Not part of the public ABI.
#pragma once

namespace dgs {

// Real spherical harmonics without the Condon-Shortley phase, index l^2+l+m;
// each constant is the normalisation of Y_lm (1/(2 sqrt(pi)), sqrt(3/(4 pi)), ...).
constexpr float SH_C0 = 0.28209479177387814f;
constexpr float SH_C1 = 0.4886025119029199f;
constexpr float SH_C2a = 1.0925484305920792f;   // (1/2) sqrt(15/pi)
constexpr float SH_C2b = 0.31539156525252005f;  // (1/4) sqrt(5/pi)
constexpr float SH_C2c = 0.5462742152960396f;   // (1/4) sqrt(15/pi)
constexpr float SH_C3a = 0.5900435899266435f;   // (1/4) sqrt(35/(2 pi))
constexpr float SH_C3b = 2.890611442640554f;    // (1/2) sqrt(105/pi)
constexpr float SH_C3c = 0.4570457994644658f;   // (1/4) sqrt(21/(2 pi))
constexpr float SH_C3d = 0.3731763325901154f;   // (1/4) sqrt(7/pi)
constexpr float SH_C3e = 1.445305721320277f;    // (1/4) sqrt(105/pi)

__device__ __forceinline__ void sh_eval(float x, float y, float z, int deg, float Y[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) Y[i] = 0.f;
    Y[0] = SH_C0;
    if (deg < 1) return;
    Y[1] = SH_C1 * y; Y[2] = SH_C1 * z; Y[3] = SH_C1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_C2a * x * y; Y[5] = SH_C2a * y * z; Y[6] = SH_C2b * (3.0f * zz - 1.0f);
    Y[7] = SH_C2a * x * z; Y[8] = SH_C2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = SH_C3a * y * (3.0f * xx - yy); Y[10] = SH_C3b * x * y * z;
    Y[11] = SH_C3c * y * (5.0f * zz - 1.0f); Y[12] = SH_C3d * z * (5.0f * zz - 3.0f);
    Y[13] = SH_C3c * x * (5.0f * zz - 1.0f); Y[14] = SH_C3e * z * (xx - yy);
    Y[15] = SH_C3a * x * (xx - 3.0f * yy);
}

// Partial derivatives of the formulas above in x, y, z (treated as free).
__device__ __forceinline__ void sh_grad(float x, float y, float z, int deg, float dX[16], float dY[16], float dZ[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) dX[i] = dY[i] = dZ[i] = 0.f;
    if (deg < 1) return;
    dX[1] = 0.f; dY[1] = SH_C1; dZ[1] = 0.f;
    dX[2] = 0.f; dY[2] = 0.f; dZ[2] = SH_C1;
    dX[3] = SH_C1; dY[3] = 0.f; dZ[3] = 0.f;
    if (deg < 2) return;
    dX[4] = SH_C2a * y; dY[4] = SH_C2a * x; dZ[4] = 0.f;
    dX[5] = 0.f; dY[5] = SH_C2a * z; dZ[5] = SH_C2a * y;
    dX[6] = 0.f; dY[6] = 0.f; dZ[6] = SH_C2b * 6.0f * z;
    dX[7] = SH_C2a * z; dY[7] = 0.f; dZ[7] = SH_C2a * x;
    dX[8] = SH_C2c * 2.0f * x; dY[8] = -SH_C2c * 2.0f * y; dZ[8] = 0.f;
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dX[9] = SH_C3a * 6.0f * x * y; dY[9] = SH_C3a * 3.0f * (xx - yy); dZ[9] = 0.f;
    dX[10] = SH_C3b * y * z; dY[10] = SH_C3b * x * z; dZ[10] = SH_C3b * x * y;
    dX[11] = 0.f; dY[11] = SH_C3c * (5.0f * zz - 1.0f); dZ[11] = SH_C3c * 10.0f * y * z;
    dX[12] = 0.f; dY[12] = 0.f; dZ[12] = SH_C3d * (15.0f * zz - 3.0f);
    dX[13] = SH_C3c * (5.0f * zz - 1.0f); dY[13] = 0.f; dZ[13] = SH_C3c * 10.0f * x * z;
    dX[14] = SH_C3e * 2.0f * x * z; dY[14] = -SH_C3e * 2.0f * y * z; dZ[14] = SH_C3e * (xx - yy);
    dX[15] = SH_C3a * 3.0f * (xx - yy); dY[15] = -SH_C3a * 6.0f * x * y; dZ[15] = 0.f;
}

// g += sum_c w[c] grad Y_c(x, y, z) (the formulas of sh_grad, without the arrays).
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, int deg, const float w[16], float g[3]) {
    if (deg < 1) return;
    g[1] += SH_C1 * w[1];
    g[2] += SH_C1 * w[2];
    g[0] += SH_C1 * w[3];
    if (deg < 2) return;
    g[0] += SH_C2a * (y * w[4] + z * w[7]) + SH_C2c * 2.0f * x * w[8];
    g[1] += SH_C2a * (x * w[4] + z * w[5]) - SH_C2c * 2.0f * y * w[8];
    g[2] += SH_C2a * (y * w[5] + x * w[7]) + SH_C2b * 6.0f * z * w[6];
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += SH_C3a * 6.0f * x * y * w[9] + SH_C3b * y * z * w[10] + SH_C3c * (5.0f * zz - 1.0f) * w[13] +
            SH_C3e * 2.0f * x * z * w[14] + SH_C3a * 3.0f * (xx - yy) * w[15];
    g[1] += SH_C3a * 3.0f * (xx - yy) * w[9] + SH_C3b * x * z * w[10] + SH_C3c * (5.0f * zz - 1.0f) * w[11] -
            SH_C3e * 2.0f * y * z * w[14] - SH_C3a * 6.0f * x * y * w[15];
    g[2] += SH_C3b * x * y * w[10] + SH_C3c * 10.0f * y * z * w[11] + SH_C3d * (15.0f * zz - 3.0f) * w[12] +
            SH_C3c * 10.0f * x * z * w[13] + SH_C3e * (xx - yy) * w[14];
}

}  // namespace dgs
