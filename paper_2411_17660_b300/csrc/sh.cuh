// sh.cuh -- real spherical harmonics up to degree 3 (SH -> RGB, Sec. 3.3:
// "c denotes the color converted from SH").  Basis with the Condon-Shortley
// phase, ordered (l, m = -l..l).  Constants are the normalisations
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0) evaluated
// in double precision; the polynomial forms below are valid on the unit
// sphere, and the backward projects out the radial derivative, so any
// extension off the sphere gives the same gradient.
#pragma once

namespace gsr {

constexpr float kC0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kC1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kC2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float kC3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float kC3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float kC3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float kC3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kC3e = 1.445305721320277f;    // sqrt(105/pi)/4

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float *Y) {
    Y[0] = kC0;
    if (DEG >= 1) {
        Y[1] = -kC1 * y;
        Y[2] = kC1 * z;
        Y[3] = -kC1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kC2a * x * y;
        Y[5] = -kC2a * y * z;
        Y[6] = kC2b * (2.f * zz - xx - yy);
        Y[7] = -kC2a * x * z;
        Y[8] = kC2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kC3a * y * (3.f * xx - yy);
            Y[10] = kC3b * x * y * z;
            Y[11] = -kC3c * y * (4.f * zz - xx - yy);
            Y[12] = kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kC3c * x * (4.f * zz - xx - yy);
            Y[14] = kC3e * z * (xx - yy);
            Y[15] = -kC3a * x * (xx - 3.f * yy);
        }
    }
}

// g = sum_k w[k] * grad Y_k at (x, y, z), with the polynomial forms above.
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float *w, float &gx, float &gy,
                                        float &gz) {
    gx = gy = gz = 0.f;
    if (DEG >= 1) {
        gy -= kC1 * w[1];
        gz += kC1 * w[2];
        gx -= kC1 * w[3];
    }
    if (DEG >= 2) {
        gx += kC2a * y * w[4];
        gy += kC2a * x * w[4];
        gy -= kC2a * z * w[5];
        gz -= kC2a * y * w[5];
        gx -= 2.f * kC2b * x * w[6];
        gy -= 2.f * kC2b * y * w[6];
        gz += 4.f * kC2b * z * w[6];
        gx -= kC2a * z * w[7];
        gz -= kC2a * x * w[7];
        gx += 2.f * kC2c * x * w[8];
        gy -= 2.f * kC2c * y * w[8];
        if (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx -= 6.f * kC3a * x * y * w[9];
            gy -= kC3a * (3.f * xx - 3.f * yy) * w[9];
            gx += kC3b * y * z * w[10];
            gy += kC3b * x * z * w[10];
            gz += kC3b * x * y * w[10];
            gx += 2.f * kC3c * x * y * w[11];
            gy -= kC3c * (4.f * zz - xx - 3.f * yy) * w[11];
            gz -= 8.f * kC3c * y * z * w[11];
            gx -= 6.f * kC3d * x * z * w[12];
            gy -= 6.f * kC3d * y * z * w[12];
            gz += kC3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            gx -= kC3c * (4.f * zz - 3.f * xx - yy) * w[13];
            gy += 2.f * kC3c * x * y * w[13];
            gz -= 8.f * kC3c * x * z * w[13];
            gx += 2.f * kC3e * x * z * w[14];
            gy -= 2.f * kC3e * y * z * w[14];
            gz += kC3e * (xx - yy) * w[14];
            gx -= kC3a * (3.f * xx - 3.f * yy) * w[15];
            gy += 6.f * kC3a * x * y * w[15];
        }
    }
}

}  // namespace gsr
