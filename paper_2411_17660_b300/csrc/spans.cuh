// spans.cuh -- exact tile coverage of one projected Gaussian.
//
// The cutoff region {d^2 <= d2max} (d2max = min(9, 2 ln(255 sigma)): beyond
// it a pixel is either past the 3-sigma cutoff or below alpha = 1/255) is an
// ellipse.  For every row of screen tiles it touches, the x-range of the
// ellipse over that row's band of pixel centres is found in closed form:
// conditioned on dy, x lies in kx*dy +- sqrt(sc (r^2 - dy^2/Syy)) with
// kx = Sxy/Syy and sc = det/Syy; the right edge is concave in dy and peaks at
// dy = r Sxy/sqrt(Sxx) (the leftmost point mirrors it), so clamping that
// point into the band gives the band's extent.  An inflation of r^2 (0.2 %
// + 0.02) and of the x-range (1e-3 px) keeps the set a superset of what the
// per-pixel FP32 test accepts, including the error of the approximate
// reciprocals and square roots used here.
//
// The preprocess (counting) and the key duplication (emitting) call this on
// the same stored FP32 inputs.  Every operation is either a round-to-nearest
// intrinsic or a single hardware approximation instruction, none of which
// the compiler may contract or reorder, so both kernels see identical spans.
#pragma once

#include "common.cuh"

namespace gsr {

template <class F>
__device__ __forceinline__ uint32_t visit_tile_spans(float u, float v, float sxx, float sxy, float syy, float m00,
                                                     float smax, int W, int H, int TS, F &&f) {
    const float d2max = __fmul_rn(smax, 1.0f / kHalfLog2e);
    const float r2 = __fmaf_rn(d2max, 1.002f, 0.02f);
    const float ey = sqrt_approx(__fmul_rn(r2, syy));
    float ylo = ceilf(__fsub_rn(v, ey));
    float yhi = floorf(__fadd_rn(v, ey));
    ylo = fmaxf(ylo, 0.f);
    yhi = fminf(yhi, (float)(H - 1));
    if (!(ylo <= yhi)) return 0u;
    const int py0 = (int)ylo, py1 = (int)yhi;
    const int tsh = 31 - __clz(TS);   // TS is a power of two; the coordinates are >= 0
    const float isyy = rcp_approx(syy);
    const float kx = __fmul_rn(sxy, isyy);
    const float sc = __fmul_rn(kHalfLog2e, rcp_approx(__fmul_rn(m00, m00)));   // det/Syy, from the stable factor
    const float dyp = __fmul_rn(__fmul_rn(sxy, sqrt_approx(r2)), rcp_approx(sqrt_approx(sxx)));
    uint32_t count = 0;
    for (int ty = py0 >> tsh; ty <= py1 >> tsh; ++ty) {
        const int yb0 = max(ty * TS, py0), yb1 = min(ty * TS + TS - 1, py1);
        const float dy0 = __fsub_rn((float)yb0, v), dy1 = __fsub_rn((float)yb1, v);
        const float dyr = fminf(fmaxf(dyp, dy0), dy1);
        const float dyl = fminf(fmaxf(-dyp, dy0), dy1);
        const float hr = sqrt_approx(fmaxf(0.f, __fmul_rn(sc, __fsub_rn(r2, __fmul_rn(__fmul_rn(dyr, dyr), isyy)))));
        const float hl = sqrt_approx(fmaxf(0.f, __fmul_rn(sc, __fsub_rn(r2, __fmul_rn(__fmul_rn(dyl, dyl), isyy)))));
        const float xr = __fadd_rn(__fmul_rn(kx, dyr), hr);
        const float xl = __fsub_rn(__fmul_rn(kx, dyl), hl);
        float xlo = ceilf(__fsub_rn(__fadd_rn(u, xl), 1e-3f));
        float xhi = floorf(__fadd_rn(__fadd_rn(u, xr), 1e-3f));
        xlo = fmaxf(xlo, 0.f);
        xhi = fminf(xhi, (float)(W - 1));
        if (!(xlo <= xhi)) continue;
        const int tx0 = (int)xlo >> tsh, tx1 = (int)xhi >> tsh;
        f(ty, tx0, tx1);
        count += (uint32_t)(tx1 - tx0 + 1);
    }
    return count;
}

}  // namespace gsr
