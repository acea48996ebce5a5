// vgr_tiletest.cuh -- tile-level preemptive alpha test (paper Sec. 4.2,
// Eq. 4, moved to binning).  Used by the counting pass (preprocess) and by
// the emission pass; every operation is an explicitly rounded intrinsic so
// both passes take bit-identical decisions.
#pragma once

#include "vgr_internal.cuh"

namespace vgr {

// rho = -1/2 (a dx^2 + c dy^2) - b dx dy
__device__ __forceinline__ float rho_rn(float a, float b, float c, float dx, float dy) {
    const float t1 = __fmul_rn(__fmul_rn(a, dx), dx);
    const float t2 = __fmul_rn(__fmul_rn(c, dy), dy);
    const float t3 = __fmul_rn(__fmul_rn(b, dx), dy);
    return __fsub_rn(__fmul_rn(-0.5f, __fadd_rn(t1, t2)), t3);
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// Keep the pair when the maximum of rho over the rectangle spanned by the
// tile's pixel centres reaches thre (= ln alpha* - ln theta - slack).  The
// maximum is 0 when the mean lies inside; otherwise it is on an edge, where
// rho is a concave quadratic in the free coordinate: on the edges x = x0, x1
// its optimum is dy* = (-b/c) dx = ry dx, on y = y0, y1 it is
// dx* = (-b/a) dy = rx dy, each clamped to the edge.
// T is the tile side in pixels (8, 16 or 32): every coordinate below is exact in FP32.
__device__ __forceinline__ bool tile_keep(float u, float v, float a, float b, float c, float rx, float ry, float thre,
                                          int tx, int ty, float W, float H, int T) {
    const float x0 = (float)(tx * T) + 0.5f;
    const float x1 = fminf((float)(tx * T) + ((float)T - 0.5f), W - 0.5f);
    const float y0 = (float)(ty * T) + 0.5f;
    const float y1 = fminf((float)(ty * T) + ((float)T - 0.5f), H - 0.5f);
    if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return thre <= 0.f;
    const float dy_lo = __fsub_rn(y0, v), dy_hi = __fsub_rn(y1, v);
    const float dx_lo = __fsub_rn(x0, u), dx_hi = __fsub_rn(x1, u);
    float best = rho_rn(a, b, c, dx_lo, clampf(__fmul_rn(ry, dx_lo), dy_lo, dy_hi));
    best = fmaxf(best, rho_rn(a, b, c, dx_hi, clampf(__fmul_rn(ry, dx_hi), dy_lo, dy_hi)));
    best = fmaxf(best, rho_rn(a, b, c, clampf(__fmul_rn(rx, dy_lo), dx_lo, dx_hi), dy_lo));
    best = fmaxf(best, rho_rn(a, b, c, clampf(__fmul_rn(rx, dy_hi), dx_lo, dx_hi), dy_hi));
    return best >= thre;
}

}  // namespace vgr
