// Per-pixel splat arithmetic shared by the compositing kernel and its
// backward, so that both take identical decisions (3-sigma test, floor) on
// identical values.  Every operation is an explicit correctly rounded
// intrinsic, so the compiler cannot contract them differently in the two
// kernels.
#pragma once
#include "common.cuh"

namespace p2e {

// Tile-relative record of a projected splat.
//   off = (0.5 - frac u, 0.5 - frac v, floor u - x0, floor v - y0)
__device__ __forceinline__ float4 splat_offset(const float4 &xy, int x0, int y0) {
    const int packed = __float_as_int(xy.w);
    const int iu = (int)(int16_t)(packed & 0xffff), iv = packed >> 16;
    return make_float4(__fsub_rn(0.5f, xy.x), __fsub_rn(0.5f, xy.y), (float)(iu - x0), (float)(iv - y0));
}

// Pixel offset d = (x - (floor u - x0)) + (0.5 - frac u): an exact integer
// plus an exact fraction.
__device__ __forceinline__ void splat_delta(const float4 &o, float x, float y, float &dx, float &dy) {
    dx = __fadd_rn(__fsub_rn(x, o.z), o.x);
    dy = __fadd_rn(__fsub_rn(y, o.w), o.y);
}

// power = -1/2 d^T Sigma_s^-1 d for conic (A, B, C)
__device__ __forceinline__ float splat_power_d(const float4 &co, float dx, float dy) {
    const float q = __fmaf_rn(co.x, __fmul_rn(dx, dx), __fmul_rn(co.z, __fmul_rn(dy, dy)));
    return __fsub_rn(__fmul_rn(-0.5f, q), __fmul_rn(co.y, __fmul_rn(dx, dy)));
}

__device__ __forceinline__ float splat_power(const float4 &o, const float4 &co, float x, float y) {
    float dx, dy;
    splat_delta(o, x, y, dx, dy);
    return splat_power_d(co, dx, dy);
}

// alpha = min(alpha_max, o exp(power)); also returns whether the clamp is
// inactive (the derivative with respect to o and power exists).
__device__ __forceinline__ float splat_alpha(float o, float power, float amax, float &e, bool &free) {
    e = __expf(power);
    const float a = __fmul_rn(o, e);
    free = !(a > amax);
    return free ? a : amax;
}

}  // namespace p2e
