// K16: the point-rasterisation baseline of Sec. 4.1 ("OpenGL": every point
// drawn as a 1-pixel square with a depth test), as a CUDA twin of the
// graphics pipeline so that it runs, and is timed, next to the splatting
// path on the same GPU.
//
// Reading of the 1-pixel square: a point covers the one pixel whose square
// [i, i+1) x [j, j+1) contains its projection (u, v) = (fx x/z + cx,
// fy y/z + cy), i = floor(u), j = floor(v); it is drawn when z > near.  The
// depth test keeps the nearest point, ties by the lower point index, and
// the pixel takes that point's colour (background elsewhere).
//
// Pass 1 (one thread per point and view): camera transform and projection
// in fp32 with explicit correctly rounded operations in a fixed order, then
// one 64-bit atomicMin of (depth bits << 32 | index) per covered pixel
// (z > 0, so the float bits order as unsigned integers).
// Pass 2 (one thread per pixel): the winning point's colour and depth.
// Bound by the atomics and HBM: 16 bytes read and one 8-byte atomic per
// point, 8 bytes read and 16 bytes written per pixel.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace p2e {

struct RasterViews {
    int32_t n_views;
    float bg[3];
    int64_t n;
    struct {
        float T[9], t[3], fx, fy, cx, cy, near_z;
        int32_t W, H;
        int64_t pix_base;
    } v[P2E_MAX_VIEWS];
};

__global__ void __launch_bounds__(256) raster_points_kernel(const float4 *__restrict__ xyz,
                                                            unsigned long long *__restrict__ zbuf,
                                                            __grid_constant__ const RasterViews R) {
    const int64_t total = R.n * R.n_views;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int vi = (int)(q / R.n);
        const int64_t i = q - (int64_t)vi * R.n;
        const auto &V = R.v[vi];
        const float4 p = __ldg(xyz + i);
        const float x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.T[0], p.x), __fmul_rn(V.T[1], p.y)),
                                            __fmul_rn(V.T[2], p.z)), V.t[0]);
        const float y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.T[3], p.x), __fmul_rn(V.T[4], p.y)),
                                            __fmul_rn(V.T[5], p.z)), V.t[1]);
        const float z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.T[6], p.x), __fmul_rn(V.T[7], p.y)),
                                            __fmul_rn(V.T[8], p.z)), V.t[2]);
        if (!(z > V.near_z) || !(z > 0.f)) continue;
        const float u = __fadd_rn(__fmul_rn(V.fx, __fdiv_rn(x, z)), V.cx);
        const float w = __fadd_rn(__fmul_rn(V.fy, __fdiv_rn(y, z)), V.cy);
        if (!(u >= 0.f) || !(w >= 0.f) || !(u < (float)V.W) || !(w < (float)V.H)) continue;
        const int px = min((int)floorf(u), V.W - 1), py = min((int)floorf(w), V.H - 1);
        const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)i;
        atomicMin(zbuf + V.pix_base + (int64_t)py * V.W + px, key);
    }
}

__global__ void __launch_bounds__(256) raster_resolve_kernel(const unsigned long long *__restrict__ zbuf,
                                                             const float4 *__restrict__ rgb, int64_t total_pix,
                                                             float *__restrict__ out_rgb, float *__restrict__ out_depth,
                                                             __grid_constant__ const RasterViews R) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total_pix;
         q += (int64_t)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < R.n_views && R.v[v + 1].pix_base <= q) ++v;
        const int64_t hw = (int64_t)R.v[v].W * R.v[v].H, p = q - R.v[v].pix_base;
        const unsigned long long key = zbuf[q];
        float c0 = R.bg[0], c1 = R.bg[1], c2 = R.bg[2], d = 0.f;
        if (key != ~0ull) {
            const float4 c = __ldg(rgb + (key & 0xffffffffull));
            c0 = c.x, c1 = c.y, c2 = c.z;
            d = __uint_as_float((uint32_t)(key >> 32));
        }
        float *o = out_rgb + 3 * R.v[v].pix_base + p;
        o[0] = c0;
        o[hw] = c1;
        o[2 * hw] = c2;
        if (out_depth) out_depth[q] = d;
    }
}

int device_sms();

}  // namespace p2e

extern "C" p2e_status p2e_point_raster(const float *xyz, const float *rgb, int64_t n, const p2e_camera *cams,
                                       int32_t n_views, const float *bg, uint64_t *zbuf, float *out_rgb,
                                       float *out_depth, void *stream) {
    using namespace p2e;
    if (!cams || n_views < 1 || n_views > P2E_MAX_VIEWS || n < 0 || n >= (int64_t(1) << 32))
        return P2E_ERR_INVALID_ARG;
    RasterViews R;
    memset(&R, 0, sizeof(R));
    R.n_views = n_views;
    R.n = n;
    for (int c = 0; c < 3; ++c) {
        R.bg[c] = bg ? bg[c] : 0.f;
        if (!isfinite(R.bg[c])) return P2E_ERR_INVALID_ARG;
    }
    int64_t pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const p2e_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 8192 || c.height > 8192) return P2E_ERR_INVALID_ARG;
        for (int k = 0; k < 12; ++k)
            if (!isfinite(c.viewmat[k])) return P2E_ERR_INVALID_ARG;
        if (!isfinite(c.fx) || !isfinite(c.fy) || !isfinite(c.cx) || !isfinite(c.cy) || !isfinite(c.near_z) ||
            c.near_z < 0.f)
            return P2E_ERR_INVALID_ARG;
        auto &V = R.v[v];
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) V.T[3 * r + k] = c.viewmat[4 * r + k];
            V.t[r] = c.viewmat[4 * r + 3];
        }
        V.fx = c.fx, V.fy = c.fy, V.cx = c.cx, V.cy = c.cy, V.near_z = c.near_z;
        V.W = c.width, V.H = c.height;
        V.pix_base = pix;
        pix += (int64_t)c.width * c.height;
    }
    if (!zbuf || !out_rgb || ((uintptr_t)zbuf & 7u)) return P2E_ERR_INVALID_ARG;
    if (n > 0 && (!xyz || !rgb || ((uintptr_t)xyz & 15u) || ((uintptr_t)rgb & 15u))) return P2E_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(zbuf, 0xff, (size_t)pix * sizeof(uint64_t), st) != cudaSuccess) return P2E_ERR_CUDA;
    const int sms = device_sms();
    if (n > 0) {
        const int64_t b1 = std::min<int64_t>((n * n_views + 255) / 256, (int64_t)sms * 16);
        raster_points_kernel<<<(unsigned)b1, 256, 0, st>>>((const float4 *)xyz,
                                                           (unsigned long long *)zbuf, R);
    }
    const int64_t b2 = std::min<int64_t>((pix + 255) / 256, (int64_t)sms * 8);
    raster_resolve_kernel<<<(unsigned)b2, 256, 0, st>>>((const unsigned long long *)zbuf, (const float4 *)rgb, pix,
                                                        out_rgb, out_depth, R);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}
