// K15: late shading from the rendered normal map (Sec. 3.1: the normal
// image, obtained by substituting n_k for c_k in Eq. 1, feeds a pixel
// shader that relights the rendered view).
//
// The paper names no shading model; the one here is Lambertian with
// directional lights and an ambient term.  Per pixel of a view:
//   C    = rgb - (1 - alpha) bg          (the composited colour, Eq. 1)
//   n^   = N / |N|                       (N the rendered normal, unnormalised)
//   s    = ambient + sum_l I_l max(0, n^ . l_l)
//   out  = C s + (1 - alpha) bg
// A pixel with |N| <= 1e-12 (no surface) keeps s = 1.  The light
// directions l_l are unit vectors in the world frame of the normals.
//
// One thread per pixel, grid-stride: every plane is read and written with
// coalesced 4-byte accesses; the kernel is bound by HBM (28 bytes read and
// 12 bytes written per pixel).
#include <algorithm>

#include "common.cuh"

namespace p2e {

struct ShadeViews {
    int32_t n_views, n_lights;
    int64_t hw[P2E_MAX_VIEWS];
    int64_t base[P2E_MAX_VIEWS];   // first pixel of the view
    float light[P2E_MAX_LIGHTS][4];  // unit direction, intensity
    float ambient;
    float bg[3];
};

__global__ void __launch_bounds__(256) relight_kernel(const float *rgb,  // may alias out
                                                      const float *__restrict__ normal,
                                                      const float *__restrict__ alpha, int64_t total,
                                                      float *out, __grid_constant__ const ShadeViews V) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < V.n_views && V.base[v + 1] <= q) ++v;
        const int64_t hw = V.hw[v], p = q - V.base[v];
        const int64_t o = 3 * V.base[v] + p;  // channel 0 of the pixel in its view's planes
        const float a = __ldg(alpha + q);
        const float ta = 1.f - a;
        const float nx = __ldg(normal + o), ny = __ldg(normal + o + hw), nz = __ldg(normal + o + 2 * hw);
        const float len2 = nx * nx + ny * ny + nz * nz;
        float s = 1.f;
        if (len2 > 1e-24f) {
            const float inv = rsqrtf(len2);
            s = V.ambient;
            for (int l = 0; l < V.n_lights; ++l) {
                const float d = (nx * V.light[l][0] + ny * V.light[l][1] + nz * V.light[l][2]) * inv;
                s = fmaf(V.light[l][3], fmaxf(d, 0.f), s);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float bgc = V.bg[c] * ta;
            const float C = rgb[o + c * hw] - bgc;
            out[o + c * hw] = fmaf(C, s, bgc);
        }
    }
}

int device_sms();

}  // namespace p2e

extern "C" p2e_status p2e_relight(const float *rgb, const float *normal, const float *alpha,
                                  const int64_t *view_pixels, int32_t n_views, const float *lights,
                                  int32_t n_lights, float ambient, const float *bg, float *out, void *stream) {
    using namespace p2e;
    if (n_views < 1 || n_views > P2E_MAX_VIEWS || !view_pixels || n_lights < 0 || n_lights > P2E_MAX_LIGHTS ||
        (n_lights > 0 && !lights) || !isfinite(ambient))
        return P2E_ERR_INVALID_ARG;
    ShadeViews V;
    V.n_views = n_views;
    V.n_lights = n_lights;
    V.ambient = ambient;
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        if (view_pixels[v] < 0) return P2E_ERR_INVALID_ARG;
        V.hw[v] = view_pixels[v];
        V.base[v] = total;
        total += view_pixels[v];
    }
    for (int l = 0; l < n_lights; ++l) {
        const float x = lights[4 * l], y = lights[4 * l + 1], z = lights[4 * l + 2], I = lights[4 * l + 3];
        const float n2 = x * x + y * y + z * z;
        if (!isfinite(n2) || !isfinite(I) || !(n2 > 0.f)) return P2E_ERR_INVALID_ARG;
        const float inv = 1.f / sqrtf(n2);
        V.light[l][0] = x * inv;
        V.light[l][1] = y * inv;
        V.light[l][2] = z * inv;
        V.light[l][3] = I;
    }
    for (int c = 0; c < 3; ++c) {
        V.bg[c] = bg ? bg[c] : 0.f;
        if (!isfinite(V.bg[c])) return P2E_ERR_INVALID_ARG;
    }
    if (total == 0) return P2E_OK;
    if (!rgb || !normal || !alpha || !out) return P2E_ERR_INVALID_ARG;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)device_sms() * 8);
    relight_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(rgb, normal, alpha, total, out, V);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}
