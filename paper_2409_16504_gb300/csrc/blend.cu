// K6: front-to-back alpha compositing (Sec. 3.1, Eq. 1-2), with the normal
// and depth images obtained by substituting n_k and z_k for c_k.
//
// One CTA per screen tile (tile x tile threads, one pixel each).  The tile's
// depth-sorted splat list is walked in batches of one splat per thread: the
// batch (up to 256 splats) is gathered (sorted index -> projected record,
// colour, normal) into shared memory with coalesced 16-byte loads, then every thread walks the
// batch from shared memory (broadcast reads).  A pixel stops at the
// transmittance cutoff; the CTA stops as soon as every pixel has stopped
// (__syncthreads_count), and a warp whose pixels have all stopped skips the
// batch.
#include "common.cuh"

namespace p2e {

template <int B>
__global__ void __launch_bounds__(B *B) blend_kernel(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
    const float4 *__restrict__ xy_depth, const float4 *__restrict__ conic_op,
    const float4 *__restrict__ rgb, const float4 *__restrict__ normal, float *__restrict__ out_rgb,
    float *__restrict__ out_nrm, float *__restrict__ out_depth, float *__restrict__ out_alpha,
    uint32_t *__restrict__ out_last, __grid_constant__ const Views P) {
    constexpr int NT = B * B;
    constexpr int BATCH = NT < 256 ? NT : 256;  // splats staged per round
    __shared__ float4 s_xy[BATCH], s_co[BATCH], s_rgb[BATCH], s_nrm[BATCH];
    const int64_t tile = blockIdx.x;
    const int vi = view_of_tile(P, tile);
    const View &V = P.v[vi];
    const int64_t lt = tile - V.tile_base;
    const int ty = (int)(lt / V.tiles_x), tx = (int)(lt - (int64_t)ty * V.tiles_x);
    const int px = tx * B + (threadIdx.x % B), py = ty * B + (threadIdx.x / B);
    const bool inside = px < V.W && py < V.H;
    const uint2 r = ranges[tile];
    const int64_t gbase = (int64_t)vi * P.n;
    const float pw_min = -0.5f * P.sigma_mult * P.sigma_mult;
    const float amax = P.alpha_max, afloor = P.alpha_floor, tmin = P.t_min;

    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f, D = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t start = r.x; start < r.y; start += BATCH) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t idx = start + threadIdx.x;
        if (threadIdx.x < BATCH && idx < r.y) {
            uint32_t g = __ldg(vals + idx);
            if (g >= (uint32_t)P.n) g = 0;  // only reachable with corrupted bins
            s_xy[threadIdx.x] = __ldg(xy_depth + gbase + g);
            s_co[threadIdx.x] = __ldg(conic_op + gbase + g);
            s_rgb[threadIdx.x] = __ldg(rgb + g);
            s_nrm[threadIdx.x] = __ldg(normal + g);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BATCH, r.y - start);
        if (__all_sync(0xffffffffu, done)) continue;
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 xy = s_xy[j];
                const int packed = __float_as_int(xy.w);
                const int iu = (int)(int16_t)(packed & 0xffff), iv = packed >> 16;
                const float dx = (float)(px - iu) + (0.5f - xy.x);
                const float dy = (float)(py - iv) + (0.5f - xy.y);
                const float4 co = s_co[j];
                const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
                if (power < pw_min) continue;
                const float alpha = fminf(amax, co.w * __expf(power));
                if (alpha < afloor) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < tmin) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                const float4 cc = s_rgb[j], nn = s_nrm[j];
                c0 = fmaf(w, cc.x, c0);
                c1 = fmaf(w, cc.y, c1);
                c2 = fmaf(w, cc.z, c2);
                n0 = fmaf(w, nn.x, n0);
                n1 = fmaf(w, nn.y, n1);
                n2 = fmaf(w, nn.z, n2);
                D = fmaf(w, xy.z, D);
                T = Tn;
                last = start + (uint32_t)j + 1u;
            }
        }
    }
    if (!inside) return;
    const int64_t HW = (int64_t)V.H * V.W;
    const int64_t p = (int64_t)py * V.W + px;
    if (out_rgb) {
        float *o = out_rgb + 3 * V.pix_base + p;
        o[0] = fmaf(T, P.bg[0], c0);
        o[HW] = fmaf(T, P.bg[1], c1);
        o[2 * HW] = fmaf(T, P.bg[2], c2);
    }
    if (out_nrm) {
        float *o = out_nrm + 3 * V.pix_base + p;
        o[0] = n0;
        o[HW] = n1;
        o[2 * HW] = n2;
    }
    if (out_depth) out_depth[V.pix_base + p] = D;
    if (out_alpha) out_alpha[V.pix_base + p] = 1.f - T;
    if (out_last) out_last[V.pix_base + p] = last;
}

cudaError_t launch_render(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                          const Views &P, float *rgb, float *nrm, float *depth, float *alpha,
                          uint32_t *last, cudaStream_t st) {
    if (P.total_tiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)P.total_tiles;
    const uint32_t *vals = bins->vals[bins->result];
    const uint2 *ranges = (const uint2 *)bins->ranges;
#define P2E_BLEND(BB)                                                                           \
    blend_kernel<BB><<<grid, BB * BB, 0, st>>>(ranges, vals, (const float4 *)proj->xy_depth,     \
                                               (const float4 *)proj->conic_op,                   \
                                               (const float4 *)g->rgb, (const float4 *)g->normal, \
                                               rgb, nrm, depth, alpha, last, P)
    switch (P.tile) {
        case 8: P2E_BLEND(8); break;
        case 16: P2E_BLEND(16); break;
        case 32: P2E_BLEND(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef P2E_BLEND
    return cudaGetLastError();
}

}  // namespace p2e
