// K7 + K8: gradient of the compositing (Eq. 1-2) and of the EWA projection
// (Eq. 3-4) with respect to the raw Gaussian parameters, with every discrete
// decision of the forward pass held fixed (differentiable splatting, used
// to train the estimator end to end, Sec. 1 and 3.3).
//
// K7 (per tile, persistent over a list of work items): each pixel first
// recomputes its final transmittance front to back over its tile list up to
// the forward's `last` (the product of (1 - alpha_k) over the contributing
// splats, re-decided with the forward's exact arithmetic, splat.cuh), then
// walks the list back to front, recovering T_k = T_{k+1} / (1 - alpha_k).
// No per-pixel lists are stored.  Lists longer than four splats per pixel
// are cut into segments walked in parallel (see bwd_items_kernel).  The final T is not taken from the alpha
// image: near saturation (T ~ 1e-4) the fp32 round trip alpha = 1 - T,
// T = 1 - alpha loses ~3e-8 absolute, a relative error of ~2.5e-4 that the
// division chain would carry to every splat of the pixel.  With
// f_k = gC.c_k + gN.n_k + gD z_k and the running tail
//   S_k = sum_{j>k} alpha_j T_j f_j + T_final (gC.bg - gA),
// dL/dalpha_k = T_k f_k - S_k / (1 - alpha_k).  Per-splat screen-space
// gradients (u, v, A, B, C, o, z, rgb, normal) are reduced over the warp
// (a transposing butterfly: 16 shuffles for the 13 channels), then over the
// CTA in shared memory, then added to global memory.
//
// K8 (per Gaussian): chain rule through conic = Sigma_s^-1,
// Sigma_s = M M^T + lowpass I, M = J T R S, R(q / |q|), and the centre
// u = fx x / z + cx (and v), summed over the views.
#include "splat.cuh"

namespace p2e {

constexpr int kG2D = 16;  // floats per (view, Gaussian) screen-space gradient slot
enum { QU = 0, QV, QA, QB, QC, QO, QZ, QR, QG, QBL, QNX, QNY, QNZ, QN };

size_t backward_scratch_bytes(int64_t n_total) {
    return ((size_t)n_total * kG2D * sizeof(float) + 255) & ~size_t(255);
}

// Sum over the warp of 16 per-lane values (q[QN..15] taken as zero),
// returned transposed: lane l gets the sum of value (l >> 1) & 15.
__device__ __forceinline__ float warp_transpose_sum(const float (&q)[QN], int lane) {
    float a[8], b[4], c[2];
#pragma unroll
    for (int i = 0; i < 8; ++i) {  // offset 16: keep half i + 8 * bit4
        const float lo = i < QN ? q[i] : 0.f, hi = i + 8 < QN ? q[i + 8] : 0.f;
        const bool up = (lane & 16) != 0;
        a[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // offset 8
        const bool up = (lane & 8) != 0;
        b[i] = (up ? a[i + 4] : a[i]) + __shfl_xor_sync(0xffffffffu, up ? a[i] : a[i + 4], 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {  // offset 4
        const bool up = (lane & 4) != 0;
        c[i] = (up ? b[i + 2] : b[i]) + __shfl_xor_sync(0xffffffffu, up ? b[i] : b[i + 2], 4);
    }
    const bool up = (lane & 2) != 0;  // offset 2
    float d = (up ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, up ? c[0] : c[1], 2);
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

template <int B>
struct BwdShape {
    static constexpr int NT = B * B;
    static constexpr int BATCH = NT < 256 ? NT : 256;
    // a tile list longer than S splats (four per pixel) is walked in
    // segments of S, each its own work item
    static constexpr uint32_t S = 4u * NT;
};

// Segments of long tile lists.  Both walks of a pixel are sums and
// products over its contributing splats in depth order, so they split at
// segment boundaries: with, per segment m, the local transmittance
// P_m = prod (1 - alpha_j) and the local weighted sum
// F_m = sum alpha_j T'_j f_j (T' the transmittance from the segment's own
// start), the transmittance entering segment s is prod_{m<s} P_m, the final
// one prod_m P_m, and the running tail S at the end of segment s is
// sum_{m>s} (prod_{l<m} P_l) F_m + T_final (gC.bg - gA).  A fold kernel
// computes (P_m, F_m) for every segment and pixel; the gradient walk of
// segment s starts from those, so a long list costs no serial walk.
//
// Only the part of a list before the tile's walk end (the largest `last` of
// its pixels) is walked, so only that part is segmented: segments past it
// have no item.
//
// Item table (in the value buffer the sort left free): header words, the
// walk end of every work tile, then (work index, segment) per item (the
// segmented tiles' items in the work list's order: longest length class
// first); the folds (float2 per item and pixel) go in the free key buffer.
// Without room (a capacity below the key count, a missing buffer) nothing
// is segmented.
enum { kBwdItems = 0, kBwdOn = 1, kBwdCtrFold = 2, kBwdHdr = 4 };

// Walk end of every work tile: the largest `last` of its pixels (at least
// the list start), one warp per tile.
template <int B>
__global__ void __launch_bounds__(256) bwd_tile_end_kernel(const uint2 *__restrict__ ranges,
                                                           const uint32_t *__restrict__ work,
                                                           const uint32_t *__restrict__ last_img, int64_t capacity,
                                                           uint32_t *__restrict__ table,
                                                           __grid_constant__ const Views P) {
    const uint32_t n_work = work[0];
    if ((int64_t)kBwdHdr + n_work > capacity) return;  // no room: nothing is segmented
    const int lane = threadIdx.x & 31;
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    for (uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_work; w += nw) {
        const int64_t tile = work[2 + w];
        const int vi = view_of_tile(P, tile);
        const View &V = P.v[vi];
        const int64_t lt = tile - V.tile_base;
        const int ty = (int)(lt / V.tiles_x), tx = (int)(lt - (int64_t)ty * V.tiles_x);
        const uint2 r = ranges[tile];
        uint32_t m = r.x;
        for (int p = lane; p < B * B; p += 32) {
            const int px = tx * B + p % B, py = ty * B + p / B;
            if (px < V.W && py < V.H) m = max(m, min(last_img[V.pix_base + (int64_t)py * V.W + px], r.y));
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) table[kBwdHdr + w] = m;
    }
}

__global__ void __launch_bounds__(1024) bwd_items_kernel(const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ work,
                                                         const int64_t *__restrict__ n_keys_dev,
                                                         int64_t capacity, uint32_t S, uint32_t NT,
                                                         uint32_t *__restrict__ table) {
    __shared__ uint32_t s_sum[32], s_off[32];
    __shared__ unsigned long long s_total;
    __shared__ uint32_t s_carry;
    const uint32_t n_work = work[0];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if (threadIdx.x == 0) {
        s_total = 0;
        s_carry = 0;
    }
    __syncthreads();
    const bool room = (int64_t)kBwdHdr + n_work <= capacity;  // the walk ends were written
    const uint32_t *tile_end = table + kBwdHdr;
    auto nseg_of = [&](uint32_t w) -> uint32_t {
        const uint32_t len = tile_end[w] - ranges[work[2 + w]].x;
        return len > S ? (len + S - 1) / S : 0u;
    };
    unsigned long long mine = 0;
    for (uint32_t w = threadIdx.x; room && w < n_work; w += blockDim.x) mine += nseg_of(w);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0 && mine) atomicAdd(&s_total, mine);  // one add per warp
    __syncthreads();
    const unsigned long long total = s_total;
    const bool fits = room && *n_keys_dev <= capacity &&
                      (long long)(kBwdHdr + n_work + 2 * total) <= capacity && (long long)(total * NT) <= capacity;
    uint32_t *items = table + kBwdHdr + n_work;
    if (threadIdx.x == 0) {
        table[kBwdItems] = fits ? (uint32_t)total : 0u;
        table[kBwdOn] = fits ? 1u : 0u;
        table[kBwdCtrFold] = 0u;
    }
    if (!fits || total == 0) return;
    for (uint32_t b0 = 0; b0 < n_work; b0 += blockDim.x) {
        const uint32_t w = b0 + threadIdx.x;
        const uint32_t v = w < n_work ? nseg_of(w) : 0u;
        // exclusive block scan of v
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const uint32_t t0 = lane < nw ? s_sum[lane] : 0u;
            uint32_t t = t0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_off[lane] = t - t0;
        }
        __syncthreads();
        const uint32_t base = s_carry + s_off[wid] + x - v;
        for (uint32_t m = 0; m < v; ++m) {
            items[2 * (base + m)] = w;
            items[2 * (base + m) + 1] = m;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = base + v;
        __syncthreads();
    }
}

// The upstream gradient of one pixel: rgb, normal, depth, alpha.
__device__ __forceinline__ void load_upstream(const View &V, int64_t pix, int64_t HW, const float *d_rgb,
                                              const float *d_nrm, const float *d_depth, const float *d_alpha,
                                              float (&up)[8]) {
    if (d_rgb)
        for (int c = 0; c < 3; ++c) up[c] = d_rgb[3 * V.pix_base + c * HW + pix];
    if (d_nrm)
        for (int c = 0; c < 3; ++c) up[3 + c] = d_nrm[3 * V.pix_base + c * HW + pix];
    if (d_depth) up[6] = d_depth[V.pix_base + pix];
    if (d_alpha) up[7] = d_alpha[V.pix_base + pix];
}

// Fold of one segment per (item, pixel): (P_m, F_m) as defined above, the
// discrete decisions exactly the forward's (splat.cuh).
template <int B>
__global__ void __launch_bounds__(BwdShape<B>::NT) bwd_fold_kernel(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ work,
    uint32_t *__restrict__ table, float2 *__restrict__ fold,
    const float4 *__restrict__ xy_depth, const float4 *__restrict__ conic_op, const ushort4 *__restrict__ rect,
    const float4 *__restrict__ rgb, const float4 *__restrict__ normal, const uint32_t *__restrict__ last_img,
    const float *__restrict__ d_rgb, const float *__restrict__ d_nrm, const float *__restrict__ d_depth,
    __grid_constant__ const Views P) {
    constexpr int NT = BwdShape<B>::NT, BATCH = BwdShape<B>::BATCH;
    constexpr uint32_t S = BwdShape<B>::S;
    __shared__ float4 s_off[BATCH], s_co[BATCH], s_cz[BATCH], s_nr[BATCH];
    __shared__ ushort4 s_rc[BATCH];
    __shared__ uint32_t s_item, s_end;
    const int tid = threadIdx.x;
    const int lx = tid % B, ly = tid / B;
    const int wy0 = (tid & ~31) / B, wy1 = ((tid & ~31) + 31) / B;
    const float lxf = (float)lx, lyf = (float)ly;
    const float pw_min = -0.5f * P.sigma_mult * P.sigma_mult;
    const float amax = P.alpha_max, afloor = P.alpha_floor;
    const uint32_t n_items = table[kBwdItems];
    const uint32_t *items = table + kBwdHdr + work[0];
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(table + kBwdCtrFold, 1u);
            s_end = 0;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) break;
        const uint32_t w = items[2 * item], seg = items[2 * item + 1];
        const int64_t tile = work[2 + w];
        const int vi = view_of_tile(P, tile);
        const View &V = P.v[vi];
        const int64_t lt = tile - V.tile_base;
        const int ty = (int)(lt / V.tiles_x), tx = (int)(lt - (int64_t)ty * V.tiles_x);
        const int x0 = tx * B, y0 = ty * B;
        const int px = x0 + lx, py = y0 + ly;
        const bool inside = px < V.W && py < V.H;
        const uint2 r = ranges[tile];
        const uint32_t lo = r.x + seg * S, hi = min(r.y, lo + S);
        const int64_t gbase = (int64_t)vi * P.n;
        const int64_t HW = (int64_t)V.H * V.W;
        const int64_t pix = (int64_t)py * V.W + px;
        float up[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        uint32_t lim = lo;
        if (inside) {
            load_upstream(V, pix, HW, d_rgb, d_nrm, d_depth, nullptr, up);
            lim = min(last_img[V.pix_base + pix], hi);
            if (lim < lo) lim = lo;
            atomicMax(&s_end, lim);
        }
        __syncthreads();
        const uint32_t end = s_end;
        float T = 1.f, F = 0.f;
        for (uint32_t bstart = lo; bstart < end; bstart += BATCH) {
            const int cnt = (int)min((uint32_t)BATCH, end - bstart);
            if (tid < cnt) {
                uint32_t g = __ldg(vals + bstart + tid);
                if (g >= (uint32_t)P.n) g = 0;
                const float4 xy = __ldg(xy_depth + gbase + g);
                const float4 cc = __ldg(rgb + g);
                s_off[tid] = splat_offset(xy, x0, y0);
                s_co[tid] = __ldg(conic_op + gbase + g);
                s_rc[tid] = __ldg(rect + gbase + g);
                s_cz[tid] = make_float4(cc.x, cc.y, cc.z, xy.z);
                s_nr[tid] = __ldg(normal + g);
            }
            __syncthreads();
            if (inside) {
                const int jend = (int)min((uint32_t)cnt, lim > bstart ? lim - bstart : 0u);
                for (int j = 0; j < jend; ++j) {
                    const ushort4 rc = s_rc[j];
                    if ((int)rc.w < y0 + wy0 || (int)rc.y > y0 + wy1) continue;  // uniform over the warp
                    const float4 o = s_off[j], co = s_co[j];
                    float dx, dy;
                    splat_delta(o, lxf, lyf, dx, dy);
                    const float power = splat_power_d(co, dx, dy);
                    if (power < pw_min) continue;
                    float e;
                    bool fr;
                    const float alpha = splat_alpha(co.w, power, amax, e, fr);
                    if (alpha < afloor) continue;
                    const float4 cz = s_cz[j], nr = s_nr[j];
                    const float f = up[0] * cz.x + up[1] * cz.y + up[2] * cz.z + up[3] * nr.x + up[4] * nr.y +
                                    up[5] * nr.z + up[6] * cz.w;
                    F = fmaf(alpha * T, f, F);
                    T *= 1.f - alpha;
                }
            }
            __syncthreads();
        }
        fold[(size_t)item * NT + tid] = make_float2(T, F);
        __syncthreads();
    }
}

template <int B>
__global__ void __launch_bounds__(BwdShape<B>::NT) blend_bwd_kernel(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ work, uint32_t *__restrict__ work_counter,
    const uint32_t *__restrict__ table, const float2 *__restrict__ fold,
    const float4 *__restrict__ xy_depth, const float4 *__restrict__ conic_op, const ushort4 *__restrict__ rect,
    const float4 *__restrict__ rgb, const float4 *__restrict__ normal,
    const float *__restrict__ alpha_img, const uint32_t *__restrict__ last_img,
    const float *__restrict__ d_rgb, const float *__restrict__ d_nrm, const float *__restrict__ d_depth,
    const float *__restrict__ d_alpha, float *__restrict__ g2d, unsigned long long *__restrict__ count,
    __grid_constant__ const Views P) {
    constexpr int NT = BwdShape<B>::NT, BATCH = BwdShape<B>::BATCH;
    constexpr uint32_t S = BwdShape<B>::S;
    __shared__ float4 s_off[BATCH], s_co[BATCH], s_cz[BATCH], s_nr[BATCH];
    __shared__ ushort4 s_rc[BATCH];
    __shared__ uint32_t s_g[BATCH];
    __shared__ float s_acc[BATCH][QN];
    __shared__ uint32_t s_item, s_end;

    const int tid = threadIdx.x, lane = tid & 31;
    const int lx = tid % B, ly = tid / B;
    // the tile rows of this warp's pixels (a splat whose pixel rectangle
    // misses them cannot touch them: the warp skips it as a whole)
    const int wy0 = (tid & ~31) / B, wy1 = ((tid & ~31) + 31) / B;
    const float lxf = (float)lx, lyf = (float)ly;
    const float pw_min = -0.5f * P.sigma_mult * P.sigma_mult;
    const float amax = P.alpha_max, afloor = P.alpha_floor;
    const uint32_t n_work = work[0];
    // items: the segments of long lists (table), then every tile whose list
    // is not segmented, walked whole
    const uint32_t n_multi = table ? table[kBwdItems] : 0u;
    const bool seg_on = table && table[kBwdOn] != 0u;
    const uint32_t *tile_end = seg_on ? table + kBwdHdr : nullptr;
    const uint32_t *items = seg_on ? table + kBwdHdr + n_work : nullptr;
    // work counts for the probe: (pixel, splat) pairs evaluated in each of
    // the two walks, the contributing ones among them, warp reductions
    uint32_t n_eval = 0, n_contrib = 0, n_red = 0;

    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(work_counter, 1u);
            s_end = 0;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_multi + n_work) break;
        const bool multi = item < n_multi;
        const uint32_t w = multi ? items[2 * item] : item - n_multi;
        const uint32_t seg = multi ? items[2 * item + 1] : 0u;
        const int64_t tile = work[2 + w];
        const uint2 r = ranges[tile];
        const uint32_t walk = seg_on ? tile_end[w] - r.x : r.y - r.x;  // length of the walked part
        if (!multi && seg_on && (walk > S || walk == 0)) {  // walked as segments, or not at all
            __syncthreads();
            continue;
        }
        const uint32_t lo = r.x + seg * S, hi = multi ? min(r.y, lo + S) : r.y;
        const int vi = view_of_tile(P, tile);
        const View &V = P.v[vi];
        const int64_t lt = tile - V.tile_base;
        const int ty = (int)(lt / V.tiles_x), tx = (int)(lt - (int64_t)ty * V.tiles_x);
        const int x0 = tx * B, y0 = ty * B;
        const int px = x0 + lx, py = y0 + ly;
        const bool inside = px < V.W && py < V.H;
        const int64_t gbase = (int64_t)vi * P.n;
        const int64_t HW = (int64_t)V.H * V.W;
        const int64_t pix = (int64_t)py * V.W + px;

        float up[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        float T = 1.f;
        uint32_t lastp = 0;
        if (inside) {
            load_upstream(V, pix, HW, d_rgb, d_nrm, d_depth, d_alpha, up);
            lastp = last_img[V.pix_base + pix];
            if (lastp > r.y) lastp = r.y;  // only reachable with mismatched inputs
            atomicMax(&s_end, min(lastp, hi));
        }
        __syncthreads();
        const uint32_t end = max(s_end, lo);
        const float cbg = up[0] * P.bg[0] + up[1] * P.bg[1] + up[2] * P.bg[2] - up[7];
        float acc;
        if (multi) {
            // entering and final transmittance and the tail from the folds
            const uint32_t nseg = (walk + S - 1) / S, first = item - seg;
            float tail = 0.f, t_in = 1.f, p_own = 1.f;
            for (uint32_t m = 0; m < nseg; ++m) {
                const float2 pf = fold[(size_t)(first + m) * NT + tid];
                if (m == seg) {
                    t_in = T;
                    p_own = pf.x;
                } else if (m > seg) {
                    tail = fmaf(T, pf.y, tail);
                }
                T *= pf.x;
            }
            acc = tail + T * cbg;
            T = t_in * p_own;
        }
        // final transmittance of a whole list, front to back over [r.x, lastp)
        for (uint32_t bstart = lo; !multi && bstart < end; bstart += BATCH) {
            const int cnt = (int)min((uint32_t)BATCH, end - bstart);
            if (tid < cnt) {
                uint32_t g = __ldg(vals + bstart + tid);
                if (g >= (uint32_t)P.n) g = 0;
                s_off[tid] = splat_offset(__ldg(xy_depth + gbase + g), x0, y0);
                s_co[tid] = __ldg(conic_op + gbase + g);
                s_rc[tid] = __ldg(rect + gbase + g);
            }
            __syncthreads();
            if (inside) {
                const int jend = (int)min((uint32_t)cnt, lastp > bstart ? lastp - bstart : 0u);
                for (int j = 0; j < jend; ++j) {
                    const ushort4 rc = s_rc[j];
                    if ((int)rc.w < y0 + wy0 || (int)rc.y > y0 + wy1) continue;  // uniform over the warp
                    const float4 o = s_off[j], co = s_co[j];
                    float dx, dy;
                    splat_delta(o, lxf, lyf, dx, dy);
                    const float power = splat_power_d(co, dx, dy);
                    if (power < pw_min) continue;
                    float e;
                    bool fr;
                    const float alpha = splat_alpha(co.w, power, amax, e, fr);
                    if (alpha < afloor) continue;
                    T *= 1.f - alpha;
                }
            }
            __syncthreads();
        }
        if (!multi) acc = T * cbg;
        // back to front over [lo, end)
        for (uint32_t bend = end; bend > lo; bend = (bend - lo > (uint32_t)BATCH) ? bend - BATCH : lo) {
            const uint32_t bstart = (bend - lo > (uint32_t)BATCH) ? bend - BATCH : lo;
            const int cnt = (int)(bend - bstart);
            for (int t = tid; t < cnt * QN; t += NT) (&s_acc[0][0])[t] = 0.f;
            if (tid < cnt) {
                uint32_t g = __ldg(vals + bstart + tid);
                if (g >= (uint32_t)P.n) g = 0;
                const float4 xy = __ldg(xy_depth + gbase + g);
                const float4 cc = __ldg(rgb + g);
                s_off[tid] = splat_offset(xy, x0, y0);
                s_co[tid] = __ldg(conic_op + gbase + g);
                s_rc[tid] = __ldg(rect + gbase + g);
                s_cz[tid] = make_float4(cc.x, cc.y, cc.z, xy.z);
                s_nr[tid] = __ldg(normal + g);
                s_g[tid] = g;
            }
            __syncthreads();
            for (int j = cnt - 1; j >= 0; --j) {
                const ushort4 rc = s_rc[j];
                if ((int)rc.w < y0 + wy0 || (int)rc.y > y0 + wy1) continue;  // uniform over the warp
                float q[QN];
#pragma unroll
                for (int c = 0; c < QN; ++c) q[c] = 0.f;
                bool contrib = false;
                if (inside && bstart + (uint32_t)j < lastp) {
                    ++n_eval;
                    const float4 o = s_off[j], co = s_co[j];
                    float dx, dy;
                    splat_delta(o, lxf, lyf, dx, dy);
                    const float power = splat_power_d(co, dx, dy);
                    if (power >= pw_min) {
                        float e;
                        bool fr;
                        const float alpha = splat_alpha(co.w, power, amax, e, fr);
                        if (alpha >= afloor) {
                            contrib = true;
                            ++n_contrib;
                            const float4 cz = s_cz[j], nr = s_nr[j];
                            // 1 - alpha >= 1 - alpha_max: the fast division keeps
                            // ~2 ulp per step over a chain of at most one segment
                            const float om = 1.f - alpha;
                            const float Tk = __fdividef(T, om);
                            const float w = alpha * Tk;
                            const float f = up[0] * cz.x + up[1] * cz.y + up[2] * cz.z + up[3] * nr.x +
                                            up[4] * nr.y + up[5] * nr.z + up[6] * cz.w;
                            const float dal = Tk * f - __fdividef(acc, om);
                            acc = fmaf(w, f, acc);
                            T = Tk;
                            q[QR] = w * up[0];
                            q[QG] = w * up[1];
                            q[QBL] = w * up[2];
                            q[QNX] = w * up[3];
                            q[QNY] = w * up[4];
                            q[QNZ] = w * up[5];
                            q[QZ] = w * up[6];
                            if (fr) {
                                q[QO] = dal * e;
                                const float dp = dal * alpha;
                                q[QA] = -0.5f * dp * dx * dx;
                                q[QC] = -0.5f * dp * dy * dy;
                                q[QB] = -dp * dx * dy;
                                q[QU] = dp * (co.x * dx + co.y * dy);
                                q[QV] = dp * (co.y * dx + co.z * dy);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    ++n_red;
                    // transposing butterfly: each step hands half of the
                    // channels a lane still holds to its partner, so 16
                    // channels take 8 + 4 + 2 + 1 + 1 shuffles; lane l ends
                    // with the warp's sum of channel (l >> 1) & 15
                    const float v = warp_transpose_sum(q, lane);
                    const int c = (lane >> 1) & 15;
                    if (!(lane & 1) && c < QN && v != 0.f) atomicAdd(&s_acc[j][c], v);
                }
            }
            __syncthreads();
            for (int t = tid; t < cnt * QN; t += NT) {
                const int j = t / QN, c = t - j * QN;
                const float v = s_acc[j][c];
                if (v != 0.f) atomicAdd(&g2d[(gbase + s_g[j]) * kG2D + c], v);
            }
            __syncthreads();
        }
        __syncthreads();
    }
    if (count) {
        const uint32_t e = __reduce_add_sync(0xffffffffu, n_eval), c = __reduce_add_sync(0xffffffffu, n_contrib);
        if (lane == 0) {
            atomicAdd(count, (unsigned long long)e);
            atomicAdd(count + 1, (unsigned long long)c);
            atomicAdd(count + 2, (unsigned long long)n_red);
        }
    }
}

// K8: screen-space gradients -> raw parameters, summed over the views.
__global__ void __launch_bounds__(256) project_bwd_kernel(
    const float4 *__restrict__ mean_op, const float4 *__restrict__ scale,
    const float4 *__restrict__ quat, const float *__restrict__ g2d, float *__restrict__ d_mean,
    float *__restrict__ d_scale, float *__restrict__ d_quat, float *__restrict__ d_opacity,
    float *__restrict__ d_rgb_g, float *__restrict__ d_normal_g, __grid_constant__ const Views P) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    const float4 m = mean_op[g], s4 = scale[g], q4 = quat[g];
    float dm[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0};
    float dop = 0.f, dc[3] = {0, 0, 0}, dn[3] = {0, 0, 0};
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float iq = qn > 0.f ? 1.f / qn : 0.f;
    const float w = q4.x * iq, a = q4.y * iq, b = q4.z * iq, c = q4.w * iq;
    float R[3][3];
    R[0][0] = 1.f - 2.f * (b * b + c * c); R[0][1] = 2.f * (a * b - w * c); R[0][2] = 2.f * (a * c + w * b);
    R[1][0] = 2.f * (a * b + w * c); R[1][1] = 1.f - 2.f * (a * a + c * c); R[1][2] = 2.f * (b * c - w * a);
    R[2][0] = 2.f * (a * c - w * b); R[2][1] = 2.f * (b * c + w * a); R[2][2] = 1.f - 2.f * (a * a + b * b);
    const float s[3] = {s4.x, s4.y, s4.z};
    float dR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int vi = 0; vi < P.n_views; ++vi) {
        const float *G = g2d + ((int64_t)vi * P.n + g) * kG2D;
        const float4 g0 = *reinterpret_cast<const float4 *>(G);
        const float4 g1 = *reinterpret_cast<const float4 *>(G + 4);
        const float4 g2 = *reinterpret_cast<const float4 *>(G + 8);
        const float g12 = G[12];
        dop += g1.y;
        dc[0] += g1.w; dc[1] += g2.x; dc[2] += g2.y;
        dn[0] += g2.z; dn[1] += g2.w; dn[2] += g12;
        if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.z == 0.f)
            continue;  // no geometric gradient from this view
        const View &V = P.v[vi];
        const float *T = V.T;
        const float x = T[0] * m.x + T[1] * m.y + T[2] * m.z + V.t[0];
        const float y = T[3] * m.x + T[4] * m.y + T[5] * m.z + V.t[1];
        const float z = T[6] * m.x + T[7] * m.y + T[8] * m.z + V.t[2];
        float Wm[3][3], Vm[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                Wm[i][k] = T[3 * i] * R[0][k] + T[3 * i + 1] * R[1][k] + T[3 * i + 2] * R[2][k];
                Vm[i][k] = Wm[i][k] * s[k];
            }
        const float iz = 1.f / z;
        const float J00 = V.fx * iz, J02 = -V.fx * x * iz * iz, J11 = V.fy * iz, J12 = -V.fy * y * iz * iz;
        float M0[3], M1[3];
        for (int k = 0; k < 3; ++k) {
            M0[k] = J00 * Vm[0][k] + J02 * Vm[2][k];
            M1[k] = J11 * Vm[1][k] + J12 * Vm[2][k];
        }
        const float sa = M0[0] * M0[0] + M0[1] * M0[1] + M0[2] * M0[2] + P.lowpass;
        const float sb = M0[0] * M1[0] + M0[1] * M1[1] + M0[2] * M1[2];
        const float sc = M1[0] * M1[0] + M1[1] * M1[1] + M1[2] * M1[2] + P.lowpass;
        const float idet = 1.f / (sa * sc - sb * sb);
        const float Q00 = sc * idet, Q01 = -sb * idet, Q11 = sa * idet;
        // dL/dSigma_s = -Q G Q with G = [[gA, gB/2], [gB/2, gC]]
        const float GA = g0.z, GB = 0.5f * g0.w, GC = g1.x;
        const float t00 = Q00 * GA + Q01 * GB, t01 = Q00 * GB + Q01 * GC;
        const float t10 = Q01 * GA + Q11 * GB, t11 = Q01 * GB + Q11 * GC;
        const float ga = -(t00 * Q00 + t01 * Q01);
        const float gc = -(t10 * Q01 + t11 * Q11);
        const float gb = -2.f * (t00 * Q01 + t01 * Q11);
        float dM0[3], dM1[3];
        for (int k = 0; k < 3; ++k) {
            dM0[k] = 2.f * ga * M0[k] + gb * M1[k];
            dM1[k] = 2.f * gc * M1[k] + gb * M0[k];
        }
        // M = J V
        const float dJ00 = dM0[0] * Vm[0][0] + dM0[1] * Vm[0][1] + dM0[2] * Vm[0][2];
        const float dJ02 = dM0[0] * Vm[2][0] + dM0[1] * Vm[2][1] + dM0[2] * Vm[2][2];
        const float dJ11 = dM1[0] * Vm[1][0] + dM1[1] * Vm[1][1] + dM1[2] * Vm[1][2];
        const float dJ12 = dM1[0] * Vm[2][0] + dM1[1] * Vm[2][1] + dM1[2] * Vm[2][2];
        float dV[3][3];
        for (int k = 0; k < 3; ++k) {
            dV[0][k] = J00 * dM0[k];
            dV[1][k] = J11 * dM1[k];
            dV[2][k] = J02 * dM0[k] + J12 * dM1[k];
        }
        float dW[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                ds[k] += dV[i][k] * Wm[i][k];
                dW[i][k] = dV[i][k] * s[k];
            }
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) dR[l][k] += T[l] * dW[0][k] + T[3 + l] * dW[1][k] + T[6 + l] * dW[2][k];
        // centre, depth image and Jacobian -> camera coordinates -> mean
        float dx = g0.x * V.fx * iz + dJ02 * (-V.fx * iz * iz);
        float dy = g0.y * V.fy * iz + dJ12 * (-V.fy * iz * iz);
        float dz = g0.x * (-V.fx * x * iz * iz) + g0.y * (-V.fy * y * iz * iz) + g1.z +
                   dJ00 * (-V.fx * iz * iz) + dJ11 * (-V.fy * iz * iz) +
                   dJ02 * (2.f * V.fx * x * iz * iz * iz) + dJ12 * (2.f * V.fy * y * iz * iz * iz);
        for (int k = 0; k < 3; ++k) dm[k] += T[k] * dx + T[3 + k] * dy + T[6 + k] * dz;
    }
    // R(w, a, b, c) -> unit quaternion -> raw quaternion
    const float gw = 2.f * (-c * dR[0][1] + b * dR[0][2] + c * dR[1][0] - a * dR[1][2] - b * dR[2][0] + a * dR[2][1]);
    const float gx = 2.f * (b * dR[0][1] + c * dR[0][2] + b * dR[1][0] - 2.f * a * dR[1][1] - w * dR[1][2] +
                            c * dR[2][0] + w * dR[2][1] - 2.f * a * dR[2][2]);
    const float gy = 2.f * (-2.f * b * dR[0][0] + a * dR[0][1] + w * dR[0][2] + a * dR[1][0] + c * dR[1][2] -
                            w * dR[2][0] + c * dR[2][1] - 2.f * b * dR[2][2]);
    const float gz = 2.f * (-2.f * c * dR[0][0] - w * dR[0][1] + a * dR[0][2] + w * dR[1][0] - 2.f * c * dR[1][1] +
                            b * dR[1][2] + a * dR[2][0] + b * dR[2][1]);
    const float dot = w * gw + a * gx + b * gy + c * gz;
    dq[0] = (gw - w * dot) * iq;
    dq[1] = (gx - a * dot) * iq;
    dq[2] = (gy - b * dot) * iq;
    dq[3] = (gz - c * dot) * iq;
    for (int k = 0; k < 3; ++k) {
        d_mean[3 * g + k] = dm[k];
        d_scale[3 * g + k] = ds[k];
        d_rgb_g[3 * g + k] = dc[k];
        d_normal_g[3 * g + k] = dn[k];
    }
    for (int k = 0; k < 4; ++k) d_quat[4 * g + k] = dq[k];
    d_opacity[g] = dop;
}

int device_sms();

template <int B>
static cudaError_t launch_bwd(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                              const Views &P, const float *alpha, const uint32_t *last,
                              const float *d_rgb, const float *d_normal, const float *d_depth,
                              const float *d_alpha, float *g2d, cudaStream_t st) {
    // persistent grids: as many CTAs as fit on an SM (64 registers a thread)
    const int grid = device_sms() * (B == 8 ? 16 : (B == 16 ? 4 : 1));
    const int other = 1 - bins->result;
    const bool seg = P.schedule == P2E_SCHEDULE_AUTO && bins->capacity >= kBwdHdr && bins->keys[other] &&
                     bins->vals[other] && bins->n_keys_dev;
    uint32_t *table = seg ? bins->vals[other] : nullptr;
    float2 *fold = seg ? (float2 *)bins->keys[other] : nullptr;
    const p2e_kernel_probe *pr = kernel_probe(P2E_PROBE_BLEND_BWD);
    probe_start(pr, st);
    if (seg) {
        bwd_tile_end_kernel<B><<<device_sms() * 2, 256, 0, st>>>((const uint2 *)bins->ranges, bins->tile_work, last,
                                                                 bins->capacity, table, P);
        bwd_items_kernel<<<1, 1024, 0, st>>>((const uint2 *)bins->ranges, bins->tile_work, bins->n_keys_dev,
                                             bins->capacity, BwdShape<B>::S, BwdShape<B>::NT, table);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        bwd_fold_kernel<B><<<grid, BwdShape<B>::NT, 0, st>>>(
            (const uint2 *)bins->ranges, bins->vals[bins->result], bins->tile_work, table, fold,
            (const float4 *)proj->xy_depth, (const float4 *)proj->conic_op, (const ushort4 *)proj->rect,
            (const float4 *)g->rgb, (const float4 *)g->normal, last, d_rgb, d_normal, d_depth, P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    blend_bwd_kernel<B><<<grid, BwdShape<B>::NT, 0, st>>>(
        (const uint2 *)bins->ranges, bins->vals[bins->result], bins->tile_work, bins->tile_work + 1, table, fold,
        (const float4 *)proj->xy_depth, (const float4 *)proj->conic_op, (const ushort4 *)proj->rect,
        (const float4 *)g->rgb,
        (const float4 *)g->normal, alpha, last, d_rgb, d_normal, d_depth, d_alpha, g2d,
        pr ? (unsigned long long *)pr->count_dev : nullptr, P);
    probe_stop(pr, st);
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const p2e_gaussians *g, const p2e_projected *proj,
                                   const p2e_bins *bins, const Views &P, const float *alpha,
                                   const uint32_t *last, const float *d_rgb, const float *d_normal,
                                   const float *d_depth, const float *d_alpha, float *d_mean,
                                   float *d_scale, float *d_quat, float *d_opacity, float *d_rgb_g,
                                   float *d_normal_g, void *scratch, cudaStream_t st) {
    if (P.n == 0) return cudaSuccess;
    float *g2d = (float *)scratch;
    cudaError_t e = cudaMemsetAsync(g2d, 0, (size_t)P.n * P.n_views * kG2D * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (P.total_tiles > 0) {
        if ((e = cudaMemsetAsync(bins->tile_work + 1, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
        switch (P.tile) {
            case 8: e = launch_bwd<8>(g, proj, bins, P, alpha, last, d_rgb, d_normal, d_depth, d_alpha, g2d, st); break;
            case 16: e = launch_bwd<16>(g, proj, bins, P, alpha, last, d_rgb, d_normal, d_depth, d_alpha, g2d, st); break;
            case 32: e = launch_bwd<32>(g, proj, bins, P, alpha, last, d_rgb, d_normal, d_depth, d_alpha, g2d, st); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    project_bwd_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, st>>>(
        (const float4 *)g->mean_op, (const float4 *)g->scale, (const float4 *)g->quat, g2d, d_mean,
        d_scale, d_quat, d_opacity, d_rgb_g, d_normal_g, P);
    return cudaGetLastError();
}

}  // namespace p2e
