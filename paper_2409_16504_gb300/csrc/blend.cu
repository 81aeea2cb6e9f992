// K6: front-to-back alpha compositing (Sec. 3.1, Eq. 1-2), with the normal
// and depth images obtained by substituting n_k and z_k for c_k.
//
// Scheduling.  A persistent grid pulls work items from the list of
// non-empty tiles that p2e_sort_bin leaves (longest list first); pixels of
// empty tiles get the background from a separate fill kernel.  A work item
// is one B x B pixel block of a binning tile: binning tiles of 16 are split
// into four 8 x 8 blocks, so that the few tiles a compact subject covers
// keep more SMs busy; each block screens its tile's whole list (next step)
// and composites only the splats that reach it.
//
// Per pixel block, the depth-sorted list is consumed in waves of up to G
// chunks of 256 splats:
//   fill     the next splats of the list are screened by their pixel
//            rectangle alone (8 bytes): only those whose rectangle meets a
//            pixel that is still compositing enter the wave, compacted in
//            list order (block-wide prefix sum).  Once the inside of a
//            surface has saturated, the rest of a long list costs one
//            rectangle load per splat instead of a full gather.
//   gather   the wave's splat records go to shared memory (16-byte loads)
//   cover    splat-parallel: every splat tests the live pixels of its pixel
//            rectangle (set bits of the live rows) against its sigma_mult
//            ellipse and sets its bit in those pixels' 256-bit chunk masks
//   blend    pixel-parallel: group k composites chunk k from T = 1, walking
//            only the set bits of its mask, in list (= depth) order
//   merge    group 0 combines the chunks in order with the associative
//            "over" rule C += T C_k, T *= T_k.  T is non-increasing, so the
//            cutoff can only fall inside chunk k when T T_k < t_min; only
//            that chunk is then re-walked from the true T with the stop
//            rule, which reproduces the sequential result.
// A splat is skipped only where it cannot contribute (outside its
// rectangle, or on a pixel that has stopped), so the result is the
// sequential one.  The tile is finished when every pixel has reached the
// cutoff or the list ends.
//
// Sub-pixel accuracy: the pixel offset is formed as
//   (x - (floor(u) - x0)) + (0.5 - frac(u)),
// an exact small integer plus an exact fraction, so it keeps ~1e-7 px at
// any image size.
#include <algorithm>

#include "splat.cuh"

namespace p2e {

template <int B>
struct BlendShape {
    static constexpr int NPIX = B * B;
    static constexpr int G = (B == 32) ? 1 : 4;    // chunk groups per CTA
    static constexpr int NT = NPIX * G;            // 256, 1024, 1024 threads
    static constexpr int NW = NT / 32;
    static constexpr int CHUNK = 256;
    static constexpr int WAVE = G * CHUNK;
    static constexpr int MW = CHUNK / 32;          // mask words per pixel and chunk
};

template <int B>
struct BlendSmem {
    using S = BlendShape<B>;
    float4 off[S::WAVE];     // (0.5 - frac u, 0.5 - frac v, floor u - x0, floor v - y0)
    float4 co[S::WAVE];      // (A, B, C, o)
    float4 cz[S::WAVE];      // (r, g, b, depth)
    float4 nr[S::WAVE];      // (nx, ny, nz, -)
    uint32_t rect[S::WAVE];  // tile-relative pixel box clamped to the tile, 4 x u8
    uint32_t gidx[S::WAVE];  // Gaussian of the wave slot
    uint32_t lpos[S::WAVE];  // list position of the wave slot
    uint32_t mask[S::G][S::MW][S::NPIX];  // word-major: conflict-free per-pixel reads
    float part[S::G][8][S::NPIX];   // per chunk: C0..2, N0..2, D, T
    uint32_t plast[S::G][S::NPIX];  // per chunk: last contributor (+1), 0 = none
    uint32_t alive[B];              // row bitmasks of the pixels still compositing
    uint32_t wscan[S::NW];          // fill: exclusive prefix of the warps' kept counts
    uint32_t wtotal, cut;
    uint8_t done[S::NPIX];
    uint32_t item;
};

__device__ __forceinline__ uint32_t row_bits(int x0, int x1) {  // bits x0..x1 (x1 <= 31)
    return (x1 >= 31 ? 0xffffffffu : ((1u << (x1 + 1)) - 1u)) & ~((1u << x0) - 1u);
}

// Row bitmasks of the live pixels from group 0's threads (pixel = thread):
// one warp holds 32 / B rows of the tile.
template <int B>
__device__ __forceinline__ void publish_alive(uint32_t *alive, int tid, bool live) {
    const uint32_t m = __ballot_sync(0xffffffffu, live);
    if ((tid & 31) == 0)
        for (int rr = 0; rr < 32 / B; ++rr)
            alive[(tid >> 5) * (32 / B) + rr] = (B == 32) ? m : ((m >> (rr * B)) & ((1u << B) - 1u));
}

template <int B>
__global__ void __launch_bounds__(BlendShape<B>::NT) blend_kernel(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ work, uint32_t *__restrict__ work_counter,
    const float4 *__restrict__ xy_depth, const float4 *__restrict__ conic_op,
    const ushort4 *__restrict__ rect, const float4 *__restrict__ rgb,
    const float4 *__restrict__ normal, float *__restrict__ out_rgb, float *__restrict__ out_nrm,
    float *__restrict__ out_depth, float *__restrict__ out_alpha, uint32_t *__restrict__ out_last,
    __grid_constant__ const Views P) {
    using S = BlendShape<B>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlendSmem<B> &sm = *reinterpret_cast<BlendSmem<B> *>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = tid / S::NPIX;
    const int pi = tid - grp * S::NPIX;     // pixel of this thread inside the tile
    const int lx = pi % B, ly = pi / B;
    const float lxf = (float)lx, lyf = (float)ly;
    const float pw_min = -0.5f * P.sigma_mult * P.sigma_mult;
    const float amax = P.alpha_max, afloor = P.alpha_floor, tmin = P.t_min;
    // work items: every non-empty binning tile (side P.tile) split into
    // sub x sub pixel blocks of side B, all blocks of a tile adjacent
    const int sub = P.tile / B;
    const uint32_t n_items = work[0] * (uint32_t)(sub * sub);

    for (;;) {
        if (tid == 0) sm.item = atomicAdd(work_counter, 1u);
        __syncthreads();
        const uint32_t item = sm.item;
        if (item >= n_items) break;
        const int64_t tile = work[2 + item / (uint32_t)(sub * sub)];
        const int blk = (int)(item % (uint32_t)(sub * sub));
        const int vi = view_of_tile(P, tile);
        const View &V = P.v[vi];
        const int64_t lt = tile - V.tile_base;
        const int ty = (int)(lt / V.tiles_x), tx = (int)(lt - (int64_t)ty * V.tiles_x);
        const int x0 = tx * P.tile + (blk % sub) * B, y0 = ty * P.tile + (blk / sub) * B;
        const int px = x0 + lx, py = y0 + ly;
        const bool inside = px < V.W && py < V.H;
        const uint2 r = ranges[tile];
        const int64_t gbase = (int64_t)vi * P.n;

        float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f, D = 0.f;
        uint32_t last = 0;
        bool done = !inside;
        if (grp == 0) {
            sm.done[pi] = done ? 1 : 0;
            publish_alive<B>(sm.alive, tid, !done);
        }

        uint32_t pos = r.x;  // next list position to screen (uniform)
        for (;;) {
            if (__syncthreads_count(grp == 0 ? done : true) == S::NT) break;
            if (pos >= r.y) break;
            // ---- fill: the next splats whose rectangle meets a live pixel
            uint32_t nfill = 0;  // uniform
            while (nfill < (uint32_t)S::WAVE && pos < r.y) {
                const uint32_t idx = pos + (uint32_t)tid;
                bool keep = false;
                uint32_t g = 0, rw = 0;
                if (idx < r.y) {
                    g = __ldg(vals + idx);
                    if (g >= (uint32_t)P.n) g = 0;  // only reachable with corrupted bins
                    const ushort4 rc = __ldg(rect + gbase + g);
                    const int rx0 = max(0, (int)rc.x - x0), rx1 = min(B - 1, (int)rc.z - x0);
                    const int ry0 = max(0, (int)rc.y - y0), ry1 = min(B - 1, (int)rc.w - y0);
                    if (rx0 <= rx1 && ry0 <= ry1) {
                        const uint32_t bits = row_bits(rx0, rx1);
                        for (int y = ry0; y <= ry1 && !keep; ++y) keep = (sm.alive[y] & bits) != 0u;
                        rw = (uint32_t)rx0 | ((uint32_t)rx1 << 8) | ((uint32_t)ry0 << 16) | ((uint32_t)ry1 << 24);
                    }
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) sm.wscan[warp] = (uint32_t)__popc(bal);
                __syncthreads();
                if (warp == 0) {
                    const uint32_t v = lane < S::NW ? sm.wscan[lane] : 0u;
                    uint32_t inc = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += u;
                    }
                    if (lane < S::NW) sm.wscan[lane] = inc - v;
                    if (lane == 31) sm.wtotal = inc;
                }
                __syncthreads();
                const uint32_t rank = nfill + sm.wscan[warp] + (uint32_t)__popc(bal & ((1u << lane) - 1u));
                if (keep && rank < (uint32_t)S::WAVE) {
                    sm.gidx[rank] = g;
                    sm.lpos[rank] = idx;
                    sm.rect[rank] = rw;
                }
                if (keep && rank == (uint32_t)S::WAVE) sm.cut = idx;  // first splat that did not fit
                __syncthreads();
                const uint32_t total = sm.wtotal;
                if (nfill + total > (uint32_t)S::WAVE) {
                    pos = sm.cut;
                    nfill = S::WAVE;
                } else {
                    pos = min(pos + (uint32_t)S::NT, r.y);
                    nfill += total;
                }
            }
            if (nfill == 0) break;  // nothing left in the list reaches a live pixel
            const int wn = (int)nfill;
            // ---- gather + clear masks
            {
                uint32_t *mw = &sm.mask[0][0][0];
                for (int t = tid; t < S::G * S::NPIX * S::MW; t += S::NT) mw[t] = 0u;
            }
            for (int t = tid; t < wn; t += S::NT) {
                const uint32_t g = sm.gidx[t];
                const float4 xy = __ldg(xy_depth + gbase + g);
                const float4 cc = __ldg(rgb + g);
                sm.off[t] = splat_offset(xy, x0, y0);
                sm.co[t] = __ldg(conic_op + gbase + g);
                sm.cz[t] = make_float4(cc.x, cc.y, cc.z, xy.z);
                sm.nr[t] = __ldg(normal + g);
            }
            __syncthreads();
            // ---- cover: splat-parallel, over the live pixels of each rectangle
            for (int t = tid; t < wn; t += S::NT) {
                const uint32_t rw = sm.rect[t];
                const int rx0 = rw & 0xff, rx1 = (rw >> 8) & 0xff, ry0 = (rw >> 16) & 0xff, ry1 = rw >> 24;
                const float4 o = sm.off[t], co = sm.co[t];
                const int k = t / S::CHUNK, b = t % S::CHUNK;
                const uint32_t bit = 1u << (b & 31);
                uint32_t *mk = &sm.mask[k][b >> 5][0];
                const uint32_t rb = row_bits(rx0, rx1);
                for (int y = ry0; y <= ry1; ++y) {
                    uint32_t m = sm.alive[y] & rb;
                    while (m) {
                        const int x = __ffs(m) - 1;
                        m &= m - 1u;
                        if (splat_power(o, co, (float)x, (float)y) < pw_min) continue;
                        atomicOr(mk + y * B + x, bit);
                    }
                }
            }
            __syncthreads();
            // ---- blend: chunk `grp`, composited from T = 1 over its set bits
            float t_ = 1.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, dd = 0.f;
            uint32_t lastl = 0;
            if (!sm.done[pi] && grp * S::CHUNK < wn) {
#pragma unroll 1
                for (int w = 0; w < S::MW; ++w) {
                    uint32_t m = sm.mask[grp][w][pi];
                    while (m) {
                        const int j = grp * S::CHUNK + w * 32 + (__ffs(m) - 1);
                        m &= m - 1u;
                        const float4 o = sm.off[j], co = sm.co[j];
                        const float power = splat_power(o, co, lxf, lyf);
                        if (power < pw_min) continue;
                        float e;
                        bool fr;
                        const float alpha = splat_alpha(co.w, power, amax, e, fr);
                        if (alpha < afloor) continue;
                        const float wgt = alpha * t_;
                        const float4 cz = sm.cz[j], nr = sm.nr[j];
                        a0 = fmaf(wgt, cz.x, a0);
                        a1 = fmaf(wgt, cz.y, a1);
                        a2 = fmaf(wgt, cz.z, a2);
                        b0 = fmaf(wgt, nr.x, b0);
                        b1 = fmaf(wgt, nr.y, b1);
                        b2 = fmaf(wgt, nr.z, b2);
                        dd = fmaf(wgt, cz.w, dd);
                        t_ = t_ * (1.f - alpha);
                        lastl = sm.lpos[j] + 1u;
                    }
                }
            }
            sm.part[grp][0][pi] = a0;
            sm.part[grp][1][pi] = a1;
            sm.part[grp][2][pi] = a2;
            sm.part[grp][3][pi] = b0;
            sm.part[grp][4][pi] = b1;
            sm.part[grp][5][pi] = b2;
            sm.part[grp][6][pi] = dd;
            sm.part[grp][7][pi] = t_;
            sm.plast[grp][pi] = lastl;
            __syncthreads();
            // ---- merge the chunks in list order (group 0)
            if (grp == 0 && !done) {
                for (int k = 0; k < S::G && k * S::CHUNK < wn; ++k) {
                    const float Tk = sm.part[k][7][pi];
                    if (T * Tk >= tmin) {
                        c0 = fmaf(T, sm.part[k][0][pi], c0);
                        c1 = fmaf(T, sm.part[k][1][pi], c1);
                        c2 = fmaf(T, sm.part[k][2][pi], c2);
                        n0 = fmaf(T, sm.part[k][3][pi], n0);
                        n1 = fmaf(T, sm.part[k][4][pi], n1);
                        n2 = fmaf(T, sm.part[k][5][pi], n2);
                        D = fmaf(T, sm.part[k][6][pi], D);
                        T = T * Tk;
                        if (sm.plast[k][pi]) last = sm.plast[k][pi];
                        continue;
                    }
                    // the cutoff falls inside chunk k: walk it from the true T
                    for (int w = 0; w < S::MW && !done; ++w) {
                        uint32_t m = sm.mask[k][w][pi];
                        while (m) {
                            const int j = k * S::CHUNK + w * 32 + (__ffs(m) - 1);
                            m &= m - 1u;
                            const float4 o = sm.off[j], co = sm.co[j];
                            const float power = splat_power(o, co, lxf, lyf);
                            if (power < pw_min) continue;
                            float e;
                            bool fr;
                            const float alpha = splat_alpha(co.w, power, amax, e, fr);
                            if (alpha < afloor) continue;
                            const float Tn = T * (1.f - alpha);
                            if (Tn < tmin) {
                                done = true;
                                break;
                            }
                            const float wgt = alpha * T;
                            const float4 cz = sm.cz[j], nr = sm.nr[j];
                            c0 = fmaf(wgt, cz.x, c0);
                            c1 = fmaf(wgt, cz.y, c1);
                            c2 = fmaf(wgt, cz.z, c2);
                            n0 = fmaf(wgt, nr.x, n0);
                            n1 = fmaf(wgt, nr.y, n1);
                            n2 = fmaf(wgt, nr.z, n2);
                            D = fmaf(wgt, cz.w, D);
                            T = Tn;
                            last = sm.lpos[j] + 1u;
                        }
                    }
                    if (done) break;
                }
                sm.done[pi] = done ? 1 : 0;
            }
            if (grp == 0) publish_alive<B>(sm.alive, tid, !done);
        }
        if (grp == 0 && inside) {
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
        __syncthreads();
    }
}

// Background for every pixel of a tile with an empty list.
__global__ void __launch_bounds__(256) fill_empty_kernel(const uint2 *__restrict__ ranges,
                                                         int64_t total_pix, float *__restrict__ out_rgb,
                                                         float *__restrict__ out_nrm,
                                                         float *__restrict__ out_depth,
                                                         float *__restrict__ out_alpha,
                                                         uint32_t *__restrict__ out_last,
                                                         __grid_constant__ const Views P) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total_pix;
         q += (int64_t)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < P.n_views && P.v[v + 1].pix_base <= q) ++v;
        const View &V = P.v[v];
        const int64_t p = q - V.pix_base;
        const int y = (int)(p / V.W), x = (int)(p - (int64_t)y * V.W);
        const int64_t tile = V.tile_base + (int64_t)(y / P.tile) * V.tiles_x + x / P.tile;
        const uint2 r = ranges[tile];
        if (r.y > r.x) continue;
        const int64_t HW = (int64_t)V.H * V.W;
        if (out_rgb) {
            float *o = out_rgb + 3 * V.pix_base + p;
            o[0] = P.bg[0];
            o[HW] = P.bg[1];
            o[2 * HW] = P.bg[2];
        }
        if (out_nrm) {
            float *o = out_nrm + 3 * V.pix_base + p;
            o[0] = 0.f;
            o[HW] = 0.f;
            o[2 * HW] = 0.f;
        }
        if (out_depth) out_depth[q] = 0.f;
        if (out_alpha) out_alpha[q] = 0.f;
        if (out_last) out_last[q] = 0u;
    }
}

int device_sms();

template <int B>
static cudaError_t launch_blend(const p2e_gaussians *g, const p2e_projected *proj,
                                const p2e_bins *bins, const Views &P, float *rgb, float *nrm,
                                float *depth, float *alpha, uint32_t *last, cudaStream_t st) {
    using S = BlendShape<B>;
    const size_t smem = sizeof(BlendSmem<B>);
    static int configured[64] = {0};
    static int per_sm[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = (dev >= 0 && dev < 64) ? dev : 0;
    if (!configured[slot]) {
        cudaError_t e = cudaFuncSetAttribute(blend_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, blend_kernel<B>, S::NT, smem);
        per_sm[slot] = nb > 0 ? nb : 1;
        configured[slot] = 1;
    }
    cudaError_t e = cudaMemsetAsync(bins->tile_work + 1, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int64_t total_pix = P.v[P.n_views - 1].pix_base +
                              (int64_t)P.v[P.n_views - 1].W * P.v[P.n_views - 1].H;
    const int sms = device_sms();
    fill_empty_kernel<<<sms * 8, 256, 0, st>>>((const uint2 *)bins->ranges, total_pix, rgb, nrm, depth,
                                               alpha, last, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t sub = P.tile / B;
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm[slot], P.total_tiles * sub * sub);
    blend_kernel<B><<<(unsigned)grid, S::NT, smem, st>>>(
        (const uint2 *)bins->ranges, bins->vals[bins->result], bins->tile_work, bins->tile_work + 1,
        (const float4 *)proj->xy_depth, (const float4 *)proj->conic_op, (const ushort4 *)proj->rect,
        (const float4 *)g->rgb, (const float4 *)g->normal, rgb, nrm, depth, alpha, last, P);
    return cudaGetLastError();
}

cudaError_t launch_render(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                          const Views &P, float *rgb, float *nrm, float *depth, float *alpha,
                          uint32_t *last, cudaStream_t st) {
    if (P.total_tiles == 0) return cudaSuccess;
    // pixel block of one CTA: 8 x 8 for binning tiles of 8 and 16 (a 16-tile
    // is shared by four CTAs, each screening the whole list against its
    // quarter), 16 x 16 for binning tiles of 32
    switch (P.tile) {
        case 8: return launch_blend<8>(g, proj, bins, P, rgb, nrm, depth, alpha, last, st);
        case 16: return launch_blend<8>(g, proj, bins, P, rgb, nrm, depth, alpha, last, st);
        case 32: return launch_blend<16>(g, proj, bins, P, rgb, nrm, depth, alpha, last, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace p2e
