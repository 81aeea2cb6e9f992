// Training kernels of the learned estimator (Sec. 3.3): the image loss of
// Eq. 5, the backward of the per-point network from the Gaussians'
// gradients, and Adam.  The renderer's own backward (backward.cu) supplies
// the Gaussians' gradients, so the network is trained end to end through
// the differentiable splatting.
//
// K13 loss_eq5:  L = w1 mean|I - I^| + w2 mean(|n x n^| + w3 min(|n - n^|, |n + n^|))
//                (mean over pixels, the L1 also over the 3 channels); writes
//                dL/dI^ and dL/dn^.
// K12 mlp_bwd:   per tile of 128 points: recompute the features and the
//                forward pass on tcgen05 (the inference head's bf16
//                roundings), back-propagate the output mapping (scale exp,
//                quaternion increment, opacity logit shift, normal = third
//                axis of R(q)) per thread, then the four layers on tcgen05
//                (bf16 operands, fp32 accumulation); weight and bias
//                gradients accumulate in TMEM per CTA and are added to the
//                global fp32 gradient once per CTA.
// K12 adam:      fp32 master weights, first/second moments, bias
//                correction; also writes the bf16 blob the forward reads.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "tcgen05.cuh"

namespace p2e {

constexpr int kIn = 96, kHid = 64, kOut = 8, kOutPad = 16, kNb = 16;
// fp32 parameter vector layout (same order as the blob): W1, W2, W3, W4 (16x64), b1, b2, b3, b4 (16)
constexpr int oW1 = 0, oW2 = oW1 + kHid * kIn, oW3 = oW2 + kHid * kHid, oW4 = oW3 + kHid * kHid,
              oB1 = oW4 + kOutPad * kHid, oB2 = oB1 + kHid, oB3 = oB2 + kHid, oB4 = oB3 + kHid,
              kNParams = oB4 + kOutPad;
static_assert(kNParams == P2E_MLP_PARAMS, "parameter layout of p2e.h");

// ------------------------------------------------------------------ loss
struct LossViews {
    int32_t n_views;
    int64_t hw[P2E_MAX_VIEWS];
    int64_t base[P2E_MAX_VIEWS];  // first pixel of the view
};

__global__ void __launch_bounds__(256) loss_eq5_kernel(const float *__restrict__ rgb, const float *__restrict__ nrm,
                                                       const float *__restrict__ grgb, const float *__restrict__ gnrm,
                                                       int64_t npix, float w1, float w2, float w3, float *loss,
                                                       float *__restrict__ d_rgb, float *__restrict__ d_nrm,
                                                       __grid_constant__ const LossViews V) {
    float acc = 0.f;
    const float inv = 1.f / (float)npix;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < V.n_views && V.base[v + 1] <= q) ++v;
        const int64_t p = q - V.base[v], HW = V.hw[v];
        const int64_t o = 3 * V.base[v] + p;
        float l1 = 0.f, a[3], b[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = rgb[o + c * HW] - grgb[o + c * HW];
            l1 += fabsf(d);
            d_rgb[o + c * HW] = w1 * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv * (1.f / 3.f);
            a[c] = gnrm[o + c * HW];  // n (ground truth)
            b[c] = nrm[o + c * HW];   // n^ (rendered)
        }
        const float cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
        const float cn = sqrtf(cx * cx + cy * cy + cz * cz);
        float dm[3], dp[3];
        for (int c = 0; c < 3; ++c) { dm[c] = b[c] - a[c]; dp[c] = b[c] + a[c]; }
        const float nm = sqrtf(dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]);
        const float np_ = sqrtf(dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
        const bool minus = nm <= np_;
        acc += w1 * l1 * (1.f / 3.f) + w2 * (cn + w3 * (minus ? nm : np_));
        // d|n x n^| / dn^ = (c x n) / |c| ; d|n^ -+ n| / dn^ = (n^ -+ n) / |n^ -+ n|
        float g[3] = {0.f, 0.f, 0.f};
        if (cn > 0.f) {
            g[0] = (cy * a[2] - cz * a[1]) / cn;
            g[1] = (cz * a[0] - cx * a[2]) / cn;
            g[2] = (cx * a[1] - cy * a[0]) / cn;
        }
        const float *dd = minus ? dm : dp;
        const float dn = minus ? nm : np_;
        if (dn > 0.f)
            for (int c = 0; c < 3; ++c) g[c] += w3 * dd[c] / dn;
        for (int c = 0; c < 3; ++c) d_nrm[o + c * HW] = w2 * g[c] * inv;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ float s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        atomicAdd(loss, t * inv);
    }
}

// ------------------------------------------------------------ SSIM term
// D = 1 - mean SSIM(I^, I) over every pixel and channel of the views, the
// structural term of an "L1 + SSIM" image loss, with its exact gradient
// with respect to the rendered image I^ (x; the target is y).  Per channel
// and pixel p, with an 11 x 11 Gaussian window w (sigma 1.5, normalised,
// zero outside the image):
//   mx = w * x, my = w * y, Exx = w * x^2, Eyy = w * y^2, Exy = w * xy,
//   vx = Exx - mx^2, vy = Eyy - my^2, cxy = Exy - mx my,
//   S = (2 mx my + C1)(2 cxy + C2) / ((mx^2 + my^2 + C1)(vx + vy + C2)),
//   C1 = 0.01^2, C2 = 0.03^2 (images in [0, 1]).
// dS_p/dx_q = w(p - q) (A_p + 2 x_q B_p + y_q C_p), A = dS/dmx, B = dS/dExx,
// C = dS/dExy, so dD/dx = -(w * A + 2 x (w * B) + y (w * C)) / N
// (w symmetric).  The blurs are separable (11 taps along a row, then along
// a column).  Two kernels, each over 32 x 16 output tiles of one (view,
// channel) plane with its 5-pixel halo staged in shared memory (zeros
// outside the image, which leave the window sums unchanged): the first
// takes the five window sums, S and the maps A, B, C; the second blurs A,
// B, C and adds the gradient.  Taps are summed in the same order (k = -5
// .. 5, row pass first) in both, one fma per tap.
constexpr int kSsimR = 5;                                  // window radius
constexpr int kSsimTX = 32, kSsimTY = 16;                  // output tile
constexpr int kSsimHX = kSsimTX + 2 * kSsimR, kSsimHY = kSsimTY + 2 * kSsimR;
constexpr int kSsimThreads = 256;

struct SsimViews {
    int32_t n_views;
    int32_t W[P2E_MAX_VIEWS], H[P2E_MAX_VIEWS];
    int64_t base[P2E_MAX_VIEWS];     // first pixel of the view
    int32_t tiles_x[P2E_MAX_VIEWS], tiles_y[P2E_MAX_VIEWS];
    int64_t block_base[P2E_MAX_VIEWS + 1];  // first block of the view (3 planes of tiles)
    int64_t npix;
    float w[2 * kSsimR + 1];
};

// The plane and output tile of block b: view v, channel c, tile origin.
struct SsimTile {
    int v, c, x0, y0, W, H;
    int64_t plane;  // offset of the (view, channel) plane
};
__device__ __forceinline__ SsimTile ssim_tile(const SsimViews &V, int64_t b) {
    SsimTile t;
    int v = 0;
    while (v + 1 < V.n_views && V.block_base[v + 1] <= b) ++v;
    const int64_t local = b - V.block_base[v];
    const int per_plane = V.tiles_x[v] * V.tiles_y[v];
    t.v = v;
    t.c = (int)(local / per_plane);
    const int k = (int)(local - (int64_t)t.c * per_plane);
    const int ty = k / V.tiles_x[v];
    t.x0 = (k - ty * V.tiles_x[v]) * kSsimTX;
    t.y0 = ty * kSsimTY;
    t.W = V.W[v];
    t.H = V.H[v];
    t.plane = 3 * V.base[v] + (int64_t)t.c * t.W * t.H;
    return t;
}

// Stage NP planes of the tile's halo region (zeros outside the image).
template <int NP>
__device__ __forceinline__ void ssim_stage(const SsimTile &t, const float *const (&src)[NP], int64_t stride,
                                           float (*dst)[kSsimHY][kSsimHX]) {
    for (int i = threadIdx.x; i < kSsimHY * kSsimHX; i += kSsimThreads) {
        const int r = i / kSsimHX, c = i - r * kSsimHX;
        const int gy = t.y0 - kSsimR + r, gx = t.x0 - kSsimR + c;
        const bool in = gy >= 0 && gy < t.H && gx >= 0 && gx < t.W;
        const int64_t o = t.plane + (int64_t)gy * t.W + gx;
#pragma unroll
        for (int p = 0; p < NP; ++p) dst[p][r][c] = in ? src[p][(int64_t)p * stride + o] : 0.f;
    }
}

// kernel 1: window sums, S (each block's sum added to an fp64 total) and
// A, B, C per pixel
__global__ void __launch_bounds__(kSsimThreads) ssim_stats_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ y,
                                                                  float *__restrict__ abc, double *s_total,
                                                                  __grid_constant__ const SsimViews V) {
    constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    __shared__ float s_in[2][kSsimHY][kSsimHX];
    __shared__ float s_row[5][kSsimHY][kSsimTX];
    __shared__ float s_red[kSsimThreads / 32];
    const SsimTile t = ssim_tile(V, blockIdx.x);
    {
        const float *const src[2] = {x, y};
        ssim_stage<2>(t, src, 0, s_in);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSsimHY * kSsimTX; i += kSsimThreads) {
        const int r = i / kSsimTX, c = i - r * kSsimTX;
        float s[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k <= 2 * kSsimR; ++k) {
            const float a = s_in[0][r][c + k], b = s_in[1][r][c + k];
            const float wk = V.w[k];
            s[0] = fmaf(wk, a, s[0]);
            s[1] = fmaf(wk, b, s[1]);
            s[2] = fmaf(wk, a * a, s[2]);
            s[3] = fmaf(wk, b * b, s[3]);
            s[4] = fmaf(wk, a * b, s[4]);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) s_row[j][r][c] = s[j];
    }
    __syncthreads();
    float acc = 0.f;
    for (int i = threadIdx.x; i < kSsimTY * kSsimTX; i += kSsimThreads) {
        const int r = i / kSsimTX, c = i - r * kSsimTX;
        const int gy = t.y0 + r, gx = t.x0 + c;
        if (gy >= t.H || gx >= t.W) continue;
        float m[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k <= 2 * kSsimR; ++k) {
            const float wk = V.w[k];
#pragma unroll
            for (int j = 0; j < 5; ++j) m[j] = fmaf(wk, s_row[j][r + k][c], m[j]);
        }
        const float mx = m[0], my = m[1];
        const float vx = m[2] - mx * mx, vy = m[3] - my * my, cxy = m[4] - mx * my;
        const float n1 = 2.f * mx * my + C1, n2 = 2.f * cxy + C2;
        const float d1 = mx * mx + my * my + C1, d2 = vx + vy + C2;
        const float S = (n1 * n2) / (d1 * d2);
        acc += S;
        const int64_t o = t.plane + (int64_t)gy * t.W + gx;
        abc[o] = S * (2.f * my / n1 - 2.f * my / n2 - 2.f * mx / d1 + 2.f * mx / d2);
        abc[3 * V.npix + o] = -S / d2;
        abc[6 * V.npix + o] = 2.f * S / n2;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int k = 0; k < kSsimThreads / 32; ++k) tsum += s_red[k];
        atomicAdd(s_total, tsum);
    }
}

// loss += weight (1 - mean S), one add of the whole term
__global__ void ssim_finish_kernel(float *loss, const double *s_total, float weight, int64_t n) {
    if (threadIdx.x == 0) atomicAdd(loss, (float)((double)weight * (1.0 - *s_total / (double)n)));
}

// kernel 2: d_rgb += weight dD/dx from the blurred A, B, C
__global__ void __launch_bounds__(kSsimThreads) ssim_grad_kernel(const float *__restrict__ x,
                                                                 const float *__restrict__ y,
                                                                 const float *__restrict__ abc, float weight,
                                                                 float *__restrict__ d_rgb,
                                                                 __grid_constant__ const SsimViews V) {
    __shared__ float s_in[3][kSsimHY][kSsimHX];
    __shared__ float s_row[3][kSsimHY][kSsimTX];
    const SsimTile t = ssim_tile(V, blockIdx.x);
    {
        const float *const src[3] = {abc, abc, abc};
        ssim_stage<3>(t, src, 3 * V.npix, s_in);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSsimHY * kSsimTX; i += kSsimThreads) {
        const int r = i / kSsimTX, c = i - r * kSsimTX;
        float s[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k <= 2 * kSsimR; ++k) {
            const float wk = V.w[k];
#pragma unroll
            for (int j = 0; j < 3; ++j) s[j] = fmaf(wk, s_in[j][r][c + k], s[j]);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) s_row[j][r][c] = s[j];
    }
    __syncthreads();
    const float scale = -weight / (float)(3 * V.npix);
    for (int i = threadIdx.x; i < kSsimTY * kSsimTX; i += kSsimThreads) {
        const int r = i / kSsimTX, c = i - r * kSsimTX;
        const int gy = t.y0 + r, gx = t.x0 + c;
        if (gy >= t.H || gx >= t.W) continue;
        float s[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k <= 2 * kSsimR; ++k) {
            const float wk = V.w[k];
#pragma unroll
            for (int j = 0; j < 3; ++j) s[j] = fmaf(wk, s_row[j][r + k][c], s[j]);
        }
        const int64_t o = t.plane + (int64_t)gy * t.W + gx;
        d_rgb[o] += scale * (s[0] + 2.f * x[o] * s[1] + y[o] * s[2]);
    }
}

size_t ssim_scratch_bytes(int64_t npix) { return (size_t)8 * 3 * (size_t)npix * sizeof(float); }

// ------------------------------------------------------------ MLP backward
// One 128-point tile per step (the UMMA M dimension), persistent CTAs of
// 128 threads (thread = point row), one CTA per SM (the weight gradients
// hold 416 TMEM columns).  All contractions run on tcgen05 (bf16 operands,
// fp32 accumulation in TMEM):
//   forward   H_l = bf16(relu(H_{l-1} W_l^T + b_l)), y = H_3 W_4^T + b_4, as
//             the inference head (same roundings)
//   output    dY = dL/dy through the output mapping (per thread, fp32),
//             rounded to bf16 for the products
//   backward  dH_{l-1} = dA_l W_l          (M = 128 points, K = out_l)
//             dA_{l-1} = dH_{l-1} (H_{l-1} > 0), bf16
//             [dW_l | db_l] += dA_l^T [H_{l-1} | 1]
//                                         (M = out_l padded to 128, K = 128
//                                          points, N = in_l + 16: a row of
//                                          ones gives the bias gradient)
// The [dW | db] accumulators stay in TMEM across the CTA's tiles and are
// added to the global fp32 gradient once per CTA.  Operands whose
// contraction runs over the points are written transposed (point-major ->
// unit-major) by the epilogues; an A operand with fewer than 128 real rows
// reads its padding rows from the next buffer (their products land in TMEM
// lanes that are never read).
// status of the last training backward on this device (P2E_OK, or
// P2E_ERR_TIMEOUT when a bounded wait gave up)
static __device__ int32_t g_train_status;

constexpr int kBT = 128;
constexpr int kInB = kIn + 16, kHidB = kHid + 16;   // B operands with the ones row (and zero padding)
constexpr uint32_t kBwdCols = 512;
constexpr uint32_t kColAcc = 0, kColW1 = 64, kColW2 = 192, kColW3 = 288, kColW4 = 384;

struct __align__(128) TrainSmem {
    __nv_bfloat16 W1[kHid * kIn], W2[kHid * kHid], W3[kHid * kHid], W4[kOutPad * kHid];   // forward B
    __nv_bfloat16 W2T[kHid * kHid], W3T[kHid * kHid], W4T[kHid * kOutPad];                 // backward B
    __nv_bfloat16 R[kBT * kIn];          // X, then H1..H3, then dA3, dA2 (point-major)
    __nv_bfloat16 dY[kBT * kOutPad];     // point-major
    __nv_bfloat16 dYT[kOutPad * kBT];    // unit-major; as a 128-row A operand it reads on into dAT, XT
    __nv_bfloat16 dAT[kHid * kBT];       // unit-major; its padding rows read on into XT
    __nv_bfloat16 XT[kInB * kBT];        // rows 96: ones, 97..111: zero
    __nv_bfloat16 HT[3][kHidB * kBT];    // rows 64: ones, 65..79: zero
    float b[3 * kHid + kOutPad];
    uint64_t bar;
    uint32_t tmem;
    int err;
};
static_assert(sizeof(TrainSmem) + 1024 <= 227 * 1024, "shared memory of the training backward");

__device__ __forceinline__ float4 qmul4(float4 a, float4 b) {
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y, a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

// value v of (unit c, point r) into a unit-major [rows][128] operand
__device__ __forceinline__ void put_t(__nv_bfloat16 *T, int c, int r, __nv_bfloat16 v) {
    T[core_off(c, r, kBT)] = v;
}

__global__ void __launch_bounds__(kBT, 1) mlp_bwd_kernel(
    const float4 *__restrict__ xyz, const float4 *__restrict__ rgb, int64_t n, const uint32_t *__restrict__ knn,
    const float4 *__restrict__ pca_scale, const float4 *__restrict__ pca_quat, float opacity0,
    const unsigned char *__restrict__ blob, const float *__restrict__ d_scale, const float *__restrict__ d_quat,
    const float *__restrict__ d_opacity, const float *__restrict__ d_normal, float *__restrict__ grad,
    int32_t *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TrainSmem &sm = *reinterpret_cast<TrainSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t ntiles = (n + kBT - 1) / kBT;

    // ---- weights: forward B operands W_l [out][in] and backward B
    // operands W_l^T [in][out], core-matrix layout, from the bf16 blob
    {
        const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(blob);
        for (int t = tid; t < kHid * kIn; t += kBT) {
            const int o = t / kIn, i = t % kIn;
            sm.W1[core_off(o, i, kIn)] = wb[oW1 + t];
        }
        for (int t = tid; t < kHid * kHid; t += kBT) {
            const int o = t / kHid, i = t % kHid;
            sm.W2[core_off(o, i, kHid)] = wb[oW2 + t];
            sm.W3[core_off(o, i, kHid)] = wb[oW3 + t];
            sm.W2T[core_off(i, o, kHid)] = wb[oW2 + t];
            sm.W3T[core_off(i, o, kHid)] = wb[oW3 + t];
        }
        for (int t = tid; t < kOutPad * kHid; t += kBT) {
            const int o = t / kHid, i = t % kHid;
            sm.W4[core_off(o, i, kHid)] = wb[oW4 + t];
            sm.W4T[core_off(i, o, kOutPad)] = wb[oW4 + t];
        }
        const float *bb = reinterpret_cast<const float *>(blob + 2 * oB1);
        for (int t = tid; t < 3 * kHid + kOutPad; t += kBT) sm.b[t] = bb[t];
        // the ones rows of the [H | 1] operands (rows in_l .. in_l + 15:
        // one row of ones, fifteen of zeros), written once
        const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
        for (int t = tid; t < 16 * kBT; t += kBT) {
            const int c = t / kBT, r = t % kBT;
            const __nv_bfloat16 v = c == 0 ? one : zero;
            put_t(sm.XT, kIn + c, r, v);
            for (int l = 0; l < 3; ++l) put_t(sm.HT[l], kHid + c, r, v);
        }
        // the dY operand's padding columns 8..15 stay zero
        for (int t = tid; t < kBT * kOutPad; t += kBT) sm.dY[t] = zero;
        for (int t = tid; t < kOutPad * kBT; t += kBT) sm.dYT[t] = zero;
    }
    if (tid == 0) {
        sm.err = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(kBwdCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    // issue (thread 0), commit, wait (everyone), uniform verdict
    auto run = [&](auto &&issue) {
        if (!ok) return;  // after a wait gave up nothing more is issued
        if (tid == 0) {
            tc_fence_after();
            issue();
            umma_commit(&sm.bar);
        }
        const bool w = mbar_wait(&sm.bar, phase);
        phase ^= 1u;
        tc_fence_after();
        ok = ok && !__syncthreads_or(!w);
    };
    // generic stores into operands -> visible to the tensor cores
    auto publish = [&]() {
        proxy_fence();
        tc_fence_before();
        __syncthreads();
    };

    bool first = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t i = tile * kBT + tid;
        const bool live = i < n;
        // ---- features of point i (bf16-rounded as the forward rounds them)
        float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), q0 = make_float4(1.f, 0.f, 0.f, 0.f);
        {
            float f[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) f[k] = 0.f;
            if (live) {
                const float4 p = __ldg(xyz + i), c = __ldg(rgb + i);
                q0 = __ldg(pca_quat + i);
                s0 = __ldg(pca_scale + i);
                const uint4 *kp = reinterpret_cast<const uint4 *>(knn + i * kNb);
                uint32_t nb[kNb];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 u = __ldg(kp + k);
                    nb[4 * k] = u.x; nb[4 * k + 1] = u.y; nb[4 * k + 2] = u.z; nb[4 * k + 3] = u.w;
                }
                float4 pn[kNb], cn[kNb];
#pragma unroll
                for (int u = 0; u < kNb; ++u) {
                    pn[u] = __ldg(xyz + nb[u]);
                    cn[u] = __ldg(rgb + nb[u]);
                }
                const float w = q0.x, x = q0.y, y = q0.z, z = q0.w;
                const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z), R02 = 2.f * (x * z + w * y);
                const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z), R12 = 2.f * (y * z - w * x);
                const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x), R22 = 1.f - 2.f * (x * x + y * y);
                const float lx = pn[kNb - 1].x - p.x, ly = pn[kNb - 1].y - p.y, lz = pn[kNb - 1].z - p.z;
                const float inv_r = 1.f / fmaxf(sqrtf(lx * lx + ly * ly + lz * lz), 1e-12f);
#pragma unroll
                for (int u = 0; u < kNb; ++u) {
                    const float dx = pn[u].x - p.x, dy = pn[u].y - p.y, dz = pn[u].z - p.z;
                    f[6 * u + 0] = (R00 * dx + R10 * dy + R20 * dz) * inv_r;
                    f[6 * u + 1] = (R01 * dx + R11 * dy + R21 * dz) * inv_r;
                    f[6 * u + 2] = (R02 * dx + R12 * dy + R22 * dz) * inv_r;
                    f[6 * u + 3] = cn[u].x - c.x;
                    f[6 * u + 4] = cn[u].y - c.y;
                    f[6 * u + 5] = cn[u].z - c.z;
                }
            }
#pragma unroll
            for (int k = 0; k < kIn; k += 8) {
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[k + 2 * e], f[k + 2 * e + 1]);
                    wv[e] = *reinterpret_cast<const uint32_t *>(&b2);
                    put_t(sm.XT, k + 2 * e, tid, b2.x);
                    put_t(sm.XT, k + 2 * e + 1, tid, b2.y);
                }
                *reinterpret_cast<uint4 *>(sm.R + core_off(tid, k, kIn)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        publish();
        // ---- forward: three hidden layers, ReLU masks kept per thread
        uint32_t mask[3][2];
        const __nv_bfloat16 *Wf[3] = {sm.W1, sm.W2, sm.W3};
        for (int L = 0; L < 3; ++L) {
            run([&] { umma_chain(tmem + kColAcc, sm.R, Wf[L], kBT, L == 0 ? kIn : kHid, kHid, false); });
            float v[kHid];
            tmem_ld64(tmem + lane_base + kColAcc, v);
            mask[L][0] = mask[L][1] = 0u;
#pragma unroll
            for (int c = 0; c < kHid; c += 8) {
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = c + 2 * e;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(fmaxf(v[k] + sm.b[L * kHid + k], 0.f),
                                                                    fmaxf(v[k + 1] + sm.b[L * kHid + k + 1], 0.f));
                    wv[e] = *reinterpret_cast<const uint32_t *>(&b2);
                    put_t(sm.HT[L], k, tid, b2.x);
                    put_t(sm.HT[L], k + 1, tid, b2.y);
                    if (__bfloat162float(b2.x) > 0.f) mask[L][k >> 5] |= 1u << (k & 31);
                    if (__bfloat162float(b2.y) > 0.f) mask[L][(k + 1) >> 5] |= 1u << ((k + 1) & 31);
                }
                *reinterpret_cast<uint4 *>(sm.R + core_off(tid, c, kHid)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            publish();
        }
        run([&] { umma_chain(tmem + kColAcc, sm.R, sm.W4, kBT, kHid, kOutPad, false); });
        // ---- output mapping backward -> dY (fp32, then bf16 operands)
        {
            float yv[16];
            tmem_ld16(tmem + lane_base + kColAcc, yv);
            float dy[kOut];
#pragma unroll
            for (int e = 0; e < kOut; ++e) dy[e] = 0.f;
            if (live) {
                float y[kOut];
#pragma unroll
                for (int e = 0; e < kOut; ++e) y[e] = yv[e] + sm.b[3 * kHid + e];
                const float s0v[3] = {s0.x, s0.y, s0.z};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float yc = fminf(fmaxf(y[k], -4.f), 4.f);
                    dy[k] = (y[k] > -4.f && y[k] < 4.f) ? d_scale[3 * i + k] * s0v[k] * __expf(yc) : 0.f;
                }
                float4 dq = make_float4(1.f + y[3], y[4], y[5], y[6]);
                const float dnorm = sqrtf(fmaxf(dq.x * dq.x + dq.y * dq.y + dq.z * dq.z + dq.w * dq.w, 1e-30f));
                const float4 dh = make_float4(dq.x / dnorm, dq.y / dnorm, dq.z / dnorm, dq.w / dnorm);
                const float4 qf = qmul4(q0, dh);
                // dL/dqf from the renderer's quaternion and from normal = third axis of R(qf)
                const float W = qf.x, X = qf.y, Y = qf.z, Z = qf.w;
                const float gn0 = d_normal[3 * i], gn1 = d_normal[3 * i + 1], gn2 = d_normal[3 * i + 2];
                float g[4] = {d_quat[4 * i], d_quat[4 * i + 1], d_quat[4 * i + 2], d_quat[4 * i + 3]};
                g[0] += 2.f * Y * gn0 - 2.f * X * gn1;
                g[1] += 2.f * Z * gn0 - 2.f * W * gn1 - 4.f * X * gn2;
                g[2] += 2.f * W * gn0 + 2.f * Z * gn1 - 4.f * Y * gn2;
                g[3] += 2.f * X * gn0 + 2.f * Y * gn1;
                // qf = L(q0) dh  ->  dL/ddh = L(q0)^T dL/dqf
                const float a0 = q0.x, a1 = q0.y, a2 = q0.z, a3 = q0.w;
                const float gh[4] = {a0 * g[0] + a1 * g[1] + a2 * g[2] + a3 * g[3],
                                     -a1 * g[0] + a0 * g[1] + a3 * g[2] - a2 * g[3],
                                     -a2 * g[0] - a3 * g[1] + a0 * g[2] + a1 * g[3],
                                     -a3 * g[0] + a2 * g[1] - a1 * g[2] + a0 * g[3]};
                const float hv[4] = {dh.x, dh.y, dh.z, dh.w};
                const float dot = hv[0] * gh[0] + hv[1] * gh[1] + hv[2] * gh[2] + hv[3] * gh[3];
#pragma unroll
                for (int k = 0; k < 4; ++k) dy[3 + k] = (gh[k] - hv[k] * dot) / dnorm;
                const float o0 = fminf(fmaxf(opacity0, 1e-6f), 1.f - 1e-6f);
                const float o = 1.f / (1.f + __expf(-(__logf(o0 / (1.f - o0)) + y[7])));
                dy[7] = d_opacity[i] * o * (1.f - o);
            }
            uint32_t wv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(dy[2 * e], dy[2 * e + 1]);
                wv[e] = *reinterpret_cast<const uint32_t *>(&b2);
                put_t(sm.dYT, 2 * e, tid, b2.x);
                put_t(sm.dYT, 2 * e + 1, tid, b2.y);
            }
            *reinterpret_cast<uint4 *>(sm.dY + core_off(tid, 0, kOutPad)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        publish();
        // ---- layer 4: dH3 = dY W4 ; [dW4 | db4] += dY^T [H3 | 1]
        run([&] {
            umma_chain(tmem + kColAcc, sm.dY, sm.W4T, kBT, kOutPad, kHid, false);
            umma_chain(tmem + kColW4, sm.dYT, sm.HT[2], kBT, kBT, kHidB, !first);
        });
        // ---- layers 3, 2: dA_l = dH_l (H_l > 0); dH_{l-1} = dA_l W_l ;
        // [dW_l | db_l] += dA_l^T [H_{l-1} | 1]
        const __nv_bfloat16 *WT[3] = {nullptr, sm.W2T, sm.W3T};
        const uint32_t colW[3] = {kColW1, kColW2, kColW3};
        for (int L = 2; L >= 0; --L) {
            float v[kHid];
            tmem_ld64(tmem + lane_base + kColAcc, v);
#pragma unroll
            for (int c = 0; c < kHid; c += 8) {
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = c + 2 * e;
                    const float g0 = (mask[L][k >> 5] >> (k & 31)) & 1u ? v[k] : 0.f;
                    const float g1 = (mask[L][(k + 1) >> 5] >> ((k + 1) & 31)) & 1u ? v[k + 1] : 0.f;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(g0, g1);
                    wv[e] = *reinterpret_cast<const uint32_t *>(&b2);
                    put_t(sm.dAT, k, tid, b2.x);
                    put_t(sm.dAT, k + 1, tid, b2.y);
                }
                if (L > 0)
                    *reinterpret_cast<uint4 *>(sm.R + core_off(tid, c, kHid)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            publish();
            run([&] {
                if (L > 0) umma_chain(tmem + kColAcc, sm.R, WT[L], kBT, kHid, kHid, false);
                umma_chain(tmem + colW[L], sm.dAT, L > 0 ? sm.HT[L - 1] : sm.XT, kBT, kBT, L > 0 ? kHidB : kInB,
                           !first);
            });
        }
        first = false;
    }
    // ---- once per CTA: [dW | db] rows 0..63 (TMEM lanes of warps 0, 1)
    if (ok && warp < 2 && !first) {
        const int row = tid;  // output unit
        float v[64], u[32], w16[16];
        // layer 1: 96 weight columns, then the bias column
        tmem_ld64(tmem + lane_base + kColW1, v);
        tmem_ld32(tmem + lane_base + kColW1 + 64, u);
        tmem_ld16(tmem + lane_base + kColW1 + 96, w16);
        for (int c = 0; c < 64; ++c) atomicAdd(&grad[oW1 + row * kIn + c], v[c]);
        for (int c = 0; c < 32; ++c) atomicAdd(&grad[oW1 + row * kIn + 64 + c], u[c]);
        atomicAdd(&grad[oB1 + row], w16[0]);
        const uint32_t cols[2] = {kColW2, kColW3};
        const int offs[2] = {oW2, oW3}, boffs[2] = {oB2, oB3};
        for (int l = 0; l < 2; ++l) {
            tmem_ld64(tmem + lane_base + cols[l], v);
            tmem_ld16(tmem + lane_base + cols[l] + 64, w16);
            for (int c = 0; c < 64; ++c) atomicAdd(&grad[offs[l] + row * kHid + c], v[c]);
            atomicAdd(&grad[boffs[l] + row], w16[0]);
        }
        tmem_ld64(tmem + lane_base + kColW4, v);
        tmem_ld16(tmem + lane_base + kColW4 + 64, w16);
        if (row < kOut) {
            for (int c = 0; c < 64; ++c) atomicAdd(&grad[oW4 + row * kHid + c], v[c]);
            atomicAdd(&grad[oB4 + row], w16[0]);
        }
    } else if (!ok && tid == 0) {
        atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
        mbar_wait(&sm.bar, phase ^ 1u);  // let an overdue MMA finish (bounded)
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBwdCols) : "memory");
    }
}

// ------------------------------------------------------------------ Adam
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ p, float *__restrict__ g,
                                                   float *__restrict__ m, float *__restrict__ v, int64_t count,
                                                   float lr, float b1, float b2, float eps, float c1, float c2,
                                                   unsigned char *__restrict__ blob) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const bool pad = (t >= oW4 + kOut * kHid && t < oB1) || (t >= oB4 + kOut);  // W4/b4 rows 8..15
        float x = p[t];
        if (!pad) {
            const float gg = g[t];
            const float mm = b1 * m[t] + (1.f - b1) * gg;
            const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
            m[t] = mm;
            v[t] = vv;
            x -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        } else {
            x = 0.f;
        }
        p[t] = x;
        g[t] = 0.f;
        if (blob) {
            if (t < oB1) reinterpret_cast<__nv_bfloat16 *>(blob)[t] = __float2bfloat16_rn(x);
            else reinterpret_cast<float *>(blob + 2 * oB1)[t - oB1] = x;
        }
    }
}

int device_sms();

}  // namespace p2e

using namespace p2e;

extern "C" {

p2e_status p2e_loss_eq5(const float *rgb, const float *normal, const float *gt_rgb, const float *gt_normal,
                        const int64_t *view_pixels, int32_t n_views, float w1, float w2, float w3,
                        float *loss_dev, float *d_rgb, float *d_normal, void *stream) {
    if (!rgb || !normal || !gt_rgb || !gt_normal || !view_pixels || !loss_dev || !d_rgb || !d_normal)
        return P2E_ERR_INVALID_ARG;
    if (n_views < 1 || n_views > P2E_MAX_VIEWS) return P2E_ERR_INVALID_ARG;
    LossViews V;
    V.n_views = n_views;
    int64_t tot = 0;
    for (int v = 0; v < n_views; ++v) {
        if (view_pixels[v] < 1) return P2E_ERR_INVALID_ARG;
        V.hw[v] = view_pixels[v];
        V.base[v] = tot;
        tot += view_pixels[v];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss_dev, 0, sizeof(float), st) != cudaSuccess) return P2E_ERR_CUDA;
    loss_eq5_kernel<<<device_sms() * 4, 256, 0, st>>>(rgb, normal, gt_rgb, gt_normal, tot, w1, w2, w3, loss_dev,
                                                      d_rgb, d_normal, V);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

p2e_status p2e_loss_ssim(const float *rgb, const float *gt_rgb, const int32_t *view_hw, int32_t n_views,
                         float weight, float *loss_dev, float *d_rgb, void *scratch, int64_t scratch_bytes,
                         void *stream) {
    if (!rgb || !gt_rgb || !view_hw || !loss_dev || !d_rgb || !scratch) return P2E_ERR_INVALID_ARG;
    if (n_views < 1 || n_views > P2E_MAX_VIEWS || !(weight == weight)) return P2E_ERR_INVALID_ARG;
    if (((uintptr_t)scratch & 255u)) return P2E_ERR_INVALID_ARG;
    SsimViews V;
    memset(&V, 0, sizeof V);
    V.n_views = n_views;
    int64_t tot = 0;
    for (int v = 0; v < n_views; ++v) {
        const int32_t h = view_hw[2 * v], w = view_hw[2 * v + 1];
        if (h < 1 || w < 1 || h > 8192 || w > 8192) return P2E_ERR_INVALID_ARG;
        V.H[v] = h;
        V.W[v] = w;
        V.base[v] = tot;
        tot += (int64_t)h * w;
    }
    V.npix = tot;
    if (scratch_bytes < (int64_t)ssim_scratch_bytes(tot)) return P2E_ERR_INVALID_ARG;
    double ws = 0.0;
    for (int k = -kSsimR; k <= kSsimR; ++k) ws += exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
    for (int k = -kSsimR; k <= kSsimR; ++k) V.w[k + kSsimR] = (float)(exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)) / ws);
    float *abc = (float *)scratch;  // A, B, C: 3 planes x 3 channels, then the fp64 sum of S
    double *s_total = (double *)((char *)scratch + (((size_t)9 * tot * sizeof(float) + 7) & ~(size_t)7));
    int64_t blocks = 0;
    for (int v = 0; v < n_views; ++v) {
        V.tiles_x[v] = (V.W[v] + kSsimTX - 1) / kSsimTX;
        V.tiles_y[v] = (V.H[v] + kSsimTY - 1) / kSsimTY;
        V.block_base[v] = blocks;
        blocks += 3 * (int64_t)V.tiles_x[v] * V.tiles_y[v];
    }
    V.block_base[n_views] = blocks;
    if (blocks > 0x7fffffff) return P2E_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(s_total, 0, sizeof(double), st) != cudaSuccess) return P2E_ERR_CUDA;
    ssim_stats_kernel<<<(unsigned)blocks, kSsimThreads, 0, st>>>(rgb, gt_rgb, abc, s_total, V);
    ssim_finish_kernel<<<1, 32, 0, st>>>(loss_dev, s_total, weight, 3 * tot);
    ssim_grad_kernel<<<(unsigned)blocks, kSsimThreads, 0, st>>>(rgb, gt_rgb, abc, weight, d_rgb, V);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

// Area term: A = weight mean_i (s_i0 s_i1) / (r_i0 r_i1), the footprint of
// each estimated splat relative to the reference estimate's; dA/ds_i0 =
// (weight / n) g_i / s_i0 and likewise for s_i1 (g_i the ratio), added to
// d_scale.  A point whose reference area is not positive and finite adds
// nothing.  The loss is summed per block (one atomic per block).
__global__ void __launch_bounds__(256) splat_area_kernel(const float4 *__restrict__ scale,
                                                         const float4 *__restrict__ ref, int64_t n, float wn,
                                                         float *__restrict__ loss_dev, float *__restrict__ d_scale) {
    __shared__ float s_part[8];
    float part = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 s = __ldg(scale + i), r = __ldg(ref + i);
        const float ra = r.x * r.y;
        if (!(ra > 0.f) || !(ra < INFINITY)) continue;
        const float g = (s.x * s.y) / ra;
        part += g;
        d_scale[3 * i] += wn * (s.y / ra);
        d_scale[3 * i + 1] += wn * (s.x / ra);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_part[k];
        atomicAdd(loss_dev, wn * t);
    }
}

p2e_status p2e_loss_splat_area(const float *scale, const float *ref_scale, int64_t n, float weight, float *loss_dev,
                               float *d_scale, void *stream) {
    if (!scale || !ref_scale || !loss_dev || !d_scale || n < 1 || !(weight >= 0.f) || !(weight < INFINITY))
        return P2E_ERR_INVALID_ARG;
    if (((uintptr_t)scale & 15u) || ((uintptr_t)ref_scale & 15u)) return P2E_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 8);
    splat_area_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const float4 *)scale, (const float4 *)ref_scale, n,
                                                              weight / (float)n, loss_dev, d_scale);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

p2e_status p2e_mlp_backward(const float *xyz, const float *rgb, int64_t n, const uint32_t *knn_idx,
                            const p2e_gaussians *pca, const void *mlp_weights, const float *d_scale,
                            const float *d_quat, const float *d_opacity, const float *d_normal, float *grad,
                            void *stream) {
    if (n < 1 || n >= (int64_t(1) << 31) || !xyz || !rgb || !knn_idx || !pca || !pca->scale || !pca->quat ||
        !pca->mean_op || !mlp_weights || !d_scale || !d_quat || !d_opacity || !d_normal || !grad)
        return P2E_ERR_INVALID_ARG;
    if (((uintptr_t)knn_idx & 15u) || ((uintptr_t)mlp_weights & 15u)) return P2E_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = sizeof(TrainSmem) + 1024;
    static int configured[64] = {0};
    static int32_t *status_addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return P2E_ERR_CUDA;
    if (!configured[dev]) {
        if (cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return P2E_ERR_CUDA;
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_train_status) != cudaSuccess || !ptr) return P2E_ERR_CUDA;
        status_addr[dev] = (int32_t *)ptr;
        configured[dev] = 1;
    }
    int32_t *status = status_addr[dev];
    const int64_t ntiles = (n + kBT - 1) / kBT;
    // one CTA per SM: its weight-gradient accumulators take 416 of the 512
    // TMEM columns
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)device_sms());
    // opacity of the PCA estimate is the same for every point (mean_op.w)
    float o0 = 0.9f;
    if (cudaMemcpyAsync(&o0, pca->mean_op + 3, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return P2E_ERR_CUDA;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return P2E_ERR_CUDA;
    mlp_bwd_kernel<<<grid, kBT, smem, st>>>((const float4 *)xyz, (const float4 *)rgb, n, knn_idx,
                                           (const float4 *)pca->scale, (const float4 *)pca->quat, o0,
                                           (const unsigned char *)mlp_weights, d_scale, d_quat, d_opacity, d_normal,
                                           grad, status);
    if (cudaGetLastError() != cudaSuccess) return P2E_ERR_CUDA;
    int32_t hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof hs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return P2E_ERR_CUDA;
    return hs != 0 ? (p2e_status)hs : P2E_OK;
}

p2e_status p2e_adam(float *params, float *grad, float *m, float *v, int64_t count, float lr, float beta1,
                    float beta2, float eps, int32_t step, void *blob, void *stream) {
    if (!params || !grad || !m || !v || count != kNParams || step < 1) return P2E_ERR_INVALID_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        params, grad, m, v, count, lr, beta1, beta2, eps, c1, c2, (unsigned char *)blob);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

}  // extern "C"
