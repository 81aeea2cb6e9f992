// Training kernels of the learned estimator (Sec. 3.3): the image loss of
// Eq. 5, the backward of the per-point network from the Gaussians'
// gradients, and Adam.  The renderer's own backward (backward.cu) supplies
// the Gaussians' gradients, so the network is trained end to end through
// the differentiable splatting.
//
// K13 loss_eq5:  L = w1 mean|I - I^| + w2 mean(|n x n^| + w3 min(|n - n^|, |n + n^|))
//                (mean over pixels, the L1 also over the 3 channels); writes
//                dL/dI^ and dL/dn^.
// K12 mlp_bwd:   per tile of 32 points: recompute the features and the
//                forward pass (bf16-rounded operands and activations, fp32
//                sums, as the tensor-core kernel), back-propagate the output
//                mapping (scale exp, quaternion increment, opacity logit
//                shift, normal = third axis of R(q)) and the four layers
//                with register-tiled shared-memory products; weight
//                gradients accumulate in shared memory per CTA and are added
//                to the global fp32 gradient once per CTA.
// K12 adam:      fp32 master weights, first/second moments, bias
//                correction; also writes the bf16 blob the forward reads.
#include <cuda_bf16.h>

#include "common.cuh"

namespace p2e {

constexpr int kIn = 96, kHid = 64, kOut = 8, kOutPad = 16, kNb = 16;
constexpr int kP = 32;  // points per tile
constexpr int kNT = 256;
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

// ------------------------------------------------------------ MLP backward
__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C[m][n] (+)= sum_k A[m*asm + k*ask] B[k*bsk + n*bsn], each thread a TM x TN block
template <int M, int N, int K, int TM, int TN>
__device__ __forceinline__ void sgemm(const float *A, int asm_, int ask, const float *B, int bsk, int bsn,
                                      float *C, int ldc, bool acc) {
    constexpr int BM = M / TM, BN = N / TN;
    for (int blk = threadIdx.x; blk < BM * BN; blk += kNT) {
        const int m0 = (blk / BN) * TM, n0 = (blk % BN) * TN;
        float c[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) c[i][j] = acc ? C[(m0 + i) * ldc + n0 + j] : 0.f;
        for (int k = 0; k < K; ++k) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = A[(m0 + i) * asm_ + k * ask];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = B[k * bsk + (n0 + j) * bsn];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) c[i][j] = fmaf(a[i], b[j], c[i][j]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) C[(m0 + i) * ldc + n0 + j] = c[i][j];
    }
}

struct BwdSmem {
    float W1[kHid * kIn], W2[kHid * kHid], W3[kHid * kHid], W4[kOut * kHid];
    float b[3 * kHid + kOut];
    float X[kP * kIn];
    float H1[kP * kHid], H2[kP * kHid], H3[kP * kHid];
    float G1[kP * kHid], G2[kP * kHid];
    float Y[kP * kOutPad], dY[kP * kOutPad];
    float dW1[kHid * kIn], dW2[kHid * kHid], dW3[kHid * kHid], dW4[kOut * kHid];
    float db[3 * kHid + kOut];
};

__device__ __forceinline__ float4 qmul4(float4 a, float4 b) {
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y, a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

__global__ void __launch_bounds__(kNT) mlp_bwd_kernel(
    const float4 *__restrict__ xyz, const float4 *__restrict__ rgb, int64_t n, const uint32_t *__restrict__ knn,
    const float4 *__restrict__ pca_scale, const float4 *__restrict__ pca_quat, float opacity0,
    const unsigned char *__restrict__ blob, const float *__restrict__ d_scale, const float *__restrict__ d_quat,
    const float *__restrict__ d_opacity, const float *__restrict__ d_normal, float *__restrict__ grad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem &sm = *reinterpret_cast<BwdSmem *>(smem_raw);
    const int tid = threadIdx.x;
    // bf16 weights -> fp32 shared memory; zero the accumulators
    {
        const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(blob);
        for (int t = tid; t < kHid * kIn; t += kNT) sm.W1[t] = __bfloat162float(wb[oW1 + t]);
        for (int t = tid; t < kHid * kHid; t += kNT) {
            sm.W2[t] = __bfloat162float(wb[oW2 + t]);
            sm.W3[t] = __bfloat162float(wb[oW3 + t]);
        }
        for (int t = tid; t < kOut * kHid; t += kNT) sm.W4[t] = __bfloat162float(wb[oW4 + t]);
        const float *bb = reinterpret_cast<const float *>(blob + 2 * oB1);
        for (int t = tid; t < 3 * kHid; t += kNT) sm.b[t] = bb[t];
        for (int t = tid; t < kOut; t += kNT) sm.b[3 * kHid + t] = bb[3 * kHid + t];
        for (int t = tid; t < kHid * kIn; t += kNT) sm.dW1[t] = 0.f;
        for (int t = tid; t < kHid * kHid; t += kNT) { sm.dW2[t] = 0.f; sm.dW3[t] = 0.f; }
        for (int t = tid; t < kOut * kHid; t += kNT) sm.dW4[t] = 0.f;
        for (int t = tid; t < 3 * kHid + kOut; t += kNT) sm.db[t] = 0.f;
    }
    __syncthreads();
    const int64_t ntiles = (n + kP - 1) / kP;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- features: 8 threads per point, 2 neighbours each
        {
            const int pt = tid >> 3, part = tid & 7;
            const int64_t i = tile * kP + pt;
            float *xr = sm.X + pt * kIn;
            if (i < n) {
                const float4 p = __ldg(xyz + i), c = __ldg(rgb + i), q = __ldg(pca_quat + i);
                const float w = q.x, x = q.y, y = q.z, z = q.w;
                const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z), R02 = 2.f * (x * z + w * y);
                const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z), R12 = 2.f * (y * z - w * x);
                const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x), R22 = 1.f - 2.f * (x * x + y * y);
                const float4 pl = __ldg(xyz + knn[i * kNb + kNb - 1]);
                const float lx = pl.x - p.x, ly = pl.y - p.y, lz = pl.z - p.z;
                const float inv_r = 1.f / fmaxf(sqrtf(lx * lx + ly * ly + lz * lz), 1e-12f);
                for (int u = 0; u < 2; ++u) {
                    const int k = part * 2 + u;
                    const uint32_t j = knn[i * kNb + k];
                    const float4 pj = __ldg(xyz + j), cj = __ldg(rgb + j);
                    const float dx = pj.x - p.x, dy = pj.y - p.y, dz = pj.z - p.z;
                    xr[6 * k + 0] = bfr((R00 * dx + R10 * dy + R20 * dz) * inv_r);
                    xr[6 * k + 1] = bfr((R01 * dx + R11 * dy + R21 * dz) * inv_r);
                    xr[6 * k + 2] = bfr((R02 * dx + R12 * dy + R22 * dz) * inv_r);
                    xr[6 * k + 3] = bfr(cj.x - c.x);
                    xr[6 * k + 4] = bfr(cj.y - c.y);
                    xr[6 * k + 5] = bfr(cj.z - c.z);
                }
            } else {
                for (int k = part * 12; k < part * 12 + 12; ++k) xr[k] = 0.f;
            }
        }
        __syncthreads();
        // ---- forward (fp32 sums of bf16-rounded operands)
        sgemm<kP, kHid, kIn, 2, 4>(sm.X, kIn, 1, sm.W1, 1, kIn, sm.H1, kHid, false);
        __syncthreads();
        for (int t = tid; t < kP * kHid; t += kNT) sm.H1[t] = bfr(fmaxf(sm.H1[t] + sm.b[t % kHid], 0.f));
        __syncthreads();
        sgemm<kP, kHid, kHid, 2, 4>(sm.H1, kHid, 1, sm.W2, 1, kHid, sm.H2, kHid, false);
        __syncthreads();
        for (int t = tid; t < kP * kHid; t += kNT) sm.H2[t] = bfr(fmaxf(sm.H2[t] + sm.b[kHid + t % kHid], 0.f));
        __syncthreads();
        sgemm<kP, kHid, kHid, 2, 4>(sm.H2, kHid, 1, sm.W3, 1, kHid, sm.H3, kHid, false);
        __syncthreads();
        for (int t = tid; t < kP * kHid; t += kNT) sm.H3[t] = bfr(fmaxf(sm.H3[t] + sm.b[2 * kHid + t % kHid], 0.f));
        __syncthreads();
        sgemm<kP, kOut, kHid, 1, 1>(sm.H3, kHid, 1, sm.W4, 1, kHid, sm.Y, kOutPad, false);
        __syncthreads();
        // ---- output mapping backward -> dY (one thread per point)
        if (tid < kP) {
            const int64_t i = tile * kP + tid;
            float *dy = sm.dY + tid * kOutPad;
            for (int e = 0; e < kOutPad; ++e) dy[e] = 0.f;
            if (i < n) {
                float y[kOut];
                for (int e = 0; e < kOut; ++e) y[e] = sm.Y[tid * kOutPad + e] + sm.b[3 * kHid + e];
                const float4 s0 = __ldg(pca_scale + i), q0 = __ldg(pca_quat + i);
                const float s0v[3] = {s0.x, s0.y, s0.z};
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
                for (int k = 0; k < 4; ++k) dy[3 + k] = (gh[k] - hv[k] * dot) / dnorm;
                const float o0 = fminf(fmaxf(opacity0, 1e-6f), 1.f - 1e-6f);
                const float o = 1.f / (1.f + __expf(-(__logf(o0 / (1.f - o0)) + y[7])));
                dy[7] = d_opacity[i] * o * (1.f - o);
            }
        }
        __syncthreads();
        // ---- layer 4
        sgemm<kOut, kHid, kP, 1, 2>(sm.dY, 1, kOutPad, sm.H3, kHid, 1, sm.dW4, kHid, true);
        if (tid < kOut) {
            float s = 0.f;
            for (int p = 0; p < kP; ++p) s += sm.dY[p * kOutPad + tid];
            sm.db[3 * kHid + tid] += s;
        }
        sgemm<kP, kHid, kOut, 2, 4>(sm.dY, kOutPad, 1, sm.W4, kHid, 1, sm.G1, kHid, false);
        __syncthreads();
        for (int t = tid; t < kP * kHid; t += kNT) sm.G1[t] = sm.H3[t] > 0.f ? sm.G1[t] : 0.f;
        __syncthreads();
        // ---- layer 3
        sgemm<kHid, kHid, kP, 4, 4>(sm.G1, 1, kHid, sm.H2, kHid, 1, sm.dW3, kHid, true);
        if (tid < kHid) {
            float s = 0.f;
            for (int p = 0; p < kP; ++p) s += sm.G1[p * kHid + tid];
            sm.db[2 * kHid + tid] += s;
        }
        sgemm<kP, kHid, kHid, 2, 4>(sm.G1, kHid, 1, sm.W3, kHid, 1, sm.G2, kHid, false);
        __syncthreads();
        for (int t = tid; t < kP * kHid; t += kNT) sm.G2[t] = sm.H2[t] > 0.f ? sm.G2[t] : 0.f;
        __syncthreads();
        // ---- layer 2
        sgemm<kHid, kHid, kP, 4, 4>(sm.G2, 1, kHid, sm.H1, kHid, 1, sm.dW2, kHid, true);
        if (tid < kHid) {
            float s = 0.f;
            for (int p = 0; p < kP; ++p) s += sm.G2[p * kHid + tid];
            sm.db[kHid + tid] += s;
        }
        sgemm<kP, kHid, kHid, 2, 4>(sm.G2, kHid, 1, sm.W2, kHid, 1, sm.G1, kHid, false);
        __syncthreads();
        for (int t = tid; t < kP * kHid; t += kNT) sm.G1[t] = sm.H1[t] > 0.f ? sm.G1[t] : 0.f;
        __syncthreads();
        // ---- layer 1
        sgemm<kHid, kIn, kP, 4, 6>(sm.G1, 1, kHid, sm.X, kIn, 1, sm.dW1, kIn, true);
        if (tid < kHid) {
            float s = 0.f;
            for (int p = 0; p < kP; ++p) s += sm.G1[p * kHid + tid];
            sm.db[tid] += s;
        }
        __syncthreads();
    }
    // ---- once per CTA: add the accumulated gradients
    for (int t = tid; t < kHid * kIn; t += kNT) atomicAdd(&grad[oW1 + t], sm.dW1[t]);
    for (int t = tid; t < kHid * kHid; t += kNT) {
        atomicAdd(&grad[oW2 + t], sm.dW2[t]);
        atomicAdd(&grad[oW3 + t], sm.dW3[t]);
    }
    for (int t = tid; t < kOut * kHid; t += kNT) atomicAdd(&grad[oW4 + t], sm.dW4[t]);
    for (int t = tid; t < 3 * kHid; t += kNT) atomicAdd(&grad[oB1 + t], sm.db[t]);
    for (int t = tid; t < kOut; t += kNT) atomicAdd(&grad[oB4 + t], sm.db[3 * kHid + t]);
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

p2e_status p2e_mlp_backward(const float *xyz, const float *rgb, int64_t n, const uint32_t *knn_idx,
                            const p2e_gaussians *pca, const void *mlp_weights, const float *d_scale,
                            const float *d_quat, const float *d_opacity, const float *d_normal, float *grad,
                            void *stream) {
    if (n < 1 || !xyz || !rgb || !knn_idx || !pca || !pca->scale || !pca->quat || !mlp_weights || !d_scale ||
        !d_quat || !d_opacity || !d_normal || !grad)
        return P2E_ERR_INVALID_ARG;
    const size_t smem = sizeof(BwdSmem);
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = (dev >= 0 && dev < 64) ? dev : 0;
    if (!configured[slot]) {
        if (cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return P2E_ERR_CUDA;
        configured[slot] = 1;
    }
    const int64_t ntiles = (n + kP - 1) / kP;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)device_sms());
    // opacity of the PCA estimate is the same for every point (mean_op.w)
    float o0 = 0.9f;
    if (cudaMemcpyAsync(&o0, pca->mean_op ? pca->mean_op + 3 : nullptr, sizeof(float), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return P2E_ERR_CUDA;
    mlp_bwd_kernel<<<grid, kNT, smem, (cudaStream_t)stream>>>(
        (const float4 *)xyz, (const float4 *)rgb, n, knn_idx, (const float4 *)pca->scale,
        (const float4 *)pca->quat, o0, (const unsigned char *)mlp_weights, d_scale, d_quat, d_opacity, d_normal,
        grad);
    return cudaGetLastError() == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
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
