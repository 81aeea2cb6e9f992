// K11: learned per-point estimator on the 5th-generation tensor cores.
//
// The paper's estimator ends in a shared per-point MLP head that predicts
// each Gaussian's scale, rotation and opacity (Sec. 3.1-3.2).  Here the
// head reads the point's 16 nearest neighbours directly:
//   features  per neighbour j (distance order): R^T (p_j - p_i) / r_i and
//             c_j - c_i, R the canonical PCA frame, r_i the 16th-neighbour
//             distance (96 inputs)
//   network   96 -> 64 -> 64 -> 64 (ReLU) -> 8, bf16 operands, fp32 accumulate
//   outputs   corrections of the PCA estimate in its own frame:
//             s = s_pca exp(clip(y0..2, -4, 4)), q = q_pca (x) normalize(1 + y3..6),
//             o = sigmoid(logit(o_pca) + y7), normal = third axis of R(q).
//
// Kernel: persistent CTAs of 128 threads; one tile = 128 points = the UMMA
// M dimension.  Each thread gathers one point's features into shared memory
// (bf16, no-swizzle K-major core-matrix layout); one elected thread issues
// tcgen05.mma (kind::f16, bf16 x bf16 -> f32 accumulator in TMEM, K = 16
// per instruction) and commits to an mbarrier; every thread then reads its
// row of the accumulator with tcgen05.ld, adds the bias, applies ReLU,
// rounds to bf16 and writes the next layer's A operand.  The weights (30 KB
// bf16) stay in shared memory for the whole kernel.  Every mbarrier wait is
// bounded; a wait that gives up records P2E_ERR_TIMEOUT, the CTA stops
// issuing work and still releases its TMEM.
#include <cuda_bf16.h>

#include "tcgen05.cuh"

namespace p2e {

constexpr int kTM = 128, kIn = 96, kHid = 64, kOutPad = 16, kNb = 16;
constexpr int kBlobW1 = 0, kBlobW2 = kBlobW1 + kHid * kIn * 2, kBlobW3 = kBlobW2 + kHid * kHid * 2,
              kBlobW4 = kBlobW3 + kHid * kHid * 2, kBlobB = kBlobW4 + kOutPad * kHid * 2;
constexpr int kBlobBytes = kBlobB + (3 * kHid + kOutPad) * 4;
static_assert(kBlobBytes == P2E_MLP_BLOB_BYTES, "weight blob layout of p2e.h");
constexpr uint32_t kTmemCols = 64;

// H (the hidden activations) aliases the front of A: layer 1 has finished
// reading A when its epilogue writes H, and each later layer has finished
// reading H when its epilogue overwrites it.  55 KB per CTA: four CTAs per SM.
struct __align__(128) MlpSmem {
    __nv_bfloat16 A[kTM * kIn];
    __nv_bfloat16 W1[kHid * kIn];
    __nv_bfloat16 W2[kHid * kHid];
    __nv_bfloat16 W3[kHid * kHid];
    __nv_bfloat16 W4[kOutPad * kHid];
    float b[3 * kHid + kOutPad];
    uint64_t mbar;
    uint32_t tmem;
    int err;
};

// bias + ReLU + bf16 of a 64-wide accumulator row into the next A operand
__device__ __forceinline__ void epilogue_hidden(uint32_t taddr, const float *bias, __nv_bfloat16 *H, int row) {
    float v[kHid];
    tmem_ld64(taddr, v);
#pragma unroll
    for (int c16 = 0; c16 < kHid / 16; ++c16) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = c16 * 16 + half * 8 + 2 * e;
                const float lo = fmaxf(v[k] + bias[k], 0.f);
                const float hi = fmaxf(v[k + 1] + bias[k + 1], 0.f);
                const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
                w[e] = *reinterpret_cast<const uint32_t *>(&p);
            }
            *reinterpret_cast<uint4 *>(H + core_off(row, c16 * 16 + half * 8, kHid)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// the per-layer MMA chain: D[128 x N] = A[128 x K] B[N x K]^T
__device__ __forceinline__ void issue_layer(uint32_t tmem, const __nv_bfloat16 *A, const __nv_bfloat16 *Bm, int K,
                                            int N, uint64_t *mbar) {
    tc_fence_after();
    const uint32_t id = idesc_bf16(kTM, N);
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t da = make_sdesc(A + s * 16 * 8, 128, (K / 8) * 128);
        const uint64_t db = make_sdesc(Bm + s * 16 * 8, 128, (K / 8) * 128);
        umma_bf16(tmem, da, db, id, s > 0 ? 1u : 0u);
    }
    umma_commit(mbar);
}

__device__ __forceinline__ float4 qmul(float4 a, float4 b) {
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w, a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y, a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

__global__ void __launch_bounds__(kTM, 3) mlp_estimate_kernel(const float4 *__restrict__ pk, int64_t n,
                                                           const unsigned char *__restrict__ blob,
                                                           const uint32_t *__restrict__ knn,
                                                           float4 *__restrict__ mean_op, float4 *__restrict__ scale,
                                                           float4 *__restrict__ quat, float4 *__restrict__ normal,
                                                           int32_t *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights -> shared memory in the core-matrix layout (16-byte pieces)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(blob);
        auto load_w = [&](__nv_bfloat16 *dst, int off, int N, int K) {
            for (int t = tid; t < N * K / 8; t += kTM) {
                const int r = t / (K / 8), c = t % (K / 8);
                *reinterpret_cast<uint4 *>(dst + core_off(r, c * 8, K)) = src[off / 16 + t];
            }
        };
        load_w(sm.W1, kBlobW1, kHid, kIn);
        load_w(sm.W2, kBlobW2, kHid, kHid);
        load_w(sm.W3, kBlobW3, kHid, kHid);
        load_w(sm.W4, kBlobW4, kOutPad, kHid);
        const float *bsrc = reinterpret_cast<const float *>(blob + kBlobB);
        for (int t = tid; t < 3 * kHid + kOutPad; t += kTM) sm.b[t] = bsrc[t];
    }
    if (tid == 0) {
        sm.err = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    __nv_bfloat16 *const H = sm.A;
    const uint32_t my_lane = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    const int64_t ntiles = (n + kTM - 1) / kTM;

    // operands of a tile that need no gather, loaded one tile ahead so that
    // their latency hides behind the previous tile's layers
    struct Ahead {
        float4 p, c, q, s0, m;
        uint4 kn[4];
    };
    auto load_ahead = [&](int64_t tile, Ahead &A) {
        const int64_t i = tile * kTM + tid;
        if (tile < ntiles && i < n) {
            A.p = __ldg(pk + 2 * i);
            A.c = __ldg(pk + 2 * i + 1);
            A.q = quat[i];
            A.s0 = scale[i];
            A.m = mean_op[i];
            const uint4 *kp = reinterpret_cast<const uint4 *>(knn + i * kNb);
#pragma unroll
            for (int k = 0; k < 4; ++k) A.kn[k] = __ldg(kp + k);
        } else {
            A.p = A.c = A.s0 = A.m = make_float4(0.f, 0.f, 0.f, 0.f);
            A.q = make_float4(1.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) A.kn[k] = make_uint4(0u, 0u, 0u, 0u);
        }
    };
    Ahead cur;
    load_ahead(blockIdx.x, cur);

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * kTM + tid;
        const bool live = i < n;
        // ---- features of point i -> row tid of A; the 16 neighbours'
        // positions and colours are all requested before any is used
        const float4 p = cur.p, c = cur.c, q = cur.q;
        const uint32_t nb[kNb] = {cur.kn[0].x, cur.kn[0].y, cur.kn[0].z, cur.kn[0].w,
                                  cur.kn[1].x, cur.kn[1].y, cur.kn[1].z, cur.kn[1].w,
                                  cur.kn[2].x, cur.kn[2].y, cur.kn[2].z, cur.kn[2].w,
                                  cur.kn[3].x, cur.kn[3].y, cur.kn[3].z, cur.kn[3].w};
        float4 pn[kNb], cn[kNb];
#pragma unroll
        for (int u = 0; u < kNb; ++u) {
            pn[u] = p;
            cn[u] = c;
            if (live) {  // both halves of one 32-byte record
                pn[u] = __ldg(pk + 2 * (size_t)nb[u]);
                cn[u] = __ldg(pk + 2 * (size_t)nb[u] + 1);
            }
        }
        const float w = q.x, x = q.y, y = q.z, z = q.w;
        const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z), R02 = 2.f * (x * z + w * y);
        const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z), R12 = 2.f * (y * z - w * x);
        const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x), R22 = 1.f - 2.f * (x * x + y * y);
        float inv_r = 0.f;
        if (live) {
            const float4 pl = pn[kNb - 1];
            const float dx = pl.x - p.x, dy = pl.y - p.y, dz = pl.z - p.z;
            inv_r = 1.f / fmaxf(sqrtf(dx * dx + dy * dy + dz * dz), 1e-12f);
        }
#pragma unroll
        for (int k = 0; k < kNb; k += 4) {
            // 4 neighbours = 24 features = 3 core-matrix rows of 8
            float f[24];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 pj = pn[k + u], cj = cn[k + u];
                const float dx = pj.x - p.x, dy = pj.y - p.y, dz = pj.z - p.z;
                f[6 * u + 0] = (R00 * dx + R10 * dy + R20 * dz) * inv_r;
                f[6 * u + 1] = (R01 * dx + R11 * dy + R21 * dz) * inv_r;
                f[6 * u + 2] = (R02 * dx + R12 * dy + R22 * dz) * inv_r;
                f[6 * u + 3] = cj.x - c.x;
                f[6 * u + 4] = cj.y - c.y;
                f[6 * u + 5] = cj.z - c.z;
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[ch * 8 + 2 * e], f[ch * 8 + 2 * e + 1]);
                    wv[e] = *reinterpret_cast<const uint32_t *>(&b2);
                }
                *reinterpret_cast<uint4 *>(sm.A + core_off(tid, k * 6 + ch * 8, kIn)) =
                    make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        Ahead nxt;
        load_ahead(tile + gridDim.x, nxt);
        // ---- four layers
        bool ok = true;
        const __nv_bfloat16 *Bs[4] = {sm.W1, sm.W2, sm.W3, sm.W4};
        for (int L = 0; L < 4 && ok; ++L) {
            if (tid == 0) issue_layer(tmem, L == 0 ? sm.A : H, Bs[L], L == 0 ? kIn : kHid, L == 3 ? kOutPad : kHid,
                                      &sm.mbar);
            if (L < 3) {
                // the layer's one barrier also makes a wait that gave up
                // known to all (the epilogue then read stale columns, unused)
                const bool waited = mbar_wait(&sm.mbar, phase);
                phase ^= 1u;
                tc_fence_after();
                epilogue_hidden(my_lane, sm.b + L * kHid, H, tid);
                proxy_fence();
                tc_fence_before();
                ok = !__syncthreads_or(!waited);
            } else {
                ok = !__syncthreads_or(!mbar_wait(&sm.mbar, phase));  // uniform decision
                phase ^= 1u;
                tc_fence_after();
            }
        }
        if (!ok) {
            atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
            sm.err = 1;
            break;
        }
        // ---- outputs: corrections of the PCA frame
        float yv[16];
        tmem_ld16(my_lane, yv);
        if (live) {
            float yy[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) yy[e] = yv[e] + sm.b[3 * kHid + e];
            const float4 s0 = cur.s0;
            scale[i] = make_float4(s0.x * __expf(fminf(fmaxf(yy[0], -4.f), 4.f)),
                                   s0.y * __expf(fminf(fmaxf(yy[1], -4.f), 4.f)),
                                   s0.z * __expf(fminf(fmaxf(yy[2], -4.f), 4.f)), 0.f);
            float4 dq = make_float4(1.f + yy[3], yy[4], yy[5], yy[6]);
            const float dn = rsqrtf(fmaxf(dq.x * dq.x + dq.y * dq.y + dq.z * dq.z + dq.w * dq.w, 1e-30f));
            dq = make_float4(dq.x * dn, dq.y * dn, dq.z * dn, dq.w * dn);
            const float4 qf = qmul(q, dq);
            quat[i] = qf;
            const float4 m = cur.m;
            const float o0 = fminf(fmaxf(m.w, 1e-6f), 1.f - 1e-6f);
            const float o = 1.f / (1.f + __expf(-(__logf(o0 / (1.f - o0)) + yy[7])));
            mean_op[i] = make_float4(m.x, m.y, m.z, o);
            const float W = qf.x, X = qf.y, Y = qf.z, Z = qf.w;
            normal[i] = make_float4(2.f * (X * Z + W * Y), 2.f * (Y * Z - W * X), 1.f - 2.f * (X * X + Y * Y), 0.f);
        }
        cur = nxt;
        tc_fence_before();
        __syncthreads();
    }
    __syncthreads();
    if (sm.err && tid == 0) mbar_wait(&sm.mbar, phase ^ 1u);  // let an overdue MMA finish (bounded)
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

cudaError_t launch_mlp_estimate(const float4 *pk, int64_t n, const void *mlp,
                                const uint32_t *knn, p2e_gaussians *out, int32_t *status, int num_sms,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(MlpSmem) + 1024;
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = (dev >= 0 && dev < 64) ? dev : 0;
    if (!configured[slot]) {
        e = cudaFuncSetAttribute(mlp_estimate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[slot] = 1;
    }
    static int per_sm[64] = {0};
    if (!per_sm[slot]) {
        // resident CTAs per SM: shared memory (1 KB reserved per CTA),
        // TMEM (64 columns per CTA of the SM's 512) and registers, so that
        // every CTA of the persistent grid is resident from the start
        int smem_sm = 0, occ = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, mlp_estimate_kernel) == cudaSuccess && fa.numRegs > 0) {
            const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocation unit: 256 per warp
            occ = 65536 / (warp_regs * (kTM / 32));
        }
        occ = std::max(occ, 1);
        per_sm[slot] = std::max(1, std::min(std::min(smem_sm / (int)(smem + 1024), 512 / (int)kTmemCols), occ));
    }
    const int64_t ntiles = (n + kTM - 1) / kTM;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms * per_sm[slot]);
    const p2e_kernel_probe *pr = kernel_probe(P2E_PROBE_MLP);
    probe_start(pr, st);
    mlp_estimate_kernel<<<grid, kTM, smem, st>>>(pk, n,
                                                 (const unsigned char *)mlp, knn, (float4 *)out->mean_op,
                                                 (float4 *)out->scale, (float4 *)out->quat, (float4 *)out->normal,
                                                 status);
    probe_stop(pr, st);
    return cudaGetLastError();
}

// Timeout self-test of the bounded mbarrier wait: one CTA initialises an
// mbarrier that expects one arrival, which never comes (no MMA is issued,
// no TMEM is allocated), and waits on it with the head's wait routine.
__global__ void selftest_mbar_kernel(int32_t *status, uint32_t limit) {
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&mbar, 0u, limit)) atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
    __syncthreads();
}

cudaError_t launch_selftest_mbar(int32_t *status, uint32_t spin_limit, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    selftest_mbar_kernel<<<1, 32, 0, st>>>(status, spin_limit);
    return cudaGetLastError();
}

}  // namespace p2e
