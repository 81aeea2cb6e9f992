// K9 + K10: per-point Gaussian estimation from the point cloud (the
// "preprocess" stage: point cloud in, one elliptical Gaussian per point out,
// Sec. 3.1-3.2).  The closed-form path sizes each splat from the local
// covariance of its 16 nearest neighbours (the prior splatting practice the
// paper contrasts with, Sec. 2.1); the learned path (mlp.cu) then corrects
// that frame with a per-point network.
//
//   bbox      one reduction: bounding box and centroid of the cloud
//   grid      uniform cells (about two cells per point at most), counting
//             sort of the points by cell (count, scan, scatter into a
//             cell-ordered copy)
//   knn       one thread per point, points taken in cell order (a
//             cell-ordered copy of the points): exact 16 nearest other
//             points (ties by index) by a two-pass threshold search of the
//             3x3x3 cell block (a counting kernel finds the trial radius, a
//             second kernel buffers and selects); the few queries that block
//             cannot certify go to a third kernel, one warp per query over
//             the 5x5x5 block (ring search beyond it)
//   pca       one thread per point in index order: the neighbours'
//             covariance, a cyclic Jacobi eigen-decomposition, scale =
//             sqrt(lambda) (smallest axis at least 0.1 of the middle one),
//             rotation in a canonical frame (normal = smallest axis turned
//             away from the centroid, first axis with its largest component
//             positive, e2 = e3 x e1) -> quaternion (Shepperd).
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace p2e {

constexpr int kK = 16;

struct GridParams {
    float lo[3];
    float h, inv_h;
    int dim[3];
    int64_t ncell;
    float cen[3];
};

struct EstScratch {
    int *bbox;            // 6 ordered-int min/max
    double *sum;          // 3
    GridParams *gp;
    uint32_t *cell;       // n
    uint32_t *counts;     // ncell_max
    uint32_t *start;      // ncell_max + 1
    uint64_t *scan_state; // scan tiles + 1
    uint32_t *ticket;
    float4 *spts;         // n points in cell order, .w = bits of the original index
    float4 *pk;           // 2n: point i's position and colour in one 32-byte record (learned path)
    uint32_t *knn;        // n * 16 (when the caller passes none)
    int64_t ncell_max, scan_tiles;
};

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
static int64_t ncell_cap(int64_t n) { return std::max<int64_t>(2 * n, 1 << 16); }
constexpr int kScanT = 4096;

static size_t est_layout(int64_t n, void *base, EstScratch *S) {
    const int64_t nc = ncell_cap(n);
    const int64_t st = (nc + 1 + kScanT - 1) / kScanT;
    size_t off = 0;
    char *b = (char *)base;
    auto take = [&](size_t bytes) {
        void *p = b ? (void *)(b + off) : nullptr;
        off += al256(bytes);
        return p;
    };
    EstScratch s;
    s.bbox = (int *)take(6 * sizeof(int));
    s.sum = (double *)take(3 * sizeof(double));
    s.gp = (GridParams *)take(sizeof(GridParams));
    s.cell = (uint32_t *)take((size_t)n * 4);
    s.counts = (uint32_t *)take((size_t)nc * 4);
    s.start = (uint32_t *)take((size_t)(nc + 1) * 4);
    s.scan_state = (uint64_t *)take((size_t)(st + 1) * 8);
    s.ticket = (uint32_t *)take(64);
    s.spts = (float4 *)take((size_t)n * 16);
    s.knn = (uint32_t *)take((size_t)n * kK * 4);
    s.pk = (float4 *)take((size_t)n * 32);
    s.ncell_max = nc;
    s.scan_tiles = st;
    if (S) *S = s;
    return off;
}

size_t estimate_scratch_bytes(int64_t n) { return est_layout(n, nullptr, nullptr); }

__device__ __forceinline__ int ord_of(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float float_of(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

__global__ void __launch_bounds__(256) bbox_kernel(const float4 *__restrict__ xyz, int64_t n, EstScratch S) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    float sm[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(xyz + i);
        const float v[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = fminf(mn[k], v[k]);
            mx[k] = fmaxf(mx[k], v[k]);
            sm[k] += v[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
            sm[k] += __shfl_xor_sync(0xffffffffu, sm[k], o);
        }
    __shared__ float s_mn[8][3], s_mx[8][3], s_sm[8][3];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) { s_mn[w][k] = mn[k]; s_mx[w][k] = mx[k]; s_sm[w][k] = sm[k]; }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int k = threadIdx.x;
        float a = INFINITY, b = -INFINITY;
        double c = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a = fminf(a, s_mn[q][k]);
            b = fmaxf(b, s_mx[q][k]);
            c += s_sm[q][k];
        }
        atomicMin(&S.bbox[k], ord_of(a));
        atomicMax(&S.bbox[3 + k], ord_of(b));
        atomicAdd(&S.sum[k], c);
    }
}

__global__ void grid_setup_kernel(int64_t n, EstScratch S) {
    GridParams g;
    float ext[3], emax = 0.f;
    for (int k = 0; k < 3; ++k) {
        g.lo[k] = float_of(S.bbox[k]);
        ext[k] = float_of(S.bbox[3 + k]) - g.lo[k];
        emax = fmaxf(emax, ext[k]);
        g.cen[k] = (float)(S.sum[k] / (double)n);
    }
    emax = fmaxf(emax, 1e-30f);
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) vol *= fmax((double)ext[k], 1e-3 * (double)emax);
    // about two cells per point: half the spacing of 4 points per cell, so
    // that a 3x3x3 block of cells almost always holds the 16 nearest
    double h = 0.5 * cbrt(vol * 4.0 / (double)n);
    for (int it = 0; it < 64; ++it) {
        double cells = 1.0;
        for (int k = 0; k < 3; ++k) {
            double d = floor(ext[k] / h) + 1.0;
            if (d > 1024.0) d = 1024.0;
            cells *= d;
        }
        bool fits = cells <= (double)S.ncell_max;
        for (int k = 0; k < 3; ++k) fits = fits && (ext[k] / h) < 1023.0;
        if (fits) break;
        h *= 1.25;
    }
    g.h = (float)h;
    g.inv_h = (float)(1.0 / h);
    g.ncell = 1;
    for (int k = 0; k < 3; ++k) {
        g.dim[k] = (int)fmin(1024.0, floor(ext[k] * g.inv_h) + 1.0);
        g.ncell *= g.dim[k];
    }
    *S.gp = g;
}

__device__ __forceinline__ void cell_of(const GridParams &g, float x, float y, float z, int c[3]) {
    const float v[3] = {x, y, z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = (int)floorf((v[k] - g.lo[k]) * g.inv_h);
        c[k] = min(max(q, 0), g.dim[k] - 1);
    }
}

// Cell of every point and the cells' counts; with rgb, also the packed
// (position, colour) records the MLP gathers (one 32-byte sector per point).
__global__ void __launch_bounds__(256) cell_count_kernel(const float4 *__restrict__ xyz,
                                                         const float4 *__restrict__ rgb, int64_t n, EstScratch S) {
    const GridParams g = *S.gp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(xyz + i);
        if (rgb) {
            S.pk[2 * i] = p;
            S.pk[2 * i + 1] = __ldg(rgb + i);
        }
        int c[3];
        cell_of(g, p.x, p.y, p.z, c);
        const uint32_t id = (uint32_t)(((int64_t)c[2] * g.dim[1] + c[1]) * g.dim[0] + c[0]);
        S.cell[i] = id;
        atomicAdd(&S.counts[id], 1u);
    }
}

__device__ __forceinline__ uint64_t ld_acq64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive scan of counts[0, len) into start[0, len] (start[len] = total),
// single pass with decoupled look-back; kScanT elements per block (16 per
// thread), the look-back by one warp over 32 predecessors at a time.
__global__ void __launch_bounds__(256) scan_counts_kernel(const uint32_t *__restrict__ counts, int64_t len,
                                                          uint32_t *__restrict__ start, EstScratch S,
                                                          int32_t *status, uint32_t spin_limit) {
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_w[8];
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(S.ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanT + threadIdx.x * 16;
    uint32_t v[16], loc = 0;
    if (base + 16 <= len) {
        const uint4 *src = reinterpret_cast<const uint4 *>(counts + base);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 u = src[k];
            v[4 * k] = u.x; v[4 * k + 1] = u.y; v[4 * k + 2] = u.z; v[4 * k + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = base + k < len ? counts[base + k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) loc += v[k];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
    for (int q = 0; q < 8; ++q) {
        if (q < w) wpre += s_w[q];
        tot += s_w[q];
    }
    if (w == 0) {
        constexpr uint64_t kAgg = 1ull << 62, kPre = 2ull << 62, kVal = (1ull << 62) - 1;
        uint64_t prefix = 0;
        if (tile == 0) {
            if (lane == 0) st_rel64(&S.scan_state[0], kPre | tot);
        } else {
            if (lane == 0) st_rel64(&S.scan_state[tile], kAgg | tot);
            int64_t p = tile - 1;  // window [p - 31, p], lane l reads p - l
            uint32_t spins = 0;
            while (true) {
                const int64_t idx = p - lane;
                const uint64_t wd = idx >= 0 ? ld_acq64(&S.scan_state[idx]) : kPre;
                const uint32_t flag = (uint32_t)(wd >> 62);
                const unsigned pre = __ballot_sync(0xffffffffu, flag == 2u);
                const unsigned notready = __ballot_sync(0xffffffffu, flag == 0u);
                const int first = pre ? __ffs(pre) - 1 : 32;  // nearest inclusive prefix
                const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                if (notready & need) {
                    if (++spins > spin_limit) {
                        if (lane == 0) atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
                        break;
                    }
                    backoff(spins);
                    continue;
                }
                uint64_t add = lane <= first ? (wd & kVal) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
                prefix += add;
                if (first < 32) break;
                p -= 32;
            }
            if (lane == 0) st_rel64(&S.scan_state[tile], kPre | (prefix + tot));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint32_t run = (uint32_t)s_prefix + wpre + x - loc;
    if (base + 16 <= len) {
        uint32_t o[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            o[k] = run;
            run += v[k];
        }
        uint4 *dst = reinterpret_cast<uint4 *>(start + base);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = make_uint4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
        if (base + 16 == len) start[len] = run;
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (base + k <= len) start[base + k] = run;
            run += v[k];
        }
    }
}

__global__ void __launch_bounds__(256) scatter_kernel(const float4 *__restrict__ xyz, int64_t n, EstScratch S) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[i];
        const uint32_t q = S.start[c] + atomicSub(&S.counts[c], 1u) - 1u;  // the count runs down to 0
        const float4 p = __ldg(xyz + i);
        S.spts[q] = make_float4(p.x, p.y, p.z, __uint_as_float((uint32_t)i));
    }
}

constexpr int kKnnThreads = 128;

// List of the 16 best (distance, index) pairs, kept sorted in shared
// memory; an insertion shifts only the entries that follow it.
struct KnnList {
    float *d;
    uint32_t *j;
    __device__ __forceinline__ float &D(int k) { return d[k]; }
    __device__ __forceinline__ uint32_t &J(int k) { return j[k]; }
    __device__ __forceinline__ void insert(float dd, uint32_t jj) {
        int k = kK - 1;
        while (k > 0 && (dd < D(k - 1) || (dd == D(k - 1) && jj < J(k - 1)))) {
            D(k) = D(k - 1);
            J(k) = J(k - 1);
            --k;
        }
        D(k) = dd;
        J(k) = jj;
    }
};

// cyclic Jacobi on a symmetric 3x3 (fp32); V columns are eigenvectors
__device__ __forceinline__ void jacobi3f(float (&A)[3][3], float (&V)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.f : 0.f;
    const float tr = fabsf(A[0][0]) + fabsf(A[1][1]) + fabsf(A[2][2]);
    for (int sweep = 0; sweep < 12; ++sweep) {
        const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
        if (!(off > 1e-7f * tr)) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            if (A[p][q] == 0.f) continue;
            const float theta = (A[q][q] - A[p][p]) / (2.f * A[p][q]);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f), s = t * c;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
}

__device__ __forceinline__ float4 shepperd_f(const float R[3][3]) {
    const float tr = R[0][0] + R[1][1] + R[2][2];
    float w, x, y, z;
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
        const float s = 2.f * sqrtf(1.f + tr);
        w = 0.25f * s; x = (R[2][1] - R[1][2]) / s; y = (R[0][2] - R[2][0]) / s; z = (R[1][0] - R[0][1]) / s;
    } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
        const float s = 2.f * sqrtf(fmaxf(1.f + R[0][0] - R[1][1] - R[2][2], 1e-30f));
        w = (R[2][1] - R[1][2]) / s; x = 0.25f * s; y = (R[0][1] + R[1][0]) / s; z = (R[0][2] + R[2][0]) / s;
    } else if (R[1][1] >= R[2][2]) {
        const float s = 2.f * sqrtf(fmaxf(1.f + R[1][1] - R[0][0] - R[2][2], 1e-30f));
        w = (R[0][2] - R[2][0]) / s; x = (R[0][1] + R[1][0]) / s; y = 0.25f * s; z = (R[1][2] + R[2][1]) / s;
    } else {
        const float s = 2.f * sqrtf(fmaxf(1.f + R[2][2] - R[0][0] - R[1][1], 1e-30f));
        w = (R[1][0] - R[0][1]) / s; x = (R[0][2] + R[2][0]) / s; y = (R[1][2] + R[2][1]) / s; z = 0.25f * s;
    }
    return make_float4(w, x, y, z);
}

constexpr int kRadA = 5;      // trial radii of the fast path, in cell sizes (0.40 .. 0.75)
constexpr int kBuf = 32;      // candidates the fast path keeps

// Iterates the candidate points of the cells of the 3x3x3 block around the
// query's cell that may hold a point within distance sqrt(R2) of the query
// (all 27 cells when R2 is infinite), taken from the cell-ordered copy.  A
// cell is skipped only when its box is farther than the radius by more than
// 1e-3 cell sizes, far above the rounding of the cell assignment.
template <typename F>
__device__ __forceinline__ void for_block(const GridParams &g, const EstScratch &S, const int c0[3],
                                          const float4 &p, float R2, F &&f) {
    const float pv[3] = {p.x, p.y, p.z};
    float lo2[3], hi2[3];  // squared distance to the own cell's lower / upper face, plus margin slack
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float face = g.lo[k] + (float)c0[k] * g.h;
        const float dl = fmaxf(pv[k] - face - 1e-3f * g.h, 0.f);
        const float dh = fmaxf(face + g.h - pv[k] - 1e-3f * g.h, 0.f);
        lo2[k] = dl * dl;
        hi2[k] = dh * dh;
    }
    for (int dz = -1; dz <= 1; ++dz) {
        const int cz = c0[2] + dz;
        if (cz < 0 || cz >= g.dim[2]) continue;
        const float ez = dz < 0 ? lo2[2] : (dz > 0 ? hi2[2] : 0.f);
        if (ez > R2) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int cy = c0[1] + dy;
            if (cy < 0 || cy >= g.dim[1]) continue;
            const float ey = ez + (dy < 0 ? lo2[1] : (dy > 0 ? hi2[1] : 0.f));
            if (ey > R2) continue;
            const int x0 = (c0[0] > 0 && ey + lo2[0] <= R2) ? c0[0] - 1 : c0[0];
            const int x1 = (c0[0] + 1 < g.dim[0] && ey + hi2[0] <= R2) ? c0[0] + 1 : c0[0];
            const uint32_t row = (uint32_t)(((int64_t)cz * g.dim[1] + cy) * g.dim[0]);
            // cells x0..x1 of a row are contiguous in the cell-ordered points
            const uint32_t s0 = __ldg(S.start + row + x0), e0 = __ldg(S.start + row + x1 + 1);
            uint32_t q = s0;
            for (; q + 4 <= e0; q += 4) {  // four independent loads in flight
                const float4 a0 = __ldg(S.spts + q), a1 = __ldg(S.spts + q + 1), a2 = __ldg(S.spts + q + 2),
                             a3 = __ldg(S.spts + q + 3);
                f(a0);
                f(a1);
                f(a2);
                f(a3);
            }
            for (; q < e0; ++q) f(__ldg(S.spts + q));
        }
    }
}

// The neighbours' covariance about their centroid, its cyclic Jacobi
// eigen-decomposition and the canonical frame, written out for query point
// i at p.  nb(k) returns neighbour k (k-th nearest; .w = bits of its
// index).
template <typename NB>
__device__ __forceinline__ void pca_out(const GridParams &g, const float4 &p, uint32_t i, float opacity, NB &&nb,
                                        const float4 *__restrict__ rgb, uint32_t *__restrict__ knn_out,
                                        float4 *__restrict__ mean_op, float4 *__restrict__ scale,
                                        float4 *__restrict__ quat, float4 *__restrict__ rgb_out,
                                        float4 *__restrict__ normal) {
    // The covariance is shift invariant; it is accumulated on the offsets
    // p_j - p_i, which are exact (or nearly: the coordinates of near
    // neighbours agree in sign and exponent), so that the centroid's rounding
    // is relative to the neighbourhood's size, not to the coordinates'
    // magnitude (a 1 mm neighbourhood at 1 m would lose ~4 digits).
    float m[3] = {0, 0, 0};
    for (int k = 0; k < kK; ++k) {
        const float4 qk = nb(k);
        if (knn_out) knn_out[(int64_t)i * kK + k] = __float_as_uint(qk.w);
        m[0] += qk.x - p.x; m[1] += qk.y - p.y; m[2] += qk.z - p.z;
    }
    for (int k = 0; k < 3; ++k) m[k] *= (1.f / kK);
    float C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < kK; ++k) {
        const float4 qk = nb(k);  // second pass, from L1
        const float d[3] = {(qk.x - p.x) - m[0], (qk.y - p.y) - m[1], (qk.z - p.z) - m[2]};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) C[a][b] = fmaf(d[a], d[b], C[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            C[a][b] *= (1.f / kK);
            C[b][a] = C[a][b];
        }
    float V[3][3];
    jacobi3f(C, V);
    // eigenpairs in descending order (static indices only)
    float l0 = C[0][0], l1 = C[1][1], l2 = C[2][2];
    float e0[3] = {V[0][0], V[1][0], V[2][0]}, e1[3] = {V[0][1], V[1][1], V[2][1]}, e2[3] = {V[0][2], V[1][2], V[2][2]};
#define P2E_SWAP_PAIR(la, lb, ua, ub)                                  \
    do {                                                               \
        const float t_ = la; la = lb; lb = t_;                         \
        _Pragma("unroll") for (int k_ = 0; k_ < 3; ++k_) {             \
            const float w_ = ua[k_]; ua[k_] = ub[k_]; ub[k_] = w_;     \
        }                                                              \
    } while (0)
    if (l1 > l0) P2E_SWAP_PAIR(l0, l1, e0, e1);
    if (l2 > l1) P2E_SWAP_PAIR(l1, l2, e1, e2);
    if (l1 > l0) P2E_SWAP_PAIR(l0, l1, e0, e1);
#undef P2E_SWAP_PAIR
    const float lamv[3] = {l0, l1, l2};
    float R[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { R[k][0] = e0[k]; R[k][1] = e1[k]; R[k][2] = e2[k]; }
    // canonical frame: normal away from the centroid, e1's largest-magnitude
    // component positive, e2 = e3 x e1
    const float sg = (p.x - g.cen[0]) * R[0][2] + (p.y - g.cen[1]) * R[1][2] + (p.z - g.cen[2]) * R[2][2];
    if (sg < 0.f)
#pragma unroll
        for (int k = 0; k < 3; ++k) R[k][2] = -R[k][2];
    {
        const float a0 = fabsf(R[0][0]), a1 = fabsf(R[1][0]), a2 = fabsf(R[2][0]);
        const float big = (a1 > a0) ? ((a2 > a1) ? R[2][0] : R[1][0]) : ((a2 > a0) ? R[2][0] : R[0][0]);
        if (big < 0.f)
#pragma unroll
            for (int k = 0; k < 3; ++k) R[k][0] = -R[k][0];
    }
    R[0][1] = R[1][2] * R[2][0] - R[2][2] * R[1][0];
    R[1][1] = R[2][2] * R[0][0] - R[0][2] * R[2][0];
    R[2][1] = R[0][2] * R[1][0] - R[1][2] * R[0][0];
    float s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = sqrtf(fmaxf(lamv[a], 0.f));
    s[2] = fmaxf(s[2], 0.1f * s[1]);
    mean_op[i] = make_float4(p.x, p.y, p.z, opacity);
    scale[i] = make_float4(s[0], s[1], s[2], 0.f);
    quat[i] = shepperd_f(R);
    rgb_out[i] = __ldg(rgb + i);
    normal[i] = make_float4(R[0][2], R[1][2], R[2][2], 0.f);
}

// Squared distance, one expression for every pass (counts and collections
// must agree bit for bit).
__device__ __forceinline__ float dist2(const float4 &a, const float4 &p) {
    const float ex = a.x - p.x, ey = a.y - p.y, ez = a.z - p.z;
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// Trial radii of the fast path, squared: (0.40 + 0.0875 k) cell sizes,
// shrunk by a relative 1e-4 and 1e-6 so that a radius never reaches a cell
// the block walk culls.
__device__ __forceinline__ float trial_r2(const GridParams &g, int k) {
    const float rr = (0.40f + 0.0875f * k) * g.h * (1.f - 1e-4f) - 1e-6f;
    return rr * rr;
}

// Fast path, one thread per query point (points taken in cell order), in
// two kernels.  Exact 16 nearest other points, ties by index:
//   knn_count_kernel  pass 1: count the candidates within five trial radii
//                     (0.40 .. 0.75 cell sizes, branch free, on the FMA
//                     pipe) over only the cells of the 3x3x3 block that the
//                     largest ball can reach, and record the smallest
//                     squared radius T that holds 16 others (and at most
//                     kBuf), or -1;
//   knn_select_kernel pass 2: keep the candidates within T (the cells that
//                     ball reaches) in shared memory as (distance bits,
//                     index) keys, check their count, select the 16
//                     smallest keys and write them as the query's list
//                     (pca_kernel computes the frames from the lists).
// The counting pass needs neither the candidate buffer nor most of the
// registers, so as a kernel of its own it runs at twice the resident warps
// with all of L1 for the cell walk.  T goes through the cell-count array,
// which the scatter has run down to zero and which holds at least n words.
// A query for which no trial radius qualifies (about 0.5 % of the points of
// a surface scan: sparse or ragged regions) is appended to a list (S.cell
// reused, its length in S.ticket[12]) for knn_slow_kernel, so that no warp
// carries one lane's long search.
__global__ void __launch_bounds__(kKnnThreads, 12) knn_count_kernel(int64_t n, EstScratch S) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const GridParams g = *S.gp;
    const float4 p = S.spts[t];
    int c0[3];
    cell_of(g, p.x, p.y, p.z, c0);
    // counts kept in fp32 on the FMA pipe: fma(-d, 2^100, r 2^100) is
    // (r - d) 2^100 rounded once (the scaling is exact): <= 0 when d >= r,
    // and for d < r at least 2^100 times the fp32 spacing at r, >= 1 for
    // any r above 2^-76, so the saturated value is 1 exactly when d < r
    // (pass 2 counts the chosen radius exactly in any case)
    float rB[kRadA], cf[kRadA];
#pragma unroll
    for (int k = 0; k < kRadA; ++k) {
        rB[k] = trial_r2(g, k) * 0x1p100f;
        cf[k] = 0.f;
    }
    for_block(g, S, c0, p, trial_r2(g, kRadA - 1), [&](const float4 &pj) {
        const float d = dist2(pj, p);
#pragma unroll
        for (int k = 0; k < kRadA; ++k) cf[k] += __saturatef(fmaf(-d, 0x1p100f, rB[k]));
    });
    float T = -1.f;
#pragma unroll
    for (int k = kRadA - 1; k >= 0; --k)
        if (cf[k] >= (float)(kK + 1) && cf[k] <= (float)(kBuf + 1)) T = trial_r2(g, k);
    if (T < 0.f) S.cell[atomicAdd(S.ticket + 12, 1u)] = (uint32_t)t;
    S.counts[t] = __float_as_uint(T);
}

__global__ void __launch_bounds__(kKnnThreads, 6) knn_select_kernel(int64_t n, EstScratch S,
                                                                 uint32_t *__restrict__ knn_out) {
    // candidates as (fp32 distance bits << 32 | index): d >= 0, so the
    // unsigned order of the keys is the order by (distance, index)
    __shared__ uint64_t s_key[kBuf * kKnnThreads];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float T = __uint_as_float(S.counts[t]);
    if (T < 0.f) return;  // listed for the slow kernel by the counting pass
    const GridParams g = *S.gp;
    const float4 p = S.spts[t];
    const uint32_t i = __float_as_uint(p.w);
    int c0[3];
    cell_of(g, p.x, p.y, p.z, c0);
    uint64_t *bk = s_key + threadIdx.x;
    int m = 0;  // candidates inside T (kept: the first kBuf)
    for_block(g, S, c0, p, T, [&](const float4 &pj) {
        const uint32_t j = __float_as_uint(pj.w);
        const float d = dist2(pj, p);
        if (d < T && j != i) {
            if (m < kBuf) bk[m * kKnnThreads] = ((uint64_t)__float_as_uint(d) << 32) | j;
            ++m;
        }
    });
    if (m < kK || m > kBuf) {  // only if the counts of pass 1 were off
        S.cell[atomicAdd(S.ticket + 12, 1u)] = (uint32_t)t;
        return;
    }
    // partial selection sort: the 16 smallest keys to the front
    for (int a = 0; a < kK; ++a) {
        int best_k = a;
        uint64_t kbst = bk[a * kKnnThreads];
#pragma unroll 4
        for (int b = a + 1; b < m; ++b) {
            const uint64_t kb = bk[b * kKnnThreads];
            if (kb < kbst) { best_k = b; kbst = kb; }
        }
        bk[best_k * kKnnThreads] = bk[a * kKnnThreads];
        bk[a * kKnnThreads] = kbst;
    }
    // the query's 16 neighbours, nearest first: one 64-byte row (16-byte
    // aligned stores) of the original index's list
    uint4 *row = reinterpret_cast<uint4 *>(knn_out + (int64_t)i * kK);
#pragma unroll
    for (int k = 0; k < kK / 4; ++k)
        row[k] = make_uint4((uint32_t)bk[(4 * k) * kKnnThreads], (uint32_t)bk[(4 * k + 1) * kKnnThreads],
                            (uint32_t)bk[(4 * k + 2) * kKnnThreads], (uint32_t)bk[(4 * k + 3) * kKnnThreads]);
}

// The neighbours' covariance, eigen-decomposition and canonical frame of
// every point, taken in the order of the original indices so that the
// Gaussians are written as whole 32-byte sectors (in cell order they were
// half-sector writes scattered over the outputs, which HBM3e, having no
// write mask, fills by reading each sector first); the neighbours come from
// the lists the selection kernels wrote.
__global__ void __launch_bounds__(256, 4) pca_kernel(const float4 *__restrict__ xyz, const float4 *__restrict__ rgb,
                                                  int64_t n, float opacity, EstScratch S,
                                                  const uint32_t *__restrict__ knn,
                                                  float4 *__restrict__ mean_op, float4 *__restrict__ scale,
                                                  float4 *__restrict__ quat, float4 *__restrict__ rgb_out,
                                                  float4 *__restrict__ normal) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GridParams g = *S.gp;
    const float4 p = __ldg(xyz + i);
    uint32_t nb[kK];
    const uint4 *row = reinterpret_cast<const uint4 *>(knn + i * kK);
#pragma unroll
    for (int k = 0; k < kK / 4; ++k) {
        const uint4 r = __ldg(row + k);
        nb[4 * k] = r.x; nb[4 * k + 1] = r.y; nb[4 * k + 2] = r.z; nb[4 * k + 3] = r.w;
    }
    pca_out(g, p, (uint32_t)i, opacity, [&](int k) {
        const uint32_t j = nb[k];
        const float4 q = __ldg(xyz + j);
        return make_float4(q.x, q.y, q.z, __uint_as_float(j));
    }, rgb, nullptr, mean_op, scale, quat, rgb_out, normal);
}

constexpr int kSlowWarps = 4;   // one query per warp at a time
constexpr int kSlowBuf = 64;    // candidates one warp keeps
constexpr int kLad = 16;        // trial radii 0.40 .. 2.00 cell sizes (ratio ~1.113)

// Slow path, one warp per listed query.  The 5x5x5 block of cells around
// the query's cell reaches at least two cell sizes from it; lane r < 25
// holds the extent of row r of the block (the row's five cells are
// contiguous in the cell-ordered copy) and the lanes stride over each row:
//   pass 1  counts within 16 trial radii, summed over the warp; T = the
//           smallest radius holding 16 others (and at most kSlowBuf);
//   pass 2  the candidates within T gathered in shared memory by ballot;
//           each candidate's rank among them by (distance, index) puts the
//           16 smallest in order.
// Where no radius qualifies (fewer than 16 others within two cell sizes,
// or many points at one distance), lane 0 searches rings of cells around
// the query's cell until the 16th distance is below the distance to the
// next ring.  The warp writes the query's neighbour list.
__global__ void __launch_bounds__(kSlowWarps * 32) knn_slow_kernel(EstScratch S, uint32_t *__restrict__ knn_out) {
    __shared__ float s_d[kSlowWarps][kSlowBuf];
    __shared__ uint32_t s_j[kSlowWarps][kSlowBuf];
    __shared__ uint32_t s_nb[kSlowWarps][kK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const GridParams g = *S.gp;
    const uint32_t nq = S.ticket[12];
    float lad[kLad];
    {
        float f = 0.40f;
#pragma unroll
        for (int k = 0; k < kLad; ++k) {
            const float rr = fminf(f, 2.f) * g.h * (1.f - 1e-4f) - 1e-6f;
            lad[k] = rr * rr;
            f *= 1.1133f;
        }
    }
    float *wd = s_d[w];
    uint32_t *wj = s_j[w];
    for (uint32_t e = blockIdx.x * kSlowWarps + w; e < nq; e += gridDim.x * kSlowWarps) {
        const uint32_t t = S.cell[e];
        const float4 p = S.spts[t];
        const uint32_t i = __float_as_uint(p.w);
        int c0[3];
        cell_of(g, p.x, p.y, p.z, c0);
        uint32_t rs = 0, re = 0;
        if (lane < 25) {
            const int cz = c0[2] + lane / 5 - 2, cy = c0[1] + lane % 5 - 2;
            if (cz >= 0 && cz < g.dim[2] && cy >= 0 && cy < g.dim[1]) {
                const int x0 = max(c0[0] - 2, 0), x1 = min(c0[0] + 2, g.dim[0] - 1);
                const uint32_t row = (uint32_t)(((int64_t)cz * g.dim[1] + cy) * g.dim[0]);
                rs = S.start[row + x0];
                re = S.start[row + x1 + 1];
            }
        }
        // ---- pass 1: counts within the trial radii
        int cnt[kLad];
#pragma unroll
        for (int k = 0; k < kLad; ++k) cnt[k] = 0;
        for (int r = 0; r < 25; ++r) {
            const uint32_t s0 = __shfl_sync(0xffffffffu, rs, r), e0 = __shfl_sync(0xffffffffu, re, r);
            for (uint32_t q = s0 + lane; q < e0; q += 32) {
                const float d = dist2(S.spts[q], p);
#pragma unroll
                for (int k = 0; k < kLad; ++k) cnt[k] += d < lad[k] ? 1 : 0;
            }
        }
        float T = -1.f;
#pragma unroll
        for (int k = kLad - 1; k >= 0; --k) {
            int c = cnt[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (c >= kK + 1 && c <= kSlowBuf + 1) T = lad[k];
        }
        if (T > 0.f) {
            // ---- pass 2: the candidates within T, ranked
            int m = 0;
            for (int r = 0; r < 25; ++r) {
                const uint32_t s0 = __shfl_sync(0xffffffffu, rs, r), e0 = __shfl_sync(0xffffffffu, re, r);
                for (uint32_t b = s0; b < e0; b += 32) {
                    const uint32_t q = b + lane;
                    bool keep = false;
                    float d = 0.f;
                    uint32_t j = 0;
                    if (q < e0) {
                        const float4 pj = S.spts[q];
                        j = __float_as_uint(pj.w);
                        d = dist2(pj, p);
                        keep = d < T && j != i;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    const int pos = m + __popc(bal & ((1u << lane) - 1u));
                    if (keep && pos < kSlowBuf) {
                        wd[pos] = d;
                        wj[pos] = j;
                    }
                    m += __popc(bal);
                }
            }
            m = min(m, kSlowBuf);
            __syncwarp();
            for (int a = lane; a < m; a += 32) {
                const float da = wd[a];
                const uint32_t ja = wj[a];
                int rank = 0;
                for (int b = 0; b < m; ++b) {
                    const float db = wd[b];
                    const uint32_t jb = wj[b];
                    rank += (db < da || (db == da && jb < ja)) ? 1 : 0;
                }
                if (rank < kK) s_nb[w][rank] = ja;
            }
        } else if (lane == 0) {
            // ---- last resort: incremental search over growing rings
            KnnList best{wd, wj};
            for (int k = 0; k < kK; ++k) { best.D(k) = INFINITY; best.J(k) = 0xffffffffu; }
            float thr = INFINITY;
            uint32_t thr_j = 0xffffffffu;
            const int rmax = max(g.dim[0], max(g.dim[1], g.dim[2]));
            for (int r = 0; r <= rmax; ++r) {
                for (int dz = -r; dz <= r; ++dz) {
                    const int cz = c0[2] + dz;
                    if (cz < 0 || cz >= g.dim[2]) continue;
                    for (int dy = -r; dy <= r; ++dy) {
                        const int cy = c0[1] + dy;
                        if (cy < 0 || cy >= g.dim[1]) continue;
                        const bool shell = (dz == -r || dz == r || dy == -r || dy == r);
                        for (int dx = -r; dx <= r; dx += (shell ? 1 : 2 * r)) {
                            const int cx = c0[0] + dx;
                            if (cx >= 0 && cx < g.dim[0]) {
                                const uint32_t c = (uint32_t)(((int64_t)cz * g.dim[1] + cy) * g.dim[0] + cx);
                                for (uint32_t q = S.start[c]; q < S.start[c + 1]; ++q) {
                                    const float4 pj = S.spts[q];
                                    const uint32_t j = __float_as_uint(pj.w);
                                    if (j == i) continue;
                                    const float d = dist2(pj, p);
                                    if (d < thr || (d == thr && j < thr_j)) {
                                        best.insert(d, j);
                                        thr = best.D(kK - 1);
                                        thr_j = best.J(kK - 1);
                                    }
                                }
                            }
                            if (r == 0) break;
                        }
                    }
                }
                const float bound = fmaxf(0.f, (float)r * g.h * (1.f - 1e-4f) - 1e-6f);
                if (thr_j != 0xffffffffu && thr < bound * bound) break;
            }
            for (int k = 0; k < kK; ++k) s_nb[w][k] = best.J(k);
        }
        __syncwarp();
        if (lane < kK) knn_out[(int64_t)i * kK + lane] = s_nb[w][lane];
        __syncwarp();
    }
}

__global__ void est_init_kernel(EstScratch S) {
    if (threadIdx.x < 3) {
        S.bbox[threadIdx.x] = ord_of(INFINITY);
        S.bbox[3 + threadIdx.x] = ord_of(-INFINITY);
        S.sum[threadIdx.x] = 0.0;
    }
}

cudaError_t launch_mlp_estimate(const float4 *pk, int64_t n, const void *mlp,
                                const uint32_t *knn, p2e_gaussians *out, int32_t *status, int num_sms,
                                cudaStream_t st);

cudaError_t launch_estimate(const float *xyz, const float *rgb, int64_t n, int32_t mode,
                            const void *mlp, float pca_opacity, p2e_gaussians *out,
                            uint32_t *knn_idx, void *scratch, int num_sms, cudaStream_t st) {
    EstScratch S;
    est_layout(n, scratch, &S);
    cudaError_t e;
    // bbox starts at (+inf, -inf); sums, counts, tickets, look-back at 0
    est_init_kernel<<<1, 32, 0, st>>>(S);
    if ((e = cudaMemsetAsync(S.counts, 0, (size_t)S.ncell_max * 4, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S.scan_state, 0, (size_t)(S.scan_tiles + 1) * 8, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S.ticket, 0, 64, st)) != cudaSuccess) return e;
    // status words (zeroed with the tickets): [8] the cell-count scan's
    // look-back, [9] the learned head's mbarrier waits
    int32_t *status = (int32_t *)(S.ticket + 8);
    const int g1 = num_sms * 4;
    bbox_kernel<<<num_sms * 2, 256, 0, st>>>((const float4 *)xyz, n, S);
    grid_setup_kernel<<<1, 1, 0, st>>>(n, S);
    cell_count_kernel<<<g1, 256, 0, st>>>((const float4 *)xyz, mode == 1 ? (const float4 *)rgb : nullptr, n, S);
    scan_counts_kernel<<<(unsigned)S.scan_tiles, 256, 0, st>>>(S.counts, S.ncell_max, S.start, S, status,
                                                               kSpinLimit);
    scatter_kernel<<<g1, 256, 0, st>>>((const float4 *)xyz, n, S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uint32_t *knn = knn_idx ? knn_idx : S.knn;
    const p2e_kernel_probe *pr = kernel_probe(P2E_PROBE_KNN);
    const unsigned kgrid = (unsigned)((n + kKnnThreads - 1) / kKnnThreads);
    probe_start(pr, st);
    knn_count_kernel<<<kgrid, kKnnThreads, 0, st>>>(n, S);
    knn_select_kernel<<<kgrid, kKnnThreads, 0, st>>>(n, S, knn);
    probe_stop(pr, st);
    // the listed queries, one warp each (their number is on the device)
    knn_slow_kernel<<<num_sms * 8, kSlowWarps * 32, 0, st>>>(S, knn);
    pca_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float4 *)xyz, (const float4 *)rgb, n, pca_opacity, S, knn, (float4 *)out->mean_op,
        (float4 *)out->scale, (float4 *)out->quat, (float4 *)out->rgb, (float4 *)out->normal);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (mode == 1) return launch_mlp_estimate(S.pk, n, mlp, knn, out, (int32_t *)(S.ticket + 9), num_sms, st);
    return cudaSuccess;
}

// Status of the last p2e_estimate (or p2e_estimate_global) call on this
// scratch: P2E_ERR_TIMEOUT if one of its bounded device waits gave up.
// Synchronises the stream.
cudaError_t estimate_status(const void *scratch, int64_t n, cudaStream_t st, int32_t *out) {
    EstScratch S;
    est_layout(n, const_cast<void *>(scratch), &S);
    int32_t w[2] = {0, 0};
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpy(w, S.ticket + 8, sizeof w, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
    *out = w[0] != 0 ? w[0] : w[1];
    return cudaSuccess;
}

// Timeout self-test of the cell-count scan: two tiles of counts whose work
// tickets start at 1, so the only CTA takes tile 1 and waits on tile 0's
// look-back word, which nothing publishes; the wait gives up after
// `spin_limit` tries and records P2E_ERR_TIMEOUT.
__global__ void selftest_scan_init_kernel(uint32_t *ticket) {
    if (threadIdx.x == 0) *ticket = 1u;
}

size_t selftest_scan_bytes() { return al256(2 * kScanT * 4) + al256((2 * kScanT + 1) * 4) + al256(64) + al256(64); }

cudaError_t launch_selftest_scan(void *scratch, int32_t *status, uint32_t spin_limit, cudaStream_t st) {
    char *p = (char *)scratch;
    EstScratch S;
    memset(&S, 0, sizeof S);
    uint32_t *counts = (uint32_t *)p;
    p += al256(2 * kScanT * 4);
    uint32_t *start = (uint32_t *)p;
    p += al256((2 * kScanT + 1) * 4);
    S.ticket = (uint32_t *)p;
    p += al256(64);
    S.scan_state = (uint64_t *)p;
    cudaError_t e = cudaMemsetAsync(scratch, 0, selftest_scan_bytes(), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    selftest_scan_init_kernel<<<1, 32, 0, st>>>(S.ticket);
    scan_counts_kernel<<<1, 256, 0, st>>>(counts, 2 * kScanT, start, S, status, spin_limit);
    return cudaGetLastError();
}

// The global isotropic baseline: the mean nearest-neighbour distance over
// the cloud (double sum, one atomic per CTA), then every Gaussian gets scale
// sigma_rel times it, the identity rotation; mean, opacity, colour and the
// PCA normal stay as the kNN-PCA pass wrote them.
__global__ void __launch_bounds__(256) nn_dist_sum_kernel(const float4 *__restrict__ xyz, int64_t n,
                                                          const uint32_t *__restrict__ knn, double *sum) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(xyz + i), q = __ldg(xyz + knn[i * kK]);
        const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
        acc += (double)sqrtf(dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
        atomicAdd(sum, t);
    }
}

__global__ void __launch_bounds__(256) global_scale_kernel(int64_t n, const double *sum, float sigma_rel,
                                                           float4 *__restrict__ scale, float4 *__restrict__ quat) {
    const float s = (float)((double)sigma_rel * (*sum / (double)n));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        scale[i] = make_float4(s, s, s, 0.f);
        quat[i] = make_float4(1.f, 0.f, 0.f, 0.f);
    }
}

cudaError_t launch_estimate_global(const float *xyz, const float *rgb, int64_t n, float sigma_rel, float opacity,
                                   p2e_gaussians *out, uint32_t *knn_idx, void *scratch, int num_sms,
                                   cudaStream_t st) {
    EstScratch S;
    est_layout(n, scratch, &S);
    uint32_t *knn = knn_idx ? knn_idx : S.knn;
    cudaError_t e = launch_estimate(xyz, rgb, n, 0, nullptr, opacity, out, knn, scratch, num_sms, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S.sum, 0, sizeof(double), st)) != cudaSuccess) return e;
    nn_dist_sum_kernel<<<num_sms * 2, 256, 0, st>>>((const float4 *)xyz, n, knn, S.sum);
    global_scale_kernel<<<num_sms * 4, 256, 0, st>>>(n, S.sum, sigma_rel, (float4 *)out->scale,
                                                     (float4 *)out->quat);
    return cudaGetLastError();
}

}  // namespace p2e
