// Shared device-side definitions of libp2e (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "p2e.h"

namespace p2e {

// Per-view constants, passed by value in a __grid_constant__ kernel
// parameter (at most P2E_MAX_VIEWS views per call).
struct View {
    float T[9];          // rotation rows of [T | t] (Eq. 3)
    float t[3];
    float fx, fy, cx, cy, near_z;
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    int64_t tile_base;   // first tile id of the view
    int64_t pix_base;    // first pixel of the view in the planar outputs
};

struct Views {
    int32_t n_views;
    int32_t tile;
    float lowpass, sigma_mult;
    float alpha_floor, alpha_max, t_min;
    float bg[3];
    int32_t schedule;    // P2E_SCHEDULE_*
    int64_t n;           // Gaussians per view
    int64_t total_tiles;
    View v[P2E_MAX_VIEWS];
};

// Upper bound on device spin iterations before a wait gives up and records
// P2E_ERR_TIMEOUT (each iteration sleeps ~32-256 ns, so a few hundred ms).
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ void backoff(uint32_t it) {
    __nanosleep(it < 8 ? 32 : 256);
}

// ---------------------------------------------------------------------------
// Error-free transformations in fp32 (Dekker/Knuth), used to carry a value
// as an unevaluated sum hi + lo with about 48 significant bits.  Explicit
// _rn intrinsics keep the compiler from contracting or reordering them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Index of the view that owns flat tile id `tile` (views are few; linear).
__device__ __forceinline__ int view_of_tile(const Views &P, int64_t tile) {
    int v = 0;
    while (v + 1 < P.n_views && P.v[v + 1].tile_base <= tile) ++v;
    return v;
}

// Measurement probe of one kernel (p2e_set_kernel_probe), or nullptr when
// the calling host thread has none set for it.
const p2e_kernel_probe *kernel_probe(int kernel);

// Events of a probe around one launch, recorded on the launching stream.
inline void probe_start(const p2e_kernel_probe *pr, cudaStream_t st) {
    if (pr && pr->start_event) cudaEventRecord((cudaEvent_t)pr->start_event, st);
}
inline void probe_stop(const p2e_kernel_probe *pr, cudaStream_t st) {
    if (pr && pr->stop_event) cudaEventRecord((cudaEvent_t)pr->stop_event, st);
}

}  // namespace p2e

#define P2E_CUDA_CHECK_LAUNCH()                                  \
    do {                                                         \
        if (cudaGetLastError() != cudaSuccess) return P2E_ERR_CUDA; \
    } while (0)
