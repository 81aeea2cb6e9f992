// C ABI of libp2e: host-side validation, per-view constants and launches.
// Declarations and the contract of every entry point are in include/p2e.h.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace p2e {
cudaError_t launch_project(const p2e_gaussians *g, const Views &P, p2e_projected *out, cudaStream_t st);
cudaError_t launch_sort_bin(const p2e_projected *proj, const Views &P, p2e_bins *io, int num_sms,
                            cudaStream_t st);
cudaError_t launch_render(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                          const Views &P, float *rgb, float *nrm, float *depth, float *alpha,
                          uint32_t *last, cudaStream_t st);
size_t sort_scratch_bytes(int64_t n_total, int64_t capacity);
int sort_passes(int64_t total_tiles);
size_t backward_scratch_bytes(int64_t n_total);
size_t estimate_scratch_bytes(int64_t n);
cudaError_t launch_estimate_global(const float *xyz, const float *rgb, int64_t n, float sigma_rel, float opacity,
                                   p2e_gaussians *out, uint32_t *knn_idx, void *scratch, int num_sms,
                                   cudaStream_t st);
cudaError_t launch_render_backward(const p2e_gaussians *g, const p2e_projected *proj,
                                   const p2e_bins *bins, const Views &P, const float *alpha,
                                   const uint32_t *last, const float *d_rgb, const float *d_normal,
                                   const float *d_depth, const float *d_alpha, float *d_mean,
                                   float *d_scale, float *d_quat, float *d_opacity, float *d_rgb_g,
                                   float *d_normal_g, void *scratch, cudaStream_t st);
cudaError_t launch_estimate(const float *xyz, const float *rgb, int64_t n, int32_t mode,
                            const void *mlp, float pca_opacity, p2e_gaussians *out,
                            uint32_t *knn_idx, void *scratch, int num_sms, cudaStream_t st);

cudaError_t estimate_status(const void *scratch, int64_t n, cudaStream_t st, int32_t *out);
size_t selftest_sort_bytes();
size_t selftest_scan_bytes();
cudaError_t launch_selftest_sort(void *scratch, int32_t *status, uint32_t spin_limit, cudaStream_t st);
cudaError_t launch_selftest_scan(void *scratch, int32_t *status, uint32_t spin_limit, cudaStream_t st);
cudaError_t launch_selftest_mbar(int32_t *status, uint32_t spin_limit, cudaStream_t st);
cudaError_t launch_selftest_queue(int which, int32_t *status, uint32_t spin_limit, cudaStream_t st);

// Probes are per host thread: a thread measuring its launches does not
// disturb launches from other threads.
static thread_local p2e_kernel_probe t_probe[P2E_PROBE_COUNT];
static thread_local bool t_probe_on[P2E_PROBE_COUNT];

const p2e_kernel_probe *kernel_probe(int kernel) {
    if (kernel < 0 || kernel >= P2E_PROBE_COUNT || !t_probe_on[kernel]) return nullptr;
    return &t_probe[kernel];
}

int device_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    if (dev >= 0 && dev < 64) cache[dev] = sms;
    return sms;
}
}  // namespace p2e

using namespace p2e;

static bool fin(float x) { return isfinite(x) != 0; }
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static p2e_status fill_views(const p2e_camera *cams, int32_t n_views, const p2e_config *cfg,
                             int64_t n, Views &P) {
    if (!cams || !cfg || n_views < 1 || n_views > P2E_MAX_VIEWS || n < 0) return P2E_ERR_INVALID_ARG;
    if (!(cfg->tile == 8 || cfg->tile == 16 || cfg->tile == 32)) return P2E_ERR_INVALID_ARG;
    if (!fin(cfg->alpha_floor) || !fin(cfg->alpha_max) || !fin(cfg->t_min) || !fin(cfg->lowpass) ||
        !fin(cfg->sigma_mult) || cfg->lowpass < 0.f || !(cfg->sigma_mult > 0.f) ||
        cfg->alpha_floor < 0.f || !(cfg->alpha_max > 0.f) || cfg->alpha_max > 1.f ||
        cfg->t_min < 0.f || !(cfg->t_min < 1.f))
        return P2E_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c)
        if (!fin(cfg->bg[c])) return P2E_ERR_INVALID_ARG;
    if (cfg->schedule != P2E_SCHEDULE_AUTO && cfg->schedule != P2E_SCHEDULE_PER_BLOCK) return P2E_ERR_INVALID_ARG;
    memset(&P, 0, sizeof(P));
    P.n_views = n_views;
    P.tile = cfg->tile;
    P.lowpass = cfg->lowpass;
    P.sigma_mult = cfg->sigma_mult;
    P.alpha_floor = cfg->alpha_floor;
    P.alpha_max = cfg->alpha_max;
    P.t_min = cfg->t_min;
    for (int c = 0; c < 3; ++c) P.bg[c] = cfg->bg[c];
    P.schedule = cfg->schedule;
    P.n = n;
    int64_t tb = 0, pb = 0;
    for (int v = 0; v < n_views; ++v) {
        const p2e_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 8192 || c.height > 8192) return P2E_ERR_INVALID_ARG;
        for (int i = 0; i < 12; ++i)
            if (!fin(c.viewmat[i])) return P2E_ERR_INVALID_ARG;
        if (!fin(c.fx) || !fin(c.fy) || !fin(c.cx) || !fin(c.cy) || !fin(c.near_z) || c.near_z < 0.f)
            return P2E_ERR_INVALID_ARG;
        View &V = P.v[v];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) V.T[3 * i + j] = c.viewmat[4 * i + j];
            V.t[i] = c.viewmat[4 * i + 3];
        }
        V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy; V.near_z = c.near_z;
        V.W = c.width; V.H = c.height;
        V.tiles_x = (c.width + cfg->tile - 1) / cfg->tile;
        V.tiles_y = (c.height + cfg->tile - 1) / cfg->tile;
        V.tile_base = tb;
        V.pix_base = pb;
        tb += (int64_t)V.tiles_x * V.tiles_y;
        pb += (int64_t)c.width * c.height;
    }
    P.total_tiles = tb;
    if (tb >= (int64_t(1) << 31)) return P2E_ERR_INVALID_ARG;
    return P2E_OK;
}

static p2e_status check_gaussians(const p2e_gaussians *g) {
    if (!g || g->n < 0 || g->n >= (int64_t(1) << 31)) return P2E_ERR_INVALID_ARG;
    if (g->n == 0) return P2E_OK;
    const void *ps[5] = {g->mean_op, g->scale, g->quat, g->rgb, g->normal};
    for (int i = 0; i < 5; ++i)
        if (!ps[i] || !aligned16(ps[i])) return P2E_ERR_INVALID_ARG;
    return P2E_OK;
}

static p2e_status check_proj(const p2e_projected *p) {
    if (!p || !p->xy_depth || !p->conic_op || !p->rect || !p->ntiles) return P2E_ERR_INVALID_ARG;
    if (!aligned16(p->xy_depth) || !aligned16(p->conic_op) || ((uintptr_t)p->rect & 7u) ||
        ((uintptr_t)p->ntiles & 3u))
        return P2E_ERR_INVALID_ARG;
    return P2E_OK;
}

extern "C" {

p2e_config p2e_default_config(void) {
    p2e_config c;
    c.tile = 16;
    c.alpha_floor = 1.0f / 255.0f;
    c.alpha_max = 0.99f;
    c.t_min = 1e-4f;
    c.lowpass = 0.3f;
    c.sigma_mult = 3.0f;
    c.bg[0] = c.bg[1] = c.bg[2] = 0.0f;
    c.schedule = P2E_SCHEDULE_AUTO;
    return c;
}

int64_t p2e_total_tiles(const p2e_camera *cams, int32_t n_views, int32_t tile) {
    p2e_config c = p2e_default_config();
    c.tile = tile;
    Views P;
    if (fill_views(cams, n_views, &c, 0, P) != P2E_OK) return -1;
    return P.total_tiles;
}

size_t p2e_scratch_bytes(int32_t which, int64_t n, int64_t capacity) {
    if (n < 0 || capacity < 0) return 0;
    switch (which) {
        case P2E_SCRATCH_SORT: return sort_scratch_bytes(n, capacity);
        case P2E_SCRATCH_ESTIMATE: return estimate_scratch_bytes(n);
        case P2E_SCRATCH_BACKWARD: return backward_scratch_bytes(n);
        default: return 0;
    }
}

const char *p2e_status_string(p2e_status s) {
    switch (s) {
        case P2E_OK: return "ok";
        case P2E_ERR_INVALID_ARG: return "invalid argument";
        case P2E_ERR_CAPACITY: return "key capacity exceeded";
        case P2E_ERR_CUDA: return "CUDA error";
        case P2E_ERR_TIMEOUT: return "device wait timed out";
        case P2E_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

p2e_status p2e_project(const p2e_gaussians *g, const p2e_camera *cams, int32_t n_views,
                       const p2e_config *cfg, p2e_projected *out, void *stream) {
    p2e_status s = check_gaussians(g);
    if (s != P2E_OK) return s;
    Views P;
    if ((s = fill_views(cams, n_views, cfg, g->n, P)) != P2E_OK) return s;
    if (g->n > 0 && (s = check_proj(out)) != P2E_OK) return s;
    return launch_project(g, P, out, (cudaStream_t)stream) == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

p2e_status p2e_sort_bin(const p2e_projected *proj, int64_t n, const p2e_camera *cams, int32_t n_views,
                        const p2e_config *cfg, p2e_bins *io, void *stream) {
    if (n < 0 || n >= (int64_t(1) << 31) || !io) return P2E_ERR_INVALID_ARG;
    Views P;
    p2e_status s = fill_views(cams, n_views, cfg, n, P);
    if (s != P2E_OK) return s;
    if (n > 0 && (s = check_proj(proj)) != P2E_OK) return s;
    if (io->capacity < 0 || io->capacity >= (int64_t(1) << 30)) return P2E_ERR_INVALID_ARG;
    if (!io->ranges || !io->tile_work || !io->n_keys_dev || !io->status_dev || !io->scratch)
        return P2E_ERR_INVALID_ARG;
    if (io->capacity > 0 && (!io->keys[0] || !io->keys[1] || !io->vals[0] || !io->vals[1]))
        return P2E_ERR_INVALID_ARG;
    if (((uintptr_t)io->scratch & 255u) || ((uintptr_t)io->ranges & 7u)) return P2E_ERR_INVALID_ARG;
    if (io->scratch_bytes < (int64_t)sort_scratch_bytes(n * n_views, io->capacity))
        return P2E_ERR_INVALID_ARG;
    if (sort_passes(P.total_tiles) > 8) return P2E_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(io->status_dev, 0, sizeof(int32_t), st) != cudaSuccess) return P2E_ERR_CUDA;
    return launch_sort_bin(proj, P, io, device_sms(), st) == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

p2e_status p2e_bins_check(const p2e_bins *io, int64_t *n_keys_host, void *stream) {
    if (!io || !io->n_keys_dev || !io->status_dev) return P2E_ERR_INVALID_ARG;
    int64_t k = 0;
    int32_t st = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return P2E_ERR_CUDA;
    if (cudaMemcpy(&k, io->n_keys_dev, sizeof k, cudaMemcpyDeviceToHost) != cudaSuccess) return P2E_ERR_CUDA;
    if (cudaMemcpy(&st, io->status_dev, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) return P2E_ERR_CUDA;
    if (n_keys_host) *n_keys_host = k;
    if (st != 0) return (p2e_status)st;
    return k > io->capacity ? P2E_ERR_CAPACITY : P2E_OK;
}

p2e_status p2e_render(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                      const p2e_camera *cams, int32_t n_views, const p2e_config *cfg, float *rgb,
                      float *normal, float *depth, float *alpha, uint32_t *last, void *stream) {
    p2e_status s = check_gaussians(g);
    if (s != P2E_OK) return s;
    Views P;
    if ((s = fill_views(cams, n_views, cfg, g->n, P)) != P2E_OK) return s;
    if (g->n > 0 && (s = check_proj(proj)) != P2E_OK) return s;
    if (!bins || !bins->ranges || !bins->tile_work || (bins->result != 0 && bins->result != 1))
        return P2E_ERR_INVALID_ARG;
    if (bins->capacity > 0 && !bins->vals[bins->result]) return P2E_ERR_INVALID_ARG;
    return launch_render(g, proj, bins, P, rgb, normal, depth, alpha, last, (cudaStream_t)stream) ==
                   cudaSuccess
               ? P2E_OK
               : P2E_ERR_CUDA;
}

p2e_status p2e_render_backward(const p2e_gaussians *g, const p2e_projected *proj,
                               const p2e_bins *bins, const p2e_camera *cams, int32_t n_views,
                               const p2e_config *cfg, const float *alpha, const uint32_t *last,
                               const float *d_rgb, const float *d_normal, const float *d_depth,
                               const float *d_alpha, float *d_mean, float *d_scale, float *d_quat,
                               float *d_opacity, float *d_rgb_g, float *d_normal_g, void *scratch,
                               int64_t scratch_bytes, void *stream) {
    p2e_status s = check_gaussians(g);
    if (s != P2E_OK) return s;
    Views P;
    if ((s = fill_views(cams, n_views, cfg, g->n, P)) != P2E_OK) return s;
    if (g->n > 0 && (s = check_proj(proj)) != P2E_OK) return s;
    if (!bins || !bins->ranges || (bins->result != 0 && bins->result != 1)) return P2E_ERR_INVALID_ARG;
    if (!last) return P2E_ERR_INVALID_ARG;
    if (g->n > 0 && (!d_mean || !d_scale || !d_quat || !d_opacity || !d_rgb_g || !d_normal_g))
        return P2E_ERR_INVALID_ARG;
    if (scratch_bytes < (int64_t)backward_scratch_bytes(g->n * n_views) ||
        (scratch_bytes > 0 && (!scratch || ((uintptr_t)scratch & 255u))))
        return P2E_ERR_INVALID_ARG;
    return launch_render_backward(g, proj, bins, P, alpha, last, d_rgb, d_normal, d_depth, d_alpha,
                                  d_mean, d_scale, d_quat, d_opacity, d_rgb_g, d_normal_g, scratch,
                                  (cudaStream_t)stream) == cudaSuccess
               ? P2E_OK
               : P2E_ERR_CUDA;
}

p2e_status p2e_estimate(const float *xyz, const float *rgb, int64_t n, int32_t mode,
                        const void *mlp_weights, float pca_opacity, p2e_gaussians *out,
                        uint32_t *knn_idx, void *scratch, int64_t scratch_bytes, void *stream) {
    if (n < 0 || n >= (int64_t(1) << 31) || !out || (mode != 0 && mode != 1)) return P2E_ERR_INVALID_ARG;
    if (!fin(pca_opacity) || pca_opacity < 0.f || pca_opacity > 1.f) return P2E_ERR_INVALID_ARG;
    if (mode == 1 && !mlp_weights) return P2E_ERR_INVALID_ARG;
    if (n == 0) return P2E_OK;
    if (n < 17) return P2E_ERR_INVALID_ARG;  // 16 neighbours need 17 points
    if (!xyz || !rgb || !aligned16(xyz) || !aligned16(rgb)) return P2E_ERR_INVALID_ARG;
    if (!out->mean_op || !out->scale || !out->quat || !out->rgb || !out->normal) return P2E_ERR_INVALID_ARG;
    if (!aligned16(out->mean_op) || !aligned16(out->scale) || !aligned16(out->quat) ||
        !aligned16(out->rgb) || !aligned16(out->normal))
        return P2E_ERR_INVALID_ARG;
    if (scratch_bytes < (int64_t)estimate_scratch_bytes(n) || !scratch || ((uintptr_t)scratch & 255u))
        return P2E_ERR_INVALID_ARG;
    if (knn_idx && !aligned16(knn_idx)) return P2E_ERR_INVALID_ARG;
    cudaError_t e = launch_estimate(xyz, rgb, n, mode, mlp_weights, pca_opacity, out, knn_idx, scratch,
                                    device_sms(), (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) return P2E_ERR_UNSUPPORTED;
    return e == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

p2e_status p2e_estimate_global(const float *xyz, const float *rgb, int64_t n, float sigma_rel, float opacity,
                               p2e_gaussians *out, uint32_t *knn_idx, void *scratch, int64_t scratch_bytes,
                               void *stream) {
    if (n < 0 || n >= (int64_t(1) << 31) || !out) return P2E_ERR_INVALID_ARG;
    if (!fin(opacity) || opacity < 0.f || opacity > 1.f || !fin(sigma_rel) || !(sigma_rel > 0.f))
        return P2E_ERR_INVALID_ARG;
    if (n == 0) return P2E_OK;
    if (n < 17) return P2E_ERR_INVALID_ARG;
    if (!xyz || !rgb || !aligned16(xyz) || !aligned16(rgb)) return P2E_ERR_INVALID_ARG;
    if (!out->mean_op || !out->scale || !out->quat || !out->rgb || !out->normal) return P2E_ERR_INVALID_ARG;
    if (!aligned16(out->mean_op) || !aligned16(out->scale) || !aligned16(out->quat) ||
        !aligned16(out->rgb) || !aligned16(out->normal))
        return P2E_ERR_INVALID_ARG;
    if (scratch_bytes < (int64_t)estimate_scratch_bytes(n) || !scratch || ((uintptr_t)scratch & 255u))
        return P2E_ERR_INVALID_ARG;
    if (knn_idx && !aligned16(knn_idx)) return P2E_ERR_INVALID_ARG;
    cudaError_t e = launch_estimate_global(xyz, rgb, n, sigma_rel, opacity, out, knn_idx, scratch, device_sms(),
                                           (cudaStream_t)stream);
    return e == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

p2e_status p2e_set_kernel_probe(int32_t kernel, const p2e_kernel_probe *probe) {
    if (kernel < 0 || kernel >= P2E_PROBE_COUNT) return P2E_ERR_INVALID_ARG;
    if (probe) {
        t_probe[kernel] = *probe;
        t_probe_on[kernel] = true;
    } else {
        t_probe_on[kernel] = false;
    }
    return P2E_OK;
}

p2e_status p2e_estimate_check(const void *scratch, int64_t scratch_bytes, int64_t n, void *stream) {
    if (n < 17 || n >= (int64_t(1) << 31) || !scratch || ((uintptr_t)scratch & 255u) ||
        scratch_bytes < (int64_t)estimate_scratch_bytes(n))
        return P2E_ERR_INVALID_ARG;
    int32_t st = 0;
    if (estimate_status(scratch, n, (cudaStream_t)stream, &st) != cudaSuccess) return P2E_ERR_CUDA;
    return st != 0 ? (p2e_status)st : P2E_OK;
}

p2e_status p2e_selftest_timeout(int32_t which, uint32_t spin_limit, void *scratch, int64_t scratch_bytes,
                                int32_t *status_dev, void *stream) {
    if (which < 0 || which > 4 || spin_limit < 1 || spin_limit > kSpinLimit || !status_dev || !scratch ||
        ((uintptr_t)scratch & 255u) || ((uintptr_t)status_dev & 3u) || scratch_bytes < P2E_SELFTEST_SCRATCH_BYTES)
        return P2E_ERR_INVALID_ARG;
    if (selftest_sort_bytes() > P2E_SELFTEST_SCRATCH_BYTES || selftest_scan_bytes() > P2E_SELFTEST_SCRATCH_BYTES)
        return P2E_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = which == 0   ? launch_selftest_sort(scratch, status_dev, spin_limit, st)
                    : which == 1 ? launch_selftest_scan(scratch, status_dev, spin_limit, st)
                    : which == 2 ? launch_selftest_mbar(status_dev, spin_limit, st)
                                 : launch_selftest_queue(which - 3, status_dev, spin_limit, st);
    return e == cudaSuccess ? P2E_OK : P2E_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// p2e_sort_bin_noalloc: p2e_sort_bin with its scratch in a fixed device
// array owned by this library, for callers that may not allocate device
// memory (see include/p2e.h).  The array lives as long as the library is
// loaded, on every device it is used on.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoallocScratchBytes = 4456448;  // 4.25 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
static void *g_noalloc_addr[64];  // device address of the array, per device, 0 = not set up
}  // namespace

extern "C" p2e_status p2e_sort_bin_noalloc(const p2e_projected *proj, int64_t n, const p2e_camera *cams,
                                           int32_t n_views, const p2e_config *cfg, p2e_bins *io,
                                           void *stream) {
    // n is bounded before it is multiplied by the view count
    if (!io || n < 0 || n > P2E_NOALLOC_MAX_N || n_views < 1 || n_views > P2E_MAX_VIEWS) return P2E_ERR_INVALID_ARG;
    if (n * n_views > P2E_NOALLOC_MAX_N || io->capacity > P2E_NOALLOC_MAX_CAPACITY || io->capacity < 0)
        return P2E_ERR_INVALID_ARG;
    if (sort_scratch_bytes(n * n_views, io->capacity) > kNoallocScratchBytes) return P2E_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return P2E_ERR_CUDA;
    if (!g_noalloc_addr[dev]) {
        // first call on this device: look up the array's device address
        // (host code cannot use the symbol itself as a device pointer)
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return P2E_ERR_CUDA;
        g_noalloc_addr[dev] = ptr;
    }
    p2e_bins local = *io;
    local.scratch = g_noalloc_addr[dev];
    local.scratch_bytes = (int64_t)kNoallocScratchBytes;
    const p2e_status s = p2e_sort_bin(proj, n, cams, n_views, cfg, &local, stream);
    io->result = local.result;
    return s;
}
