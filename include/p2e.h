/*
 * p2e.h -- C ABI of libp2e.so, the GB300 (sm_103a) splatting renderer and
 * point-to-ellipsoid estimator of "Low Latency Point Cloud Rendering with
 * Learned Splatting" (arXiv 2409.16504).
 *
 * Problem statement (Sec. 3.1): a coloured point cloud P = {(p_i, c_i)} and a
 * viewpoint in; RGB, normal and depth images out.  Each point becomes a 3D
 * Gaussian <G(p, Sigma), o, c, n> (Sec. 3.1, 3.2); the Gaussians are splatted
 * with the EWA screen covariance (Eq. 3-4), bounded at three standard
 * deviations, depth-ordered and alpha-composited front to back (Eq. 1-2).
 *
 * Conventions shared by every call
 *   * Ownership: every pointer is caller-owned.  Pointers named *_dev or
 *     documented as "device" are CUDA device memory; structs passed by
 *     pointer (p2e_camera, p2e_config and the descriptor structs themselves)
 *     live in host memory.  The library never allocates or frees device
 *     memory and keeps no state between calls.
 *   * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Every call only enqueues work on it and returns without synchronising,
 *     except p2e_bins_check (documented below).
 *   * Errors: arguments are validated on the host before anything is
 *     enqueued; an invalid argument returns P2E_ERR_INVALID_ARG and enqueues
 *     nothing.  A failed launch returns P2E_ERR_CUDA.  Key-capacity overflow
 *     is detected on the device (see p2e_sort_bin) and reported by
 *     p2e_bins_check.  No call traps, asserts or spins without bound on the
 *     device: bounded waits record P2E_ERR_TIMEOUT in a device status word.
 *   * Layout: per-Gaussian arrays are float4 structure-of-arrays (16-byte
 *     aligned, coalesced 16-byte loads).  Images are planar fp32, views
 *     concatenated in order; view v occupies H_v*W_v pixels per plane.
 */
#ifndef P2E_H
#define P2E_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    P2E_OK = 0,
    P2E_ERR_INVALID_ARG = 1,
    P2E_ERR_CAPACITY = 2,
    P2E_ERR_CUDA = 3,
    P2E_ERR_TIMEOUT = 4,
    P2E_ERR_UNSUPPORTED = 5
} p2e_status;

#define P2E_MAX_VIEWS 64
#define P2E_MAX_LIGHTS 8

/* Pinhole camera (Sec. 3.1, Eq. 3-4), host memory.
 * viewmat: row-major 3x4 [T | t] mapping world to camera coordinates
 * (OpenCV axes: x right, y down, z forward).  fx, fy, cx, cy in pixels;
 * pixel (i, j) has its centre at (i + 0.5, j + 0.5).  Gaussians with camera
 * depth z <= near_z are culled.  1 <= width, height <= 8192. */
typedef struct {
    float viewmat[12];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;
} p2e_camera;

/* Renderer constants (host memory).  The paper fixes none of them; the
 * defaults (p2e_default_config) are those of the 3D Gaussian splatting
 * renderer the paper follows (Sec. 3.1):
 *   tile        8, 16 or 32 pixels (square screen tiles for binning)
 *   alpha_floor splats with alpha < alpha_floor are skipped   (1/255)
 *   alpha_max   alpha = min(alpha_max, o exp(power))           (0.99)
 *   t_min       compositing stops before T would drop below    (1e-4)
 *   lowpass     px^2 added to the screen covariance diagonal   (0.3)
 *   sigma_mult  splat boundary in standard deviations (Sec. 3.1: 3)
 *   bg          background colour composited with the final T  (0,0,0)
 *   schedule    compositing work schedule (no effect on the images, which
 *               are bit-identical either way): P2E_SCHEDULE_AUTO (0) chains
 *               the segments of long tile lists across warps, longest
 *               tiles first, while their states fit in the free half of
 *               the key buffers (8 bytes per key of a chained segment), and
 *               has one warp per (tile, pixel block) take the rest;
 *               P2E_SCHEDULE_PER_BLOCK (1) has one warp composite all
 *               segments of every (tile, pixel block) in turn.  In
 *               p2e_render_backward AUTO walks tile lists longer than
 *               4 x tile^2 splats as segments of that length in parallel
 *               (gradients equal up to fp32 rounding order), PER_BLOCK
 *               walks every list whole. */
enum { P2E_SCHEDULE_AUTO = 0, P2E_SCHEDULE_PER_BLOCK = 1 };
typedef struct {
    int32_t tile;
    float alpha_floor, alpha_max, t_min, lowpass, sigma_mult;
    float bg[3];
    int32_t schedule;
} p2e_config;

/* Gaussian set, device memory, n entries each (Sec. 3.1, 11 parameters plus
 * colour and normal):
 *   mean_op  float4 (x, y, z, opacity o in [0,1])
 *   scale    float4 (sx, sy, sz, unused), linear standard deviations > 0
 *   quat     float4 (w, x, y, z), any non-zero quaternion (normalised
 *            inside; the zero quaternion culls the Gaussian).
 *            Sigma = R diag(s^2) R^T, R the rotation of the unit quaternion.
 *   rgb      float4 (r, g, b, unused)
 *   normal   float4 (nx, ny, nz, unused) */
typedef struct {
    const float *mean_op;
    const float *scale;
    const float *quat;
    const float *rgb;
    const float *normal;
    int64_t n;
} p2e_gaussians;

/* Projected splats, device memory, n_views * n entries (view-major):
 *   xy_depth float4 (u - floor(u), v - floor(v), depth key, bits of
 *            int16 floor(u) | int16 floor(v) << 16); floor(u), floor(v)
 *            are clamped to [-32768, 32767].
 *   conic_op float4 (A, B, C, o): Sigma_s^{-1} = [[A, B], [B, C]]
 *   rect     ushort4 (x0, y0, x1, y1): inclusive pixel rectangle of the
 *            splat's sigma_mult ellipse box.  Its tiles (x / tile, y / tile)
 *            are exact; the pixel bounds are exact or a superset clamped to
 *            those tiles (used only to skip splats early).
 *   ntiles   uint32 number of tiles touched (0 = culled) */
typedef struct {
    float *xy_depth;
    float *conic_op;
    uint16_t *rect;
    uint32_t *ntiles;
} p2e_projected;

/* Binning buffers, device memory, caller-owned.
 *   keys[2], vals[2]  double buffers of `capacity` entries each
 *   ranges            uint2 per tile of all views: [start, end) into the
 *                     sorted arrays; empty tiles hold [0, 0)
 *   scratch           p2e_scratch_bytes(P2E_SCRATCH_SORT, n*n_views,
 *                     capacity) bytes, 256-byte aligned
 *   n_keys_dev        int64: number of keys the views need (may exceed
 *                     capacity, in which case nothing past capacity is
 *                     written and the sorted result is invalid)
 *   status_dev        int32 device status word (P2E_OK, or P2E_ERR_TIMEOUT
 *                     when a bounded device wait gave up)
 *   tile_work         uint32[total tiles + 2]: written by p2e_sort_bin
 *                     ([0] = number of non-empty tiles, [1] = a counter
 *                     p2e_render resets, then the non-empty tile ids,
 *                     longest list first) and consumed by p2e_render
 *   result            written by p2e_sort_bin (host field): index (0 or 1)
 *                     of the buffer pair that holds the sorted keys/vals */
typedef struct {
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint32_t *ranges;
    uint32_t *tile_work;
    void *scratch;
    int64_t scratch_bytes;
    int64_t capacity;
    int64_t *n_keys_dev;
    int32_t *status_dev;
    int32_t result;
} p2e_bins;

enum { P2E_SCRATCH_SORT = 0, P2E_SCRATCH_ESTIMATE = 1, P2E_SCRATCH_BACKWARD = 2 };

#define P2E_MLP_BLOB_BYTES 31552

/* Defaults of p2e_config (see above). */
p2e_config p2e_default_config(void);

/* Total tile count of the views for a tile size (sum over views of
 * ceil(W/tile) * ceil(H/tile)). Returns -1 on invalid input. */
int64_t p2e_total_tiles(const p2e_camera *cams, int32_t n_views, int32_t tile);

/* Bytes of device scratch a call needs (`which` = P2E_SCRATCH_*; n = number
 * of Gaussians (times views for SORT), capacity = key capacity). */
size_t p2e_scratch_bytes(int32_t which, int64_t n, int64_t capacity);

/* p2e_project -- EWA projection (Sec. 3.1, Eq. 3-4) and 3-sigma footprint.
 * For every view v and Gaussian g: camera transform, near cull,
 * Sigma = R diag(s^2) R^T, Sigma_s = J T Sigma T^T J^T + lowpass I, conic,
 * screen centre, and the tile rectangle of the exact bounding box of the
 * sigma_mult ellipse.  Integer results (cull, rectangle, depth key =
 * fp32 of the double-precision camera depth) equal those of an IEEE double
 * evaluation: an fp32 fast path carries an error bound and hands ambiguous
 * Gaussians to a double-precision path.
 * Writes out->* for n_views * g->n entries. */
p2e_status p2e_project(const p2e_gaussians *g, const p2e_camera *cams, int32_t n_views,
                       const p2e_config *cfg, p2e_projected *out, void *stream);

/* p2e_sort_bin -- duplication into (tile id | depth) keys, device radix sort
 * and per-tile ranges (Sec. 3.1: splats covering a pixel sorted by depth).
 * key = ((tile_base_v + ty * ceil(W_v/tile) + tx) << 32) | bits(depth key),
 * val = g; the result is the keys in ascending order, equal keys in
 * ascending Gaussian order (views in order).  When io->capacity >= n *
 * n_views the Gaussians are first sorted by depth (stable LSD passes on
 * the depth bits) and the keys, emitted in that order, are sorted stably
 * on the tile bits only; otherwise the keys, emitted in (view, Gaussian)
 * order, are sorted stably on all 32 + ceil(log2(total tiles)) significant
 * bits.  Both give the same result.  n = g->n used by p2e_project.
 * Writes io->n_keys_dev, the sorted pair io->keys/vals[io->result] and
 * io->ranges; the other key/value buffers are overwritten (scratch).  If
 * the key count exceeds io->capacity nothing is written past it and
 * p2e_bins_check reports P2E_ERR_CAPACITY. */
p2e_status p2e_sort_bin(const p2e_projected *proj, int64_t n, const p2e_camera *cams,
                        int32_t n_views, const p2e_config *cfg, p2e_bins *io, void *stream);

/* p2e_sort_bin_noalloc -- the same binning as p2e_sort_bin for callers that
 * are not allowed to allocate device memory: code running inside a host
 * application that owns the GPU's memory budget (an engine or compositor
 * plugin that is handed its buffers), or a latency-critical loop where a
 * cudaMalloc/cudaFree could stall or synchronise the device.  The paper has
 * no counterpart; this is a deployment convenience.
 * Its scratch is a fixed 4.25 MiB array inside libp2e that every GPU using
 * the library keeps until the process exits; io->scratch and
 * io->scratch_bytes are ignored, everything else in io is used as in
 * p2e_sort_bin and still belongs to the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * The address is kept for the life of the process, so this entry point
 * must not be used on a device after cudaDeviceReset of that device (the
 * reloaded module may place the array elsewhere).
 * Limits: n * n_views <= P2E_NOALLOC_MAX_N and io->capacity <=
 * P2E_NOALLOC_MAX_CAPACITY, otherwise P2E_ERR_INVALID_ARG is returned and
 * nothing is enqueued.  All calls share the one array (the call clears what
 * must start at zero), so calls whose work overlaps on the GPU -- on
 * different streams, or on different host threads -- race and give wrong
 * results; serialise them. */
#define P2E_NOALLOC_MAX_N (1 << 22)
#define P2E_NOALLOC_MAX_CAPACITY (1 << 21)
p2e_status p2e_sort_bin_noalloc(const p2e_projected *proj, int64_t n, const p2e_camera *cams,
                                int32_t n_views, const p2e_config *cfg, p2e_bins *io, void *stream);

/* p2e_bins_check -- synchronises `stream`, copies the key count to
 * *n_keys_host and returns P2E_ERR_CAPACITY if it exceeded io->capacity,
 * P2E_ERR_TIMEOUT if a device wait gave up, else P2E_OK. */
p2e_status p2e_bins_check(const p2e_bins *io, int64_t *n_keys_host, void *stream);

/* p2e_render -- front-to-back alpha compositing (Sec. 3.1, Eq. 1-2) of
 * colour, and by substitution of n_k and z_k for c_k, of normal and depth.
 * Per pixel over its tile's depth-sorted list: splats with
 * power = -0.5 d^T Sigma_s^{-1} d < -sigma_mult^2/2 are outside the splat;
 * alpha = min(alpha_max, o exp(power)); alpha < alpha_floor skipped;
 * compositing stops before a splat with T (1 - alpha) < t_min.
 * Outputs (device, planar fp32, views concatenated):
 *   rgb[3][H][W] = C + T bg, normal[3][H][W], depth[H][W], alpha[H][W] =
 *   1 - T, last[H][W] uint32 = one past the position of the pixel's last
 *   contributing splat in this call's sorted value array
 *   bins->vals[bins->result] (0 = none); vals[last - 1] is that splat's
 *   Gaussian index.  Positions count every view of the call, so `last`
 *   (unlike the other planes) depends on the batch a view is rendered in.
 *   Any output pointer may be NULL except `last` when a backward pass
 *   will follow.
 * Scratch: the free half of the key double buffer, keys[1 - result] and
 * vals[1 - result], is overwritten (the work-item table, per-segment
 * compositing states, arrival counters and flags); the sorted
 * keys/vals[result] are left intact.
 * Device waits are bounded (the chained schedule's warps wait for deferred
 * re-walks of other warps' segments); one that gives up sets
 * *bins->status_dev to P2E_ERR_TIMEOUT, which p2e_bins_check reports when
 * called after p2e_render (the next p2e_sort_bin clears it).  With
 * bins->status_dev NULL the one-warp-per-block schedule runs. */
p2e_status p2e_render(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                      const p2e_camera *cams, int32_t n_views, const p2e_config *cfg,
                      float *rgb, float *normal, float *depth, float *alpha, uint32_t *last,
                      void *stream);

/* p2e_render_backward -- exact gradient of p2e_render's outputs with
 * respect to the Gaussian parameters (the differentiable splatting used to
 * train the estimator, Sec. 1 and 3.3), with the discrete decisions (cull,
 * rectangle, 3-sigma test, floor, stop) held fixed.  Per tile and pixel
 * the transmittance is recomputed from the tile's sorted list and `last`:
 * front to back for the final T, then back to front through the
 * contributing splats; no per-pixel lists are stored.  A list longer than
 * 4 x tile^2 splats is split into segments of that length: a fold of each
 * segment (its transmittance product and weighted sum per pixel) gives
 * every segment's entering T and tail, and the segments' backward walks
 * run in parallel.  The item table and the folds use the free halves of
 * the bins' buffers (keys[1 - result], vals[1 - result], which
 * p2e_render uses as scratch too); with cfg->schedule PER_BLOCK, or with
 * no room there, lists are walked whole.  `alpha` (the
 * forward's alpha image) is not read and may be NULL: recovering T as
 * 1 - alpha would lose ~2.5e-4 relative accuracy on saturated pixels.
 * Inputs: the forward's arguments and outputs plus the upstream gradients
 * d_rgb[3][H][W], d_normal[3][H][W], d_depth[H][W], d_alpha[H][W] (any may
 * be NULL = zero).  Outputs (device, written, not accumulated; n entries):
 * d_mean[3n], d_scale[3n], d_quat[4n] (w.r.t. the raw quaternion),
 * d_opacity[n], d_rgb_g[3n], d_normal_g[3n].  scratch: p2e_scratch_bytes(
 * P2E_SCRATCH_BACKWARD, n * n_views, 0) bytes. */
p2e_status p2e_render_backward(const p2e_gaussians *g, const p2e_projected *proj,
                               const p2e_bins *bins, const p2e_camera *cams, int32_t n_views,
                               const p2e_config *cfg, const float *alpha, const uint32_t *last,
                               const float *d_rgb, const float *d_normal, const float *d_depth,
                               const float *d_alpha, float *d_mean, float *d_scale, float *d_quat,
                               float *d_opacity, float *d_rgb_g, float *d_normal_g,
                               void *scratch, int64_t scratch_bytes, void *stream);

/* p2e_estimate -- per-point ellipsoid estimation (Sec. 3.2 role: point cloud
 * in, <G(p, Sigma), o, n> out).  xyz, rgb: device float4[n] (w unused).
 * mode 0: closed-form kNN-PCA (k = 16 nearest neighbours, the local
 *   covariance prior of Sec. 2.1): Sigma from the neighbours' covariance,
 *   normal = smallest principal axis, opacity = pca_opacity.
 * mode 1: the learned per-point MLP (16 x (offset, colour) -> 64 -> 64 -> 64
 *   -> 8, bf16 weights, fp32 accumulation on tcgen05 tensor cores) predicting
 *   corrections of the PCA frame, scale, rotation and opacity.
 * mlp_weights: device blob of P2E_MLP_BLOB_BYTES (mode 1; 16-byte aligned),
 * else NULL.  Layout: bf16 W1[64][96], W2[64][64], W3[64][64], W4[16][64]
 * (row = output unit; rows 8..15 of W4 are padding and must be zero), then
 * fp32 b1[64], b2[64], b3[64], b4[16].  Features per point: for each of the
 * 16 nearest neighbours j in distance order, R^T (p_j - p_i) / r_i and
 * c_j - c_i (R the canonical PCA frame, r_i the 16th-neighbour distance).
 * Outputs y[0..7] correct the PCA estimate in its frame:
 * s = s_pca exp(clip(y0..2, -4, 4)), q = q_pca (x) normalize(1 + y3, y4, y5, y6),
 * o = sigmoid(logit(pca_opacity) + y7), normal = third axis of R(q).
 * out: device Gaussian set (mean_op, scale, quat, rgb, normal) of n entries
 * (the const qualifiers of p2e_gaussians are cast away for output).
 * knn_idx (optional, may be NULL): device uint32[n*16] neighbour indices,
 * 16-byte aligned, row i the 16 nearest other points of point i in
 * ascending distance (ties by index).
 * scratch: p2e_scratch_bytes(P2E_SCRATCH_ESTIMATE, n, 0) bytes. */
p2e_status p2e_estimate(const float *xyz, const float *rgb, int64_t n, int32_t mode,
                        const void *mlp_weights, float pca_opacity, p2e_gaussians *out,
                        uint32_t *knn_idx, void *scratch, int64_t scratch_bytes, void *stream);

/* ---- training of the learned estimator (Sec. 3.3) ------------------- */

/* p2e_loss_eq5 -- the training loss of Eq. 5 and its gradient:
 *   L = w1 mean|I - I^| + w2 mean(|n x n^| + w3 min(|n - n^|, |n + n^|))
 * (the L1 mean is over pixels and the 3 channels, the normal term's over
 * pixels; the paper uses w1 = 1, w2 = 10, w3 = 0.1).  rgb/normal: the
 * rendered planar images of p2e_render, gt_rgb/gt_normal the targets in the
 * same layout; view_pixels (host) holds H*W of each of n_views views.
 * Writes *loss_dev (device float, overwritten), d_rgb and d_normal
 * (dL/dI^, dL/dn^, same layout).  The gradient of |.| at 0 is taken as 0. */
p2e_status p2e_loss_eq5(const float *rgb, const float *normal, const float *gt_rgb,
                        const float *gt_normal, const int64_t *view_pixels, int32_t n_views,
                        float w1, float w2, float w3, float *loss_dev, float *d_rgb,
                        float *d_normal, void *stream);

/* p2e_loss_splat_area -- a rendering-cost term for training the estimator
 * (not in the paper; an option of this implementation's training):
 *   A = weight * mean_i (s_i0 s_i1) / (r_i0 r_i1)
 * the footprint of each estimated splat (its two largest axes) relative to
 * a reference estimate's, typically the kNN-PCA frame the network
 * corrects: compositing screens and evaluates every splat over its
 * footprint, so A tracks the frame's compositing work.  scale: the
 * estimate's device float4[n] (s0, s1, s2, -); ref_scale: the reference's,
 * both 16-byte aligned.  ADDS A to *loss_dev and dA/ds to d_scale (device
 * float[3n], s0 s1 s2 per point, the layout p2e_render_backward writes).
 * A point whose reference area is not positive and finite adds nothing.
 * weight >= 0. */
p2e_status p2e_loss_splat_area(const float *scale, const float *ref_scale, int64_t n, float weight,
                               float *loss_dev, float *d_scale, void *stream);

/* p2e_loss_ssim -- the structural term of an "L1 + SSIM" image loss on the
 * rendered colour (the training objective of the differentiable splatting
 * this renderer follows; the paper's Eq. 5 is the L1 + normal loss above):
 *   D = 1 - mean over pixels and channels of SSIM(I^, I)
 * with, per channel and pixel, local statistics over an 11 x 11 Gaussian
 * window (sigma 1.5, normalised; pixels outside the image count as zero):
 *   SSIM = (2 mx my + C1)(2 cxy + C2) / ((mx^2 + my^2 + C1)(vx + vy + C2)),
 *   C1 = 0.01^2, C2 = 0.03^2 (images in [0, 1]).
 * ACCUMULATES: *loss_dev += weight D and d_rgb += weight dD/dI^ (so that it
 * adds to p2e_loss_eq5's outputs).  rgb, gt_rgb, d_rgb: device planar
 * [3][H][W] per view, views concatenated; view_hw (host): H, W of each of
 * n_views views.  scratch: device, >= 96 bytes per pixel of all views,
 * 256-byte aligned. */
p2e_status p2e_loss_ssim(const float *rgb, const float *gt_rgb, const int32_t *view_hw, int32_t n_views,
                         float weight, float *loss_dev, float *d_rgb, void *scratch, int64_t scratch_bytes,
                         void *stream);

/* p2e_mlp_backward -- gradient of a loss with respect to the estimator's
 * parameters, given its gradient with respect to the estimated Gaussians
 * (d_scale[3n], d_quat[4n] w.r.t. the output quaternion, d_opacity[n],
 * d_normal[3n] w.r.t. the output normal; as p2e_render_backward writes
 * them).  xyz, rgb: the cloud (device float4[n]); knn_idx: the 16
 * neighbours of p2e_estimate (device uint32[n*16]); pca: the mode-0
 * estimate of the same cloud (its scale, quat and mean_op.w are read);
 * mlp_weights: the blob the forward used.  The network is re-evaluated
 * with the forward's bf16 roundings.  grad: device float[P2E_MLP_PARAMS]
 * in blob order (W1, W2, W3, W4 16x64, b1, b2, b3, b4 16), ACCUMULATED
 * into.  The products run on the tensor cores with bf16 operands (the
 * gradients flowing back are rounded to bf16 before each product) and fp32
 * accumulation.  Synchronises the stream twice (reads the PCA opacity
 * before the launch, and the kernel's status after it): returns
 * P2E_ERR_TIMEOUT if a bounded device wait gave up (grad is then invalid). */
#define P2E_MLP_PARAMS 15568
p2e_status p2e_mlp_backward(const float *xyz, const float *rgb, int64_t n, const uint32_t *knn_idx,
                            const p2e_gaussians *pca, const void *mlp_weights, const float *d_scale,
                            const float *d_quat, const float *d_opacity, const float *d_normal,
                            float *grad, void *stream);

/* p2e_adam -- one Adam step (bias-corrected) on the fp32 parameter vector
 * (count must be P2E_MLP_PARAMS; W4/b4 rows 8..15 are kept at zero), zeroes
 * grad, and, if blob is not NULL, rewrites the P2E_MLP_BLOB_BYTES weight
 * blob (bf16 weights rounded to nearest even, fp32 biases).  step >= 1. */
p2e_status p2e_adam(float *params, float *grad, float *m, float *v, int64_t count, float lr,
                    float beta1, float beta2, float eps, int32_t step, void *blob, void *stream);

/* ---- the global isotropic baseline and relighting ------------------- */

/* p2e_estimate_global -- the comparison estimator of Sec. 4.1 ("surface
 * splatting using the same isotropic Gaussian representing each point"):
 * every Gaussian gets the isotropic scale sigma_rel * d, d the average
 * distance of a point to its nearest neighbour over the cloud (the global
 * point density), the identity rotation and opacity `opacity`; the normal
 * is the kNN-PCA normal (so the normal image can still be rendered).
 * sigma_rel > 0 (the paper compares 1.2, 1.5 and 1.7).  Arguments
 * otherwise as p2e_estimate (same scratch size). */
p2e_status p2e_estimate_global(const float *xyz, const float *rgb, int64_t n, float sigma_rel, float opacity,
                               p2e_gaussians *out, uint32_t *knn_idx, void *scratch, int64_t scratch_bytes,
                               void *stream);

/* p2e_relight -- late shading of rendered views from their normal images
 * (Sec. 3.1: the normal map feeds a pixel shader).  Lambertian with
 * directional lights and an ambient term, per pixel:
 *   C = rgb - (1 - alpha) bg,  n^ = normal / |normal|,
 *   s = ambient + sum_l I_l max(0, n^ . l_l),  out = C s + (1 - alpha) bg;
 * a pixel whose |normal| <= 1e-12 keeps s = 1.
 * rgb, normal, alpha: device planar images as p2e_render writes them (views
 * concatenated); view_pixels (host) holds H*W of each of n_views views.
 * lights (host): n_lights (<= P2E_MAX_LIGHTS) x (dx, dy, dz, intensity),
 * directions in the normals' (world) frame, normalised here; bg (host,
 * 3 floats) or NULL for black.  out: device planar rgb (may alias rgb). */
p2e_status p2e_relight(const float *rgb, const float *normal, const float *alpha, const int64_t *view_pixels,
                       int32_t n_views, const float *lights, int32_t n_lights, float ambient, const float *bg,
                       float *out, void *stream);

/* p2e_point_raster -- the point-rasterisation baseline of Sec. 4.1 (each
 * point drawn as a 1-pixel square with a depth test, "OpenGL"): a point
 * covers the pixel (floor(u), floor(v)) containing its projection
 * u = fx x/z + cx, v = fy y/z + cy (camera transform and projection in
 * fp32, each operation correctly rounded, in the order written: x = ((T00 px
 * + T01 py) + T02 pz) + t0, ...), when z > near_z and the pixel is in the
 * image; the nearest point wins, ties by the lower index; the pixel gets
 * its colour, uncovered pixels get bg (host, 3 floats, or NULL for black).
 * xyz, rgb: device float4[n].  zbuf: device uint64 scratch of the total
 * pixel count (overwritten).  out_rgb: device planar rgb, views
 * concatenated as p2e_render; out_depth (may be NULL): the winning z, 0
 * where uncovered. */
p2e_status p2e_point_raster(const float *xyz, const float *rgb, int64_t n, const p2e_camera *cams,
                            int32_t n_views, const float *bg, uint64_t *zbuf, float *out_rgb, float *out_depth,
                            void *stream);

/* ---- measurement and diagnostics (no counterpart in the paper) -------- */

/* p2e_set_kernel_probe -- attaches measurement to the launches of one
 * kernel made by the calling host thread, until it is called again with
 * probe = NULL.  This is the one piece of state the library keeps between
 * calls (thread-local, host memory only); with no probe set nothing is
 * recorded.
 *   kernel   P2E_PROBE_KNN       the kNN search of p2e_estimate (its fast
 *                                path: the counting and selection kernels;
 *                                the few listed queries and the PCA run after)
 *            P2E_PROBE_BLEND     the compositing kernel of p2e_render
 *            P2E_PROBE_MLP       the learned head of p2e_estimate (mode 1)
 *            P2E_PROBE_BLEND_BWD the per-tile kernel of p2e_render_backward
 *   probe    start_event / stop_event: cudaEvent_t (or NULL) recorded on
 *            the launching stream immediately before / after the kernel;
 *            count_dev: device uint64 counters (or NULL) the kernel adds
 *            its work counts to.  BLEND: one, the (pixel, splat) pairs it
 *            evaluated, every pass included.  BLEND_BWD: three, the pairs
 *            evaluated by each of its two walks (front to back, back to
 *            front: the same set), the contributing pairs among them, and
 *            the warp reductions of per-splat gradients.  Ignored by the
 *            other kernels.
 * The probe struct is copied; the events and counters stay caller-owned. */
enum { P2E_PROBE_KNN = 0, P2E_PROBE_BLEND = 1, P2E_PROBE_MLP = 2, P2E_PROBE_BLEND_BWD = 3, P2E_PROBE_COUNT = 4 };
typedef struct {
    void *start_event;
    void *stop_event;
    uint64_t *count_dev;
} p2e_kernel_probe;
p2e_status p2e_set_kernel_probe(int32_t kernel, const p2e_kernel_probe *probe);

/* p2e_estimate_check -- synchronises `stream` and returns P2E_ERR_TIMEOUT if
 * a bounded device wait of the last p2e_estimate / p2e_estimate_global
 * call on this scratch gave up (its outputs are then invalid), else P2E_OK.
 * n and scratch as passed to that call. */
p2e_status p2e_estimate_check(const void *scratch, int64_t scratch_bytes, int64_t n, void *stream);

/* p2e_selftest_timeout -- drives one of the library's bounded device waits
 * to its limit, so that tests can check that the wait gives up, the kernel
 * returns and the timeout is reported, without faulting or hanging the GPU.
 *   which 0  a radix-sort pass of p2e_sort_bin whose first tile is never
 *            published: the next tile's decoupled look-back gives up;
 *         1  the cell-count scan of p2e_estimate, likewise;
 *         2  the learned head's mbarrier wait for an MMA completion that is
 *            never issued;
 *         3  p2e_render's wait for the deferred re-walks of its CTA, with
 *            a CTA that never leaves its item;
 *         4  the lock of that re-walk queue, held and never released.
 *   spin_limit  wait rounds before giving up, 1 .. 2^22 (the library's
 *            own default limit is 2^22 rounds, a few hundred ms).
 *   scratch  device, >= P2E_SELFTEST_SCRATCH_BYTES, 256-byte aligned.
 *   status_dev  device int32: P2E_ERR_TIMEOUT once the wait gave up.
 * Asynchronous on `stream`; read status_dev after synchronising (for
 * example through p2e_bins_check with a p2e_bins whose status_dev it is). */
#define P2E_SELFTEST_SCRATCH_BYTES (1 << 20)
p2e_status p2e_selftest_timeout(int32_t which, uint32_t spin_limit, void *scratch, int64_t scratch_bytes,
                                int32_t *status_dev, void *stream);

/* Human-readable name of a status code (static storage). */
const char *p2e_status_string(p2e_status s);

#ifdef __cplusplus
}
#endif
#endif /* P2E_H */
