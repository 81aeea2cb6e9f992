/*
 * FP64 CPU oracle for the splatting renderer.  TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path.
 *
 * It evaluates the plain definition of the rendered image (Sec. 3.1):
 * every Gaussian projected with the EWA approximation (Eq. 3-4), bounded by
 * its 3-sigma ellipse, ordered by camera depth, and alpha-composited front to
 * back (Eq. 1-2); the normal and depth images substitute n_k and z_k for c_k
 * (Sec. 3.1, last paragraph).  No tiles take part in the image; tiles appear
 * only in the binning reference (the (tile | depth) keys).
 *
 * All arithmetic is IEEE double (compile with -ffp-contract=off) on the fp32
 * inputs widened exactly.  The statement order inside rect_arith() is the
 * reference order for the integer decisions (cull, pixel rectangle, tile
 * rectangle); it is written out plainly and kept stable.
 *
 * Readings where the paper is silent (all documented with the renderer):
 *   near plane cull z <= near; Sigma = R diag(s^2) R^T with R the Hamilton
 *   rotation of the normalised quaternion (w, x, y, z); a low-pass dilation
 *   of `lowpass` px^2 added to the screen covariance; J not clamped; pixel
 *   centres at (i + 0.5, j + 0.5); the 3-sigma bound is the exact bounding
 *   box of the Mahalanobis-3 ellipse for binning and power >= -sigma^2/2 per
 *   pixel; alpha = min(alpha_max, o exp(power)); splats with alpha <
 *   alpha_floor are skipped; compositing stops before a splat that would take
 *   T below t_min; depth key = fp32 of z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double T[3][3], t[3];
    double fx, fy, cx, cy, near_z;
    int W, H;
} cam_t;

static void load_cam(cam_t *c, const float *cam /* 17 floats */, int W, int H)
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) c->T[i][j] = (double)cam[4 * i + j];
        c->t[i] = (double)cam[4 * i + 3];
    }
    c->fx = cam[12]; c->fy = cam[13]; c->cx = cam[14]; c->cy = cam[15];
    c->near_z = cam[16];
    c->W = W; c->H = H;
}

/* Result of the per-Gaussian projection (R1-R4). */
typedef struct {
    int visible;
    double x, y, z;          /* camera-space centre            */
    double u, v;             /* screen-space centre (pixels)   */
    double a, b, c;          /* screen covariance Sigma_s      */
    double A, B, C;          /* conic = Sigma_s^{-1}           */
    int i0, i1, j0, j1;      /* pixel rectangle, inclusive     */
} proj_t;

/*
 * Projection of one Gaussian.  The statement order here is the reference
 * order for every decision taken from floating point.
 */
static void rect_arith(const cam_t *cm, double lowpass, double k,
                       const float *mean, const float *scale, const float *quat,
                       proj_t *p)
{
    const double mx = mean[0], my = mean[1], mz = mean[2];
    p->visible = 0;
    /* R1: viewing transform W = [T t; 0 1] (Eq. 3) */
    const double z = fma(cm->T[2][0], mx, fma(cm->T[2][1], my, fma(cm->T[2][2], mz, cm->t[2])));
    const double x = fma(cm->T[0][0], mx, fma(cm->T[0][1], my, fma(cm->T[0][2], mz, cm->t[0])));
    const double y = fma(cm->T[1][0], mx, fma(cm->T[1][1], my, fma(cm->T[1][2], mz, cm->t[1])));
    p->x = x; p->y = y; p->z = z;
    if (!(z > cm->near_z)) return;

    /* R2: Sigma = R S S R^T, R from the normalised quaternion (Sec. 3.1) */
    const double qw = quat[0], qx = quat[1], qy = quat[2], qz = quat[3];
    if (qw == 0.0 && qx == 0.0 && qy == 0.0 && qz == 0.0) return;
    const double qn = sqrt(((qw * qw + qx * qx) + qy * qy) + qz * qz);
    const double w = qw / qn, xx = qx / qn, yy = qy / qn, zz = qz / qn;
    double R[3][3];
    R[0][0] = 1.0 - 2.0 * (yy * yy + zz * zz);
    R[0][1] = 2.0 * (xx * yy - w * zz);
    R[0][2] = 2.0 * (xx * zz + w * yy);
    R[1][0] = 2.0 * (xx * yy + w * zz);
    R[1][1] = 1.0 - 2.0 * (xx * xx + zz * zz);
    R[1][2] = 2.0 * (yy * zz - w * xx);
    R[2][0] = 2.0 * (xx * zz - w * yy);
    R[2][1] = 2.0 * (yy * zz + w * xx);
    R[2][2] = 1.0 - 2.0 * (xx * xx + yy * yy);
    const double s[3] = {scale[0], scale[1], scale[2]};

    /* R3: Sigma_s = J T Sigma T^T J^T + lowpass I (Eq. 4), computed as
     * M M^T with M = J (T R) S. */
    double V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            V[i][j] = ((cm->T[i][0] * R[0][j] + cm->T[i][1] * R[1][j]) + cm->T[i][2] * R[2][j]) * s[j];
    const double xs = x / z, ys = y / z;
    const double j00 = cm->fx / z, j02 = -(cm->fx * xs) / z;
    const double j11 = cm->fy / z, j12 = -(cm->fy * ys) / z;
    double M0[3], M1[3];
    for (int j = 0; j < 3; ++j) {
        M0[j] = j00 * V[0][j] + j02 * V[2][j];
        M1[j] = j11 * V[1][j] + j12 * V[2][j];
    }
    const double a = ((M0[0] * M0[0] + M0[1] * M0[1]) + M0[2] * M0[2]) + lowpass;
    const double b = (M0[0] * M1[0] + M0[1] * M1[1]) + M0[2] * M1[2];
    const double c = ((M1[0] * M1[0] + M1[1] * M1[1]) + M1[2] * M1[2]) + lowpass;
    const double det = a * c - b * b;
    const double u = cm->fx * xs + cm->cx;
    const double v = cm->fy * ys + cm->cy;
    if (!(det > 0.0) || !isfinite(det) || !isfinite(a) || !isfinite(c) ||
        !isfinite(b) || !isfinite(u) || !isfinite(v))
        return;

    /* R4: exact bounding box of the k-sigma ellipse, pixel centres at +0.5 */
    const double ex = k * sqrt(a), ey = k * sqrt(c);
    const double lox = (u - ex) - 0.5, hix = (u + ex) - 0.5;
    const double loy = (v - ey) - 0.5, hiy = (v + ey) - 0.5;
    const double i0 = fmax(0.0, ceil(lox)), i1 = fmin((double)(cm->W - 1), floor(hix));
    const double j0 = fmax(0.0, ceil(loy)), j1 = fmin((double)(cm->H - 1), floor(hiy));
    if (!(i0 <= i1) || !(j0 <= j1)) return;

    p->u = u; p->v = v;
    p->a = a; p->b = b; p->c = c;
    p->A = c / det; p->B = -b / det; p->C = a / det;
    p->i0 = (int)i0; p->i1 = (int)i1; p->j0 = (int)j0; p->j1 = (int)j1;
    p->visible = 1;
}

/*
 * or_project: R1-R4 for n Gaussians.
 * cam: 17 floats (viewmat[12] row-major [T|t], fx, fy, cx, cy, near).
 * Outputs (each n entries, or n*k for vectors):
 *   vis[n] u8, xyz[3n] f64 camera coords, uv[2n], cov2[3n] (a,b,c),
 *   conic[3n] (A,B,C), prect[4n] i32 (i0,i1,j0,j1), trect[4n] i32
 *   (tx0,tx1,ty0,ty1), ntiles[n] i32, zkey[n] f32.
 */
void or_project(int64_t n, const float *mean, const float *scale, const float *quat,
                const float *cam, int W, int H, double lowpass, double k, int tile,
                uint8_t *vis, double *xyz, double *uv, double *cov2, double *conic,
                int32_t *prect, int32_t *trect, int32_t *ntiles, float *zkey)
{
    cam_t cm;
    load_cam(&cm, cam, W, H);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        proj_t p;
        memset(&p, 0, sizeof p);
        rect_arith(&cm, lowpass, k, mean + 3 * g, scale + 3 * g, quat + 4 * g, &p);
        vis[g] = (uint8_t)p.visible;
        xyz[3 * g] = p.x; xyz[3 * g + 1] = p.y; xyz[3 * g + 2] = p.z;
        zkey[g] = (float)p.z;
        if (!p.visible) {
            ntiles[g] = 0;
            for (int q = 0; q < 4; ++q) { prect[4 * g + q] = 0; trect[4 * g + q] = 0; }
            for (int q = 0; q < 3; ++q) { cov2[3 * g + q] = 0; conic[3 * g + q] = 0; }
            uv[2 * g] = 0; uv[2 * g + 1] = 0;
            continue;
        }
        uv[2 * g] = p.u; uv[2 * g + 1] = p.v;
        cov2[3 * g] = p.a; cov2[3 * g + 1] = p.b; cov2[3 * g + 2] = p.c;
        conic[3 * g] = p.A; conic[3 * g + 1] = p.B; conic[3 * g + 2] = p.C;
        prect[4 * g] = p.i0; prect[4 * g + 1] = p.i1; prect[4 * g + 2] = p.j0; prect[4 * g + 3] = p.j1;
        const int tx0 = p.i0 / tile, tx1 = p.i1 / tile, ty0 = p.j0 / tile, ty1 = p.j1 / tile;
        trect[4 * g] = tx0; trect[4 * g + 1] = tx1; trect[4 * g + 2] = ty0; trect[4 * g + 3] = ty1;
        ntiles[g] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Binning reference (R5): keys emitted in Gaussian-index order, then sorted */
/* by (key, value); since values are Gaussian indices, this is the stable     */
/* sort of the keys.                                                          */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t val; } kv_t;

static int kv_cmp(const void *pa, const void *pb)
{
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->val < b->val ? -1 : (a->val > b->val);
}

/* Emits the keys of one view into keys/vals starting at `offset`; returns
 * the number written.  tiles_x = ceil(W / tile). */
int64_t or_emit_keys(int64_t n, const int32_t *trect, const int32_t *ntiles,
                     const float *zkey, int tiles_x, int64_t tile_base,
                     uint64_t *keys, uint32_t *vals, int64_t offset)
{
    int64_t o = offset;
    for (int64_t g = 0; g < n; ++g) {
        if (ntiles[g] == 0) continue;
        uint32_t zb;
        memcpy(&zb, &zkey[g], 4);
        for (int ty = trect[4 * g + 2]; ty <= trect[4 * g + 3]; ++ty)
            for (int tx = trect[4 * g]; tx <= trect[4 * g + 1]; ++tx) {
                const uint64_t tid = (uint64_t)(tile_base + (int64_t)ty * tiles_x + tx);
                keys[o] = (tid << 32) | (uint64_t)zb;
                vals[o] = (uint32_t)g;
                ++o;
            }
    }
    return o - offset;
}

/* Sorts (key, val) pairs and writes per-tile [start, end) ranges
 * (ranges[2*t], ranges[2*t+1]); empty tiles get [0, 0). */
void or_sort_ranges(int64_t K, uint64_t *keys, uint32_t *vals, int64_t n_tiles_total,
                    uint32_t *ranges)
{
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (K > 0 ? K : 1));
    for (int64_t i = 0; i < K; ++i) { kv[i].key = keys[i]; kv[i].val = vals[i]; }
    qsort(kv, (size_t)K, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < K; ++i) { keys[i] = kv[i].key; vals[i] = kv[i].val; }
    free(kv);
    for (int64_t t = 0; t < n_tiles_total; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t i = 0; i < K; ++i) {
        const int64_t t = (int64_t)(keys[i] >> 32);
        if (t < 0 || t >= n_tiles_total) continue;
        if (i == 0 || (keys[i - 1] >> 32) != (uint64_t)t) ranges[2 * t] = (uint32_t)i;
        ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Compositing (R6-R7)                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    double alpha_floor, alpha_max, t_min, k, bg[3];
    double flag_power, flag_alpha, flag_t;   /* knife-edge flag half-widths */
} blend_cfg_t;

/* Depth order: fp32 depth key, ties by Gaussian index. */
static const float *g_sort_z;
static int ord_cmp(const void *pa, const void *pb)
{
    const int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    const float za = g_sort_z[a], zb = g_sort_z[b];
    if (za != zb) return za < zb ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/*
 * Composites one pixel over the candidates `list[0..m)` (already in depth
 * order).  A candidate contributes when the pixel lies in its rectangle and
 * power >= -k^2/2.
 * The pixel is flagged when a floating-point knife edge (power at the
 * 3-sigma boundary, alpha at the floor, T at the cutoff) lies within the
 * flag half-widths of a candidate it reaches; candidates in a one-pixel
 * border around the rectangle are inspected for the power edge.
 */
static void composite_pixel(int i, int j, const int64_t *list, int64_t m,
                            const uint8_t *vis, const double *uv, const double *conic,
                            const int32_t *prect, const double *xyz, const float *opac,
                            const float *rgb, const float *nrm, const blend_cfg_t *bc,
                            double out[8], int32_t *ncontrib, int32_t *last, uint8_t *flag)
{
    double T = 1.0, Cc[3] = {0, 0, 0}, N[3] = {0, 0, 0}, D = 0.0;
    int32_t nc = 0, lg = -1;
    uint8_t fl = 0;
    const double pw_min = -0.5 * bc->k * bc->k;
    const double px = i + 0.5, py = j + 0.5;
    for (int64_t q = 0; q < m; ++q) {
        const int64_t g = list[q];
        if (!vis[g]) continue;
        const int32_t *r = prect + 4 * g;
        if (i < r[0] - 1 || i > r[1] + 1 || j < r[2] - 1 || j > r[3] + 1) continue;
        const double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
        const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
        const double power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
        if (fabs(power - pw_min) < bc->flag_power) fl = 1;
        if (i < r[0] || i > r[1] || j < r[2] || j > r[3]) continue;
        if (power < pw_min) continue;
        double alpha = (double)opac[g] * exp(power);
        if (alpha > bc->alpha_max) alpha = bc->alpha_max;
        if (fabs(alpha - bc->alpha_floor) < bc->flag_alpha) fl = 1;
        if (alpha < bc->alpha_floor) continue;
        const double Tn = T * (1.0 - alpha);
        if (fabs(Tn - bc->t_min) < bc->flag_t) fl = 1;
        if (Tn < bc->t_min) break;
        const double w = alpha * T;
        for (int ch = 0; ch < 3; ++ch) {
            Cc[ch] += w * (double)rgb[3 * g + ch];
            N[ch] += w * (double)nrm[3 * g + ch];
        }
        D += w * xyz[3 * g + 2];
        T = Tn;
        ++nc;
        lg = (int32_t)g;
    }
    for (int ch = 0; ch < 3; ++ch) {
        out[ch] = Cc[ch] + T * bc->bg[ch];
        out[3 + ch] = N[ch];
    }
    out[6] = D;
    out[7] = 1.0 - T;
    *ncontrib = nc;
    *last = lg;
    *flag = fl;
}

/*
 * or_render: one view.  Inputs are the or_project outputs plus the
 * per-Gaussian opacity, rgb (3n) and normal (3n).  Outputs are planar
 * doubles: img[8][H][W] = rgb(3), normal(3), depth, alpha, and per pixel
 * ncontrib, last (Gaussian index or -1), flag.
 * brute != 0: every visible Gaussian is a candidate of every pixel (the
 * literal definition).  brute == 0: candidates come from per-row lists
 * built from the rectangles (exact, because a Gaussian outside its
 * rectangle never contributes).
 * params: alpha_floor, alpha_max, t_min, k, bg0, bg1, bg2, flag_power,
 * flag_alpha, flag_t.
 */
int or_render(int64_t n, int W, int H, const uint8_t *vis, const double *xyz,
              const double *uv, const double *conic, const int32_t *prect,
              const float *zkey, const float *opac, const float *rgb, const float *nrm,
              const double *params, int brute, double *img, int32_t *ncontrib,
              int32_t *last, uint8_t *flag)
{
    blend_cfg_t bc;
    bc.alpha_floor = params[0]; bc.alpha_max = params[1]; bc.t_min = params[2];
    bc.k = params[3]; bc.bg[0] = params[4]; bc.bg[1] = params[5]; bc.bg[2] = params[6];
    bc.flag_power = params[7]; bc.flag_alpha = params[8]; bc.flag_t = params[9];
    const int64_t HW = (int64_t)H * W;

    /* depth order of the visible Gaussians */
    int64_t nv = 0;
    for (int64_t g = 0; g < n; ++g) nv += vis[g] ? 1 : 0;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (nv > 0 ? nv : 1));
    nv = 0;
    for (int64_t g = 0; g < n; ++g) if (vis[g]) order[nv++] = g;
    g_sort_z = zkey;
    qsort(order, (size_t)nv, sizeof(int64_t), ord_cmp);

    int64_t *rowptr = NULL, *rowlist = NULL;
    if (!brute) {
        /* per-row candidate lists (rows r0-1 .. r1+1), in depth order */
        rowptr = (int64_t *)calloc((size_t)H + 1, sizeof(int64_t));
        for (int64_t q = 0; q < nv; ++q) {
            const int32_t *r = prect + 4 * order[q];
            const int a = r[2] - 1 < 0 ? 0 : r[2] - 1, b = r[3] + 1 > H - 1 ? H - 1 : r[3] + 1;
            for (int j = a; j <= b; ++j) rowptr[j + 1]++;
        }
        for (int j = 0; j < H; ++j) rowptr[j + 1] += rowptr[j];
        rowlist = (int64_t *)malloc(sizeof(int64_t) * (rowptr[H] > 0 ? rowptr[H] : 1));
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)H);
        for (int j = 0; j < H; ++j) fill[j] = rowptr[j];
        for (int64_t q = 0; q < nv; ++q) {
            const int32_t *r = prect + 4 * order[q];
            const int a = r[2] - 1 < 0 ? 0 : r[2] - 1, b = r[3] + 1 > H - 1 ? H - 1 : r[3] + 1;
            for (int j = a; j <= b; ++j) rowlist[fill[j]++] = order[q];
        }
        free(fill);
    }

#pragma omp parallel
    {
        int64_t *plist = NULL;
        int64_t *pcnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(W + 1));
#pragma omp for schedule(dynamic, 1)
        for (int j = 0; j < H; ++j) {
            const int64_t *cand;
            int64_t m;
            if (brute) { cand = order; m = nv; }
            else { cand = rowlist + rowptr[j]; m = rowptr[j + 1] - rowptr[j]; }
            /* per-pixel lists of this row, kept in depth order */
            int64_t tot = 0;
            memset(pcnt, 0, sizeof(int64_t) * (size_t)(W + 1));
            if (!brute) {
                for (int64_t q = 0; q < m; ++q) {
                    const int32_t *r = prect + 4 * cand[q];
                    const int a = r[0] - 1 < 0 ? 0 : r[0] - 1, b = r[1] + 1 > W - 1 ? W - 1 : r[1] + 1;
                    for (int i = a; i <= b; ++i) pcnt[i + 1]++;
                }
                for (int i = 0; i < W; ++i) pcnt[i + 1] += pcnt[i];
                tot = pcnt[W];
                plist = (int64_t *)realloc(plist, sizeof(int64_t) * (size_t)(tot > 0 ? tot : 1));
                int64_t *pf = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
                for (int i = 0; i < W; ++i) pf[i] = pcnt[i];
                for (int64_t q = 0; q < m; ++q) {
                    const int32_t *r = prect + 4 * cand[q];
                    const int a = r[0] - 1 < 0 ? 0 : r[0] - 1, b = r[1] + 1 > W - 1 ? W - 1 : r[1] + 1;
                    for (int i = a; i <= b; ++i) plist[pf[i]++] = cand[q];
                }
                free(pf);
            }
            for (int i = 0; i < W; ++i) {
                double o8[8];
                const int64_t pix = (int64_t)j * W + i;
                const int64_t *lst = brute ? cand : plist + pcnt[i];
                const int64_t len = brute ? m : pcnt[i + 1] - pcnt[i];
                composite_pixel(i, j, lst, len, vis, uv, conic, prect, xyz, opac, rgb, nrm,
                                &bc, o8, &ncontrib[pix], &last[pix], &flag[pix]);
                for (int ch = 0; ch < 8; ++ch) img[ch * HW + pix] = o8[ch];
            }
        }
        free(plist);
        free(pcnt);
    }
    free(order);
    free(rowptr);
    free(rowlist);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gradient (R8): exact derivative of one view's images with respect to the  */
/* raw inputs, holding every discrete decision (cull, rectangle, 3-sigma      */
/* test, floor, stop) fixed.  The images are linearised by upstream weights:  */
/*   L = sum gC . rgb + gN . normal + gD depth + gA alpha.                    */
/* ------------------------------------------------------------------------ */

/* per-Gaussian screen-space gradient slots */
enum { GU = 0, GV, GA, GB, GC, GO, GZ, GR, GG, GBL, GNX, GNY, GNZ, G2D };

typedef struct { int64_t g; double alpha, T, power, dx, dy; } contrib_t;

/* Forward + backward of one pixel; adds into g2d[n][G2D]. */
static void grad_pixel(int i, int j, const int64_t *list, int64_t m, const uint8_t *vis,
                       const double *uv, const double *conic, const int32_t *prect,
                       const double *xyz, const float *opac, const float *rgb, const float *nrm,
                       const blend_cfg_t *bc, const double up[8], double *g2d,
                       contrib_t **buf, int64_t *cap)
{
    double T = 1.0;
    int64_t nk = 0;
    const double pw_min = -0.5 * bc->k * bc->k;
    const double px = i + 0.5, py = j + 0.5;
    for (int64_t q = 0; q < m; ++q) {
        const int64_t g = list[q];
        if (!vis[g]) continue;
        const int32_t *r = prect + 4 * g;
        if (i < r[0] || i > r[1] || j < r[2] || j > r[3]) continue;
        const double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
        const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
        const double power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
        if (power < pw_min) continue;
        double alpha = (double)opac[g] * exp(power);
        if (alpha > bc->alpha_max) alpha = bc->alpha_max;
        if (alpha < bc->alpha_floor) continue;
        const double Tn = T * (1.0 - alpha);
        if (Tn < bc->t_min) break;
        if (nk == *cap) {
            *cap = *cap ? 2 * *cap : 64;
            *buf = (contrib_t *)realloc(*buf, sizeof(contrib_t) * (size_t)*cap);
        }
        contrib_t c = {g, alpha, T, power, dx, dy};
        (*buf)[nk++] = c;
        T = Tn;
    }
    /* up = gC[3], gN[3], gD, gA */
    const double bgterm = up[0] * bc->bg[0] + up[1] * bc->bg[1] + up[2] * bc->bg[2];
    double acc = T * (bgterm - up[7]);
    for (int64_t q = nk - 1; q >= 0; --q) {
        const contrib_t *c = &(*buf)[q];
        const int64_t g = c->g;
        const double w = c->alpha * c->T;
        const double f = up[0] * rgb[3 * g] + up[1] * rgb[3 * g + 1] + up[2] * rgb[3 * g + 2] +
                         up[3] * nrm[3 * g] + up[4] * nrm[3 * g + 1] + up[5] * nrm[3 * g + 2] +
                         up[6] * xyz[3 * g + 2];
        double *G = g2d + G2D * g;
        G[GR] += w * up[0]; G[GG] += w * up[1]; G[GBL] += w * up[2];
        G[GNX] += w * up[3]; G[GNY] += w * up[4]; G[GNZ] += w * up[5];
        G[GZ] += w * up[6];
        const double dalpha = c->T * f - acc / (1.0 - c->alpha);
        acc += w * f;
        /* alpha = o exp(power) unless clamped at alpha_max */
        if ((double)opac[g] * exp(c->power) > bc->alpha_max) continue;
        const double e = exp(c->power);
        G[GO] += dalpha * e;
        const double dp = dalpha * c->alpha;
        const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
        G[GA] += dp * (-0.5 * c->dx * c->dx);
        G[GC] += dp * (-0.5 * c->dy * c->dy);
        G[GB] += dp * (-c->dx * c->dy);
        G[GU] += dp * (A * c->dx + B * c->dy);
        G[GV] += dp * (B * c->dx + C * c->dy);
    }
}

/*
 * or_render_grad: screen-space gradients of one view (single thread, for
 * test scenes).  up_img: 8 planes (gC[3], gN[3], gD, gA) of H*W doubles.
 * Writes g2d[n][13] (u, v, A, B, C, o, z, r, g, b, nx, ny, nz).
 */
void or_render_grad(int64_t n, int W, int H, const uint8_t *vis, const double *xyz,
                    const double *uv, const double *conic, const int32_t *prect,
                    const float *zkey, const float *opac, const float *rgb, const float *nrm,
                    const double *params, const double *up_img, double *g2d)
{
    blend_cfg_t bc;
    bc.alpha_floor = params[0]; bc.alpha_max = params[1]; bc.t_min = params[2];
    bc.k = params[3]; bc.bg[0] = params[4]; bc.bg[1] = params[5]; bc.bg[2] = params[6];
    const int64_t HW = (int64_t)H * W;
    int64_t nv = 0;
    for (int64_t g = 0; g < n; ++g) nv += vis[g] ? 1 : 0;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (nv > 0 ? nv : 1));
    nv = 0;
    for (int64_t g = 0; g < n; ++g) if (vis[g]) order[nv++] = g;
    g_sort_z = zkey;
    qsort(order, (size_t)nv, sizeof(int64_t), ord_cmp);
    for (int64_t q = 0; q < n * G2D; ++q) g2d[q] = 0.0;
    contrib_t *buf = NULL;
    int64_t cap = 0;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            const int64_t pix = (int64_t)j * W + i;
            double up[8];
            for (int ch = 0; ch < 8; ++ch) up[ch] = up_img[ch * HW + pix];
            grad_pixel(i, j, order, nv, vis, uv, conic, prect, xyz, opac, rgb, nrm, &bc, up, g2d,
                       &buf, &cap);
        }
    free(buf);
    free(order);
}

/*
 * or_project_grad: chain rule from the screen-space gradients g2d[n][13]
 * of one view to the raw inputs (Eq. 3-4 backwards): adds into
 * d_mean[3n], d_scale[3n], d_quat[4n], d_opac[n], d_rgb[3n], d_nrm[3n].
 */
void or_project_grad(int64_t n, const float *mean, const float *scale, const float *quat,
                     const float *cam, int W, int H, double lowpass, const uint8_t *vis,
                     const double *g2d, double *d_mean, double *d_scale, double *d_quat,
                     double *d_opac, double *d_rgb, double *d_nrm)
{
    cam_t cm;
    load_cam(&cm, cam, W, H);
    (void)lowpass;
    for (int64_t g = 0; g < n; ++g) {
        const double *G = g2d + G2D * g;
        d_opac[g] += G[GO];
        for (int c = 0; c < 3; ++c) {
            d_rgb[3 * g + c] += G[GR + c];
            d_nrm[3 * g + c] += G[GNX + c];
        }
        if (!vis[g]) continue;
        const double mx = mean[3 * g], my = mean[3 * g + 1], mz = mean[3 * g + 2];
        double p[3];
        for (int i = 0; i < 3; ++i)
            p[i] = cm.T[i][0] * mx + cm.T[i][1] * my + cm.T[i][2] * mz + cm.t[i];
        const double x = p[0], y = p[1], z = p[2];
        const double qw = quat[4 * g], qx = quat[4 * g + 1], qy = quat[4 * g + 2], qz = quat[4 * g + 3];
        const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        const double w = qw / qn, a = qx / qn, b = qy / qn, c = qz / qn;
        double R[3][3];
        R[0][0] = 1 - 2 * (b * b + c * c); R[0][1] = 2 * (a * b - w * c); R[0][2] = 2 * (a * c + w * b);
        R[1][0] = 2 * (a * b + w * c); R[1][1] = 1 - 2 * (a * a + c * c); R[1][2] = 2 * (b * c - w * a);
        R[2][0] = 2 * (a * c - w * b); R[2][1] = 2 * (b * c + w * a); R[2][2] = 1 - 2 * (a * a + b * b);
        const double s[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        double Wm[3][3], V[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                Wm[i][k] = cm.T[i][0] * R[0][k] + cm.T[i][1] * R[1][k] + cm.T[i][2] * R[2][k];
                V[i][k] = Wm[i][k] * s[k];
            }
        const double fx = cm.fx, fy = cm.fy;
        double J[2][3] = {{fx / z, 0, -fx * x / (z * z)}, {0, fy / z, -fy * y / (z * z)}};
        double M[2][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) M[r][k] = J[r][0] * V[0][k] + J[r][1] * V[1][k] + J[r][2] * V[2][k];
        const double sa = M[0][0] * M[0][0] + M[0][1] * M[0][1] + M[0][2] * M[0][2] + lowpass;
        const double sb = M[0][0] * M[1][0] + M[0][1] * M[1][1] + M[0][2] * M[1][2];
        const double sc = M[1][0] * M[1][0] + M[1][1] * M[1][1] + M[1][2] * M[1][2] + lowpass;
        const double det = sa * sc - sb * sb;
        const double Q[2][2] = {{sc / det, -sb / det}, {-sb / det, sa / det}};
        /* dL/dQ as a symmetric matrix: B enters twice in the quadratic form */
        const double Gq[2][2] = {{G[GA], 0.5 * G[GB]}, {0.5 * G[GB], G[GC]}};
        double QG[2][2], GM[2][2];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 2; ++k) QG[r][k] = Q[r][0] * Gq[0][k] + Q[r][1] * Gq[1][k];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 2; ++k) GM[r][k] = -(QG[r][0] * Q[0][k] + QG[r][1] * Q[1][k]);
        const double ga = GM[0][0], gc = GM[1][1], gb = GM[0][1] + GM[1][0];
        double dM[2][3];
        for (int k = 0; k < 3; ++k) {
            dM[0][k] = 2 * ga * M[0][k] + gb * M[1][k];
            dM[1][k] = 2 * gc * M[1][k] + gb * M[0][k];
        }
        double dJ[2][3], dV[3][3];
        for (int r = 0; r < 2; ++r)
            for (int i = 0; i < 3; ++i) dJ[r][i] = dM[r][0] * V[i][0] + dM[r][1] * V[i][1] + dM[r][2] * V[i][2];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) dV[i][k] = J[0][i] * dM[0][k] + J[1][i] * dM[1][k];
        double dW[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                d_scale[3 * g + k] += dV[i][k] * Wm[i][k];
                dW[i][k] = dV[i][k] * s[k];
            }
        double dR[3][3];
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) dR[l][k] = cm.T[0][l] * dW[0][k] + cm.T[1][l] * dW[1][k] + cm.T[2][l] * dW[2][k];
        /* R(w, a, b, c) -> gradient w.r.t. the unit quaternion */
        const double dw = 2 * (-c * dR[0][1] + b * dR[0][2] + c * dR[1][0] - a * dR[1][2] - b * dR[2][0] + a * dR[2][1]);
        const double da = 2 * (b * dR[0][1] + c * dR[0][2] + b * dR[1][0] - 2 * a * dR[1][1] - w * dR[1][2] +
                               c * dR[2][0] + w * dR[2][1] - 2 * a * dR[2][2]);
        const double db = 2 * (-2 * b * dR[0][0] + a * dR[0][1] + w * dR[0][2] + a * dR[1][0] + c * dR[1][2] -
                               w * dR[2][0] + c * dR[2][1] - 2 * b * dR[2][2]);
        const double dc = 2 * (-2 * c * dR[0][0] - w * dR[0][1] + a * dR[0][2] + w * dR[1][0] - 2 * c * dR[1][1] +
                               b * dR[1][2] + a * dR[2][0] + b * dR[2][1]);
        const double qh[4] = {w, a, b, c}, dq[4] = {dw, da, db, dc};
        const double dot = qh[0] * dq[0] + qh[1] * dq[1] + qh[2] * dq[2] + qh[3] * dq[3];
        for (int k = 0; k < 4; ++k) d_quat[4 * g + k] += (dq[k] - qh[k] * dot) / qn;
        /* camera-space centre: through u, v, the depth image and J */
        double dx_ = 0, dy_ = 0, dz_ = 0;
        dx_ += G[GU] * fx / z;
        dz_ += G[GU] * (-fx * x / (z * z));
        dy_ += G[GV] * fy / z;
        dz_ += G[GV] * (-fy * y / (z * z));
        dz_ += G[GZ];
        dz_ += dJ[0][0] * (-fx / (z * z)) + dJ[1][1] * (-fy / (z * z));
        dx_ += dJ[0][2] * (-fx / (z * z));
        dz_ += dJ[0][2] * (2 * fx * x / (z * z * z));
        dy_ += dJ[1][2] * (-fy / (z * z));
        dz_ += dJ[1][2] * (2 * fy * y / (z * z * z));
        for (int k = 0; k < 3; ++k)
            d_mean[3 * g + k] += cm.T[0][k] * dx_ + cm.T[1][k] * dy_ + cm.T[2][k] * dz_;
    }
}
