/*
 * Exact FP64 ground-truth views of the analytic scenes.  TEST / TRAINING
 * INFRASTRUCTURE ONLY (see oracle/__init__.py).  Stands in for the paper's
 * ground-truth images rasterised from meshes (Sec. 3.3): one ray through
 * each pixel centre, nearest positive intersection with the union of the
 * primitives (the first surface a ray enters is on the union's boundary).
 *   ellipsoid  |R^T (o + t d - c) / radii|^2 = 1, normal from the gradient
 *   capped     tube |(x - p0) - ((x - p0).a) a| = r with 0 <= (x - p0).a <= h,
 *   cylinder   plus the two end disks
 * The camera direction of pixel (i, j) is T^T ((i+.5-cx)/fx, (j+.5-cy)/fy, 1),
 * so the ray parameter t at a hit is the camera depth z.
 */
#include <math.h>
#include <stdint.h>

/* primitive record: 20 doubles
 *   [0] kind (0 ellipsoid, 1 capped cylinder)
 *   ellipsoid: [1..3] centre, [4..6] radii, [7..15] rotation (row-major,
 *              columns = local axes)
 *   cylinder:  [1..3] p0, [4..6] p1, [7] radius */
enum { PREC = 20 };

static void hit_ellipsoid(const double *P, const double o[3], const double d[3], double *tbest,
                          double nbest[3])
{
    const double *c = P + 1, *rad = P + 4, *R = P + 7;
    double ol[3], dl[3];
    for (int k = 0; k < 3; ++k) {
        double so = 0, sd = 0;
        for (int m = 0; m < 3; ++m) {          /* R^T v: column k of R dotted with v */
            so += R[3 * m + k] * (o[m] - c[m]);
            sd += R[3 * m + k] * d[m];
        }
        ol[k] = so / rad[k];
        dl[k] = sd / rad[k];
    }
    const double a = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
    const double b = 2 * (ol[0] * dl[0] + ol[1] * dl[1] + ol[2] * dl[2]);
    const double cc = ol[0] * ol[0] + ol[1] * ol[1] + ol[2] * ol[2] - 1;
    const double disc = b * b - 4 * a * cc;
    if (disc < 0) return;
    const double sq = sqrt(disc);
    double t = (-b - sq) / (2 * a);
    if (t <= 0) t = (-b + sq) / (2 * a);
    if (t <= 0 || t >= *tbest) return;
    *tbest = t;
    double g[3];
    for (int k = 0; k < 3; ++k) g[k] = (ol[k] + t * dl[k]) / rad[k];   /* local x / radii^2 (scaled) */
    double nn = 0;
    for (int m = 0; m < 3; ++m) {
        nbest[m] = R[3 * m] * g[0] + R[3 * m + 1] * g[1] + R[3 * m + 2] * g[2];
        nn += nbest[m] * nbest[m];
    }
    nn = sqrt(nn);
    for (int m = 0; m < 3; ++m) nbest[m] /= nn;
}

static void hit_cylinder(const double *P, const double o[3], const double d[3], double *tbest,
                         double nbest[3])
{
    const double *p0 = P + 1, *p1 = P + 4;
    const double r = P[7];
    double a[3], h = 0;
    for (int k = 0; k < 3; ++k) { a[k] = p1[k] - p0[k]; h += a[k] * a[k]; }
    h = sqrt(h);
    for (int k = 0; k < 3; ++k) a[k] /= h;
    double w[3], wa = 0, da = 0;
    for (int k = 0; k < 3; ++k) { w[k] = o[k] - p0[k]; wa += w[k] * a[k]; da += d[k] * a[k]; }
    double wp[3], dp[3];
    for (int k = 0; k < 3; ++k) { wp[k] = w[k] - wa * a[k]; dp[k] = d[k] - da * a[k]; }
    const double A = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    const double B = 2 * (wp[0] * dp[0] + wp[1] * dp[1] + wp[2] * dp[2]);
    const double Cc = wp[0] * wp[0] + wp[1] * wp[1] + wp[2] * wp[2] - r * r;
    if (A > 0) {
        const double disc = B * B - 4 * A * Cc;
        if (disc >= 0) {
            const double sq = sqrt(disc);
            const double ts[2] = {(-B - sq) / (2 * A), (-B + sq) / (2 * A)};
            for (int q = 0; q < 2; ++q) {
                const double t = ts[q];
                if (t <= 0 || t >= *tbest) continue;
                const double s = wa + t * da;
                if (s < 0 || s > h) continue;
                *tbest = t;
                for (int k = 0; k < 3; ++k) nbest[k] = (wp[k] + t * dp[k]) / r;
                break;
            }
        }
    }
    if (da != 0) {
        for (int end = 0; end < 2; ++end) {
            const double s = end ? h : 0.0;
            const double t = (s - wa) / da;
            if (t <= 0 || t >= *tbest) continue;
            double q2 = 0;
            for (int k = 0; k < 3; ++k) { const double v = wp[k] + t * dp[k]; q2 += v * v; }
            if (q2 > r * r) continue;
            *tbest = t;
            for (int k = 0; k < 3; ++k) nbest[k] = end ? a[k] : -a[k];
        }
    }
}

/*
 * or_raycast: cam = 17 floats (as the renderer's), prims[np * 20].
 * Outputs per pixel (row-major H x W): hit u8, depth (= camera z), normal[3]
 * (world, outward), point[3] (world hit position).
 */
void or_raycast(const float *cam, int W, int H, const double *prims, int np, uint8_t *hit,
                double *depth, double *normal, double *point)
{
    double T[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T[i][j] = cam[4 * i + j];
        t[i] = cam[4 * i + 3];
    }
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    double o[3];
    for (int k = 0; k < 3; ++k) o[k] = -(T[0][k] * t[0] + T[1][k] * t[1] + T[2][k] * t[2]);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            const double dc[3] = {(i + 0.5 - cx) / fx, (j + 0.5 - cy) / fy, 1.0};
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = T[0][k] * dc[0] + T[1][k] * dc[1] + T[2][k] * dc[2];
            double tb = INFINITY, nb[3] = {0, 0, 0};
            for (int q = 0; q < np; ++q) {
                const double *P = prims + PREC * q;
                if (P[0] == 0) hit_ellipsoid(P, o, d, &tb, nb);
                else hit_cylinder(P, o, d, &tb, nb);
            }
            const int64_t pix = (int64_t)j * W + i;
            const int h = isfinite(tb);
            hit[pix] = (uint8_t)h;
            depth[pix] = h ? tb : 0.0;
            for (int k = 0; k < 3; ++k) {
                normal[3 * pix + k] = h ? nb[k] : 0.0;
                point[3 * pix + k] = h ? o[k] + tb * d[k] : 0.0;
            }
        }
}
