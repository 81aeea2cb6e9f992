/*
 * FP64 kNN-PCA oracle.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
 *
 * The closed-form per-point covariance estimate that the paper cites as the
 * prior way of sizing splats (local covariance of the point coordinates,
 * Sec. 2.1), used here as the estimator's fallback and as the judge of the
 * learned estimate:
 *   neighbours  the 16 nearest other points by Euclidean distance, ties by
 *               the smaller index (exact search on a uniform grid);
 *   covariance  Cov = 1/16 sum (p_j - pbar)(p_j - pbar)^T, pbar the mean of
 *               the 16 neighbours;
 *   axes        cyclic Jacobi eigen-decomposition, l1 >= l2 >= l3;
 *   Gaussian    s_a = kappa sqrt(l_a), s3 = max(s3, flat s2); rotation
 *               [e1 e2 e3] in a canonical frame (e3 = normal turned away
 *               from the cloud centroid, e1 with its largest-magnitude
 *               component positive, e2 = e3 x e1), quaternion by Shepperd's
 *               method.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KNN 16

typedef struct { double d; int64_t i; } cand_t;

static int cand_less(const cand_t *a, const cand_t *b) {
    return a->d < b->d || (a->d == b->d && a->i < b->i);
}

/* insert into a sorted array of at most KNN candidates */
static void cand_push(cand_t *best, int *nb, cand_t c) {
    if (*nb == KNN && !cand_less(&c, &best[KNN - 1])) return;
    int k = *nb < KNN ? (*nb)++ : KNN - 1;
    while (k > 0 && cand_less(&c, &best[k - 1])) { best[k] = best[k - 1]; --k; }
    best[k] = c;
}

/*
 * or_knn: idx[n*16] (ascending distance, ties by index), d2[n*16].
 */
void or_knn(int64_t n, const float *xyz, int64_t *idx, double *d2)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            const double v = xyz[3 * i + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) vol *= (hi[k] - lo[k]) + 1e-9;
    double h = cbrt(vol * 4.0 / (double)n);   /* ~4 points per cell in a filled box */
    int dim[3];
    for (int k = 0; k < 3; ++k) {
        double c = floor((hi[k] - lo[k]) / h) + 1;
        if (c > 1024) c = 1024;
        dim[k] = (int)c;
    }
    for (int k = 0; k < 3; ++k)
        if ((hi[k] - lo[k]) / h > dim[k]) h = (hi[k] - lo[k]) / dim[k] * 1.000001;
    const int64_t ncell = (int64_t)dim[0] * dim[1] * dim[2];
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * n);
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        for (int k = 0; k < 3; ++k) {
            int v = (int)floor((xyz[3 * i + k] - lo[k]) / h);
            c[k] = v < 0 ? 0 : (v >= dim[k] ? dim[k] - 1 : v);
        }
        cell[i] = ((int64_t)c[2] * dim[1] + c[1]) * dim[0] + c[0];
        start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ncell);
    memcpy(fill, start, sizeof(int64_t) * ncell);
    for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
    free(fill);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        cand_t best[KNN];
        int nb = 0;
        const double px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2];
        int c0[3];
        for (int k = 0; k < 3; ++k) {
            int v = (int)floor((xyz[3 * i + k] - lo[k]) / h);
            c0[k] = v < 0 ? 0 : (v >= dim[k] ? dim[k] - 1 : v);
        }
        const int rmax = dim[0] > dim[1] ? (dim[0] > dim[2] ? dim[0] : dim[2]) : (dim[1] > dim[2] ? dim[1] : dim[2]);
        for (int r = 0; r <= rmax; ++r) {
            for (int dz = -r; dz <= r; ++dz)
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        if (abs(dx) != r && abs(dy) != r && abs(dz) != r) continue;  /* ring r only */
                        const int cx = c0[0] + dx, cy = c0[1] + dy, cz = c0[2] + dz;
                        if (cx < 0 || cy < 0 || cz < 0 || cx >= dim[0] || cy >= dim[1] || cz >= dim[2]) continue;
                        const int64_t c = ((int64_t)cz * dim[1] + cy) * dim[0] + cx;
                        for (int64_t q = start[c]; q < start[c + 1]; ++q) {
                            const int64_t j = order[q];
                            if (j == i) continue;
                            const double ex = (double)xyz[3 * j] - px, ey = (double)xyz[3 * j + 1] - py,
                                         ez = (double)xyz[3 * j + 2] - pz;
                            cand_t cd = {ex * ex + ey * ey + ez * ez, j};
                            cand_push(best, &nb, cd);
                        }
                    }
            /* every point outside rings 0..r is at least r*h away */
            if (nb == KNN && best[KNN - 1].d < (r * h) * (r * h)) break;
        }
        for (int k = 0; k < KNN; ++k) {
            idx[KNN * i + k] = k < nb ? best[k].i : -1;
            d2[KNN * i + k] = k < nb ? best[k].d : -1.0;
        }
    }
    free(cell); free(start); free(order);
}

/* cyclic Jacobi on a symmetric 3x3; V columns are the eigenvectors */
static void jacobi3(double A[3][3], double V[3][3], double lam[3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    const double tr = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        if (off <= 1e-14 * tr || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {       /* A <- A J */
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {       /* A <- J^T A */
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {       /* V <- V J */
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int k = 0; k < 3; ++k) lam[k] = A[k][k];
}

/* Shepperd: unit quaternion (w, x, y, z) of a proper rotation matrix */
static void shepperd(const double R[3][3], double q[4])
{
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
        const double s = 2.0 * sqrt(1.0 + tr);
        q[0] = 0.25 * s; q[1] = (R[2][1] - R[1][2]) / s; q[2] = (R[0][2] - R[2][0]) / s; q[3] = (R[1][0] - R[0][1]) / s;
    } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
        const double s = 2.0 * sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]);
        q[0] = (R[2][1] - R[1][2]) / s; q[1] = 0.25 * s; q[2] = (R[0][1] + R[1][0]) / s; q[3] = (R[0][2] + R[2][0]) / s;
    } else if (R[1][1] >= R[2][2]) {
        const double s = 2.0 * sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]);
        q[0] = (R[0][2] - R[2][0]) / s; q[1] = (R[0][1] + R[1][0]) / s; q[2] = 0.25 * s; q[3] = (R[1][2] + R[2][1]) / s;
    } else {
        const double s = 2.0 * sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]);
        q[0] = (R[1][0] - R[0][1]) / s; q[1] = (R[0][2] + R[2][0]) / s; q[2] = (R[1][2] + R[2][1]) / s; q[3] = 0.25 * s;
    }
}

/*
 * or_pca: from idx[n*16]: cov[n*6] (xx, xy, xz, yy, yz, zz), lam[n*3]
 * (descending), scale[n*3], quat[n*4], normal[n*3].
 */
void or_pca(int64_t n, const float *xyz, const int64_t *idx, double kappa, double flat,
            double *cov, double *lam, double *scale, double *quat, double *normal)
{
    double cen[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) cen[k] += xyz[3 * i + k];
    for (int k = 0; k < 3; ++k) cen[k] /= (double)n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double mu[3] = {0, 0, 0};
        for (int a = 0; a < KNN; ++a)
            for (int k = 0; k < 3; ++k) mu[k] += xyz[3 * idx[KNN * i + a] + k];
        for (int k = 0; k < 3; ++k) mu[k] /= KNN;
        double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < KNN; ++a) {
            const int64_t j = idx[KNN * i + a];
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = xyz[3 * j + k] - mu[k];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) C[r][c] += d[r] * d[c];
        }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) C[r][c] /= KNN;
        double *cv = cov + 6 * i;
        cv[0] = C[0][0]; cv[1] = C[0][1]; cv[2] = C[0][2]; cv[3] = C[1][1]; cv[4] = C[1][2]; cv[5] = C[2][2];
        double A[3][3], V[3][3], l[3];
        memcpy(A, C, sizeof A);
        jacobi3(A, V, l);
        int o[3] = {0, 1, 2};                       /* sort descending */
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b)
                if (l[o[b]] > l[o[a]]) { int t = o[a]; o[a] = o[b]; o[b] = t; }
        double R[3][3];
        for (int a = 0; a < 3; ++a) {
            lam[3 * i + a] = l[o[a]];
            for (int k = 0; k < 3; ++k) R[k][a] = V[k][o[a]];
        }
        /* canonical frame: e3 (normal) away from the cloud centroid, e1 with
         * its largest-magnitude component positive, e2 = e3 x e1 */
        double sg = 0;
        for (int k = 0; k < 3; ++k) sg += (xyz[3 * i + k] - cen[k]) * R[k][2];
        if (sg < 0)
            for (int k = 0; k < 3; ++k) R[k][2] = -R[k][2];
        int km = 0;
        for (int k = 1; k < 3; ++k)
            if (fabs(R[k][0]) > fabs(R[km][0])) km = k;
        if (R[km][0] < 0)
            for (int k = 0; k < 3; ++k) R[k][0] = -R[k][0];
        R[0][1] = R[1][2] * R[2][0] - R[2][2] * R[1][0];
        R[1][1] = R[2][2] * R[0][0] - R[0][2] * R[2][0];
        R[2][1] = R[0][2] * R[1][0] - R[1][2] * R[0][0];
        for (int k = 0; k < 3; ++k) normal[3 * i + k] = R[k][2];
        double s[3];
        for (int a = 0; a < 3; ++a) s[a] = kappa * sqrt(lam[3 * i + a] > 0 ? lam[3 * i + a] : 0.0);
        if (s[2] < flat * s[1]) s[2] = flat * s[1];
        for (int a = 0; a < 3; ++a) scale[3 * i + a] = s[a];
        shepperd(R, quat + 4 * i);
    }
}
