// K1: EWA projection and 3-sigma tile footprint (Sec. 3.1, Eq. 3-4).
//
// One thread per (view, Gaussian).  The integer results -- cull, tile
// rectangle and the fp32 depth key -- must equal those of an IEEE double
// evaluation in a fixed statement order.  They are taken from an fp32 fast
// path that carries a forward error bound; whenever the bound straddles a
// decision boundary (or anything is non-finite) the thread recomputes the
// Gaussian in double precision in that exact statement order.  GB300's FP64
// rate is low, so the fallback is kept to the rare ambiguous Gaussians.
//
// Continuous outputs for the blend (sub-pixel centre, conic) come from the
// fast path: the centre is carried in float-float so that pixel offsets keep
// ~1e-7 px accuracy at 2048 px, which the 1e-4 image tolerance needs.
#include "common.cuh"

namespace p2e {

struct ProjOut {
    bool visible;
    int tx0, ty0, tx1, ty1;   // exact tile rectangle (inclusive)
    int px0, py0, px1, py1;   // pixel rectangle: exact (double path) or a superset
                              // of it clamped to the exact tile rectangle
    float fu, fv;          // sub-pixel parts of the centre, in [0, 1)
    int iu, iv;            // floor of the centre
    float zkey;            // fp32 of the double camera depth
    float A, B, C;         // conic
};

// Integer footprint of one axis from the ellipse box [lo, hi] (both already
// shifted by -0.5 so that pixel i is inside iff lo <= i <= hi).
__device__ __forceinline__ void axis_rect(float lo, float hi, int W, int B, int &t0, int &t1,
                                          bool &empty) {
    const float c0 = fmaxf(0.f, ceilf(lo));
    const float c1 = fminf((float)(W - 1), floorf(hi));
    empty = !(c0 <= c1);
    t0 = empty ? 0 : (int)c0 / B;
    t1 = empty ? 0 : (int)c1 / B;
}

__device__ __forceinline__ void axis_rect_d(double lo, double hi, int W, int B, int &t0, int &t1,
                                            bool &empty) {
    const double c0 = fmax(0.0, ceil(lo));
    const double c1 = fmin((double)(W - 1), floor(hi));
    empty = !(c0 <= c1);
    t0 = empty ? 0 : (int)c0 / B;
    t1 = empty ? 0 : (int)c1 / B;
}

// Double-precision projection in the reference statement order (every
// operation an explicit correctly rounded intrinsic, nothing contracted).
__device__ __noinline__ void project_fp64(const View &V, const Views &P, float4 m, float4 s4,
                                          float4 q4, ProjOut &o) {
    o.visible = false;
    const double mx = m.x, my = m.y, mz = m.z;
    double T[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T[i][j] = (double)V.T[3 * i + j];
        t[i] = (double)V.t[i];
    }
    const double z = __fma_rn(T[2][0], mx, __fma_rn(T[2][1], my, __fma_rn(T[2][2], mz, t[2])));
    const double x = __fma_rn(T[0][0], mx, __fma_rn(T[0][1], my, __fma_rn(T[0][2], mz, t[0])));
    const double y = __fma_rn(T[1][0], mx, __fma_rn(T[1][1], my, __fma_rn(T[1][2], mz, t[1])));
    o.zkey = __double2float_rn(z);
    if (!(z > (double)V.near_z)) return;
    const double qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
    if (qw == 0.0 && qx == 0.0 && qy == 0.0 && qz == 0.0) return;
    const double qn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(qw, qw), __dmul_rn(qx, qx)),
                                                     __dmul_rn(qy, qy)),
                                           __dmul_rn(qz, qz)));
    const double w = __ddiv_rn(qw, qn), xx = __ddiv_rn(qx, qn), yy = __ddiv_rn(qy, qn),
                 zz = __ddiv_rn(qz, qn);
    double R[3][3];
    R[0][0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(yy, yy), __dmul_rn(zz, zz))));
    R[0][1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(xx, yy), __dmul_rn(w, zz)));
    R[0][2] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(xx, zz), __dmul_rn(w, yy)));
    R[1][0] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(xx, yy), __dmul_rn(w, zz)));
    R[1][1] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(xx, xx), __dmul_rn(zz, zz))));
    R[1][2] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(yy, zz), __dmul_rn(w, xx)));
    R[2][0] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(xx, zz), __dmul_rn(w, yy)));
    R[2][1] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(yy, zz), __dmul_rn(w, xx)));
    R[2][2] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(xx, xx), __dmul_rn(yy, yy))));
    const double s[3] = {(double)s4.x, (double)s4.y, (double)s4.z};
    double Vm[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Vm[i][j] = __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn(T[i][0], R[0][j]), __dmul_rn(T[i][1], R[1][j])),
                                           __dmul_rn(T[i][2], R[2][j])),
                                 s[j]);
    const double fx = V.fx, fy = V.fy, cx = V.cx, cy = V.cy;
    const double xs = __ddiv_rn(x, z), ys = __ddiv_rn(y, z);
    const double j00 = __ddiv_rn(fx, z), j02 = __ddiv_rn(-__dmul_rn(fx, xs), z);
    const double j11 = __ddiv_rn(fy, z), j12 = __ddiv_rn(-__dmul_rn(fy, ys), z);
    double M0[3], M1[3];
    for (int j = 0; j < 3; ++j) {
        M0[j] = __dadd_rn(__dmul_rn(j00, Vm[0][j]), __dmul_rn(j02, Vm[2][j]));
        M1[j] = __dadd_rn(__dmul_rn(j11, Vm[1][j]), __dmul_rn(j12, Vm[2][j]));
    }
    const double lp = (double)P.lowpass;
    const double a = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(M0[0], M0[0]), __dmul_rn(M0[1], M0[1])),
                                         __dmul_rn(M0[2], M0[2])),
                               lp);
    const double b = __dadd_rn(__dadd_rn(__dmul_rn(M0[0], M1[0]), __dmul_rn(M0[1], M1[1])),
                               __dmul_rn(M0[2], M1[2]));
    const double c = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(M1[0], M1[0]), __dmul_rn(M1[1], M1[1])),
                                         __dmul_rn(M1[2], M1[2])),
                               lp);
    const double det = __dsub_rn(__dmul_rn(a, c), __dmul_rn(b, b));
    const double u = __dadd_rn(__dmul_rn(fx, xs), cx);
    const double v = __dadd_rn(__dmul_rn(fy, ys), cy);
    if (!(det > 0.0) || !isfinite(det) || !isfinite(a) || !isfinite(c) || !isfinite(b) ||
        !isfinite(u) || !isfinite(v))
        return;
    const double k = (double)P.sigma_mult;
    const double ex = __dmul_rn(k, __dsqrt_rn(a)), ey = __dmul_rn(k, __dsqrt_rn(c));
    const double lox = __dsub_rn(__dsub_rn(u, ex), 0.5), hix = __dsub_rn(__dadd_rn(u, ex), 0.5);
    const double loy = __dsub_rn(__dsub_rn(v, ey), 0.5), hiy = __dsub_rn(__dadd_rn(v, ey), 0.5);
    bool ex_, ey_;
    axis_rect_d(lox, hix, V.W, P.tile, o.tx0, o.tx1, ex_);
    axis_rect_d(loy, hiy, V.H, P.tile, o.ty0, o.ty1, ey_);
    if (ex_ || ey_) return;
    o.visible = true;
    o.px0 = (int)fmax(0.0, ceil(lox));
    o.px1 = (int)fmin((double)(V.W - 1), floor(hix));
    o.py0 = (int)fmax(0.0, ceil(loy));
    o.py1 = (int)fmin((double)(V.H - 1), floor(hiy));
    const double fu = floor(u), fv = floor(v);
    o.fu = (float)(u - fu);
    o.fv = (float)(v - fv);
    o.iu = (int)fmax(-32768.0, fmin(32767.0, fu));
    o.iv = (int)fmax(-32768.0, fmin(32767.0, fv));
    if ((double)o.iu != fu) o.fu = (float)(u - (double)o.iu);
    if ((double)o.iv != fv) o.fv = (float)(v - (double)o.iv);
    o.A = (float)(c / det);
    o.B = (float)(-b / det);
    o.C = (float)(a / det);
}

// x = r . m + t as a float-float (hi, lo) plus the magnitude sum |terms|.
__device__ __forceinline__ void ff_affine(float r0, float r1, float r2, float t, float mx, float my,
                                          float mz, float &hi, float &lo, float &mag) {
    float p0, e0, p1, e1, p2, e2, s, c, err;
    two_prod(r0, mx, p0, e0);
    two_prod(r1, my, p1, e1);
    two_prod(r2, mz, p2, e2);
    two_sum(t, p0, s, c);
    err = c;
    two_sum(s, p1, s, c);
    err = __fadd_rn(err, c);
    two_sum(s, p2, s, c);
    err = __fadd_rn(err, c);
    err = __fadd_rn(err, __fadd_rn(e0, __fadd_rn(e1, e2)));
    fast_two_sum(s, err, hi, lo);
    mag = fabsf(t) + fabsf(p0) + fabsf(p1) + fabsf(p2);
}

// (xh + xl) / (zh + zl) as a float-float.
__device__ __forceinline__ void ff_div(float xh, float xl, float zh, float zl, float &qh, float &ql) {
    const float q1 = __fdiv_rn(xh, zh);
    float r = __fmaf_rn(-q1, zh, xh);                 // exact remainder
    r = __fadd_rn(r, __fsub_rn(xl, __fmul_rn(q1, zl)));
    const float q2 = __fdiv_rn(r, zh);
    fast_two_sum(q1, q2, qh, ql);
}

// f * (qh + ql) + c as a float-float.
__device__ __forceinline__ void ff_affine1(float f, float qh, float ql, float c, float &uh, float &ul) {
    float p, e, s, t;
    two_prod(f, qh, p, e);
    e = __fmaf_rn(f, ql, e);
    two_sum(p, c, s, t);
    fast_two_sum(s, __fadd_rn(t, e), uh, ul);
}

// floor of hi + lo and the fractional part in [0, 1).
__device__ __forceinline__ void ff_floor(float hi, float lo, int &i, float &f) {
    float fl = floorf(hi);
    float fr = __fadd_rn(__fsub_rn(hi, fl), lo);
    if (fr >= 1.f) { fl += 1.f; fr = __fsub_rn(fr, 1.f); }
    if (fr < 0.f) { fl -= 1.f; fr = __fadd_rn(fr, 1.f); }
    if (fr >= 1.f) fr = 0x1.fffffep-1f;
    const float cl = fmaxf(-32768.f, fminf(32767.f, fl));
    if (cl != fl) fr = __fadd_rn(__fsub_rn(hi, cl), lo);
    i = (int)cl;
    f = fr;
}

// fp32 fast path.  Returns false when a decision is not certain.
__device__ __forceinline__ bool project_fp32(const View &V, const Views &P, float4 m, float4 s4,
                                             float4 q4, ProjOut &o) {
    o.visible = false;
    float xh, xl, xm, yh, yl, ym, zh, zl, zm;
    ff_affine(V.T[0], V.T[1], V.T[2], V.t[0], m.x, m.y, m.z, xh, xl, xm);
    ff_affine(V.T[3], V.T[4], V.T[5], V.t[1], m.x, m.y, m.z, yh, yl, ym);
    ff_affine(V.T[6], V.T[7], V.T[8], V.t[2], m.x, m.y, m.z, zh, zl, zm);
    if (!isfinite(zh) || !isfinite(xh) || !isfinite(yh)) return false;
    // depth key: fp32(z) is zh unless hi + lo sits within the error bound of
    // a rounding midpoint (then the double path decides).
    {
        const float ez = zm * 0x1p-42f;
        const float up = __fsub_rn(nextafterf(zh, INFINITY), zh);
        const float dn = __fsub_rn(zh, nextafterf(zh, -INFINITY));
        const float gap = zl >= 0.f ? 0.5f * up : 0.5f * dn;
        if (!(fabsf(zl) + ez < gap)) return false;
        o.zkey = zh;
    }
    // near-plane cull
    {
        const float d = __fsub_rn(zh, V.near_z);
        const float e = (fabsf(zh) + fabsf(V.near_z)) * 0x1p-22f + fabsf(zl) + zm * 0x1p-40f;
        if (fabsf(d) <= e) return false;
        if (d < 0.f) return true;  // culled for certain
    }
    if (q4.x == 0.f && q4.y == 0.f && q4.z == 0.f && q4.w == 0.f) return true;  // culled
    // rotation of the normalised quaternion (Hamilton, w first)
    const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
    if (!(qn2 > 0x1p-100f) || !isfinite(qn2)) return false;
    const float rq = 1.f / sqrtf(qn2);
    const float w = q4.x * rq, x = q4.y * rq, y = q4.z * rq, z = q4.w * rq;
    float R[3][3];
    R[0][0] = 1.f - 2.f * (y * y + z * z);
    R[0][1] = 2.f * (x * y - w * z);
    R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);
    R[1][1] = 1.f - 2.f * (x * x + z * z);
    R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);
    R[2][1] = 2.f * (y * z + w * x);
    R[2][2] = 1.f - 2.f * (x * x + y * y);
    const float s[3] = {s4.x, s4.y, s4.z};
    // M = J (T R) S and its magnitude bound |J| (|T| (|R| + eps)) |S|
    float xs, xsl, ys, ysl;
    ff_div(xh, xl, zh, zl, xs, xsl);
    ff_div(yh, yl, zh, zl, ys, ysl);
    const float iz = 1.f / zh;
    const float j00 = V.fx * iz, j02 = -(V.fx * xs) * iz;
    const float j11 = V.fy * iz, j12 = -(V.fy * ys) * iz;
    float M0[3], M1[3], A0[3], A1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float vr[3], va[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            vr[i] = (V.T[3 * i] * R[0][j] + V.T[3 * i + 1] * R[1][j] + V.T[3 * i + 2] * R[2][j]) * s[j];
            // |T|(|R| + 1)|s|: the +1 makes the bound absolute in the scale
            // of |T||s|, which covers the O(u) error of the computed R.
            va[i] = (fabsf(V.T[3 * i]) * (fabsf(R[0][j]) + 1.f) +
                     fabsf(V.T[3 * i + 1]) * (fabsf(R[1][j]) + 1.f) +
                     fabsf(V.T[3 * i + 2]) * (fabsf(R[2][j]) + 1.f)) * fabsf(s[j]);
        }
        M0[j] = j00 * vr[0] + j02 * vr[2];
        M1[j] = j11 * vr[1] + j12 * vr[2];
        A0[j] = fabsf(j00) * va[0] + fabsf(j02) * va[2];
        A1[j] = fabsf(j11) * va[1] + fabsf(j12) * va[2];
    }
    const float lp = P.lowpass;
    const float a = M0[0] * M0[0] + M0[1] * M0[1] + M0[2] * M0[2] + lp;
    const float b = M0[0] * M1[0] + M0[1] * M1[1] + M0[2] * M1[2];
    const float c = M1[0] * M1[0] + M1[1] * M1[1] + M1[2] * M1[2] + lp;
    // Each computed M entry is within 2^-20 of its magnitude bound A (R, J,
    // T R and the sums each add a few ulp); a, b, c inherit 2|M| err(M) plus
    // their own rounding.  The constants carry a 2x margin.
    const float ea = 0x1p-18f * (A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2]) + 0x1p-21f * a;
    const float ec = 0x1p-18f * (A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2]) + 0x1p-21f * c;
    const float eb = 0x1p-18f * (A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2]) + 0x1p-21f * fabsf(b);
    const float det = a * c - b * b;
    if (!isfinite(a) || !isfinite(b) || !isfinite(c) || !isfinite(det) || !isfinite(ea) ||
        !isfinite(ec))
        return false;
    const float edet = ea * c + ec * a + 2.f * fabsf(b) * eb + ea * ec + eb * eb +
                       0x1p-21f * (a * c + b * b);
    if (fabsf(det) <= edet) return false;
    if (det < 0.f) return true;  // culled for certain
    // screen centre, float-float
    float uh, ul, vh, vl;
    ff_affine1(V.fx, xs, xsl, V.cx, uh, ul);
    ff_affine1(V.fy, ys, ysl, V.cy, vh, vl);
    if (!isfinite(uh) || !isfinite(vh)) return false;
    // k-sigma box and its error bound
    const float k = P.sigma_mult;
    const float sa = sqrtf(a), sc = sqrtf(c);
    const float ex = k * sa, ey = k * sc;
    const float dex = k * (sqrtf(a + ea) - sqrtf(fmaxf(a - ea, 0.f))) + 0x1p-21f * ex;
    const float dey = k * (sqrtf(c + ec) - sqrtf(fmaxf(c - ec, 0.f))) + 0x1p-21f * ey;
    const float lox = __fadd_rn(__fsub_rn(__fsub_rn(uh, 0.5f), ex), ul);
    const float hix = __fadd_rn(__fadd_rn(__fsub_rn(uh, 0.5f), ex), ul);
    const float loy = __fadd_rn(__fsub_rn(__fsub_rn(vh, 0.5f), ey), vl);
    const float hiy = __fadd_rn(__fadd_rn(__fsub_rn(vh, 0.5f), ey), vl);
    // three fp32 roundings of at most 2^-24 |value| each (the two in lo/hi
    // and the +-eps below), plus an absolute term for the float-float centre
    // and the double evaluation's own rounding.
    const float epx = dex + 0x1p-21f * (fabsf(uh) + ex + 1.f) + 1e-6f;
    const float epy = dey + 0x1p-21f * (fabsf(vh) + ey + 1.f) + 1e-6f;
    if (!isfinite(lox + hix + loy + hiy + epx + epy)) return false;
    int a0, a1, b0, b1, c0, c1, d0, d1;
    bool ea_, eb_, ec_, ed_;
    axis_rect(lox - epx, hix + epx, V.W, P.tile, a0, a1, ea_);
    axis_rect(lox + epx, hix - epx, V.W, P.tile, b0, b1, eb_);
    axis_rect(loy - epy, hiy + epy, V.H, P.tile, c0, c1, ec_);
    axis_rect(loy + epy, hiy - epy, V.H, P.tile, d0, d1, ed_);
    if (ea_ != eb_ || ec_ != ed_) return false;
    if (ea_ || ec_) return true;  // culled for certain (empty box)
    if (a0 != b0 || a1 != b1 || c0 != d0 || c1 != d1) return false;
    o.tx0 = a0; o.tx1 = a1; o.ty0 = c0; o.ty1 = c1;
    // pixel rectangle of the widened box, clamped into the exact tile
    // rectangle: a superset of the exact pixel rectangle with the same tiles
    {
        const int B = P.tile;
        const float fx0 = fmaxf(0.f, fminf(ceilf(lox - epx), (float)(V.W - 1)));
        const float fx1 = fmaxf(0.f, fminf(floorf(hix + epx), (float)(V.W - 1)));
        const float fy0 = fmaxf(0.f, fminf(ceilf(loy - epy), (float)(V.H - 1)));
        const float fy1 = fmaxf(0.f, fminf(floorf(hiy + epy), (float)(V.H - 1)));
        o.px0 = max((int)fx0, a0 * B);
        o.px1 = min((int)fx1, a1 * B + B - 1);
        o.py0 = max((int)fy0, c0 * B);
        o.py1 = min((int)fy1, c1 * B + B - 1);
    }
    ff_floor(uh, ul, o.iu, o.fu);
    ff_floor(vh, vl, o.iv, o.fv);
    const float idet = 1.f / det;
    o.A = c * idet;
    o.B = -b * idet;
    o.C = a * idet;
    o.visible = true;
    return true;
}

__global__ void __launch_bounds__(256, 4) project_kernel(const float4 *__restrict__ mean_op,
                                                      const float4 *__restrict__ scale,
                                                      const float4 *__restrict__ quat,
                                                      float4 *__restrict__ xy_depth,
                                                      float4 *__restrict__ conic_op,
                                                      ushort4 *__restrict__ rect,
                                                      uint32_t *__restrict__ ntiles,
                                                      __grid_constant__ const Views P) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int vi = blockIdx.y;
    if (g >= P.n) return;
    const View &V = P.v[vi];
    const float4 m = __ldg(mean_op + g);
    const float4 s = __ldg(scale + g);
    const float4 q = __ldg(quat + g);
    ProjOut o;
    o.zkey = 0.f;
    if (!project_fp32(V, P, m, s, q, o)) project_fp64(V, P, m, s, q, o);
    const int64_t e = (int64_t)vi * P.n + g;
    if (!o.visible) {
        ntiles[e] = 0u;
        rect[e] = make_ushort4(0, 0, 0, 0);
        xy_depth[e] = make_float4(0.f, 0.f, o.zkey, 0.f);
        conic_op[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    ntiles[e] = (uint32_t)((o.tx1 - o.tx0 + 1) * (o.ty1 - o.ty0 + 1));
    rect[e] = make_ushort4((unsigned short)o.px0, (unsigned short)o.py0, (unsigned short)o.px1,
                           (unsigned short)o.py1);
    const uint32_t packed = ((uint32_t)(uint16_t)(int16_t)o.iu) | ((uint32_t)(uint16_t)(int16_t)o.iv << 16);
    xy_depth[e] = make_float4(o.fu, o.fv, o.zkey, __uint_as_float(packed));
    conic_op[e] = make_float4(o.A, o.B, o.C, m.w);
}

cudaError_t launch_project(const p2e_gaussians *g, const Views &P, p2e_projected *out,
                           cudaStream_t st) {
    if (P.n == 0) return cudaSuccess;
    dim3 grid((unsigned)((P.n + 255) / 256), (unsigned)P.n_views);
    project_kernel<<<grid, 256, 0, st>>>((const float4 *)g->mean_op, (const float4 *)g->scale,
                                         (const float4 *)g->quat, (float4 *)out->xy_depth,
                                         (float4 *)out->conic_op, (ushort4 *)out->rect,
                                         out->ntiles, P);
    return cudaGetLastError();
}

}  // namespace p2e
