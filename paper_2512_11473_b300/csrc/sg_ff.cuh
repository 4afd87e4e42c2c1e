// sg_ff.cuh -- float-float ("double-float") arithmetic and analytic signed
// distance functions evaluated in it.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The error-free transforms are Knuth's TwoSum,
// Dekker's Fast2Sum and the FMA-based TwoProduct; division and square root
// take one Newton correction on a float estimate (Dekker 1971; Karp &
// Markstein 1997).  All primitive operations use the round-to-nearest
// intrinsics so that no compiler contraction can break an error-free step.
//
// The band predicate |d(cell centre)| < T decides which packages exist, so it
// must agree with an exact evaluation; float-float keeps the error near
// 1e-14 relative, far below the margin between any cell and the threshold.
// The initial level set is evaluated the same way and rounded to float once.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace sg {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    ff t = two_sum(x.lo, y.lo);
    float e = __fadd_rn(s.lo, t.hi);
    ff u = fast_two_sum(s.hi, e);
    float e2 = __fadd_rn(u.lo, t.lo);
    return fast_two_sum(u.hi, e2);
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = two_prod(x.hi, y.hi);
    float c = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    return fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}

__device__ __forceinline__ ff ff_mul_f(ff x, float b) {
    ff p = two_prod(x.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

__device__ __forceinline__ ff ff_sqr(ff x) { return ff_mul(x, x); }

// sqrt(x) for x >= 0, after Karp and Markstein ("High-precision division
// and square root", 1997): a reciprocal square root r of hi refined by one
// Newton step, a float root s = hi r corrected once, then
// sqrt(x) = s + (x - s^2) r / 2 with x - s^2 formed exactly (two_prod and
// Sterbenz); relative error about 2^-46.
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.0f)) return ff{0.0f, 0.0f};
    if (x.hi < 0x1p-100f) return ff{__fsqrt_rn(x.hi), 0.0f};  // far below any grid length; keeps rsqrtf normal
    float r = rsqrtf(x.hi);
    r = __fmul_rn(r, __fmaf_rn(__fmul_rn(-0.5f, x.hi), __fmul_rn(r, r), 1.5f));
    const float hr = __fmul_rn(0.5f, r);
    float s = __fmul_rn(x.hi, r);
    s = __fmaf_rn(__fmaf_rn(-s, s, x.hi), hr, s);
    const ff p = two_prod(s, s);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    return fast_two_sum(s, __fmul_rn(d, hr));
}

__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return ff_lt(b, a); }
__device__ __forceinline__ bool ff_neg_p(ff a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f); }
__device__ __forceinline__ ff ff_abs(ff a) { return ff_neg_p(a) ? ff_neg(a) : a; }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(a, b) ? a : b; }
__device__ __forceinline__ ff ff_clamp01(ff t) {
    if (ff_neg_p(t)) return ff{0.0f, 0.0f};
    if (ff_gt(t, ff{1.0f, 0.0f})) return ff{1.0f, 0.0f};
    return t;
}
__device__ __forceinline__ float ff_to_float(ff a) { return __fadd_rn(a.hi, a.lo); }

// ---------------------------------------------------------------------------
// Shapes, pre-split on the host into float-float constants.
// ---------------------------------------------------------------------------
enum { SHAPE_SPHERE = 0, SHAPE_PLANE = 1, SHAPE_TORUS = 2, SHAPE_PRISM = 3, SHAPE_ROUNDED_BOX = 4, SHAPE_SHELL = 5 };

struct ShapeFF {
    int kind;
    int plain;  // rotation is the identity and the centre the origin: q = x
    ff centre[3];
    ff rot[9];  // row-major, local -> world
    ff p[8];
    float cf[3], rf[9], pf[8];  // the same in float, for the float pre-filter
    // prism: per edge k (a -> b: 0 -> 1, 1 -> 2, 2 -> 0) e = b - a and
    // 1 / |e|^2 (seg[3k .. 3k+2]), and the sign of the triangle's orientation
    ff seg[9];
    int orient;
    ff zc, hz;  // prism: centre and half height of the z extent
};

// local coordinates q = R^T (x - centre)
__device__ __forceinline__ void ff_to_local(const ShapeFF& s, const ff x[3], ff q[3]) {
    ff d[3] = {ff_sub(x[0], s.centre[0]), ff_sub(x[1], s.centre[1]), ff_sub(x[2], s.centre[2])};
#pragma unroll
    for (int i = 0; i < 3; ++i)
        q[i] = ff_add(ff_add(ff_mul(s.rot[i], d[0]), ff_mul(s.rot[3 + i], d[1])), ff_mul(s.rot[6 + i], d[2]));
}


__device__ __forceinline__ ff ff_cross(ff ax, ff ay, ff bx, ff by) { return ff_sub(ff_mul(ax, by), ff_mul(ay, bx)); }

// squared distance from p to the edge from a along e, with 1 / |e|^2 given
__device__ __forceinline__ ff ff_edge_dist2(ff px, ff py, ff ax, ff ay, ff ex, ff ey, ff inv_len2) {
    ff wx = ff_sub(px, ax), wy = ff_sub(py, ay);
    ff t = ff_clamp01(ff_mul(ff_add(ff_mul(wx, ex), ff_mul(wy, ey)), inv_len2));
    ff dx = ff_sub(wx, ff_mul(t, ex)), dy = ff_sub(wy, ff_mul(t, ey));
    return ff_add(ff_sqr(dx), ff_sqr(dy));
}

__device__ __forceinline__ float f_edge_dist2(float px, float py, float ax, float ay, float ex, float ey, float inv_len2);

// upper estimate of sqrt(x) for x >= 0 (hardware approximation, relative
// error below 2^-22, inflated by 2^-20)
__device__ __forceinline__ float f_sqrt_up(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r * 1.000001f;
}

// Signed distance to a triangle (negative inside) in float-float.  A float
// pass first bounds each edge's squared distance (error below
// 2 |d| delta + delta^2 + 2.4e-7 d^2 with delta = 1e-6 (1 + |p|), generous
// for these few operations on inputs rounded to float): only the edges that
// can hold the minimum are evaluated in float-float.  The inside test is
// decided by float cross products when all three are clear of zero by their
// error bound, else in float-float.
__device__ inline ff ff_triangle_sdf(ff px, ff py, const ShapeFF& s) {
    const ff* t = s.p;
    const float* tf = s.pf;
    const float fx = px.hi, fy = py.hi;
    const float scale = 1.0f + fabsf(fx) + fabsf(fy), delta = 1e-6f * scale;
    float d[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        d[k] = f_edge_dist2(fx, fy, tf[2 * k], tf[2 * k + 1], s.seg[3 * k].hi, s.seg[3 * k + 1].hi, s.seg[3 * k + 2].hi);
    float tol[3], up = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        tol[k] = 2.0f * f_sqrt_up(d[k]) * delta + delta * delta + 2.4e-7f * d[k];
        hi[k] = d[k] + tol[k];
        up = fminf(up, hi[k]);
    }
    ff d2{INFINITY, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] - tol[k] > up) continue;  // cannot be the nearest edge
        const int a = 2 * k;
        d2 = ff_min(d2, ff_edge_dist2(px, py, t[a], t[a + 1], s.seg[3 * k], s.seg[3 * k + 1], s.seg[3 * k + 2]));
    }
    const float ctol = 8e-6f * scale * scale;
    float c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = 2 * k, b = (2 * k + 2) % 6;
        c[k] = (tf[b] - tf[a]) * (fy - tf[a + 1]) - (tf[b + 1] - tf[a + 1]) * (fx - tf[a]);
    }
    bool inside;
    if (fabsf(c[0]) > ctol && fabsf(c[1]) > ctol && fabsf(c[2]) > ctol) {
        inside = s.orient > 0 ? (c[0] > 0.0f && c[1] > 0.0f && c[2] > 0.0f) : (c[0] < 0.0f && c[1] < 0.0f && c[2] < 0.0f);
    } else {
        ff c0 = ff_cross(ff_sub(t[2], t[0]), ff_sub(t[3], t[1]), ff_sub(px, t[0]), ff_sub(py, t[1]));
        ff c1 = ff_cross(ff_sub(t[4], t[2]), ff_sub(t[5], t[3]), ff_sub(px, t[2]), ff_sub(py, t[3]));
        ff c2 = ff_cross(ff_sub(t[0], t[4]), ff_sub(t[1], t[5]), ff_sub(px, t[4]), ff_sub(py, t[5]));
        const ff zero{0.0f, 0.0f};
        inside = s.orient > 0 ? (ff_gt(c0, zero) && ff_gt(c1, zero) && ff_gt(c2, zero))
                              : (ff_lt(c0, zero) && ff_lt(c1, zero) && ff_lt(c2, zero));
    }
    ff dd = ff_sqrt(d2);
    return inside ? ff_neg(dd) : dd;
}

// The torus and the prism split into a part of the local (x, y) alone, the
// same for every point of a column along the local z axis, and a finish
// with z: the torus's in-plane distance to its core circle
// a = |(x, y)| - R, then sqrt(a^2 + z^2) - r; the prism's triangle distance
// w0, then its combination with the slab distance w1 = |z - zc| - hz.
template <int K>
__device__ __forceinline__ ff ff_column_k(const ShapeFF& s, ff qx, ff qy) {
    if (K == SHAPE_TORUS) return ff_sub(ff_sqrt(ff_add(ff_sqr(qx), ff_sqr(qy))), s.p[0]);
    return ff_triangle_sdf(qx, qy, s);
}

template <int K>
__device__ __forceinline__ ff ff_finish_k(const ShapeFF& s, ff col, ff qz) {
    if (K == SHAPE_TORUS) return ff_sub(ff_sqrt(ff_add(ff_sqr(col), ff_sqr(qz))), s.p[1]);
    const ff zero{0.0f, 0.0f};
    const ff w1 = ff_sub(ff_abs(ff_sub(qz, s.zc)), s.hz);
    // max(w0, w1) where at most one is positive, else the distance to the
    // rim sqrt(w0^2 + w1^2)
    if (!(ff_gt(col, zero) && ff_gt(w1, zero))) return ff_max(col, w1);
    return ff_sqrt(ff_add(ff_sqr(col), ff_sqr(w1)));
}

// Exact signed distance (negative inside) of primitive K, in float-float.
template <int K>
__device__ inline ff ff_sdf_k(const ShapeFF& s, const ff x[3]) {
    ff q[3];
    if (s.plain) {
        q[0] = x[0], q[1] = x[1], q[2] = x[2];
    } else {
        ff_to_local(s, x, q);
    }
    const ff zero{0.0f, 0.0f};
    switch (K) {
    case SHAPE_SPHERE:
        return ff_sub(ff_sqrt(ff_add(ff_add(ff_sqr(q[0]), ff_sqr(q[1])), ff_sqr(q[2]))), s.p[0]);
    case SHAPE_PLANE:
        return q[2];
    case SHAPE_SHELL: {  // | |q| - (r0 + r1)/2 | - (r1 - r0)/2
        ff r = ff_sqrt(ff_add(ff_add(ff_sqr(q[0]), ff_sqr(q[1])), ff_sqr(q[2])));
        ff mid = ff_mul_f(ff_add(s.p[0], s.p[1]), 0.5f), half = ff_mul_f(ff_sub(s.p[1], s.p[0]), 0.5f);
        return ff_sub(ff_abs(ff_sub(r, mid)), half);
    }
    case SHAPE_TORUS:
    case SHAPE_PRISM:
        return ff_finish_k<K>(s, ff_column_k<K>(s, q[0], q[1]), q[2]);
    case SHAPE_ROUNDED_BOX: {
        ff r = s.p[3];
        ff o = zero, m = ff{-INFINITY, 0.0f};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ff d = ff_sub(ff_abs(q[i]), ff_sub(s.p[i], r));
            if (ff_gt(d, zero)) o = ff_add(o, ff_sqr(d));
            if (ff_gt(d, m)) m = d;
        }
        return ff_sub(ff_add(ff_sqrt(o), ff_min(m, zero)), r);
    }
    default:
        return ff{NAN, 0.0f};
    }
}

// ---------------------------------------------------------------------------
// The same distances in plain float, for the pre-filter of the band
// predicate: decisions far from the thresholds are taken here, the rest in
// float-float.
// ---------------------------------------------------------------------------
// squared distance from p to the edge from a along e, with 1 / |e|^2 given
// (an error in the clamped parameter t changes the distance to second order)
__device__ __forceinline__ float f_edge_dist2(float px, float py, float ax, float ay, float ex, float ey, float inv_len2) {
    const float wx = px - ax, wy = py - ay;
    const float t = fminf(fmaxf((wx * ex + wy * ey) * inv_len2, 0.0f), 1.0f);
    const float dx = wx - t * ex, dy = wy - t * ey;
    return dx * dx + dy * dy;
}

template <int K>
__device__ inline float f_sdf_k(const ShapeFF& s, const float x[3]) {
    float q[3];
    if (s.plain) {
        q[0] = x[0], q[1] = x[1], q[2] = x[2];
    } else {
        const float d0 = x[0] - s.cf[0], d1 = x[1] - s.cf[1], d2 = x[2] - s.cf[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) q[i] = s.rf[i] * d0 + s.rf[3 + i] * d1 + s.rf[6 + i] * d2;
    }
    const float* p = s.pf;
    switch (K) {
    case SHAPE_SPHERE:
        return sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - p[0];
    case SHAPE_PLANE:
        return q[2];
    case SHAPE_SHELL:
        return fabsf(sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - 0.5f * (p[0] + p[1])) - 0.5f * (p[1] - p[0]);
    case SHAPE_TORUS: {
        const float a = sqrtf(q[0] * q[0] + q[1] * q[1]) - p[0];
        return sqrtf(a * a + q[2] * q[2]) - p[1];
    }
    case SHAPE_PRISM: {
        float d2 = INFINITY;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            d2 = fminf(d2, f_edge_dist2(q[0], q[1], p[2 * k], p[2 * k + 1], s.seg[3 * k].hi, s.seg[3 * k + 1].hi,
                                        s.seg[3 * k + 2].hi));
        const float orient = (p[2] - p[0]) * (p[5] - p[1]) - (p[3] - p[1]) * (p[4] - p[0]);
        const float c0 = (p[2] - p[0]) * (q[1] - p[1]) - (p[3] - p[1]) * (q[0] - p[0]);
        const float c1 = (p[4] - p[2]) * (q[1] - p[3]) - (p[5] - p[3]) * (q[0] - p[2]);
        const float c2 = (p[0] - p[4]) * (q[1] - p[5]) - (p[1] - p[5]) * (q[0] - p[4]);
        const bool inside = orient > 0.0f ? (c0 > 0.0f && c1 > 0.0f && c2 > 0.0f) : (c0 < 0.0f && c1 < 0.0f && c2 < 0.0f);
        const float w0 = inside ? -sqrtf(d2) : sqrtf(d2);
        const float w1 = fabsf(q[2] - 0.5f * (p[6] + p[7])) - 0.5f * (p[7] - p[6]);
        const float a = fmaxf(w0, 0.0f), b = fmaxf(w1, 0.0f);
        return fminf(fmaxf(w0, w1), 0.0f) + sqrtf(a * a + b * b);
    }
    case SHAPE_ROUNDED_BOX: {
        float o = 0.0f, m = -INFINITY;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float d = fabsf(q[i]) - (p[i] - p[3]);
            if (d > 0.0f) o += d * d;
            m = fmaxf(m, d);
        }
        return sqrtf(o) + fminf(m, 0.0f) - p[3];
    }
    default:
        return NAN;
    }
}

}  // namespace sg
