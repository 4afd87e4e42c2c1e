// sg_sur.cuh -- device code of the kernel-integral surrogate shared by its
// inference (sg_kernel_integrals mode 1, single grid and batch), its training
// samples and its training kernel (sg_mlp.cu): the exact class decision, the
// symmetry canonicalisation of the 27 inputs, and the three layers of one
// 128-row tile on the tcgen05 tensor cores.
//
// Symmetries of the exact integral (no paper counterpart; they follow from
// the definitions of W and G^): the tap weights depend on |s| alone, so a
// signed permutation T of the axes maps the inputs v(s) -> v(T^-1 s) and the
// outputs W -> W, G^ -> T G^; the smoothed Heaviside is antisymmetric,
// H(-z) = 1 - H(z), so v -> -v maps W -> 1 - W, G^ -> -G^.  The network
// therefore only sees canonical inputs: centre value positive (phi >= h),
// central differences g_a = phi(+a) - phi(-a) non-negative and ordered
// g_0 >= g_1 >= g_2, and its outputs are carried back.  The decisions use
// exact arithmetic (a difference of two floats is held exactly as a
// float-float pair), ties between |g_a| keep the lower axis first, so every
// implementation of the definition picks the same transform.
#pragma once
#include "sg_integrals.cuh"
#include "sg_mlp.cuh"
#include "sg_umma.cuh"

namespace sg {
namespace {

__device__ __forceinline__ float tanh_approx(float x) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// logistic sigmoid through the hardware tanh: 1 / (1 + e^-z) = (1 + tanh(z/2)) / 2
__device__ __forceinline__ float sigmoidf_(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }
// SiLU z sigmoid(z) = h + h tanh(h) with h = z/2
__device__ __forceinline__ float silu_(float z) {
    const float h = 0.5f * z;
    return fmaf(h, tanh_approx(h), h);
}

// silu_(v + b) of two values at once on paired FP32 instructions (each lane
// the same rounded operations as the scalar form, so the same bits)
__device__ __forceinline__ float2 silu2_bias(float2 v, float2 b) {
    const float2 h = __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(v, b));
    return __ffma2_rn(h, make_float2(tanh_approx(h.x), tanh_approx(h.y)), h);
}

// v[i] = silu_(v[i] + bias[i]) for 32 consecutive columns (bias 8-byte aligned)
__device__ __forceinline__ void silu32_bias(float (&v)[32], const float* bias) {
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
        const float2 s = silu2_bias(make_float2(v[i], v[i + 1]), *reinterpret_cast<const float2*>(bias + i));
        v[i] = s.x;
        v[i + 1] = s.y;
    }
}

// ---------------------------------------------------------------------------
// Class decision (see SurConst): exact on the real values of the float phi.
// ---------------------------------------------------------------------------

// |kappa| h > 0.1 with kappa the 7-point Laplacian (sum of the six face
// neighbours - 6 phi) / h^2, i.e. |a| > 0.1 h for the numerator a: the float
// sum a is within 7 roundings, 2^-21 S, of the exact one (S the float sum of
// the terms' magnitudes); only when |a| falls within 2^-19 S of the bound is
// the numerator re-formed in float-float (error about 2^-44 S).
__device__ __forceinline__ bool curvature_exceeds(float xp, float xm, float yp, float ym, float zp, float zm, float c,
                                                  const SurConst& C) {
    const float a = __fadd_rn(__fadd_rn(__fadd_rn(xp, xm), __fadd_rn(yp, ym)),
                              __fsub_rn(__fadd_rn(zp, zm), __fmul_rn(6.0f, c)));
    const float S = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(xp), fabsf(xm)), __fadd_rn(fabsf(yp), fabsf(ym))),
                              __fadd_rn(__fadd_rn(fabsf(zp), fabsf(zm)), __fmul_rn(6.0f, fabsf(c))));
    const float d = __fsub_rn(fabsf(a), C.kap_thr);
    if (fabsf(d) > __fmul_rn(0x1p-19f, S) + __fmul_rn(0x1p-22f, C.kap_thr)) return d > 0.0f;
    ff s = ff_add(two_sum(xp, xm), two_sum(yp, ym));
    s = ff_add(s, two_sum(zp, zm));
    s = ff_add(s, two_prod(-6.0f, c));  // -6 phi exactly
    if (s.hi < 0.0f) s = ff_neg(s);
    return ff_gt(s, C.kap_thr_ff);
}

// Class of the data point at e0 of a phi tile (rows of TILE_Y, planes of
// TILE_Z): trivial where every tap has |phi_s| >= h on one side (the
// Heaviside saturates), fallback where |phi| < h or |kappa| h > 0.1, network
// else.
__device__ __forceinline__ int sur_class_at(const float* tile, int e0, const SurConst& C) {
    bool all_in = true, all_out = true;
#pragma unroll
    for (int n = 0; n < MLP_IN; ++n) {
        const int sx = n % 3 - 1, sy = (n / 3) % 3 - 1, sz = n / 9 - 1;
        const float f = tile[e0 + sx + TILE_Y * sy + TILE_Z * sz];
        all_in &= -f >= C.h_up;
        all_out &= f >= C.h_up;
    }
    if (all_in) return SG_SUR_TRIVIAL_IN;
    if (all_out) return SG_SUR_TRIVIAL_OUT;
    const float c = tile[e0];
    if (fabsf(c) < C.h_up) return SG_SUR_FALLBACK;
    if (curvature_exceeds(tile[e0 + 1], tile[e0 - 1], tile[e0 + TILE_Y], tile[e0 - TILE_Y], tile[e0 + TILE_Z],
                          tile[e0 - TILE_Z], c, C))
        return SG_SUR_FALLBACK;
    return SG_SUR_NETWORK;
}

// The fallback test of a point that is not trivial: |phi| < h, or
// |kappa| h > 0.1 (the last two steps of sur_class_at).
__device__ __forceinline__ bool sur_fallback_at(const float* tile, int e0, const SurConst& C) {
    const float c = tile[e0];
    if (fabsf(c) < C.h_up) return true;
    return curvature_exceeds(tile[e0 + 1], tile[e0 - 1], tile[e0 + TILE_Y], tile[e0 - TILE_Y], tile[e0 + TILE_Z],
                             tile[e0 - TILE_Z], c, C);
}

__device__ __forceinline__ int tile_e0(int d) { return ((d & 3) + 1) + TILE_Y * (((d >> 2) & 3) + 1) + TILE_Z * ((d >> 4) + 1); }

// ---------------------------------------------------------------------------
// Canonical transform.  code = flip | reflections << 1 | perm << 4:
//   flip        the centre value is negative (inputs and W, G^ negate)
//   reflections bit a: original axis a reversed
//   perm        which of the six axis permutations (lexicographic order):
//               canonical axis k is original axis perm_axis(perm, k)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int perm_axis(int perm, int k) {
    // (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0): two bits per entry,
    // six bits per permutation, in one register-held constant
    constexpr uint64_t tab = 0x24ull | 0x18ull << 6 | 0x21ull << 12 | 0x09ull << 18 | 0x12ull << 24 | 0x06ull << 30;
    return (int)((tab >> (6 * perm + 2 * k)) & 3u);
}

// Index of the permutation (p0, p1, 3 - p0 - p1).
__device__ __forceinline__ int perm_index(int p0, int p1) { return 2 * p0 + (p1 > 3 - p0 - p1 ? 1 : 0); }

// Canonical input position of original input n (offset s, n = (sx+1) +
// 3 (sy+1) + 9 (sz+1)) under reflections rb and permutation perm.
__device__ __forceinline__ int canon_pos(int n, int rb, int perm) {
    int s[3] = {n % 3 - 1, (n / 3) % 3 - 1, n / 9 - 1};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (rb >> a & 1) s[a] = -s[a];
    int m = 0, w = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k, w *= 3) m += (s[perm_axis(perm, k)] + 1) * w;
    return m;
}

__device__ __forceinline__ bool ff_abs_gt(ff a, ff b) {  // |a| > |b| for exact differences
    if (a.hi < 0.0f) a = ff_neg(a);
    if (b.hi < 0.0f) b = ff_neg(b);
    return ff_gt(a, b);
}

// Canonical code of a point from its centre and six face neighbours.
__device__ __forceinline__ int canon_code(float c, float xp, float xm, float yp, float ym, float zp, float zm) {
    const bool flip = c < 0.0f;
    ff g[3] = {two_sum(xp, -xm), two_sum(yp, -ym), two_sum(zp, -zm)};  // exact differences
    int rb = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (flip) g[a] = ff_neg(g[a]);
        if (g[a].hi < 0.0f) rb |= 1 << a;
    }
    // stable sort of the axes by decreasing |g| (equal magnitudes keep the
    // lower axis first), the values moving with their axes
    ff ga = g[0], gb = g[1], gc = g[2];
    int p0 = 0, p1 = 1, p2 = 2;
    if (ff_abs_gt(gb, ga)) {
        const ff u = ga; ga = gb; gb = u;
        const int v = p0; p0 = p1; p1 = v;
    }
    if (ff_abs_gt(gc, gb)) {
        const ff u = gb; gb = gc; gc = u;
        const int v = p1; p1 = p2; p2 = v;
    }
    if (ff_abs_gt(gb, ga)) {
        const int v = p0; p0 = p1; p1 = v;
    }
    (void)p2;
    return (flip ? 1 : 0) | (rb << 1) | (perm_index(p0, p1) << 4);
}

// Network outputs (canonical frame) -> (W, G^) of the point.
__device__ __forceinline__ void uncanon_outputs(int code, const float (&y)[4], float (&o)[4]) {
    const bool flip = code & 1;
    const int rb = (code >> 1) & 7, perm = code >> 4;
    o[0] = flip ? __fsub_rn(1.0f, y[0]) : y[0];
    // output axis b takes the canonical component k with perm_axis(perm, k)
    // = b (selects, so that o stays in registers)
    const int a0 = perm_axis(perm, 0), a1 = perm_axis(perm, 1);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float v = a0 == b ? y[1] : (a1 == b ? y[2] : y[3]);
        const bool neg = ((rb >> b) & 1) != flip;
        o[1 + b] = neg ? -v : v;
    }
}

// (W, G^) of a point -> training targets in its canonical frame.
__device__ __forceinline__ void canon_targets(int code, const float (&o)[4], float (&y)[4]) {
    const bool flip = code & 1;
    const int rb = (code >> 1) & 7, perm = code >> 4;
    y[0] = flip ? __fsub_rn(1.0f, o[0]) : o[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = perm_axis(perm, k);
        const bool neg = ((rb >> a) & 1) != flip;
        y[1 + k] = neg ? -o[1 + a] : o[1 + a];
    }
}

}  // namespace
}  // namespace sg
