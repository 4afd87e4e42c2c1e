// sg_rows.cuh -- per-package face-stencil code shared by the single-grid
// sweeps (sg_sweep.cu, sg_reinit.cu) and the batched persistent sweeps
// (sg_batch.cu), so that both run the same arithmetic per data point and
// agree bit for bit.
//
// Face stencils: a half-warp owns one package and each lane one row of four
// x-values (float4, row r = j + 4k).  x neighbours inside the row are in
// registers; rows j +- 1 and k +- 1 are 16-byte loads of the package's own
// rows (served by L1 once the half-warp has read the package); across a
// package face the neighbour package named by the 27-entry table (Listing 2,
// kept as a 32-byte face row) supplies one value (x faces) or one row (y, z
// faces).
#pragma once
#include "sg_internal.cuh"

namespace sg {

constexpr int ROW_THREADS = 256;
constexpr int ROW_PKGS = ROW_THREADS / 16;  // packages per CTA (a half-warp each)

namespace {


// Listing 2: shift s per axis in [-4, 7] -> (package, data index)
__device__ __forceinline__ int64_t shift_index(const int* nb27, int sx, int sy, int sz) {
    int nx = (sx + PKG) >> 2, ny = (sy + PKG) >> 2, nz = (sz + PKG) >> 2;
    int pkg = nb27[nx + 3 * ny + 9 * nz];
    int dx = sx + PKG - nx * PKG, dy = sy + PKG - ny * PKG, dz = sz + PKG - nz * PKG;
    return (int64_t)pkg * PKG3 + dx + PKG * dy + PKG * PKG * dz;
}


__device__ __forceinline__ float get(const float4& v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ void set(float4& v, int i, float a) {
    if (i == 0) v.x = a;
    else if (i == 1) v.y = a;
    else if (i == 2) v.z = a;
    else v.w = a;
}

// A lane's row and its six neighbours.
struct Rows {
    float4 c;       // own row, i = 0..3
    float xm, xp;   // x - 1 of i = 0 and x + 1 of i = 3
    float4 ym, yp;  // rows j - 1, j + 1
    float4 zm, zp;  // rows k - 1, k + 1
};

// Package of a half-warp and row of a lane.  Offsets are kept in float4
// units in 32 bits: P < 2^31 / 27 packages, so 16 P < 2^31.
struct RowSlot {
    int64_t p;
    int q4;  // float4 index of this lane's row: 16 p + r
    int r;
    bool valid;
};

__device__ __forceinline__ RowSlot make_slot(int64_t p, bool valid) {
    RowSlot s;
    s.r = threadIdx.x & 15;
    s.p = p;
    s.valid = valid;
    s.q4 = (int)p * 16 + s.r;
    return s;
}

// Gather a lane's row and neighbours of field f.  faces[p][8] holds the six
// face neighbours of package p (-x, +x, -y, +y, -z, +z), one 32-byte row
// read by every lane of the half-warp (one broadcast transaction).  Rows
// j +- 1 and k +- 1 are loaded from the package itself (L1 hits: the
// half-warp reads the whole package) or, on its boundary, from the face
// neighbour; each lane also takes one value from the -x and +x packages.
// Lanes of an invalid package get zeros.
// Loads of field values: read-only for the whole kernel (the non-coherent
// path), or written by a grid this kernel was launched to depend on (plain
// loads, visible once the dependency wait has returned).
template <bool Dependent>
__device__ __forceinline__ float4 ld_f4(const float4* p) { return Dependent ? __ldca(p) : __ldg(p); }
template <bool Dependent>
__device__ __forceinline__ float ld_f1(const float* p) { return Dependent ? __ldca(p) : __ldg(p); }

template <bool Dependent>
__device__ __forceinline__ Rows load_rows_t(const float* f, const int32_t* __restrict__ faces, const RowSlot& s) {
    const int j = s.r & 3, k = s.r >> 2;
    const float4* f4 = reinterpret_cast<const float4*>(f);
    Rows w;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!s.valid) {
        w.c = w.ym = w.yp = w.zm = w.zp = zero;
        w.xm = w.xp = 0.f;
        return w;
    }
    const int4 fa = __ldg(reinterpret_cast<const int4*>(faces + s.p * 8));
    const int2 fb = __ldg(reinterpret_cast<const int2*>(faces + s.p * 8 + 4));
    const int q = s.q4;
    w.c = ld_f4<Dependent>(f4 + q);
    w.xm = ld_f1<Dependent>(reinterpret_cast<const float*>(f4 + (fa.x * 16 + s.r)) + 3);
    w.xp = ld_f1<Dependent>(reinterpret_cast<const float*>(f4 + (fa.y * 16 + s.r)));
    w.ym = ld_f4<Dependent>(f4 + (j > 0 ? q - 1 : fa.z * 16 + s.r + 3));
    w.yp = ld_f4<Dependent>(f4 + (j < 3 ? q + 1 : fa.w * 16 + s.r - 3));
    w.zm = ld_f4<Dependent>(f4 + (k > 0 ? q - 4 : fb.x * 16 + s.r + 12));
    w.zp = ld_f4<Dependent>(f4 + (k < 3 ? q + 4 : fb.y * 16 + s.r - 12));
    return w;
}

__device__ __forceinline__ Rows load_rows(const float* __restrict__ f, const int32_t* __restrict__ faces,
                                          const RowSlot& s) {
    return load_rows_t<false>(f, faces, s);
}

__device__ __forceinline__ float row_xm(const Rows& w, int i) { return i > 0 ? get(w.c, i - 1) : w.xm; }
__device__ __forceinline__ float row_xp(const Rows& w, int i) { return i < 3 ? get(w.c, i + 1) : w.xp; }

// Listing 5 with (p + m) / (2h) per axis.
__device__ __forceinline__ void gradient_row(const Rows& w, float inv2h, float4& ox, float4& oy, float4& oz) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = get(w.c, i);
        set(ox, i, ((row_xp(w, i) - c) + (c - row_xm(w, i))) * inv2h);
        set(oy, i, ((get(w.yp, i) - c) + (c - get(w.ym, i))) * inv2h);
        set(oz, i, ((get(w.zp, i) - c) + (c - get(w.zm, i))) * inv2h);
    }
}

__device__ __forceinline__ float4 laplacian_row(const Rows& w, float inv_h2) {
    float4 o;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = get(w.c, i);
        float a = (row_xp(w, i) - 2.0f * c) + row_xm(w, i);
        a += (get(w.yp, i) - 2.0f * c) + get(w.ym, i);
        a += (get(w.zp, i) - 2.0f * c) + get(w.zm, i);
        set(o, i, a * inv_h2);
    }
    return o;
}

// One Godunov sweep.  With sigma = sign(S0) the upwind pair of each axis is
// u = max(sigma (c - phi(-e)), 0) and v = max(sigma (c - phi(+e)), 0): for
// S0 > 0 these are max(D-, 0) h and -min(D+, 0) h, for S0 < 0 -min(D-, 0) h
// and max(D+, 0) h, so max(u^2, v^2) = max(u, v)^2 is the Godunov term of
// that axis times h^2.  Then dt sqrt(G) = cfl sqrt(sum h^2 terms) and
// phi <- phi - S0 (cfl sqrt(.) - dt), which leaves phi unchanged where S0 = 0.
__device__ __forceinline__ float godunov_axis(float cs, float sigma, float m, float p) {
    const float u = fmaf(-sigma, m, cs), v = fmaf(-sigma, p, cs);
    return fmaxf(fmaxf(u, v), 0.0f);
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float4 reinit_row(const Rows& w, const float4& sg, float cfl, float dt) {
    float4 o;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = get(w.c, i), sv = get(sg, i);
        const float sigma = copysignf(1.0f, sv), cs = sigma * c;
        const float mx = godunov_axis(cs, sigma, row_xm(w, i), row_xp(w, i));
        const float my = godunov_axis(cs, sigma, get(w.ym, i), get(w.yp, i));
        const float mz = godunov_axis(cs, sigma, get(w.zm, i), get(w.zp, i));
        const float g2 = fmaf(mx, mx, fmaf(my, my, mz * mz));
        set(o, i, fmaf(-sv, fmaf(cfl, sqrt_approx(g2), -dt), c));
    }
    return o;
}

// Smoothed sign S0 = phi / sqrt(phi^2 + h^2).
__device__ __forceinline__ float smoothed_sign(float v, float h2) { return v / sqrtf(v * v + h2); }

// The slot of this lane in a single-grid launch: CTA b owns packages
// 2 + 16 b .. 2 + 16 b + 15, a half-warp each.
__device__ __forceinline__ RowSlot row_slot(int64_t P) {
    const int64_t p = 2 + (int64_t)blockIdx.x * ROW_PKGS + (threadIdx.x >> 4);
    return make_slot(p, p < P);
}

// The same with the CTAs taken in reverse order when `reverse` is set (CTA
// b owns the packages of CTA gridDim.x - 1 - b): a sweep that follows one
// in the other direction starts on the packages whose data the previous
// sweep touched last, still in L2.
__device__ __forceinline__ RowSlot row_slot_dir(int64_t P, int reverse) {
    const int64_t b = reverse ? (int64_t)gridDim.x - 1 - blockIdx.x : (int64_t)blockIdx.x;
    const int64_t p = 2 + b * ROW_PKGS + (threadIdx.x >> 4);
    return make_slot(p, p < P);
}

inline unsigned row_blocks(int64_t P) { return (unsigned)((P - 2 + ROW_PKGS - 1) / ROW_PKGS); }

}  // namespace
}  // namespace sg
