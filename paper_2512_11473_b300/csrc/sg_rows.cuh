// sg_rows.cuh -- per-package device code shared by the single-grid sweeps
// (sg_sweep.cu) and the batched persistent sweeps (sg_batch.cu), so that both
// run the same arithmetic per data point and agree bit for bit.
//
// Face stencils: a half-warp owns one package and each lane one row of four
// x-values (float4, row r = j + 4k).  x neighbours inside the row are in
// registers; rows j +- 1 and k +- 1 are 16-byte loads of the package's own
// rows (served by L1 once the half-warp has read the package); across a
// package face the neighbour package named by the 27-entry table (Listing 2,
// kept as a 32-byte face row) supplies one value (x faces) or one row (y, z
// faces).
//
// Kernel integrals: 64 threads own a package, stage the smoothed Heaviside of
// a 6^3 tile (package plus a one-point halo) in shared memory, one x-row of
// six per thread (four interior points from one package by a 16-byte load,
// the two halo points from the -x and +x packages of the index shift), and
// sum the 27 non-zero taps from there.
#pragma once
#include "sg_internal.cuh"

namespace sg {

// Kernel integrals.  Tap weights by squared distance |s|^2 in {0..12} (the
// 5^3 stencil): cw = w(|s|) / sum w, ck = w'(|s|) / |s| / sum w, for the
// Wendland C2 of support R h, w(q) = (1 - q/R)^4 (1 + 4q/R) (0 at q >= R).
struct KernelCoef {
    float cw[13];
    float ck[13];
};

// host: the tap coefficients for support R h (R <= 3), normalised by the
// discrete sum of the taps
KernelCoef kernel_coef(double R = 2.0);

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
__device__ __forceinline__ Rows load_rows(const float* __restrict__ f, const int32_t* __restrict__ faces,
                                          const RowSlot& s) {
    const int j = s.r & 3, k = s.r >> 2;
    const float4* __restrict__ f4 = reinterpret_cast<const float4*>(f);
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
    w.c = __ldg(f4 + q);
    w.xm = __ldg(reinterpret_cast<const float*>(f4 + (fa.x * 16 + s.r)) + 3);
    w.xp = __ldg(reinterpret_cast<const float*>(f4 + (fa.y * 16 + s.r)));
    w.ym = __ldg(f4 + (j > 0 ? q - 1 : fa.z * 16 + s.r + 3));
    w.yp = __ldg(f4 + (j < 3 ? q + 1 : fa.w * 16 + s.r - 3));
    w.zm = __ldg(f4 + (k > 0 ? q - 4 : fb.x * 16 + s.r + 12));
    w.zp = __ldg(f4 + (k < 3 ? q + 4 : fb.y * 16 + s.r - 12));
    return w;
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

__device__ __forceinline__ float heaviside_neg(float phi, float inv_eps) {
    // H(z) at z = -phi with half width eps: 0 below -eps, 1 above eps,
    // 1/2 (1 + z/eps + sin(pi z/eps)/pi) between; the sine is the hardware
    // approximation (absolute error about 5e-7 on [-pi, pi], far below the
    // 1e-5 the integrals are held to)
    float t = -phi * inv_eps;
    if (t < -1.0f) return 0.0f;
    if (t > 1.0f) return 1.0f;
    return 0.5f * (1.0f + t + __sinf(3.14159265358979323846f * t) * 0.318309886183790672f);
}

// Fill the 6^3 Heaviside tile of package p (64 threads, d = thread index in
// the package); nb27 holds the package's neighbourhood in shared memory.
// Stage the package's 6^3 tile (the package plus a one-point halo) by
// x-rows, one row of six per thread d < 36: four interior points from one
// package (a 16-byte load) and the two halo points from the -x and +x
// packages of the index shift (Listing 2).  Writes phi to tphi and the
// smoothed Heaviside to tH (either may be null); returns the saturation
// bits of the H values this thread staged: bit 0 unless all were 0, bit 1
// unless all were 1 (a tile whose bits OR to 1 is all ones, to 2 all zeros).
__device__ __forceinline__ unsigned stage_rows(const int* nb27, const float* __restrict__ phi, float inv_eps, int d,
                                               float* tphi, float* tH) {
    unsigned bits = 0;
    if (d < 36) {
        const int y = d % 6 - 1, z = d / 6 - 1;
        const int oy = ((y + 4) >> 2) - 1, oz = ((z + 4) >> 2) - 1;
        const int d0 = 4 * (y - 4 * oy) + 16 * (z - 4 * oz);
        const int nb = 3 * (oy + 1) + 9 * (oz + 1);
        const float4 v = __ldg(reinterpret_cast<const float4*>(phi + (int64_t)nb27[nb + 1] * PKG3 + d0));
        const float vm = __ldg(phi + (int64_t)nb27[nb] * PKG3 + d0 + 3);
        const float vp = __ldg(phi + (int64_t)nb27[nb + 2] * PKG3 + d0);
        const int e0 = 6 * (y + 1) + 36 * (z + 1);
        const float f[6] = {vm, v.x, v.y, v.z, v.w, vp};
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (tphi) tphi[e0 + i] = f[i];
            if (tH) {
                const float hv = heaviside_neg(f[i], inv_eps);
                tH[e0 + i] = hv;
                bits |= (hv != 0.0f ? 1u : 0u) | (hv != 1.0f ? 2u : 0u);
            }
        }
    }
    return bits;
}

// Supports above 2h reach two points: the package's 8^3 tile (a two-point
// halo) is staged by x-rows, one per thread (64 rows of eight: four interior
// points by a 16-byte load, two from the -x and two from the +x package by
// 8-byte loads).  Returns saturation bits as stage_rows.
__device__ __forceinline__ unsigned stage_rows_wide(const int* nb27, const float* __restrict__ phi, float inv_eps,
                                                    int d, float* tH) {
    const int y = d % 8 - 2, z = d / 8 - 2;
    const int oy = ((y + 4) >> 2) - 1, oz = ((z + 4) >> 2) - 1;
    const int d0 = 4 * (y - 4 * oy) + 16 * (z - 4 * oz);
    const int nb = 3 * (oy + 1) + 9 * (oz + 1);
    const float2 m = __ldg(reinterpret_cast<const float2*>(phi + (int64_t)nb27[nb] * PKG3 + d0 + 2));
    const float4 v = __ldg(reinterpret_cast<const float4*>(phi + (int64_t)nb27[nb + 1] * PKG3 + d0));
    const float2 pp = __ldg(reinterpret_cast<const float2*>(phi + (int64_t)nb27[nb + 2] * PKG3 + d0));
    const float f[8] = {m.x, m.y, v.x, v.y, v.z, v.w, pp.x, pp.y};
    float* t = tH + 8 * (y + 2) + 64 * (z + 2);
    unsigned bits = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float hv = heaviside_neg(f[i], inv_eps);
        t[i] = hv;
        bits |= (hv != 0.0f ? 1u : 0u) | (hv != 1.0f ? 2u : 0u);
    }
    return bits;
}

// The 5^3 tap sums of data point d from an 8^3 tile (taps with |s|^2 >= 9
// carry no weight for supports up to 3h).
__device__ __forceinline__ void integrals_point_wide(const float* tile, int d, const KernelCoef& K, float& w,
                                                     float& ax, float& ay, float& az) {
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    const float* H = tile + (i + 2) + 8 * (j + 2) + 64 * (k + 2);
    w = 0.0f;
    ax = ay = az = 0.0f;
#pragma unroll
    for (int sz = -2; sz <= 2; ++sz)
#pragma unroll
        for (int sy = -2; sy <= 2; ++sy)
#pragma unroll
            for (int sx = -2; sx <= 2; ++sx) {
                const int q2 = sx * sx + sy * sy + sz * sz;
                if (q2 >= 9) continue;
                const float h = H[sx + 8 * sy + 64 * sz];
                w = fmaf(K.cw[q2], h, w);
                if (q2 > 0) {
                    const float kh = K.ck[q2] * h;
                    if (sx) ax = fmaf(kh, (float)(-sx), ax);
                    if (sy) ay = fmaf(kh, (float)(-sy), ay);
                    if (sz) az = fmaf(kh, (float)(-sz), az);
                }
            }
}

// The Heaviside tile of the kernel integrals (see stage_rows).
__device__ __forceinline__ unsigned integrals_stage(const int* nb27, const float* __restrict__ phi, float inv_eps,
                                                    int d, float* tile) {
    return stage_rows(nb27, phi, inv_eps, d, nullptr, tile);
}

// The 27 taps around data point d of a staged tile.
// A saturated tile (every H in it 0, or every H 1) gives W = that value and
// G = 0 exactly (the normalised weights sum to one): the taps are skipped.
__device__ __forceinline__ bool integrals_saturated(unsigned tile_bits, float& w, float& ax, float& ay, float& az) {
    if (tile_bits == 3u) return false;
    w = tile_bits == 1u ? 1.0f : 0.0f;
    ax = ay = az = 0.0f;
    return true;
}

__device__ __forceinline__ void integrals_point(const float* tile, int d, const KernelCoef& K, float& w,
                                                float& ax, float& ay, float& az) {
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    const float* H = tile + (i + 1) + 6 * (j + 1) + 36 * (k + 1);
    w = 0.0f;
    ax = ay = az = 0.0f;
#pragma unroll
    for (int sz = -1; sz <= 1; ++sz)
#pragma unroll
        for (int sy = -1; sy <= 1; ++sy)
#pragma unroll
            for (int sx = -1; sx <= 1; ++sx) {
                const int q2 = sx * sx + sy * sy + sz * sz;
                const float h = H[sx + 6 * sy + 36 * sz];
                w = fmaf(K.cw[q2], h, w);
                if (q2 > 0) {
                    const float kh = K.ck[q2] * h;
                    if (sx) ax = fmaf(kh, (float)(-sx), ax);
                    if (sy) ay = fmaf(kh, (float)(-sy), ay);
                    if (sz) az = fmaf(kh, (float)(-sz), az);
                }
            }
}

}  // namespace
}  // namespace sg
