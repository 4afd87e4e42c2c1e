// sg_integrals.cuh -- kernel-integral device code shared by the exact
// integrals (sg_sweep.cu), the batched sweeps (sg_batch.cu) and the
// surrogate's staging and fallback (sg_mlp.cu).
//
// Kernel integrals: 64 threads own a package, stage the smoothed Heaviside of
// a 6^3 tile (package plus a one-point halo) in shared memory, one x-row of
// six per thread (four interior points from one package by a 16-byte load,
// the two halo points from the -x and +x packages of the index shift), and
// sum the 27 non-zero taps from there; supports above 2h use 8^3 tiles and
// the 5^3 taps.
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

// A package's 6^3 tile (the package plus a one-point halo) in shared
// memory: rows of 6 along x, planes of 40 (6 x 6 padded), 242 floats per
// package, so that every row starts on an 8-byte boundary.  When 16 threads
// of a package take one row (j, k) each and read 8-byte pairs, a warp's two
// packages are served in two half-warp phases and each phase meets 16
// distinct bank pairs (the rows 6 j + 40 k: 3 j + 20 k pairs, distinct mod
// 16); 6 x 36 x 216 gave 3-way conflicts.
constexpr int TILE_Y = 6;
constexpr int TILE_Z = 40;
constexpr int TILE_N = 242;

namespace {

__device__ __forceinline__ float heaviside_neg(float phi, float inv_eps) {
    // H(z) at z = -phi with half width eps: 0 below -eps, 1 above eps,
    // 1/2 (1 + z/eps + sin(pi z/eps)/pi) between; the sine is the hardware
    // approximation (absolute error about 5e-7 on [-pi, pi], far below the
    // 1e-5 the integrals are held to).  Every operation is an explicitly
    // rounded one, so that all kernels that stage H agree bit for bit.
    const float t = __fmul_rn(-phi, inv_eps);
    if (t < -1.0f) return 0.0f;
    if (t > 1.0f) return 1.0f;
    const float sn = __sinf(__fmul_rn(3.14159265358979323846f, t));
    return __fmul_rn(0.5f, __fmaf_rn(sn, 0.318309886183790672f, __fadd_rn(1.0f, t)));
}

// Stage the package's 6^3 tile (the package plus a one-point halo) by
// x-rows, one row of six per thread d < 36: four interior points from one
// package (a 16-byte load) and the two halo points from the -x and +x
// packages of the index shift (Listing 2).  Writes phi to tphi and the
// smoothed Heaviside to tH (either may be null); returns the saturation
// bits of the H values this thread staged: bit 0 unless all were 0, bit 1
// unless all were 1 (a tile whose bits OR to 1 is all ones, to 2 all zeros).
// The tiles (8-byte aligned, TILE_N floats apart) take the row as three pairs.
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
        const int e0 = TILE_Y * (y + 1) + TILE_Z * (z + 1);  // even: rows start on 8-byte boundaries
        const float f[6] = {vm, v.x, v.y, v.z, v.w, vp};
#pragma unroll
        for (int i = 0; i < 6; i += 2) {
            if (tphi) *reinterpret_cast<float2*>(tphi + e0 + i) = make_float2(f[i], f[i + 1]);
            if (tH) {
                const float h0 = heaviside_neg(f[i], inv_eps), h1 = heaviside_neg(f[i + 1], inv_eps);
                *reinterpret_cast<float2*>(tH + e0 + i) = make_float2(h0, h1);
                bits |= (h0 != 0.0f ? 1u : 0u) | (h0 != 1.0f ? 2u : 0u) | (h1 != 0.0f ? 1u : 0u) | (h1 != 1.0f ? 2u : 0u);
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

// A saturated tile (every H in it 0, or every H 1) gives W = that value and
// G = 0 exactly (the normalised weights sum to one): the taps are skipped.
__device__ __forceinline__ bool integrals_saturated(unsigned tile_bits, float& w, float& ax, float& ay, float& az) {
    if (tile_bits == 3u) return false;
    w = tile_bits == 1u ? 1.0f : 0.0f;
    ax = ay = az = 0.0f;
    return true;
}

// The 27 taps of data point d, summed plane by plane (sz = -1, 0, 1).  In a
// plane each row sy holds the centre tap h0 and the pair x -+ 1, taken as
// its sum a and difference b (x - 1 minus x + 1); with the weights grouped
// by |s|^2 = sz^2 + sy^2 + sx^2:
//   W  += cw[s2] h0(0) + cw[s2+1] (a(0) + h0(-1) + h0(+1)) + cw[s2+2] (a(-1) + a(+1))
//   Gx += ck[s2+1] b(0) + ck[s2+2] (b(-1) + b(+1))
//   Gy += ck[s2+1] (h0(-1) - h0(+1)) + ck[s2+2] (a(-1) - a(+1))
//   Gz -= sz (ck[s2] h0(0) + ck[s2+1] (a(0) + h0(-1) + h0(+1)) + ck[s2+2] (a(-1) + a(+1)))
// with s2 = sz^2: the same sums as tap by tap (G = sum of ck(|s|^2) (-s) H),
// in about half the operations.
__device__ __forceinline__ void integrals_point(const float* tile, int d, const KernelCoef& K, float& w,
                                                float& ax, float& ay, float& az) {
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    const float* H = tile + (i + 1) + TILE_Y * (j + 1) + TILE_Z * (k + 1);
    w = 0.0f;
    ax = ay = az = 0.0f;
#pragma unroll
    for (int sz = -1; sz <= 1; ++sz) {
        const int s2 = sz * sz;
        float h0[3], a[3], b[3];
#pragma unroll
        for (int sy = -1; sy <= 1; ++sy) {
            const float* row = H + TILE_Y * sy + TILE_Z * sz;
            const float m = row[-1], p = row[1];
            h0[sy + 1] = row[0];
            a[sy + 1] = m + p;
            b[sy + 1] = m - p;
        }
        const float t = a[1] + (h0[0] + h0[2]), sa = a[0] + a[2];
        w = fmaf(K.cw[s2], h0[1], w);
        w = fmaf(K.cw[s2 + 1], t, w);
        w = fmaf(K.cw[s2 + 2], sa, w);
        ax = fmaf(K.ck[s2 + 1], b[1], ax);
        ax = fmaf(K.ck[s2 + 2], b[0] + b[2], ax);
        ay = fmaf(K.ck[s2 + 1], h0[0] - h0[2], ay);
        ay = fmaf(K.ck[s2 + 2], a[0] - a[2], ay);
        if (sz != 0) {
            const float kz = fmaf(K.ck[s2 + 2], sa, fmaf(K.ck[s2 + 1], t, K.ck[s2] * h0[1]));
            az = sz < 0 ? az + kz : az - kz;
        }
    }
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// Points d and d + 1 (x-neighbours of one package row) at once: the sums of
// integrals_point, operation for operation, on pairs of floats (each lane of
// a paired instruction is the same rounded operation), so both points come
// out bit for bit as integrals_point gives them.
__device__ __forceinline__ void integrals_point2(const float* tile, int d, const KernelCoef& K, float2& w, float2& ax,
                                                 float2& ay, float2& az) {
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    const float* H = tile + (i + 1) + TILE_Y * (j + 1) + TILE_Z * (k + 1);
    w = ax = ay = az = f2(0.0f);
#pragma unroll
    for (int sz = -1; sz <= 1; ++sz) {
        const int s2 = sz * sz;
        float2 h0[3], a[3], b[3];
#pragma unroll
        for (int sy = -1; sy <= 1; ++sy) {
            const float* row = H + TILE_Y * sy + TILE_Z * sz;  // row - 1 is 8-byte aligned (d even)
            const float2 m = *reinterpret_cast<const float2*>(row - 1), p = *reinterpret_cast<const float2*>(row + 1);
            h0[sy + 1] = make_float2(m.y, p.x);
            a[sy + 1] = __fadd2_rn(m, p);
            b[sy + 1] = __fadd2_rn(m, neg2(p));
        }
        const float2 t = __fadd2_rn(a[1], __fadd2_rn(h0[0], h0[2])), sa = __fadd2_rn(a[0], a[2]);
        w = __ffma2_rn(f2(K.cw[s2]), h0[1], w);
        w = __ffma2_rn(f2(K.cw[s2 + 1]), t, w);
        w = __ffma2_rn(f2(K.cw[s2 + 2]), sa, w);
        ax = __ffma2_rn(f2(K.ck[s2 + 1]), b[1], ax);
        ax = __ffma2_rn(f2(K.ck[s2 + 2]), __fadd2_rn(b[0], b[2]), ax);
        ay = __ffma2_rn(f2(K.ck[s2 + 1]), __fadd2_rn(h0[0], neg2(h0[2])), ay);
        ay = __ffma2_rn(f2(K.ck[s2 + 2]), __fadd2_rn(a[0], neg2(a[2])), ay);
        if (sz != 0) {
            const float2 kz = __ffma2_rn(f2(K.ck[s2 + 2]), sa,
                                         __ffma2_rn(f2(K.ck[s2 + 1]), t, __fmul2_rn(f2(K.ck[s2]), h0[1])));
            az = sz < 0 ? __fadd2_rn(az, kz) : __fadd2_rn(az, neg2(kz));
        }
    }
}

}  // namespace
}  // namespace sg
