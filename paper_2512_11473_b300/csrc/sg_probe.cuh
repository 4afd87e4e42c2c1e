// sg_probe.cuh -- per-particle probe arithmetic ("Grid-Particle Coupling"),
// shared by the single-grid probe (sg_probe.cu) and the batched relaxation
// (sg_batch.cu) so that both locate and interpolate identically.
#pragma once
#include "sg_internal.cuh"

namespace sg {
namespace {

// Fine lattice coordinate u = (x - lo)/h - 1/2 = x (1/h) - (lo/h + 1/2) in
// float-float, about 44 significant bits: ih = 1/h and c = lo/h + 1/2 are
// float-float constants, x ih.hi is formed exactly (TwoProduct) and c.hi is
// subtracted exactly (TwoSum).  i0 = floor(u) then agrees with the exact
// decision unless u lies within about 1e-10 of an integer, and t = u - i0
// is correct to float rounding.  i0 is clamped to +-2^24 (t = 0 there:
// the particle is far outside any domain).
__device__ __forceinline__ void lattice(float x, const ff& c, const ff& ih, int& i0, float& t) {
    const ff p = two_prod(x, ih.hi);
    const ff s = two_sum(p.hi, -c.hi);
    const float e = __fadd_rn(__fadd_rn(s.lo, p.lo), __fsub_rn(__fmul_rn(x, ih.lo), c.lo));
    const ff u = two_sum(s.hi, e);
    float f = floorf(u.hi);
    if (f == u.hi && u.lo < 0.0f) f = __fsub_rn(f, 1.0f);  // an integer hi with the rest below it
    float tt = __fadd_rn(__fsub_rn(u.hi, f), u.lo);       // u.hi - f is exact
    if (!(fabsf(f) < 16777216.0f)) {
        f = fminf(fmaxf(f, -16777216.0f), 16777216.0f);
        tt = 0.0f;
    }
    i0 = (int)f;
    t = tt;
}

// Where a particle sits: home package (the package of its home coarse cell
// I = floor(i0 / 4), or `outside` when I leaves the domain), the local index
// l = i0 - 4 I of the lower interpolation corner and the weights t.
struct ProbeAt {
    int64_t home;
    int l[3];
    float t[3];
};

__device__ __forceinline__ ProbeAt probe_locate(const ff (&lat_c)[3], const ff& lat_ih, const int (&dims)[3],
                                                const int32_t* __restrict__ cell_pkg, int64_t outside,
                                                const float (&pos)[3]) {
    ProbeAt A;
    int i0[3];
    bool inside = true;
    int64_t c = 0, stride = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lattice(pos[a], lat_c[a], lat_ih, i0[a], A.t[a]);
        int I = i0[a] >> 2;  // floor division by 4
        A.l[a] = i0[a] & 3;
        inside &= I >= 0 && I < dims[a];
        c += (int64_t)I * stride;
        stride *= dims[a];
    }
    A.home = inside ? (int64_t)__ldg(cell_pkg + c) : outside;
    return A;
}

// Trilinear interpolation of the first NF probe fields (phi, gx, gy, gz, W,
// Gx, Gy, Gz) from the 8 corners, reached from the home package by the
// index shift.  Per axis the lower corner l lies in the home package's
// column and the upper one, l + 1, in the next package when l = 3, so a
// corner's neighbourhood slot is 13 + (up_x + 3 up_y + 9 up_z) and the home
// package itself needs no table read.
template <int NF>
__device__ __forceinline__ void probe_interp(const int32_t* __restrict__ nbr, const ProbeFields& F, const ProbeAt& A,
                                             float (&acc)[8]) {
    const int32_t* nb = nbr + A.home * NB;
    int up[3], lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        up[a] = A.l[a] == 3 ? 1 : 0;
        lo[a] = A.l[a];
        hi[a] = up[a] ? 0 : A.l[a] + 1;
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) acc[f] = 0.0f;
#pragma unroll
    for (int cr = 0; cr < 8; ++cr) {
        const int a0 = cr & 1, a1 = (cr >> 1) & 1, a2 = (cr >> 2) & 1;
        const float w = (a0 ? A.t[0] : 1.0f - A.t[0]) * (a1 ? A.t[1] : 1.0f - A.t[1]) * (a2 ? A.t[2] : 1.0f - A.t[2]);
        const int slot = (a0 ? up[0] : 0) + 3 * (a1 ? up[1] : 0) + 9 * (a2 ? up[2] : 0);
        const int64_t pkg = slot == 0 ? A.home : (int64_t)__ldg(nb + 13 + slot);
        const int64_t at =
            pkg * PKG3 + ((a0 ? hi[0] : lo[0]) + PKG * (a1 ? hi[1] : lo[1]) + PKG * PKG * (a2 ? hi[2] : lo[2]));
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = fmaf(w, __ldg(F.f[f] + at), acc[f]);
    }
}

// probe_interp with 32-bit byte offsets (for stores of fewer than 2^24
// packages): a corner's offset is formed once and each field's load adds it
// to that field's base address, without 64-bit address arithmetic per load.
// Same sums in the same order.
template <int NF>
__device__ __forceinline__ void probe_interp32(const int32_t* __restrict__ nbr, const ProbeFields& F, const ProbeAt& A,
                                               float (&acc)[8]) {
    const int32_t* nb = nbr + A.home * NB;
    const uint32_t home = (uint32_t)A.home;
    int up[3], lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        up[a] = A.l[a] == 3 ? 1 : 0;
        lo[a] = A.l[a];
        hi[a] = up[a] ? 0 : A.l[a] + 1;
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) acc[f] = 0.0f;
#pragma unroll
    for (int cr = 0; cr < 8; ++cr) {
        const int a0 = cr & 1, a1 = (cr >> 1) & 1, a2 = (cr >> 2) & 1;
        const float w = (a0 ? A.t[0] : 1.0f - A.t[0]) * (a1 ? A.t[1] : 1.0f - A.t[1]) * (a2 ? A.t[2] : 1.0f - A.t[2]);
        const int slot = (a0 ? up[0] : 0) + 3 * (a1 ? up[1] : 0) + 9 * (a2 ? up[2] : 0);
        const uint32_t pkg = slot == 0 ? home : (uint32_t)__ldg(nb + 13 + slot);
        const uint32_t off =
            4u * (pkg * PKG3 + (uint32_t)((a0 ? hi[0] : lo[0]) + PKG * (a1 ? hi[1] : lo[1]) + PKG * PKG * (a2 ? hi[2] : lo[2])));
#pragma unroll
        for (int f = 0; f < NF; ++f)
            acc[f] = fmaf(w, __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(F.f[f]) + off)), acc[f]);
    }
}

// The same interpolation from the point-interleaved probe table: data
// point d of package p holds (phi, gx, gy, gz) in tab[64 p + d] and
// (W, Gx, Gy, Gz) in tab[half + 64 p + d] (half = 64 P), so a corner's first
// four fields come in one 16-byte load and the other four in a second.
// Same sums in the same order as probe_interp.
template <int NF>
__device__ __forceinline__ void probe_interp_quad(const int32_t* __restrict__ nbr, const float4* __restrict__ tab,
                                                  int64_t half, const ProbeAt& A, float (&acc)[8]) {
    static_assert(NF == 4 || NF == 8, "four or eight fields");
    const int32_t* nb = nbr + A.home * NB;
    int up[3], lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        up[a] = A.l[a] == 3 ? 1 : 0;
        lo[a] = A.l[a];
        hi[a] = up[a] ? 0 : A.l[a] + 1;
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) acc[f] = 0.0f;
#pragma unroll
    for (int cr = 0; cr < 8; ++cr) {
        const int a0 = cr & 1, a1 = (cr >> 1) & 1, a2 = (cr >> 2) & 1;
        const float w = (a0 ? A.t[0] : 1.0f - A.t[0]) * (a1 ? A.t[1] : 1.0f - A.t[1]) * (a2 ? A.t[2] : 1.0f - A.t[2]);
        const int slot = (a0 ? up[0] : 0) + 3 * (a1 ? up[1] : 0) + 9 * (a2 ? up[2] : 0);
        const int64_t pkg = slot == 0 ? A.home : (int64_t)__ldg(nb + 13 + slot);
        const float4* q = tab + pkg * PKG3 + (a0 ? hi[0] : lo[0]) + PKG * (a1 ? hi[1] : lo[1]) +
                          PKG * PKG * (a2 ? hi[2] : lo[2]);
        const float4 v = __ldg(q);
        acc[0] = fmaf(w, v.x, acc[0]);
        acc[1] = fmaf(w, v.y, acc[1]);
        acc[2] = fmaf(w, v.z, acc[2]);
        acc[3] = fmaf(w, v.w, acc[3]);
        if (NF == 8) {
            const float4 u = __ldg(q + half);
            acc[4] = fmaf(w, u.x, acc[4]);
            acc[5] = fmaf(w, u.y, acc[5]);
            acc[6] = fmaf(w, u.z, acc[6]);
            acc[7] = fmaf(w, u.w, acc[7]);
        }
    }
}

// probe_interp_quad with 32-bit byte offsets into the table (tables of fewer
// than 2^21 packages; half_bytes = 16 half).  Same sums in the same order.
template <int NF>
__device__ __forceinline__ void probe_interp_quad32(const int32_t* __restrict__ nbr, const float4* __restrict__ tab,
                                                    uint32_t half_bytes, const ProbeAt& A, float (&acc)[8]) {
    static_assert(NF == 4 || NF == 8, "four or eight fields");
    const int32_t* nb = nbr + A.home * NB;
    const uint32_t home = (uint32_t)A.home;
    int up[3], lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        up[a] = A.l[a] == 3 ? 1 : 0;
        lo[a] = A.l[a];
        hi[a] = up[a] ? 0 : A.l[a] + 1;
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) acc[f] = 0.0f;
#pragma unroll
    for (int cr = 0; cr < 8; ++cr) {
        const int a0 = cr & 1, a1 = (cr >> 1) & 1, a2 = (cr >> 2) & 1;
        const float w = (a0 ? A.t[0] : 1.0f - A.t[0]) * (a1 ? A.t[1] : 1.0f - A.t[1]) * (a2 ? A.t[2] : 1.0f - A.t[2]);
        const int slot = (a0 ? up[0] : 0) + 3 * (a1 ? up[1] : 0) + 9 * (a2 ? up[2] : 0);
        const uint32_t pkg = slot == 0 ? home : (uint32_t)__ldg(nb + 13 + slot);
        const uint32_t off = 16u * (pkg * PKG3 + (uint32_t)((a0 ? hi[0] : lo[0]) + PKG * (a1 ? hi[1] : lo[1]) +
                                                            PKG * PKG * (a2 ? hi[2] : lo[2])));
        const char* base = reinterpret_cast<const char*>(tab);
        const float4 v = __ldg(reinterpret_cast<const float4*>(base + off));
        acc[0] = fmaf(w, v.x, acc[0]);
        acc[1] = fmaf(w, v.y, acc[1]);
        acc[2] = fmaf(w, v.z, acc[2]);
        acc[3] = fmaf(w, v.w, acc[3]);
        if (NF == 8) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(base + (off + half_bytes)));
            acc[4] = fmaf(w, u.x, acc[4]);
            acc[5] = fmaf(w, u.y, acc[5]);
            acc[6] = fmaf(w, u.z, acc[6]);
            acc[7] = fmaf(w, u.w, acc[7]);
        }
    }
}

// n = g / |g|, or 0 where |g| = 0
__device__ __forceinline__ float probe_inv_norm(const float (&acc)[8]) {
    const float gn = sqrtf(acc[1] * acc[1] + acc[2] * acc[2] + acc[3] * acc[3]);
    return gn > 0.0f ? 1.0f / gn : 0.0f;
}

}  // namespace
}  // namespace sg
