// sg_sweep.cu -- per-package stencil sweeps over the active packages
// ("MeshPackageDynamics" / package_for, Listing 4): gradient (Listing 5),
// 7-point Laplacian, Godunov reinitialisation step, kernel integrals.
//
// Face stencils (gradient, Laplacian, reinit): a half-warp owns one package
// and each lane one row of four x-values (float4, row r = j + 4k).  x
// neighbours inside the row are in registers; rows j +- 1 and k +- 1 come
// from lanes r -+ 1 and r -+ 4 by warp shuffles; across a package face the
// neighbour package named by the 27-entry table (Listing 2) supplies one
// value (x faces) or one row (y, z faces).  The six face ids are read once
// per package by six lanes and broadcast by shuffles.
//
// Kernel integrals (27 taps, edges and corners included): a CTA of 256
// threads owns 4 packages, stages the smoothed Heaviside of a 6^3 tile
// (package plus a one-point halo, reached by the index shift) in shared
// memory and sums the taps from there.
#include "sg_internal.cuh"

namespace sg {
namespace {

constexpr int SW_THREADS = 256;
constexpr int SW_PKGS = SW_THREADS / PKG3;  // packages per CTA

// neighbourhood entries of the six faces: -x, +x, -y, +y, -z, +z
__constant__ int c_face_n[6] = {12, 14, 10, 16, 4, 22};

// Listing 2: shift s per axis in [-4, 7] -> (package, data index)
__device__ __forceinline__ int64_t shift_index(const int* nb27, int sx, int sy, int sz) {
    int nx = (sx + PKG) >> 2, ny = (sy + PKG) >> 2, nz = (sz + PKG) >> 2;
    int pkg = nb27[nx + 3 * ny + 9 * nz];
    int dx = sx + PKG - nx * PKG, dy = sy + PKG - ny * PKG, dz = sz + PKG - nz * PKG;
    return (int64_t)pkg * PKG3 + dx + PKG * dy + PKG * PKG * dz;
}

__global__ void __launch_bounds__(SW_THREADS) k_set_far(float* f, float v_in, float v_out) {
    f[threadIdx.x] = threadIdx.x < PKG3 ? v_in : v_out;
}

__global__ void __launch_bounds__(SW_THREADS) k_reinit_s0(const float* __restrict__ phi, float* __restrict__ s0,
                                                           int64_t n_act, float h2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x) {
        float v = phi[2 * PKG3 + e];
        s0[2 * PKG3 + e] = v / sqrtf(v * v + h2);
    }
}

// ---------------------------------------------------------------------------
// Row-per-lane face stencils
// ---------------------------------------------------------------------------
constexpr int ROW_THREADS = 256;
constexpr int ROW_PKGS = ROW_THREADS / 16;  // packages per CTA
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float4 shfl_up4(float4 v, int d) {
    v.x = __shfl_up_sync(FULL, v.x, d, 16);
    v.y = __shfl_up_sync(FULL, v.y, d, 16);
    v.z = __shfl_up_sync(FULL, v.z, d, 16);
    v.w = __shfl_up_sync(FULL, v.w, d, 16);
    return v;
}

__device__ __forceinline__ float4 shfl_down4(float4 v, int d) {
    v.x = __shfl_down_sync(FULL, v.x, d, 16);
    v.y = __shfl_down_sync(FULL, v.y, d, 16);
    v.z = __shfl_down_sync(FULL, v.z, d, 16);
    v.w = __shfl_down_sync(FULL, v.w, d, 16);
    return v;
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

// Package of this half-warp and row of this lane.  Offsets are kept in
// float4 units in 32 bits: P < 2^31 / 27 packages, so 16 P < 2^31.
struct RowSlot {
    int64_t p;
    int q4;  // float4 index of this lane's row: 16 p + r
    int r;
    bool valid;
};

__device__ __forceinline__ RowSlot row_slot(int64_t P) {
    RowSlot s;
    s.r = threadIdx.x & 15;
    s.p = 2 + (int64_t)blockIdx.x * ROW_PKGS + (threadIdx.x >> 4);
    s.valid = s.p < P;
    s.q4 = (int)s.p * 16 + s.r;
    return s;
}

// Gather a lane's row and neighbours of field f.  All lanes of the warp must
// call this (shuffles); lanes of a package past the end get zeros.
__device__ __forceinline__ Rows load_rows(const float* __restrict__ f, const int32_t* __restrict__ nbr,
                                          const RowSlot& s) {
    const int lane = threadIdx.x & 31, base = lane & 16;
    const int j = s.r & 3, k = s.r >> 2;
    const float4* __restrict__ f4 = reinterpret_cast<const float4*>(f);
    int nid = 0;
    if (s.valid && s.r < 6) nid = __ldg(nbr + s.p * NB + c_face_n[s.r]);
    Rows w;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    w.c = s.valid ? __ldg(f4 + s.q4) : zero;
    const int n_xm = __shfl_sync(FULL, nid, base + 0), n_xp = __shfl_sync(FULL, nid, base + 1);
    const int n_ym = __shfl_sync(FULL, nid, base + 2), n_yp = __shfl_sync(FULL, nid, base + 3);
    const int n_zm = __shfl_sync(FULL, nid, base + 4), n_zp = __shfl_sync(FULL, nid, base + 5);
    w.xm = s.valid ? __ldg(reinterpret_cast<const float*>(f4 + (n_xm * 16 + s.r)) + 3) : 0.f;
    w.xp = s.valid ? __ldg(reinterpret_cast<const float*>(f4 + (n_xp * 16 + s.r))) : 0.f;
    const float4 ym = shfl_up4(w.c, 1), yp = shfl_down4(w.c, 1);
    const float4 zm = shfl_up4(w.c, 4), zp = shfl_down4(w.c, 4);
    w.ym = j > 0 ? ym : (s.valid ? __ldg(f4 + (n_ym * 16 + s.r + 3)) : zero);
    w.yp = j < 3 ? yp : (s.valid ? __ldg(f4 + (n_yp * 16 + s.r - 3)) : zero);
    w.zm = k > 0 ? zm : (s.valid ? __ldg(f4 + (n_zm * 16 + s.r + 12)) : zero);
    w.zp = k < 3 ? zp : (s.valid ? __ldg(f4 + (n_zp * 16 + s.r - 12)) : zero);
    return w;
}

__device__ __forceinline__ float row_xm(const Rows& w, int i) { return i > 0 ? get(w.c, i - 1) : w.xm; }
__device__ __forceinline__ float row_xp(const Rows& w, int i) { return i < 3 ? get(w.c, i + 1) : w.xp; }

__global__ void __launch_bounds__(ROW_THREADS) k_gradient(const int32_t* __restrict__ nbr, const float* __restrict__ phi,
                                                           float* __restrict__ gx, float* __restrict__ gy,
                                                           float* __restrict__ gz, int64_t P, float inv2h) {
    const RowSlot s = row_slot(P);
    const Rows w = load_rows(phi, nbr, s);
    if (!s.valid) return;
    float4 ox, oy, oz;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = get(w.c, i);
        set(ox, i, ((row_xp(w, i) - c) + (c - row_xm(w, i))) * inv2h);
        set(oy, i, ((get(w.yp, i) - c) + (c - get(w.ym, i))) * inv2h);
        set(oz, i, ((get(w.zp, i) - c) + (c - get(w.zm, i))) * inv2h);
    }
    reinterpret_cast<float4*>(gx)[s.q4] = ox;
    reinterpret_cast<float4*>(gy)[s.q4] = oy;
    reinterpret_cast<float4*>(gz)[s.q4] = oz;
}

__global__ void __launch_bounds__(ROW_THREADS) k_laplacian(const int32_t* __restrict__ nbr,
                                                            const float* __restrict__ phi, float* __restrict__ lap,
                                                            int64_t P, float inv_h2) {
    const RowSlot s = row_slot(P);
    const Rows w = load_rows(phi, nbr, s);
    if (!s.valid) return;
    float4 o;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = get(w.c, i);
        float a = (row_xp(w, i) - 2.0f * c) + row_xm(w, i);
        a += (get(w.yp, i) - 2.0f * c) + get(w.ym, i);
        a += (get(w.zp, i) - 2.0f * c) + get(w.zm, i);
        set(o, i, a * inv_h2);
    }
    reinterpret_cast<float4*>(lap)[s.q4] = o;
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

__global__ void __launch_bounds__(ROW_THREADS) k_reinit_step(const int32_t* __restrict__ nbr,
                                                              const float* __restrict__ s0,
                                                              const float* __restrict__ phi_in,
                                                              float* __restrict__ phi_out, int64_t P, float cfl,
                                                              float dt) {
    const RowSlot s = row_slot(P);
    const float4 sg = s.valid ? __ldg(reinterpret_cast<const float4*>(s0) + s.q4) : make_float4(0.f, 0.f, 0.f, 0.f);
    const Rows w = load_rows(phi_in, nbr, s);
    if (!s.valid) return;
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
    reinterpret_cast<float4*>(phi_out)[s.q4] = o;
}

__global__ void __launch_bounds__(SW_THREADS) k_copy(const float* __restrict__ src, float* __restrict__ dst,
                                                      int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// Kernel integrals.  Tap weights by squared distance |s|^2 in {0,1,2,3}:
// cw = w(|s|) / sum w, ck = w'(|s|) / |s| / sum w (taps at |s| >= 2 vanish).
struct KernelCoef {
    float cw[4];
    float ck[4];
    float inv_eps;
};

__device__ __forceinline__ float heaviside_neg(float phi, float inv_eps) {
    // H(z) at z = -phi with half width eps: 0 below -eps, 1 above eps,
    // 1/2 (1 + z/eps + sin(pi z/eps)/pi) between
    float t = -phi * inv_eps;
    if (t < -1.0f) return 0.0f;
    if (t > 1.0f) return 1.0f;
    return 0.5f * (1.0f + t + sinpif(t) * 0.318309886183790672f);
}

__global__ void __launch_bounds__(SW_THREADS) k_kernel_integrals(const int32_t* __restrict__ nbr,
                                                                  const float* __restrict__ phi, float* __restrict__ W,
                                                                  float* __restrict__ gx, float* __restrict__ gy,
                                                                  float* __restrict__ gz, int64_t P, KernelCoef K) {
    __shared__ int s_nb[SW_PKGS][NB];
    __shared__ float s_H[SW_PKGS][216];  // 6^3 tile: package plus a one-point halo
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t p = 2 + (int64_t)blockIdx.x * SW_PKGS + lp;
    const bool valid = p < P;
    if (valid && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
    __syncthreads();
    if (valid) {
        for (int e = d; e < 216; e += PKG3) {
            int x = e % 6 - 1, y = (e / 6) % 6 - 1, z = e / 36 - 1;
            s_H[lp][e] = heaviside_neg(__ldg(phi + shift_index(s_nb[lp], x, y, z)), K.inv_eps);
        }
    }
    __syncthreads();
    if (!valid) return;
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    const float* H = s_H[lp] + (i + 1) + 6 * (j + 1) + 36 * (k + 1);
    float w = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
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
    const int64_t at = p * PKG3 + d;
    W[at] = w;
    gx[at] = ax;
    gy[at] = ay;
    gz[at] = az;
}

unsigned pkg_blocks(int64_t P) {
    int64_t n = P - 2;
    return (unsigned)((n + SW_PKGS - 1) / SW_PKGS);
}

unsigned row_blocks(int64_t P) {
    int64_t n = P - 2;
    return (unsigned)((n + ROW_PKGS - 1) / ROW_PKGS);
}

unsigned flat_blocks(int64_t n) {
    int64_t b = (n + SW_THREADS - 1) / SW_THREADS;
    if (b < 1) b = 1;
    if (b > 148 * 64) b = 148 * 64;
    return (unsigned)b;
}

double wendland(double q) {
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return t * t * t * t * (1.0 + 2.0 * q);
}

double wendland_dq(double q) {
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * q * t * t * t;
}

}  // namespace

cudaError_t launch_set_far(float* f, float v_in, float v_out, cudaStream_t s) {
    k_set_far<<<1, 2 * PKG3, 0, s>>>(f, v_in, v_out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gradient(const GridF& G, const int32_t* nbr, const float* phi, float* gx, float* gy, float* gz,
                            int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    k_gradient<<<row_blocks(P), ROW_THREADS, 0, s>>>(nbr, phi, gx, gy, gz, P, (float)(1.0 / (2.0 * G.h_d)));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_laplacian(const GridF& G, const int32_t* nbr, const float* phi, float* lap, int64_t P,
                             cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    k_laplacian<<<row_blocks(P), ROW_THREADS, 0, s>>>(nbr, phi, lap, P, (float)(1.0 / (G.h_d * G.h_d)));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_reinit_s0(const GridF& G, const float* phi, float* s0, int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    int64_t n = (P - 2) * PKG3;
    k_reinit_s0<<<flat_blocks(n), SW_THREADS, 0, s>>>(phi, s0, n, (float)(G.h_d * G.h_d));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_reinit_step(const GridF& G, const int32_t* nbr, const float* s0, const float* phi_in,
                               float* phi_out, float dt, int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    // dt sqrt(G) = (dt / h) sqrt(h^2 G) and dt / h is the CFL number
    k_reinit_step<<<row_blocks(P), ROW_THREADS, 0, s>>>(nbr, s0, phi_in, phi_out, P, (float)(dt / G.h_d), dt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_copy_active(const float* src, float* dst, int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    int64_t n = (P - 2) * PKG3;
    k_copy<<<flat_blocks(n), SW_THREADS, 0, s>>>(src + 2 * PKG3, dst + 2 * PKG3, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_kernel_integrals(const GridF& G, const int32_t* nbr, const float* phi, float* W, float* gx,
                                    float* gy, float* gz, int64_t P, cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_set_far(W, 1.0f, 0.0f, s)) != cudaSuccess) return e;
    if ((e = launch_set_far(gx, 0.0f, 0.0f, s)) != cudaSuccess) return e;
    if ((e = launch_set_far(gy, 0.0f, 0.0f, s)) != cudaSuccess) return e;
    if ((e = launch_set_far(gz, 0.0f, 0.0f, s)) != cudaSuccess) return e;
    if (P <= 2) return cudaSuccess;
    KernelCoef K;
    const double q[4] = {0.0, 1.0, 1.4142135623730951, 1.7320508075688772};
    double den = wendland(q[0]) + 6 * wendland(q[1]) + 12 * wendland(q[2]) + 8 * wendland(q[3]);
    for (int c = 0; c < 4; ++c) {
        K.cw[c] = (float)(wendland(q[c]) / den);
        K.ck[c] = c == 0 ? 0.0f : (float)(wendland_dq(q[c]) / q[c] / den);
    }
    K.inv_eps = (float)(1.0 / G.h_d);
    k_kernel_integrals<<<pkg_blocks(P), SW_THREADS, 0, s>>>(nbr, phi, W, gx, gy, gz, P, K);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sg
