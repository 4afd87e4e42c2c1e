// sg_sweep.cu -- per-package stencil sweeps over the active packages
// ("MeshPackageDynamics" / package_for, Listing 4): gradient (Listing 5),
// 7-point Laplacian, Godunov reinitialisation step, kernel integrals.
//
// Layout: a CTA of 256 threads owns 4 consecutive packages, one thread per
// data point (d = i + 4j + 16k).  The CTA stages its own packages in shared
// memory; values across a package face come from the neighbour package
// named by the 27-entry table through the index shift of Listing 2.
// Packages are numbered in cell order, so a CTA's face neighbours along x
// are usually its own packages and the rest sit in L2.
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

struct Nbr6 {
    float xm, xp, ym, yp, zm, zp;
};

// The six face neighbours of data point d of a package whose own values are
// staged in s (64 floats) and whose face neighbour packages are nb6.
__device__ __forceinline__ Nbr6 face_values(const float* s, const int* nb6, const float* __restrict__ f, int d) {
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    Nbr6 r;
    r.xm = i > 0 ? s[d - 1] : __ldg(f + (int64_t)nb6[0] * PKG3 + d + 3);
    r.xp = i < 3 ? s[d + 1] : __ldg(f + (int64_t)nb6[1] * PKG3 + d - 3);
    r.ym = j > 0 ? s[d - 4] : __ldg(f + (int64_t)nb6[2] * PKG3 + d + 12);
    r.yp = j < 3 ? s[d + 4] : __ldg(f + (int64_t)nb6[3] * PKG3 + d - 12);
    r.zm = k > 0 ? s[d - 16] : __ldg(f + (int64_t)nb6[4] * PKG3 + d + 48);
    r.zp = k < 3 ? s[d + 16] : __ldg(f + (int64_t)nb6[5] * PKG3 + d - 48);
    return r;
}

// Stage the CTA's packages of field f and their face neighbour ids.
// Returns the package id of this thread (>= P when past the end).
__device__ __forceinline__ int64_t stage_faces(const float* __restrict__ f, const int32_t* __restrict__ nbr, int64_t P,
                                               float (*s_f)[PKG3], int (*s_nb)[6], float& own) {
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t p = 2 + (int64_t)blockIdx.x * SW_PKGS + lp;
    own = 0.0f;
    if (p < P) {
        own = __ldg(f + p * PKG3 + d);
        if (d < 6) s_nb[lp][d] = __ldg(nbr + p * NB + c_face_n[d]);
    }
    s_f[lp][d] = own;
    __syncthreads();
    return p;
}

__global__ void __launch_bounds__(SW_THREADS) k_set_far(float* f, float v_in, float v_out) {
    f[threadIdx.x] = threadIdx.x < PKG3 ? v_in : v_out;
}

__global__ void __launch_bounds__(SW_THREADS) k_gradient(const int32_t* __restrict__ nbr, const float* __restrict__ phi,
                                                          float* __restrict__ gx, float* __restrict__ gy,
                                                          float* __restrict__ gz, int64_t P, float inv2h) {
    __shared__ float s_f[SW_PKGS][PKG3];
    __shared__ int s_nb[SW_PKGS][6];
    float c;
    const int64_t p = stage_faces(phi, nbr, P, s_f, s_nb, c);
    if (p >= P) return;
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    Nbr6 n = face_values(s_f[lp], s_nb[lp], phi, d);
    const int64_t at = p * PKG3 + d;
    gx[at] = ((n.xp - c) + (c - n.xm)) * inv2h;
    gy[at] = ((n.yp - c) + (c - n.ym)) * inv2h;
    gz[at] = ((n.zp - c) + (c - n.zm)) * inv2h;
}

__global__ void __launch_bounds__(SW_THREADS) k_laplacian(const int32_t* __restrict__ nbr, const float* __restrict__ phi,
                                                           float* __restrict__ lap, int64_t P, float inv_h2) {
    __shared__ float s_f[SW_PKGS][PKG3];
    __shared__ int s_nb[SW_PKGS][6];
    float c;
    const int64_t p = stage_faces(phi, nbr, P, s_f, s_nb, c);
    if (p >= P) return;
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    Nbr6 n = face_values(s_f[lp], s_nb[lp], phi, d);
    float s = ((n.xp - 2.0f * c) + n.xm);
    s += ((n.yp - 2.0f * c) + n.ym);
    s += ((n.zp - 2.0f * c) + n.zm);
    lap[p * PKG3 + d] = s * inv_h2;
}

__global__ void __launch_bounds__(SW_THREADS) k_reinit_s0(const float* __restrict__ phi, float* __restrict__ s0,
                                                           int64_t n_act, float h2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x) {
        float v = phi[2 * PKG3 + e];
        s0[2 * PKG3 + e] = v / sqrtf(v * v + h2);
    }
}

// One Godunov component: the upwind pair (u, v) chosen by the sign of S0.
__device__ __forceinline__ float godunov_term(float a, float b, bool pos) {
    float u = pos ? fmaxf(a, 0.0f) : fminf(a, 0.0f);
    float v = pos ? fminf(b, 0.0f) : fmaxf(b, 0.0f);
    return fmaxf(u * u, v * v);
}

__global__ void __launch_bounds__(SW_THREADS) k_reinit_step(const int32_t* __restrict__ nbr, const float* __restrict__ s0,
                                                             const float* __restrict__ phi_in,
                                                             float* __restrict__ phi_out, int64_t P, float inv_h,
                                                             float dt) {
    __shared__ float s_f[SW_PKGS][PKG3];
    __shared__ int s_nb[SW_PKGS][6];
    float c;
    const int64_t p = stage_faces(phi_in, nbr, P, s_f, s_nb, c);
    if (p >= P) return;
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t at = p * PKG3 + d;
    const float s = __ldg(s0 + at);
    Nbr6 n = face_values(s_f[lp], s_nb[lp], phi_in, d);
    const bool pos = s > 0.0f;
    float G = godunov_term((c - n.xm) * inv_h, (n.xp - c) * inv_h, pos);
    G += godunov_term((c - n.ym) * inv_h, (n.yp - c) * inv_h, pos);
    G += godunov_term((c - n.zm) * inv_h, (n.zp - c) * inv_h, pos);
    phi_out[at] = s == 0.0f ? c : c - dt * s * (sqrtf(G) - 1.0f);
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
    k_gradient<<<pkg_blocks(P), SW_THREADS, 0, s>>>(nbr, phi, gx, gy, gz, P, (float)(1.0 / (2.0 * G.h_d)));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_laplacian(const GridF& G, const int32_t* nbr, const float* phi, float* lap, int64_t P,
                             cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    k_laplacian<<<pkg_blocks(P), SW_THREADS, 0, s>>>(nbr, phi, lap, P, (float)(1.0 / (G.h_d * G.h_d)));
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
    k_reinit_step<<<pkg_blocks(P), SW_THREADS, 0, s>>>(nbr, s0, phi_in, phi_out, P, (float)(1.0 / G.h_d), dt);
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
