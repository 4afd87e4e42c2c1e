// sg_sweep.cu -- per-package stencil sweeps over the active packages of one
// grid ("MeshPackageDynamics" / package_for, Listing 4): gradient
// (Listing 5), 7-point Laplacian, the sequential update, kernel integrals.
// The per-package arithmetic lives in sg_rows.cuh and sg_integrals.cuh; the
// reinitialisation sweep has its own file, sg_reinit.cu.
#include <algorithm>
#include <cmath>

#include "sg_integrals.cuh"
#include "sg_rows.cuh"

namespace sg {
namespace {

constexpr int SW_THREADS = 256;
constexpr int SW_PKGS = SW_THREADS / PKG3;  // packages per CTA (64 threads each)


__global__ void __launch_bounds__(SW_THREADS) k_set_far(float* f, float v_in, float v_out) {
    f[threadIdx.x] = threadIdx.x < PKG3 ? v_in : v_out;
}

__global__ void __launch_bounds__(ROW_THREADS) k_gradient(const int32_t* __restrict__ faces, const float* __restrict__ phi,
                                                           float* __restrict__ gx, float* __restrict__ gy,
                                                           float* __restrict__ gz, int64_t P, float inv2h) {
    pdl_enter();
    write_far(gx, 0.0f, 0.0f);
    write_far(gy, 0.0f, 0.0f);
    write_far(gz, 0.0f, 0.0f);
    const RowSlot s = row_slot(P);
    const Rows w = load_rows(phi, faces, s);
    if (!s.valid) return;
    float4 ox, oy, oz;
    gradient_row(w, inv2h, ox, oy, oz);
    reinterpret_cast<float4*>(gx)[s.q4] = ox;
    reinterpret_cast<float4*>(gy)[s.q4] = oy;
    reinterpret_cast<float4*>(gz)[s.q4] = oz;
}

// 32-register launch bounds (8 CTAs of 256 per SM) as for the reinit sweep;
// the far packages of the output are written by the first CTA.
__global__ void __launch_bounds__(ROW_THREADS, 8) k_laplacian(const int32_t* __restrict__ faces,
                                                               const float* __restrict__ phi, float* __restrict__ lap,
                                                               int64_t P, float inv_h2) {
    write_far(lap, 0.0f, 0.0f);
    const RowSlot s = row_slot(P);
    const Rows w = load_rows(phi, faces, s);
    if (!s.valid) return;
    reinterpret_cast<float4*>(lap)[s.q4] = laplacian_row(w, inv_h2);
}

// One float4 row per thread, grid-stride over the active packages.
__global__ void __launch_bounds__(SW_THREADS) k_sequential(float4* __restrict__ phi, float delta, int64_t rows) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows; q += (int64_t)gridDim.x * blockDim.x) {
        float4 v = phi[32 + q];  // skip the two far packages (32 rows)
        v.x += delta;
        v.y += delta;
        v.z += delta;
        v.w += delta;
        phi[32 + q] = v;
    }
}

__global__ void __launch_bounds__(SW_THREADS) k_copy(const float* __restrict__ src, float* __restrict__ dst,
                                                      int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// Each warp takes pairs of packages in turn (a persistent loop): it stages
// the two packages' smoothed Heaviside tiles (6^3: the package plus a
// one-point halo; 72 rows of six, a 16-byte interior load and two halo
// values per row, rows fixed per lane so their index arithmetic is done
// once), then each half-warp sums the taps of one package, a row of four
// points per lane, as two x-neighbour pairs on paired FP32 instructions,
// and writes four outputs per field as 16-byte stores.  Warps never wait for
// one another; a tile that is all 0 or all 1 writes W = that value and G = 0
// without the taps.
constexpr int IW_WARPS = 8;  // warps per CTA
constexpr int IW_ROWS = 72;  // staged rows per package pair
#ifndef SG_IW_MIN_CTAS
#define SG_IW_MIN_CTAS 4
#endif

// With BATCH the store is a batch's: packages of type < 2 (every body's far
// packages) are skipped and left as they are, and each package takes the
// Heaviside width of its body, ieps_b[body[p] * ieps_stride].
template <bool OFF32, bool BATCH>
__global__ void __launch_bounds__(IW_WARPS * 32, SG_IW_MIN_CTAS) k_kernel_integrals(const int32_t* __restrict__ nbr,
                                                                     const float* __restrict__ phi,
                                                                     float* __restrict__ W, float* __restrict__ gx,
                                                                     float* __restrict__ gy, float* __restrict__ gz,
                                                                     int64_t P, KernelCoef K, float inv_eps,
                                                                     const uint8_t* __restrict__ type,
                                                                     const int32_t* __restrict__ body,
                                                                     const float* __restrict__ ieps_b,
                                                                     int ieps_stride) {
    pdl_enter();
    __shared__ __align__(16) float s_H[IW_WARPS][2][TILE_N];
    __shared__ int s_nb[IW_WARPS][2][32];  // rows of 27, padded: the two packages' rows start on bank 0
    if (!BATCH) {
        write_far(W, 1.0f, 0.0f);
        write_far(gx, 0.0f, 0.0f);
        write_far(gy, 0.0f, 0.0f);
        write_far(gz, 0.0f, 0.0f);
    }
    constexpr int first = BATCH ? 0 : 2;  // a single grid's far packages are 0 and 1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float(*tH)[TILE_N] = s_H[warp];
    int(*tnb)[32] = s_nb[warp];
    // staging rows of this lane: e = lane, lane + 32, lane + 64 (< 72): package e / 36, row e % 36
    int r_pk[3], r_nb[3], r_d0[3], r_e0[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = lane + 32 * q, rr = e % 36;
        const int y = rr % 6 - 1, z = rr / 6 - 1;
        const int oy = ((y + 4) >> 2) - 1, oz = ((z + 4) >> 2) - 1;
        r_pk[q] = e < IW_ROWS ? e / 36 : -1;
        r_nb[q] = 3 * (oy + 1) + 9 * (oz + 1);
        r_d0[q] = 4 * (y - 4 * oy) + 16 * (z - 4 * oz);
        r_e0[q] = TILE_Y * (y + 1) + TILE_Z * (z + 1);
    }
    const int half = lane >> 4, r = lane & 15;
    const int64_t pairs = (P - first + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * IW_WARPS;
    // the neighbourhood rows of the next pair are loaded while this pair's taps are summed
    int nb_next[2] = {0, 0};
    int64_t pr = (int64_t)blockIdx.x * IW_WARPS + warp;
    if (pr < pairs && lane < NB) {
        nb_next[0] = __ldg(nbr + (first + 2 * pr) * NB + lane);
        if (first + 1 + 2 * pr < P) nb_next[1] = __ldg(nbr + (first + 1 + 2 * pr) * NB + lane);
    }
    for (; pr < pairs; pr += stride) {
        const int64_t p0 = first + 2 * pr;
        const bool two = p0 + 1 < P;
        // which of the two packages take part (bit k: package p0 + k), and
        // their Heaviside widths (lane k holds package k's)
        unsigned okm = two ? 3u : 1u;
        float ie_l = inv_eps;
        if (BATCH) {
            bool ok = lane < 2 && (lane == 0 || two);
            if (ok) {
                ok = __ldg(type + p0 + lane) >= 2;
                if (ok) ie_l = __ldg(ieps_b + (int64_t)__ldg(body + p0 + lane) * ieps_stride);
            }
            okm = __ballot_sync(0xffffffffu, ok);
        }
        if (lane < NB) {
            tnb[0][lane] = nb_next[0];
            tnb[1][lane] = nb_next[1];
        }
        __syncwarp();
        const int64_t pn = pr + stride;
        if (pn < pairs && lane < NB) {
            nb_next[0] = __ldg(nbr + (first + 2 * pn) * NB + lane);
            if (first + 1 + 2 * pn < P) nb_next[1] = __ldg(nbr + (first + 1 + 2 * pn) * NB + lane);
        }
        unsigned bits[2] = {0u, 0u};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int pk = r_pk[q];
            const float ie = BATCH ? __shfl_sync(0xffffffffu, ie_l, pk < 0 ? 0 : pk) : inv_eps;
            if (pk < 0 || !((okm >> pk) & 1u)) continue;
            const int* nb = tnb[pk];
            float4 v;
            float vm, vp;
            if (OFF32) {  // 32-bit byte offsets (stores of fewer than 2^24 packages)
                const char* pb = reinterpret_cast<const char*>(phi) + 4u * (uint32_t)r_d0[q];
                v = __ldg(reinterpret_cast<const float4*>(pb + 4u * PKG3 * (uint32_t)nb[r_nb[q] + 1]));
                vm = __ldg(reinterpret_cast<const float*>(pb + 4u * (PKG3 * (uint32_t)nb[r_nb[q]] + 3u)));
                vp = __ldg(reinterpret_cast<const float*>(pb + 4u * PKG3 * (uint32_t)nb[r_nb[q] + 2]));
            } else {
                v = __ldg(reinterpret_cast<const float4*>(phi + (int64_t)nb[r_nb[q] + 1] * PKG3 + r_d0[q]));
                vm = __ldg(phi + (int64_t)nb[r_nb[q]] * PKG3 + r_d0[q] + 3);
                vp = __ldg(phi + (int64_t)nb[r_nb[q] + 2] * PKG3 + r_d0[q]);
            }
            const float f[6] = {vm, v.x, v.y, v.z, v.w, vp};
            float2* t = reinterpret_cast<float2*>(tH[pk] + r_e0[q]);  // rows start on 8-byte boundaries
            unsigned b = 0;
#pragma unroll
            for (int i = 0; i < 6; i += 2) {
                const float h0 = heaviside_neg(f[i], ie), h1 = heaviside_neg(f[i + 1], ie);
                t[i / 2] = make_float2(h0, h1);
                b |= (h0 != 0.0f ? 1u : 0u) | (h0 != 1.0f ? 2u : 0u) | (h1 != 0.0f ? 1u : 0u) | (h1 != 1.0f ? 2u : 0u);
            }
            bits[pk] |= b;
        }
        bits[0] = __reduce_or_sync(0xffffffffu, bits[0]);
        bits[1] = __reduce_or_sync(0xffffffffu, bits[1]);
        __syncwarp();
        if ((okm >> half) & 1u) {
            const int64_t p = p0 + half;
            float w[4], ax[4], ay[4], az[4];
            if (!integrals_saturated(bits[half], w[0], ax[0], ay[0], az[0])) {
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    float2 w2, x2, y2, z2;
                    integrals_point2(tH[half], 4 * r + 2 * pp, K, w2, x2, y2, z2);
                    w[2 * pp] = w2.x, w[2 * pp + 1] = w2.y;
                    ax[2 * pp] = x2.x, ax[2 * pp + 1] = x2.y;
                    ay[2 * pp] = y2.x, ay[2 * pp + 1] = y2.y;
                    az[2 * pp] = z2.x, az[2 * pp + 1] = z2.y;
                }
            } else {
#pragma unroll
                for (int i = 1; i < 4; ++i) w[i] = w[0], ax[i] = ax[0], ay[i] = ay[0], az[i] = az[0];
            }
            if (OFF32) {
                const uint32_t ob = 16u * (uint32_t)(p * 16 + r);
                auto row = [ob](float* a) { return reinterpret_cast<float4*>(reinterpret_cast<char*>(a) + ob); };
                *row(W) = make_float4(w[0], w[1], w[2], w[3]);
                *row(gx) = make_float4(ax[0], ax[1], ax[2], ax[3]);
                *row(gy) = make_float4(ay[0], ay[1], ay[2], ay[3]);
                *row(gz) = make_float4(az[0], az[1], az[2], az[3]);
            } else {
                const int64_t q4 = p * 16 + r;
                reinterpret_cast<float4*>(W)[q4] = make_float4(w[0], w[1], w[2], w[3]);
                reinterpret_cast<float4*>(gx)[q4] = make_float4(ax[0], ax[1], ax[2], ax[3]);
                reinterpret_cast<float4*>(gy)[q4] = make_float4(ay[0], ay[1], ay[2], ay[3]);
                reinterpret_cast<float4*>(gz)[q4] = make_float4(az[0], az[1], az[2], az[3]);
            }
        }
        __syncwarp();  // the next pair's staging overwrites the tiles
    }
}

// Supports above 2h: 8^3 tiles, 5^3 taps.
__global__ void __launch_bounds__(SW_THREADS) k_kernel_integrals_wide(const int32_t* __restrict__ nbr,
                                                                       const float* __restrict__ phi,
                                                                       float* __restrict__ W, float* __restrict__ gx,
                                                                       float* __restrict__ gy, float* __restrict__ gz,
                                                                       int64_t P, KernelCoef K, float inv_eps) {
    __shared__ int s_nb[SW_PKGS][NB];
    __shared__ float s_H[SW_PKGS][512];  // 8^3 tile: package plus a two-point halo
    __shared__ unsigned s_sat[SW_PKGS];
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t p = 2 + (int64_t)blockIdx.x * SW_PKGS + lp;
    const bool valid = p < P;
    if (valid && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
    if (d == 0) s_sat[lp] = 0;
    __syncthreads();
    const unsigned bits = __reduce_or_sync(0xffffffffu, valid ? stage_rows_wide(s_nb[lp], phi, inv_eps, d, s_H[lp]) : 0u);
    if ((threadIdx.x & 31) == 0 && bits) atomicOr(&s_sat[lp], bits);
    __syncthreads();
    if (!valid) return;
    float w, ax, ay, az;
    if (!integrals_saturated(s_sat[lp], w, ax, ay, az)) integrals_point_wide(s_H[lp], d, K, w, ax, ay, az);
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

double wendland(double q, double R) {
    if (q >= R) return 0.0;
    const double t = 1.0 - q / R;
    return t * t * t * t * (1.0 + 4.0 * q / R);
}

double wendland_dq(double q, double R) {
    if (q >= R) return 0.0;
    const double t = 1.0 - q / R;
    return -20.0 * q / (R * R) * t * t * t;
}

}  // namespace

KernelCoef kernel_coef(double R) {
    KernelCoef K;
    double den = 0.0;
    for (int sz = -2; sz <= 2; ++sz)
        for (int sy = -2; sy <= 2; ++sy)
            for (int sx = -2; sx <= 2; ++sx) den += wendland(std::sqrt((double)(sx * sx + sy * sy + sz * sz)), R);
    for (int c = 0; c < 13; ++c) {
        const double q = std::sqrt((double)c);
        K.cw[c] = (float)(wendland(q, R) / den);
        K.ck[c] = c == 0 ? 0.0f : (float)(wendland_dq(q, R) / q / den);
    }
    return K;
}

cudaError_t launch_set_far(float* f, float v_in, float v_out, cudaStream_t s) {
    k_set_far<<<1, 2 * PKG3, 0, s>>>(f, v_in, v_out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gradient(const GridF& G, const int32_t* faces, const float* phi, float* gx, float* gy, float* gz,
                            int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    return launch_pdl(k_gradient, row_blocks(P), ROW_THREADS, 0, s, faces, phi, gx, gy, gz, P, (float)(1.0 / (2.0 * G.h_d)));
}

cudaError_t launch_laplacian(const GridF& G, const int32_t* faces, const float* phi, float* lap, int64_t P,
                             cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    k_laplacian<<<row_blocks(P), ROW_THREADS, 0, s>>>(faces, phi, lap, P, (float)(1.0 / (G.h_d * G.h_d)));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sequential(float* phi, float delta, int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    const int64_t rows = (P - 2) * 16;
    int64_t b = (rows + SW_THREADS - 1) / SW_THREADS;
    if (b > 148 * 16) b = 148 * 16;
    k_sequential<<<(unsigned)b, SW_THREADS, 0, s>>>(reinterpret_cast<float4*>(phi), delta, rows);
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

// Persistent grid of k_kernel_integrals: the CTAs resident on every SM at
// once, at most one warp per package pair.
unsigned integrals_grid(int64_t P) {
    static int per_sm = 0, sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kernel_integrals<true, false>, IW_WARPS * 32, 0) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int64_t pairs = (P - 2 + 1) / 2;
    const int64_t need = (pairs + IW_WARPS - 1) / IW_WARPS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)per_sm * sms));
}

cudaError_t launch_kernel_integrals(const GridF& G, const int32_t* nbr, const float* phi, float* W, float* gx,
                                    float* gy, float* gz, int64_t P, double R, double eps, cudaStream_t s) {
    cudaError_t e;
    if (P <= 2 || R > 2.0) {  // the narrow kernel writes the far packages itself
        if ((e = launch_set_far(W, 1.0f, 0.0f, s)) != cudaSuccess) return e;
        if ((e = launch_set_far(gx, 0.0f, 0.0f, s)) != cudaSuccess) return e;
        if ((e = launch_set_far(gy, 0.0f, 0.0f, s)) != cudaSuccess) return e;
        if ((e = launch_set_far(gz, 0.0f, 0.0f, s)) != cudaSuccess) return e;
    }
    if (P <= 2) return cudaSuccess;
    if (R > 2.0)
        k_kernel_integrals_wide<<<pkg_blocks(P), SW_THREADS, 0, s>>>(nbr, phi, W, gx, gy, gz, P, kernel_coef(R),
                                                                      (float)(1.0 / eps));
    else if (P < ((int64_t)1 << 24) && !force_wide_offsets())  // byte offsets of every field fit 32 bits
        return launch_pdl(k_kernel_integrals<true, false>, integrals_grid(P), IW_WARPS * 32, 0, s, nbr, phi, W, gx, gy, gz,
                          P, kernel_coef(R), (float)(1.0 / eps), nullptr, nullptr, nullptr, 0);
    else
        return launch_pdl(k_kernel_integrals<false, false>, integrals_grid(P), IW_WARPS * 32, 0, s, nbr, phi, W, gx, gy,
                          gz, P, kernel_coef(R), (float)(1.0 / eps), nullptr, nullptr, nullptr, 0);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_kernel_integrals(const int32_t* nbr, const uint8_t* type, const int32_t* body,
                                          const float* ieps_b, int ieps_stride, const float* phi, float* W, float* gx,
                                          float* gy, float* gz, int64_t P, double R, cudaStream_t s) {
    if (P < 1) return cudaSuccess;
    const KernelCoef K = kernel_coef(R);
    if (P < ((int64_t)1 << 24) && !force_wide_offsets())
        k_kernel_integrals<true, true><<<integrals_grid(P + 2), IW_WARPS * 32, 0, s>>>(
            nbr, phi, W, gx, gy, gz, P, K, 0.0f, type, body, ieps_b, ieps_stride);
    else
        k_kernel_integrals<false, true><<<integrals_grid(P + 2), IW_WARPS * 32, 0, s>>>(
            nbr, phi, W, gx, gy, gz, P, K, 0.0f, type, body, ieps_b, ieps_stride);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sg
