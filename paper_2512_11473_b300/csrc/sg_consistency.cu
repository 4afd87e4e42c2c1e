// sg_consistency.cu -- consistency (sign) correction ("Consistency
// Correction"): the sign of phi is trusted only within tau of the surface
// and carried from there to the rest of the domain by two diffusion steps,
// one over the data points of the active packages and one over the
// background cells.  Each step is a Jacobi flood over face neighbours (an
// unknown entry takes the sign of the sum of its labelled neighbours'
// signs), run in batches of sweeps until a sweep changes nothing.
//  - points: trusted points (|phi| < tau) start with their sign; the flood
//    stays inside active packages; then phi <- sign |phi| where known;
//  - cells: core cells are blocked, an inner cell starts with the sign its
//    package's points share, far cells take their flooded label (package 0
//    inside, 1 outside) and the neighbour table is rebuilt.
// The point step runs first: every data point within h of the surface lies
// in a core cell, so the cells have no trusted sign until the points have.
#include "sg_internal.cuh"

namespace sg {
namespace {

constexpr int CC_THREADS = 256;
constexpr int8_t CC_BLOCK = 2;

unsigned cc_blocks(int64_t n) {
    int64_t b = (n + CC_THREADS - 1) / CC_THREADS;
    if (b < 1) b = 1;
    if (b > 148 * 64) b = 148 * 64;
    return (unsigned)b;
}

__device__ __forceinline__ void flag_if_any(bool changed, int* flag) {
    const unsigned any = __ballot_sync(0xffffffffu, changed);
    if (any && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// trusted points keep their sign; every other entry starts unknown
__global__ void __launch_bounds__(CC_THREADS) k_cc_seed_points(const float* __restrict__ phi, int8_t* __restrict__ sg,
                                                                int64_t n_act, float tau) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = 2 * PKG3 + e;
        const float v = phi[q];
        sg[q] = fabsf(v) < tau ? (int8_t)(v > 0.0f ? 1 : (v < 0.0f ? -1 : 0)) : (int8_t)0;
    }
}

// one Jacobi sweep of the point flood; neighbours across a package face come
// from the face table, neighbours in far packages do not count
__global__ void __launch_bounds__(CC_THREADS) k_cc_flood_points(const int32_t* __restrict__ faces,
                                                                 const int8_t* __restrict__ src,
                                                                 int8_t* __restrict__ dst, int64_t n_act, int* flag) {
    bool changed = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = 2 * PKG3 + e, p = q >> 6;
        const int d = (int)(q & 63);
        int8_t s = src[q];
        if (s == 0) {
            const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
            const int32_t* fc = faces + p * 8;
            int sum = 0;
            int64_t pp;
            pp = i > 0 ? p : __ldg(fc + 0);
            if (pp >= 2) sum += src[pp * PKG3 + (i > 0 ? d - 1 : d + 3)];
            pp = i < 3 ? p : __ldg(fc + 1);
            if (pp >= 2) sum += src[pp * PKG3 + (i < 3 ? d + 1 : d - 3)];
            pp = j > 0 ? p : __ldg(fc + 2);
            if (pp >= 2) sum += src[pp * PKG3 + (j > 0 ? d - 4 : d + 12)];
            pp = j < 3 ? p : __ldg(fc + 3);
            if (pp >= 2) sum += src[pp * PKG3 + (j < 3 ? d + 4 : d - 12)];
            pp = k > 0 ? p : __ldg(fc + 4);
            if (pp >= 2) sum += src[pp * PKG3 + (k > 0 ? d - 16 : d + 48)];
            pp = k < 3 ? p : __ldg(fc + 5);
            if (pp >= 2) sum += src[pp * PKG3 + (k < 3 ? d + 16 : d - 48)];
            if (sum != 0) {
                s = sum > 0 ? 1 : -1;
                changed = true;
            }
        }
        dst[q] = s;
    }
    flag_if_any(changed, flag);
}

// phi <- sign |phi| where the flood found a sign; counts the flips
__global__ void __launch_bounds__(CC_THREADS) k_cc_apply(float* __restrict__ phi, const int8_t* __restrict__ sg,
                                                          int64_t n_act, unsigned long long* count) {
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = 2 * PKG3 + e;
        const int8_t s = sg[q];
        const float v = phi[q];
        if ((s > 0 && v < 0.0f) || (s < 0 && v > 0.0f)) {
            phi[q] = -v;
            ++c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// cell labels: core cells blocked, inner cells from their package's signs
__global__ void __launch_bounds__(CC_THREADS) k_cc_seed_cells(const int32_t* __restrict__ cell_pkg,
                                                               const uint8_t* __restrict__ pkg_type,
                                                               const int8_t* __restrict__ sg, int8_t* __restrict__ lab,
                                                               int64_t nc) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = cell_pkg[c];
        int8_t l = 0;
        if (p >= 2) {
            if (pkg_type[p] == 2) {
                l = CC_BLOCK;
            } else {
                // bytes are 0x01 (+), 0xff (-) or 0: bit 7 marks -, bit 0 without bit 7 marks +
                const uint4* r = reinterpret_cast<const uint4*>(sg + p * PKG3);
                unsigned pos = 0, neg = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 v = r[k];
                    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        neg |= w[m] & 0x80808080u;
                        pos |= w[m] & 0x01010101u & ~((w[m] >> 7) & 0x01010101u);
                    }
                }
                l = (pos && neg) ? CC_BLOCK : (pos ? 1 : (neg ? -1 : 0));
            }
        }
        lab[c] = l;
    }
}

// one Jacobi sweep of the cell flood over the background mesh
__global__ void __launch_bounds__(CC_THREADS) k_cc_flood_cells(const int8_t* __restrict__ src, int8_t* __restrict__ dst,
                                                                int nx, int ny, int nz, int* flag) {
    const int64_t nc = (int64_t)nx * ny * nz;
    bool changed = false;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        int8_t s = src[c];
        if (s == 0) {
            // 32-bit index arithmetic: grids hold fewer than 2^31 cells
            const uint32_t u = (uint32_t)c, q = u / (uint32_t)nx, kk = q / (uint32_t)ny;
            const int I = (int)(u - q * (uint32_t)nx), J = (int)(q - kk * (uint32_t)ny), K = (int)kk;
            const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
            int sum = 0;
            int8_t v;
            if (I > 0 && ((v = src[c - sx]) == 1 || v == -1)) sum += v;
            if (I < nx - 1 && ((v = src[c + sx]) == 1 || v == -1)) sum += v;
            if (J > 0 && ((v = src[c - sy]) == 1 || v == -1)) sum += v;
            if (J < ny - 1 && ((v = src[c + sy]) == 1 || v == -1)) sum += v;
            if (K > 0 && ((v = src[c - sz]) == 1 || v == -1)) sum += v;
            if (K < nz - 1 && ((v = src[c + sz]) == 1 || v == -1)) sum += v;
            if (sum != 0) {
                s = sum > 0 ? 1 : -1;
                changed = true;
            }
        }
        dst[c] = s;
    }
    flag_if_any(changed, flag);
}

// far cells take their label's far package; counts the moves
__global__ void __launch_bounds__(CC_THREADS) k_cc_far(int32_t* __restrict__ cell_pkg, const int8_t* __restrict__ lab,
                                                        int64_t nc, unsigned long long* count) {
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = cell_pkg[e];
        const int8_t l = lab[e];
        if (p < 2 && (l == 1 || l == -1)) {
            const int32_t want = l < 0 ? 0 : 1;
            if (p != want) {
                cell_pkg[e] = want;
                ++c;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Jacobi sweeps in batches of CC_BATCH until one changes nothing; `a` ends
// on the fixed point.  Host-synchronising.
constexpr int CC_BATCH = 8;

template <class Sweep>
cudaError_t flood(Sweep sweep, int8_t*& a, int8_t*& b, int* dflag, int* hflag, int64_t max_sweeps, int64_t& sweeps,
                  cudaStream_t s) {
    for (;;) {
        cudaError_t e = cudaMemsetAsync(dflag, 0, CC_BATCH * sizeof(int), s);
        for (int k = 0; k < CC_BATCH && e == cudaSuccess; ++k) {
            sweep(a, b, dflag + k);
            e = cudaGetLastError();
            int8_t* t = a;
            a = b;
            b = t;
            ++sweeps;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, dflag, CC_BATCH * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (hflag[CC_BATCH - 1] == 0) return cudaSuccess;
        if (sweeps > max_sweeps) return cudaErrorLaunchTimeout;  // cannot happen: every sweep labels an entry
    }
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t consistency_scratch_bytes(int64_t P, int64_t nc) {
    return 2 * al256((size_t)P * PKG3) + 2 * al256((size_t)nc) + 256;
}

cudaError_t run_consistency(const GridFF& G, int64_t P, int64_t nc, int32_t* cell_pkg, const int32_t* pkg_cell,
                            const uint8_t* pkg_type, int32_t* nbr, int32_t* faces, float* phi, float tau,
                            void* scratch, void* host_pin, int64_t out[4], cudaStream_t s) {
    char* sp = (char*)scratch;
    int8_t* sa = (int8_t*)sp;
    sp += al256((size_t)P * PKG3);
    int8_t* sb = (int8_t*)sp;
    sp += al256((size_t)P * PKG3);
    int8_t* la = (int8_t*)sp;
    sp += al256((size_t)nc);
    int8_t* lb = (int8_t*)sp;
    sp += al256((size_t)nc);
    int* dflag = (int*)sp;                                               // CC_BATCH ints
    unsigned long long* cnt = (unsigned long long*)(sp + 64);            // 2 counters
    int* hflag = (int*)host_pin;                                         // CC_BATCH ints
    unsigned long long* hcnt = (unsigned long long*)((char*)host_pin + 64);  // 2 counters
    const int64_t n_act = (P - 2) * PKG3;
    cudaError_t e;
    if ((e = cudaMemsetAsync(sa, 0, (size_t)P * PKG3, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sb, 0, (size_t)P * PKG3, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    int64_t sweeps_pt = 0, sweeps_cell = 0;
    if (n_act > 0) {
        k_cc_seed_points<<<cc_blocks(n_act), CC_THREADS, 0, s>>>(phi, sa, n_act, tau);
        note_launch();
        const unsigned nb = cc_blocks(n_act);
        e = flood(
            [&](const int8_t* src, int8_t* dst, int* flag) {
                k_cc_flood_points<<<nb, CC_THREADS, 0, s>>>(faces, src, dst, n_act, flag);
                note_launch();
            },
            sa, sb, dflag, hflag, n_act + 1, sweeps_pt, s);
        if (e != cudaSuccess) return e;
        k_cc_apply<<<cc_blocks(n_act), CC_THREADS, 0, s>>>(phi, sa, n_act, cnt);
        note_launch();
    }
    k_cc_seed_cells<<<cc_blocks(nc), CC_THREADS, 0, s>>>(cell_pkg, pkg_type, sa, la, nc);
    note_launch();
    const unsigned cb = cc_blocks(nc);
    e = flood(
        [&](const int8_t* src, int8_t* dst, int* flag) {
            k_cc_flood_cells<<<cb, CC_THREADS, 0, s>>>(src, dst, G.dims[0], G.dims[1], G.dims[2], flag);
            note_launch();
        },
        la, lb, dflag, hflag, nc + 1, sweeps_cell, s);
    if (e != cudaSuccess) return e;
    k_cc_far<<<cc_blocks(nc), CC_THREADS, 0, s>>>(cell_pkg, la, nc, cnt + 1);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the neighbour and face tables name far packages by their cells
    if ((e = launch_fill_nbr(G, cell_pkg, pkg_cell, nbr, P, s)) != cudaSuccess) return e;
    if ((e = launch_fill_faces(nbr, faces, P, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hcnt, cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (out) {
        out[0] = (int64_t)hcnt[0];
        out[1] = (int64_t)hcnt[1];
        out[2] = sweeps_pt;
        out[3] = sweeps_cell;
    }
    return cudaSuccess;
}

}  // namespace sg
