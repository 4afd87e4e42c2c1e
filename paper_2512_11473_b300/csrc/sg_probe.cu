// sg_probe.cu -- particle probe ("Grid-Particle Coupling"): trilinear
// interpolation of the package fields at particle positions, with particles
// optionally walked in Morton order, and the Morton sort itself (an LSD radix
// sort written for this library: per-tile digit histograms, an exclusive scan
// of the digit-major histogram table, and a stable scatter staged through
// shared memory so that global writes of one digit run are contiguous).
#include <cmath>
#include <mutex>

#include "sg_probe.cuh"
#include <algorithm>

namespace sg {
namespace {

constexpr int PR_THREADS = 256;
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_WARPS = RS_THREADS / 32;

__device__ __forceinline__ uint64_t spread3(uint64_t v) {  // bit b -> bit 3b (21 bits)
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t morton_key(const GridF& G, float x, float y, float z) {
    const float pos[3] = {x, y, z};
    uint64_t key = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int i0;
        float t;
        lattice(pos[a], G.lat_c[a], G.lat_ih, i0, t);
        int k = i0 + 1;
        k = k < 0 ? 0 : (k > 4 * G.dims[a] + 1 ? 4 * G.dims[a] + 1 : k);
        key |= spread3((uint64_t)k) << a;
    }
    return key;
}

// Sortedness check, reading the positions only: *unsorted is set when some
// key exceeds its successor's (one atomic per warp that finds one, and none
// once the flag is seen set).  The successor's key comes from the next lane.
__global__ void __launch_bounds__(RS_THREADS) k_morton_check(GridF G, int64_t n, const float* __restrict__ x,
                                                             const float* __restrict__ y, const float* __restrict__ z,
                                                             int* unsorted) {
    pdl_enter();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = (n + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    for (int64_t it = 0; it < iters; ++it) {  // uniform trip count: every lane takes part in the vote
        const int64_t q = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const uint64_t k = q < n ? morton_key(G, x[q], y[q], z[q]) : 0;
        uint64_t next = __shfl_down_sync(0xffffffffu, k, 1);
        if (lane == 31 && q + 1 < n) next = morton_key(G, x[q + 1], y[q + 1], z[q + 1]);
        const bool bad = q + 1 < n && k > next;
        const unsigned m = __ballot_sync(0xffffffffu, bad);
        if (m && lane == __ffs(m) - 1 && *(volatile int*)unsorted == 0) atomicOr(unsorted, 1);
    }
}

// Keys and identity indices for the radix passes (skipped when the input is
// already in order), and the caller's copy of the keys when asked for.
// Sampled sortedness check: only the pairs (q, q + 1) with q a multiple of
// `stride` are compared.  Used where the walk order is a matter of speed
// only (the probe): an input that passes is walked as it is.
__global__ void __launch_bounds__(RS_THREADS) k_morton_check_sampled(GridF G, int64_t n, const float* __restrict__ x,
                                                                     const float* __restrict__ y,
                                                                     const float* __restrict__ z, int stride,
                                                                     int* unsorted) {
    pdl_enter();
    const int64_t pairs = (n - 1 + stride - 1) / stride;
    bool bad = false;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < pairs; m += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = m * stride;
        bad |= morton_key(G, x[q], y[q], z[q]) > morton_key(G, x[q + 1], y[q + 1], z[q + 1]);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(unsorted, 1);
}

template <typename KeyT>
__global__ void __launch_bounds__(RS_THREADS) k_morton_keys(GridF G, int64_t n, const float* __restrict__ x,
                                                            const float* __restrict__ y, const float* __restrict__ z,
                                                            KeyT* __restrict__ keys, uint32_t* __restrict__ vals,
                                                            uint64_t* __restrict__ keys_out, const int* unsorted) {
    pdl_enter();
    const bool sort = *unsorted != 0;
    if (!sort && !keys_out) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = morton_key(G, x[q], y[q], z[q]);
        if (sort) {
            keys[q] = (KeyT)k;
            vals[q] = (uint32_t)q;
        }
        if (keys_out) keys_out[q] = k;
    }
}

__global__ void k_identity_if_sorted(const int* __restrict__ unsorted, int32_t* __restrict__ order, int64_t n) {
    pdl_enter();
    if (*unsorted) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        order[q] = (int32_t)q;
}

// Per-tile digit histogram, written digit-major: hist[d * nb + tile].
template <typename KeyT>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const KeyT* __restrict__ keys, int64_t n, int shift,
                                                        uint32_t* __restrict__ hist, int64_t nb, const int* run) {
    pdl_enter();
    if (*run == 0) return;  // keys already in order
    __shared__ uint32_t h[256];
    for (int64_t tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = tile * RS_TILE;
#pragma unroll 4
        for (int r = 0; r < RS_ITEMS; ++r) {
            int64_t i = base + r * RS_THREADS + threadIdx.x;
            if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[(int64_t)threadIdx.x * nb + tile] = h[threadIdx.x];
        __syncthreads();
    }
}

// Stable scatter of one 8-bit digit.  Warp w ranks its own contiguous 512
// keys of the tile in 16 rounds of 32 (match_any groups equal digits; a
// warp-private counter per digit gives the rank), so the rank order is the
// input order.  A block pass turns the per-warp counts into tile offsets, the
// keys are staged in shared memory in digit order and written out so that
// each digit's run is one contiguous global range.
template <typename KeyT>
__global__ void __launch_bounds__(RS_THREADS, 2) k_rs_scatter(const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           KeyT* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           int64_t n, int shift, const uint32_t* __restrict__ offs,
                                                           int64_t nb, const int* run) {
    pdl_enter();
    if (*run == 0) return;  // keys already in order
    extern __shared__ __align__(16) unsigned char smem[];
    KeyT* s_k = (KeyT*)smem;
    uint32_t* s_v = (uint32_t*)(smem + RS_TILE * sizeof(KeyT));
    __shared__ uint32_t s_cnt[RS_WARPS][256];
    __shared__ uint32_t s_start[256], s_goff[256];
    __shared__ uint32_t s_wsum[RS_WARPS];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // blocks loop over the tiles (a bounded grid, so that a launch whose
    // run flag is clear ends at once)
    for (int64_t tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        const int64_t tile0 = tile * RS_TILE;
        const int tile_n = (int)min((int64_t)RS_TILE, n - tile0);
        const int wbase = warp * (RS_TILE / RS_WARPS);

#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) s_cnt[w][t] = 0;
        KeyT key[RS_ITEMS];
        uint32_t val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            const int i = wbase + 32 * r + lane;
            key[r] = i < tile_n ? kin[tile0 + i] : (KeyT)0;
            val[r] = i < tile_n ? vin[tile0 + i] : 0u;
        }
        __syncthreads();
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            const bool valid = wbase + 32 * r + lane < tile_n;
            const uint32_t dg = valid ? ((uint32_t)(key[r] >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, dg);
            const uint32_t below = __popc(peers & lt);
            const uint32_t before = valid ? s_cnt[warp][dg] : 0u;
            __syncwarp();
            if (valid && below == 0) s_cnt[warp][dg] = before + __popc(peers);
            __syncwarp();
            rank[r] = before + below;
        }
        __syncthreads();
        {  // per digit t: exclusive prefix over warps, then over digits
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = s_cnt[w][t];
                s_cnt[w][t] = run;
                run += c;
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            uint32_t wpre = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) wpre += w < warp ? s_wsum[w] : 0u;
            const uint32_t start = wpre + incl - run;
            s_start[t] = start;
            s_goff[t] = offs[(int64_t)t * nb + tile] - start;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            if (wbase + 32 * r + lane < tile_n) {
                const uint32_t dg = (uint32_t)(key[r] >> shift) & 255u;
                const uint32_t pos = s_start[dg] + s_cnt[warp][dg] + rank[r];
                s_k[pos] = key[r];
                s_v[pos] = val[r];
            }
        }
        __syncthreads();
        for (int j = t; j < tile_n; j += RS_THREADS) {
            const KeyT k = s_k[j];
            const uint32_t g = s_goff[(uint32_t)(k >> shift) & 255u] + (uint32_t)j;
            kout[g] = k;
            vout[g] = s_v[j];
        }
        __syncthreads();
    }
}

// Point-interleaved probe table of n data points: tab[e] = (phi, gx, gy,
// gz) and tab[n + e] = (W, Gx, Gy, Gz) of data point e.
__global__ void __launch_bounds__(PR_THREADS) k_pack_probe(ProbeFields F, float4* __restrict__ tab, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        tab[e] = make_float4(__ldg(F.f[0] + e), __ldg(F.f[1] + e), __ldg(F.f[2] + e), __ldg(F.f[3] + e));
        tab[n + e] = make_float4(__ldg(F.f[4] + e), __ldg(F.f[5] + e), __ldg(F.f[6] + e), __ldg(F.f[7] + e));
    }
}

// Bounded to 40 registers, six CTAs per SM, without spills (50M probes on
// the h = 0.002 torus: 1.05 ms, against 1.07 ms at 43 registers and five
// CTAs and 1.15 ms at seven CTAs).
constexpr int PR_MIN_CTAS = 6;

template <bool OFF32>
__global__ void __launch_bounds__(PR_THREADS, PR_MIN_CTAS) k_probe(GridF G, const int32_t* __restrict__ cell_pkg,
                                                       const int32_t* __restrict__ nbr, ProbeFields F, int64_t n,
                                                       const float* __restrict__ x, const float* __restrict__ y,
                                                       const float* __restrict__ z, const int32_t* __restrict__ order,
                                                       const int* __restrict__ unsorted, ProbeOut out) {
    pdl_enter();
    // with the input already in Morton order the walk is the input order
    const bool use_order = order && (!unsorted || *unsorted != 0);
    // each CTA walks one contiguous stretch of the walk, so that a warp's
    // successive particles are near each other and hit the packages L1 holds
    // (a grid-stride walk measured 8% slower)
    const int64_t per = ((n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
    const int64_t r1 = min(n, (int64_t)blockIdx.x * per + per);
    for (int64_t r = (int64_t)blockIdx.x * per + threadIdx.x; r < r1; r += blockDim.x) {
        const int64_t q = use_order ? (int64_t)__ldg(order + r) : r;
        float acc[8];
        if (OFF32) {
            // particle arrays of fewer than 2^30 entries: 32-bit byte offsets here too
            const uint32_t qb = 4u * (uint32_t)q;
            auto at = [qb](const float* a) { return reinterpret_cast<const float*>(reinterpret_cast<const char*>(a) + qb); };
            auto st = [qb](float* a, float v) { *reinterpret_cast<float*>(reinterpret_cast<char*>(a) + qb) = v; };
            const float pos[3] = {__ldg(at(x)), __ldg(at(y)), __ldg(at(z))};
            const ProbeAt A = probe_locate(G.lat_c, G.lat_ih, G.dims, cell_pkg, 1, pos);
            probe_interp32<8>(nbr, F, A, acc);
            const float inv = probe_inv_norm(acc);
            if (out.o[0]) st(out.o[0], acc[0]);
            if (out.o[1]) st(out.o[1], acc[1] * inv);
            if (out.o[2]) st(out.o[2], acc[2] * inv);
            if (out.o[3]) st(out.o[3], acc[3] * inv);
#pragma unroll
            for (int f = 4; f < 8; ++f)
                if (out.o[f]) st(out.o[f], acc[f]);
        } else {
            const float pos[3] = {__ldg(x + q), __ldg(y + q), __ldg(z + q)};
            const ProbeAt A = probe_locate(G.lat_c, G.lat_ih, G.dims, cell_pkg, 1, pos);
            probe_interp<8>(nbr, F, A, acc);
            const float inv = probe_inv_norm(acc);
            if (out.o[0]) out.o[0][q] = acc[0];
            if (out.o[1]) out.o[1][q] = acc[1] * inv;
            if (out.o[2]) out.o[2][q] = acc[2] * inv;
            if (out.o[3]) out.o[3][q] = acc[3] * inv;
#pragma unroll
            for (int f = 4; f < 8; ++f)
                if (out.o[f]) out.o[f][q] = acc[f];
        }
    }
}

unsigned blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 148 * 64) b = 148 * 64;
    return (unsigned)b;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename KeyT>
cudaError_t sort_impl(const GridF& G, int64_t n, int key_bits, const float* x, const float* y, const float* z,
                      uint64_t* keys_out, int32_t* order_out, void* scratch, cudaStream_t s, bool identity_out,
                      const int** unsorted_out, int check_stride) {
    const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    char* sp = (char*)scratch;
    int* unsorted = (int*)sp;
    sp += 256;
    KeyT* k0 = (KeyT*)sp;
    sp += align256(n * sizeof(KeyT));
    KeyT* k1 = (KeyT*)sp;
    sp += align256(n * sizeof(KeyT));
    uint32_t* v0 = (uint32_t*)sp;
    sp += align256(n * sizeof(uint32_t));
    uint32_t* v1 = (uint32_t*)sp;
    sp += align256(n * sizeof(uint32_t));
    uint32_t* hist = (uint32_t*)sp;
    sp += align256(256 * nb * sizeof(uint32_t));
    void* scan_scratch = sp;

    cudaError_t e = cudaMemsetAsync(unsorted, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (check_stride > 1)
        e = launch_pdl(k_morton_check_sampled, blocks_for((n + check_stride - 1) / check_stride, RS_THREADS), RS_THREADS,
                       0, s, G, n, x, y, z, check_stride, unsorted);
    else
        e = launch_pdl(k_morton_check, blocks_for(n, RS_THREADS), RS_THREADS, 0, s, G, n, x, y, z, unsorted);
    if (e != cudaSuccess) return e;
    // grid-stride kernels that may find nothing to do: a bounded grid ends at once
    const unsigned small_grid = blocks_for(n, RS_THREADS) < 148 * 8 ? blocks_for(n, RS_THREADS) : 148 * 8;
    if ((e = launch_pdl(k_morton_keys<KeyT>, small_grid, RS_THREADS, 0, s, G, n, x, y, z, k0, v0, keys_out, unsorted)) !=
        cudaSuccess)
        return e;
    const int passes = (key_bits + 7) / 8;
    const size_t smem = RS_TILE * (sizeof(KeyT) + sizeof(uint32_t));
    e = cudaFuncSetAttribute(k_rs_scatter<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    KeyT* K[2] = {k0, k1};
    uint32_t* V[2] = {v0, v1};
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        uint32_t* vout = (p == passes - 1) ? (uint32_t*)order_out : V[1 - cur];
        if ((e = launch_pdl(k_rs_hist<KeyT>, (unsigned)(nb < 148 * 8 ? nb : 148 * 8), RS_THREADS, 0, s,
                            (const KeyT*)K[cur], n, shift, hist, nb, unsorted)) != cudaSuccess)
            return e;
        if ((e = exclusive_scan_u32(hist, hist, 256 * nb, nullptr, scan_scratch, s, unsorted)) != cudaSuccess)
            return e;
        // two blocks of the scatter fit on an SM (128 registers, 42-74 KB of shared memory)
        if ((e = launch_pdl(k_rs_scatter<KeyT>, (unsigned)(nb < 148 * 2 ? nb : 148 * 2), RS_THREADS, smem, s, K[cur],
                            V[cur], K[1 - cur], vout, n, shift, hist, nb, unsorted)) != cudaSuccess)
            return e;
        cur = 1 - cur;
    }
    if (passes == 0) {
        if ((e = cudaMemcpyAsync(order_out, V[0], n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
    } else if (identity_out) {
        if ((e = launch_pdl(k_identity_if_sorted, small_grid, RS_THREADS, 0, s, (const int*)unsorted, order_out, n)) !=
            cudaSuccess)
            return e;
    }
    if (unsorted_out) *unsorted_out = unsorted;
    return cudaSuccess;
}

}  // namespace

int morton_bits(const GridF& G) {
    int m = 0;
    for (int a = 0; a < 3; ++a) {
        int v = 4 * G.dims[a] + 1, b = 0;
        while ((1 << b) <= v) ++b;
        if (b > m) m = b;
    }
    return 3 * m;
}

size_t sort_scratch_bytes(int64_t n, int key_bits) {
    const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    size_t ks = key_bits <= 32 ? 4 : 8;
    return 2 * align256(n * ks) + 2 * align256(n * 4) + align256(256 * nb * 4) + scan_scratch_bytes(256 * nb) + 256;
}

cudaError_t morton_sort(const GridF& G, int64_t n, const float* x, const float* y, const float* z, uint64_t* keys_out,
                        int32_t* order_out, void* scratch, cudaStream_t s, bool identity_out,
                        const int** unsorted_out, int check_stride) {
    if (n <= 0) return cudaSuccess;
    const int bits = morton_bits(G);
    if (bits <= 32)
        return sort_impl<uint32_t>(G, n, bits, x, y, z, keys_out, order_out, scratch, s, identity_out, unsorted_out,
                                   check_stride);
    return sort_impl<uint64_t>(G, n, bits, x, y, z, keys_out, order_out, scratch, s, identity_out, unsorted_out,
                               check_stride);
}

cudaError_t launch_pack_probe(const ProbeFields& F, float4* tab, int64_t n_points, cudaStream_t s) {
    if (n_points <= 0) return cudaSuccess;
    k_pack_probe<<<blocks_for(n_points, PR_THREADS), PR_THREADS, 0, s>>>(F, tab, n_points);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_probe(const GridF& G, const int32_t* cell_pkg, const int32_t* nbr, const ProbeFields& F,
                         int64_t P, int64_t n, const float* x, const float* y, const float* z, const int32_t* order,
                         const int* unsorted, const ProbeOut& out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // up to 148 x 128 CTAs, each a contiguous stretch of about 2.6k particles
    // at 50M (9,472 CTAs measured 2% slower on the torus)
    const int64_t ctas = std::min<int64_t>((n + PR_THREADS - 1) / PR_THREADS, 148 * 128);
    if (P < ((int64_t)1 << 24) && n < ((int64_t)1 << 30) && !force_wide_offsets())
        return launch_pdl(k_probe<true>, (unsigned)ctas, PR_THREADS, 0, s, G, cell_pkg, nbr, F, n, x, y, z, order,
                          unsorted, out);
    return launch_pdl(k_probe<false>, (unsigned)ctas, PR_THREADS, 0, s, G, cell_pkg, nbr, F, n, x, y, z, order, unsorted,
                      out);
}

}  // namespace sg

// ---------------------------------------------------------------------------
// Allocation-free Morton order.  The scratch of the radix sort (two key and
// two index buffers, the digit histograms and the scan partials) lives in one
// file-scope device array sized for SG_NOALLOC_MAX_PARTICLES particles with
// 64-bit keys.  Every device that loads the library holds it until exit.
// ---------------------------------------------------------------------------
namespace sg {
namespace {

constexpr size_t na_align(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr size_t noalloc_scratch_size() {
    const size_t n = (size_t)SG_NOALLOC_MAX_PARTICLES;
    const size_t tiles = (n + RS_TILE - 1) / RS_TILE;
    const size_t hist = 256 * tiles;
    const size_t scan_partials = (hist + 2047) / 2048 + 64;  // bound of scan_scratch_bytes(hist)
    return 2 * na_align(n * 8) + 2 * na_align(n * 4) + na_align(hist * 4) + na_align(scan_partials * 4) + 256;
}

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

}  // namespace
}  // namespace sg

static __device__ __align__(256) unsigned char g_noalloc_scratch[sg::noalloc_scratch_size()];

extern "C" sg_status sg_morton_order_noalloc(const sg_grid_desc* desc, int64_t n, const float* x, const float* y,
                                             const float* z, uint64_t* keys, int32_t* order, void* stream) {
    using namespace sg;
    if (!desc || n < 0 || (n > 0 && (!x || !y || !z || !order))) return SG_ERR_INVALID;
    if (!(desc->h > 0.0) || !std::isfinite(desc->h)) return SG_ERR_INVALID;
    for (int a = 0; a < 3; ++a) {
        if (desc->dims[a] < 1) return SG_ERR_INVALID;
        if (4LL * desc->dims[a] + 1 >= (1LL << 21)) return SG_ERR_CAPACITY;
    }
    if (n > SG_NOALLOC_MAX_PARTICLES) return SG_ERR_CAPACITY;
    if (n == 0) return SG_OK;
    GridF G;
    for (int a = 0; a < 3; ++a) {
        G.lo[a] = (float)desc->lo[a];
        G.dims[a] = desc->dims[a];
    }
    G.h = (float)desc->h;
    G.h_d = desc->h;
    G.F = 0.0f;
    G.inv_h = (float)(1.0 / desc->h);
    set_lattice(G.lat_c, G.lat_ih, desc->lo, desc->h);
    if (sort_scratch_bytes(n, morton_bits(G)) > sizeof(g_noalloc_scratch)) return SG_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SG_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SG_ERR_CAPACITY;
    // the arrays must live on the current device (the scratch array used is that device's)
    for (const void* ptr : {(const void*)x, (const void*)y, (const void*)z, (const void*)order, (const void*)keys}) {
        if (!ptr) continue;
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, ptr) != cudaSuccess) {
            cudaGetLastError();
            return SG_ERR_INVALID;
        }
        if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return SG_ERR_INVALID;
        if (pa.device != dev) return SG_ERR_INVALID;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            // host code cannot use the array's name as a device address: look
            // the address up once, with this device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SG_ERR_CUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    if (morton_sort(G, n, x, y, z, keys, order, scratch, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return SG_ERR_CUDA;
    }
    return SG_OK;
}
