// sg_scan.cu -- exclusive prefix sum of uint32 values (reduce, scan of the
// tile sums, down-sweep).  Three launches and no inter-block waiting, so no
// block ever spins on another.  Used to number the active cells (package ids
// in cell order) and to turn radix-sort histograms into scatter offsets.
#include "sg_internal.cuh"

namespace sg {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SPINE_THREADS = 1024;
constexpr int64_t SCAN_GRID = 148 * 8;  // 8 blocks of 256 on each of the 148 SMs

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread over the block; returns the
// block total through *total
template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < THREADS / 32 ? warp_sums[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < THREADS / 32) warp_sums[lane] = wi - w;
        if (lane == THREADS / 32 - 1) warp_sums[THREADS / 32] = wi;  // slot past the warp sums
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - v;
    *total = warp_sums[THREADS / 32];
    __syncthreads();
    return r;
}

// Tile sums; blocks loop over the tiles (a grid of at most SCAN_GRID blocks,
// so that a launch whose `go` flag is clear ends at once).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, int64_t nb,
                                                               uint32_t* __restrict__ partial, const int* go) {
    pdl_enter();
    if (go && *go == 0) return;
    __shared__ uint32_t red[SCAN_THREADS / 32];
    for (int64_t tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        uint32_t s = 0;
#pragma unroll
        for (int r = 0; r < SCAN_ITEMS; ++r)
            if (base + r < n) s += in[base + r];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t v = threadIdx.x < SCAN_THREADS / 32 ? red[threadIdx.x] : 0u;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) partial[tile] = v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SPINE_THREADS) k_scan_spine(uint32_t* __restrict__ partial, int64_t nb,
                                                               uint32_t* __restrict__ total, const int* go) {
    pdl_enter();
    if (go && *go == 0) return;
    __shared__ uint32_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SPINE_THREADS) {
        int64_t i = base + threadIdx.x;
        uint32_t v = i < nb ? partial[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan<SPINE_THREADS>(v, &tot);
        uint32_t carry = carry_s;
        if (i < nb) partial[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry_s;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t* in, uint32_t* out, int64_t n, int64_t nb,
                                                             const uint32_t* __restrict__ partial, const int* go) {
    pdl_enter();
    if (go && *go == 0) return;
    for (int64_t tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS];
        uint32_t s = 0;
#pragma unroll
        for (int r = 0; r < SCAN_ITEMS; ++r) {
            v[r] = base + r < n ? in[base + r] : 0u;
            s += v[r];
        }
        uint32_t tot;
        uint32_t run = block_excl_scan<SCAN_THREADS>(s, &tot) + partial[tile];
#pragma unroll
        for (int r = 0; r < SCAN_ITEMS; ++r) {
            if (base + r < n) out[base + r] = run;
            run += v[r];
        }
    }
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)((nb + 64) * sizeof(uint32_t) + 255) & ~(size_t)255;
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* scratch,
                               cudaStream_t s, const int* go) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return cudaSuccess;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* partial = (uint32_t*)scratch;
    const unsigned grid = (unsigned)(nb < SCAN_GRID ? nb : SCAN_GRID);
    cudaError_t e = launch_pdl(k_scan_reduce, grid, SCAN_THREADS, 0, s, in, n, nb, partial, go);
    if (e == cudaSuccess) e = launch_pdl(k_scan_spine, 1, SPINE_THREADS, 0, s, partial, nb, total, go);
    if (e == cudaSuccess) e = launch_pdl(k_scan_down, grid, SCAN_THREADS, 0, s, in, out, n, nb, partial, go);
    return e;
}

}  // namespace sg
