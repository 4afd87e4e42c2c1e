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
// Labels are kept as bit planes (a 64-bit word per package for the points,
// 32-cell words of the mesh's x-rows for the cells) and a sweep counts the
// + and - neighbours of every bit with bit-sliced adders: a few dozen word
// operations per 64 or 32 entries, the same labels sweep by sweep as the
// entry-by-entry rule.
#include <algorithm>

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

// Both floods run on bit planes of labels, `plus` and `minus`.  Points: a
// package's 64 data points are the bits of one 64-bit word (bit d = i + 4j +
// 16k), so a plane is P words, seen as 2P 32-bit halves by the kernels that
// work point by point.

// count of set inputs per bit, bit-sliced: n = n0 + 2 n1 + 4 n2 (at most 6)
template <class W>
__device__ __forceinline__ void count6(W a1, W a2, W a3, W a4, W a5, W a6, W& n0, W& n1, W& n2) {
    const W x1 = a1 ^ a2, s1 = x1 ^ a3, c1 = (a1 & a2) | (a3 & x1);
    const W x2 = a4 ^ a5, s2 = x2 ^ a6, c2 = (a4 & a5) | (a6 & x2);
    n0 = s1 ^ s2;
    const W k = s1 & s2, x3 = c1 ^ c2;
    n1 = x3 ^ k;
    n2 = (c1 & c2) | (k & x3);
}

// From the per-bit counts of + and - neighbours (bit-sliced, three bits
// each) the bits where + outnumbers - (gt) and where - outnumbers + (lt):
// the sign of the sum of the neighbours' signs.
template <class W>
__device__ __forceinline__ void majority(const W (&pa)[6], const W (&ma)[6], W& gt, W& lt) {
    W p0, p1, p2, m0, m1, m2;
    count6(pa[0], pa[1], pa[2], pa[3], pa[4], pa[5], p0, p1, p2);
    count6(ma[0], ma[1], ma[2], ma[3], ma[4], ma[5], m0, m1, m2);
    const W e2 = ~(p2 ^ m2), e1 = ~(p1 ^ m1);
    gt = (p2 & ~m2) | (e2 & ((p1 & ~m1) | (e1 & p0 & ~m0)));
    lt = (m2 & ~p2) | (e2 & ((m1 & ~p1) | (e1 & m0 & ~p0)));
}

// trusted points (|phi| < tau, phi != 0) start with their sign, every other
// point unknown; a warp forms one 32-bit half of a package's words by ballots
__global__ void __launch_bounds__(CC_THREADS) k_cc_seed_points(const float* __restrict__ phi,
                                                                uint32_t* __restrict__ plus,
                                                                uint32_t* __restrict__ minus, int64_t n_act,
                                                                float tau) {
    // n_act and the grid stride are multiples of 32: a warp is in or out as a whole
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = 2 * PKG3 + e;
        const float v = phi[q];
        const bool trusted = fabsf(v) < tau;
        const unsigned po = __ballot_sync(0xffffffffu, trusted && v > 0.0f);
        const unsigned mo = __ballot_sync(0xffffffffu, trusted && v < 0.0f);
        if ((threadIdx.x & 31) == 0) {
            plus[q >> 5] = po;
            minus[q >> 5] = mo;
        }
    }
}

// The six face-neighbour words of a package word v (bit d = i + 4j + 16k):
// bit d of the result is the neighbour's bit, from v inside the package and
// from the neighbour package's word (0 for a far package) across a face.
__device__ __forceinline__ void point_neighbours(uint64_t v, const uint64_t (&nb)[6], uint64_t (&out)[6]) {
    constexpr uint64_t I0 = 0x1111111111111111ull, I3 = 0x8888888888888888ull;  // i = 0, i = 3
    constexpr uint64_t J0 = 0x000F000F000F000Full, J3 = 0xF000F000F000F000ull;  // j = 0, j = 3
    out[0] = ((v << 1) & ~I0) | ((nb[0] >> 3) & I0);    // -x: d - 1, or d + 3 of the -x package
    out[1] = ((v >> 1) & ~I3) | ((nb[1] << 3) & I3);    // +x: d + 1, or d - 3 of the +x package
    out[2] = ((v << 4) & ~J0) | ((nb[2] >> 12) & J0);   // -y: d - 4, or d + 12
    out[3] = ((v >> 4) & ~J3) | ((nb[3] << 12) & J3);   // +y: d + 4, or d - 12
    out[4] = (v << 16) | (nb[4] >> 48);                 // -z: d - 16, or d + 48
    out[5] = (v >> 16) | (nb[5] << 48);                 // +z: d + 16, or d - 48
}

// Label loads: plain in the one-sweep kernels, from L2 (ld.global.cg) in
// the persistent ones, where another SM may have rewritten a line this SM
// still holds in L1 since an earlier sweep.
template <bool L2, class W>
__device__ __forceinline__ W ld_lab(const W* p) { return L2 ? __ldcg(p) : *p; }

// One package of a point sweep: an unknown point takes the sign of the sum
// of its labelled face neighbours' signs; neighbours across a package face
// come from the face table, those in far packages do not count.  Returns
// whether a label was set.
template <bool L2>
__device__ __forceinline__ bool point_sweep_one(const int32_t* __restrict__ faces, const uint64_t* p_in,
                                                const uint64_t* m_in, uint64_t* p_out, uint64_t* m_out, int64_t p) {
    const uint64_t Pw = ld_lab<L2>(p_in + p), Mw = ld_lab<L2>(m_in + p), U = ~(Pw | Mw);
    uint64_t Pn = Pw, Mn = Mw;
    bool changed = false;
    if (U) {
        const int4 f0 = __ldg(reinterpret_cast<const int4*>(faces + p * 8));
        const int2 f1 = __ldg(reinterpret_cast<const int2*>(faces + p * 8 + 4));
        const int32_t fc[6] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y};
        uint64_t pn[6], mn[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            pn[a] = fc[a] >= 2 ? ld_lab<L2>(p_in + fc[a]) : 0ull;
            mn[a] = fc[a] >= 2 ? ld_lab<L2>(m_in + fc[a]) : 0ull;
        }
        uint64_t pa[6], ma[6], gt, lt;
        point_neighbours(Pw, pn, pa);
        point_neighbours(Mw, mn, ma);
        majority(pa, ma, gt, lt);
        Pn |= U & gt;
        Mn |= U & lt;
        changed = (U & (gt | lt)) != 0ull;
    }
    p_out[p] = Pn;
    m_out[p] = Mn;
    return changed;
}

// one Jacobi sweep of the point flood, a thread per active package
__global__ void __launch_bounds__(CC_THREADS) k_cc_flood_points(const int32_t* __restrict__ faces,
                                                                 const uint64_t* __restrict__ p_in,
                                                                 const uint64_t* __restrict__ m_in,
                                                                 uint64_t* __restrict__ p_out,
                                                                 uint64_t* __restrict__ m_out, int64_t P, int* flag) {
    bool changed = false;
    for (int64_t p = 2 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
        changed |= point_sweep_one<false>(faces, p_in, m_in, p_out, m_out, p);
    flag_if_any(changed, flag);
}

// phi <- sign |phi| where the flood found a sign; counts the flips.  A
// thread per row of four points (one float4 of phi, four bits of each
// plane); rows without a label are not read.
__device__ __forceinline__ float apply_sign(float v, uint32_t pos, uint32_t neg, unsigned long long& c) {
    if ((pos && v < 0.0f) || (neg && v > 0.0f)) {
        ++c;
        return -v;
    }
    return v;
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_apply(float4* __restrict__ phi4, const uint32_t* __restrict__ plus,
                                                          const uint32_t* __restrict__ minus, int64_t n_rows,
                                                          unsigned long long* count) {
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_rows; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = 2 * PKG3 + 4 * e;  // first point of the row
        const uint32_t sh = (uint32_t)q & 31u;
        const uint32_t pb = (plus[q >> 5] >> sh) & 0xFu, mb = (minus[q >> 5] >> sh) & 0xFu;
        if ((pb | mb) == 0u) continue;
        const float4 v = phi4[q >> 2];
        float4 o;
        o.x = apply_sign(v.x, pb & 1u, mb & 1u, c);
        o.y = apply_sign(v.y, pb & 2u, mb & 2u, c);
        o.z = apply_sign(v.z, pb & 4u, mb & 4u, c);
        o.w = apply_sign(v.w, pb & 8u, mb & 8u, c);
        if (o.x != v.x || o.y != v.y || o.z != v.z || o.w != v.w) phi4[q >> 2] = o;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// The label of one background cell at the start of the cell flood: 0 for a
// far cell (unknown), CC_BLOCK for a core cell or an inner cell whose points
// carry both signs, else the sign its package's points share (or 0).
__device__ __forceinline__ int cell_label(const int32_t* __restrict__ cell_pkg, const uint8_t* __restrict__ pkg_type,
                                          const uint64_t* __restrict__ pt_plus, const uint64_t* __restrict__ pt_minus,
                                          int64_t c) {
    const int64_t p = cell_pkg[c];
    if (p < 2) return 0;
    if (pkg_type[p] == 2) return CC_BLOCK;
    const bool pos = pt_plus[p] != 0ull, neg = pt_minus[p] != 0ull;
    return (pos && neg) ? CC_BLOCK : (pos ? 1 : (neg ? -1 : 0));
}

// The cell flood runs on bit planes: each x-row of the background mesh is
// cut into nwx = ceil(nx / 32) words, bit b of word x of row r = J + ny K
// standing for cell I = 32 x + b (bits at I >= nx are 0 in every plane).
// `open` marks the cells that are not blocked, `plus` and `minus` the
// labelled ones.  Seeding: a lane per bit (rows padded to whole words, so a
// warp covers one word), the three words formed by ballots.
__global__ void __launch_bounds__(CC_THREADS) k_cc_seed_words(const int32_t* __restrict__ cell_pkg,
                                                               const uint8_t* __restrict__ pkg_type,
                                                               const uint64_t* __restrict__ pt_plus,
                                                               const uint64_t* __restrict__ pt_minus,
                                                               uint32_t* __restrict__ open,
                                                               uint32_t* __restrict__ plus, uint32_t* __restrict__ minus,
                                                               int nx, int nwx, int64_t n_lanes) {
    // n_lanes and the grid stride are multiples of 32: a warp is in or out as a whole
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_lanes; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row_lanes = 32 * (int64_t)nwx, r = t / row_lanes;
        const int I = (int)(t - r * row_lanes);
        const int l = I < nx ? cell_label(cell_pkg, pkg_type, pt_plus, pt_minus, (int64_t)I + (int64_t)nx * r) : CC_BLOCK;
        const unsigned po = __ballot_sync(0xffffffffu, l == 1);
        const unsigned mo = __ballot_sync(0xffffffffu, l == -1);
        const unsigned op = __ballot_sync(0xffffffffu, l != CC_BLOCK);
        if ((threadIdx.x & 31) == 0) {
            const int64_t w = t >> 5;
            open[w] = op;
            plus[w] = po;
            minus[w] = mo;
        }
    }
}

// One word of a cell sweep: an unknown open cell takes + where more of its
// face neighbours are + than -, - where more are -, exactly as the sign of
// the sum of their signs (blocked and unknown neighbours count 0;
// neighbours outside the mesh do not exist).  Returns whether a label was
// set.
template <bool L2>
__device__ __forceinline__ bool cell_sweep_one(const uint32_t* __restrict__ open, const uint32_t* p_in,
                                               const uint32_t* m_in, uint32_t* p_out, uint32_t* m_out, int64_t w,
                                               int nwx, int ny, int nz) {
    const uint32_t P = ld_lab<L2>(p_in + w), M = ld_lab<L2>(m_in + w);
    const uint32_t U = __ldg(open + w) & ~(P | M);
    uint32_t Pn = P, Mn = M;
    bool changed = false;
    if (U) {
        // 32-bit index arithmetic: nw <= nx ny nz < 2^31
        const uint32_t u = (uint32_t)w, r = u / (uint32_t)nwx, x = u - r * (uint32_t)nwx;
        const uint32_t K = r / (uint32_t)ny, J = r - K * (uint32_t)ny;
        const int64_t sy = nwx, sz = (int64_t)nwx * ny;
        const bool xl = x > 0, xr = x + 1 < (uint32_t)nwx, yl = J > 0, yr = J + 1 < (uint32_t)ny, zl = K > 0,
                   zr = K + 1 < (uint32_t)nz;
        const uint32_t Pl = xl ? ld_lab<L2>(p_in + w - 1) : 0u, Pr = xr ? ld_lab<L2>(p_in + w + 1) : 0u;
        const uint32_t Ml = xl ? ld_lab<L2>(m_in + w - 1) : 0u, Mr = xr ? ld_lab<L2>(m_in + w + 1) : 0u;
        const uint32_t pa[6] = {(P << 1) | (Pl >> 31), (P >> 1) | (Pr << 31),
                                yl ? ld_lab<L2>(p_in + w - sy) : 0u, yr ? ld_lab<L2>(p_in + w + sy) : 0u,
                                zl ? ld_lab<L2>(p_in + w - sz) : 0u, zr ? ld_lab<L2>(p_in + w + sz) : 0u};
        const uint32_t ma[6] = {(M << 1) | (Ml >> 31), (M >> 1) | (Mr << 31),
                                yl ? ld_lab<L2>(m_in + w - sy) : 0u, yr ? ld_lab<L2>(m_in + w + sy) : 0u,
                                zl ? ld_lab<L2>(m_in + w - sz) : 0u, zr ? ld_lab<L2>(m_in + w + sz) : 0u};
        uint32_t gt, lt;
        majority(pa, ma, gt, lt);
        Pn |= U & gt;
        Mn |= U & lt;
        changed = (U & (gt | lt)) != 0u;
    }
    p_out[w] = Pn;
    m_out[w] = Mn;
    return changed;
}

// one Jacobi sweep of the cell flood, a thread per word
__global__ void __launch_bounds__(CC_THREADS) k_cc_flood_words(const uint32_t* __restrict__ open,
                                                                const uint32_t* __restrict__ p_in,
                                                                const uint32_t* __restrict__ m_in,
                                                                uint32_t* __restrict__ p_out, uint32_t* __restrict__ m_out,
                                                                int nwx, int ny, int nz, int* flag) {
    const int64_t nw = (int64_t)nwx * ny * nz;
    bool changed = false;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
        changed |= cell_sweep_one<false>(open, p_in, m_in, p_out, m_out, w, nwx, ny, nz);
    flag_if_any(changed, flag);
}

// ---------------------------------------------------------------------------
// Persistent floods: every sweep of a flood in one cooperative launch (all
// CTAs resident), the sweeps separated by a grid barrier of the library's
// own whose waits are bounded: a CTA that waits longer than CC_SPIN_LIMIT
// polls sets `err` and returns, and the others then give up at their next
// barrier, so the launch always ends.  `chg` rotates over three slots: the
// slot of sweep s is final after barrier s, read by every CTA, and cleared
// (as slot s + 2) by CTA 0 after barrier s + 1, when every CTA has read it.
struct FloodSync {
    unsigned arrive;   // CTAs arrived at the current barrier
    unsigned gen;      // barriers completed
    int chg[3];        // per-sweep change flags
    int err;           // 1: a barrier wait gave up, 2: no fixed point within the sweep bound
    int sweeps;        // sweeps up to and including the first that changed nothing
    unsigned absent;   // CTAs counted at every barrier that never arrive: 0, or 1 to test the bounded waits
};
// 2^21 polls, each a load of the barrier word and a __nanosleep(32): at least
// 67 ms; 0.54 s measured on a B300 for the small sphere (the give-up is timed
// by the consistency tests)
constexpr unsigned CC_SPIN_LIMIT = 1u << 21;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// all CTAs of the launch; false when a wait gave up (then `err` is set)
__device__ bool grid_barrier(FloodSync* fs, unsigned& gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gen + 1;
        __threadfence();  // this CTA's label stores and flag updates before its arrival
        if (atomicAdd(&fs->arrive, 1u) == gridDim.x - 1 + fs->absent) {
            atomicExch(&fs->arrive, 0u);  // reset before the release: no CTA arrives again before it
            __threadfence();
            atomicExch(&fs->gen, target);
        } else {
            unsigned polls = 0;
            while (ld_acquire(&fs->gen) != target) {
                if (++polls > CC_SPIN_LIMIT) {
                    atomicExch(&fs->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        gen = target;
        s_ok = ok && ld_acquire((const unsigned*)&fs->err) == 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

// after barrier `sw`: whether the flood goes on (CTA 0 records the end)
__device__ __forceinline__ bool flood_continues(FloodSync* fs, int64_t sw) {
    const unsigned c = ld_acquire((const unsigned*)&fs->chg[sw % 3]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        fs->chg[(sw + 2) % 3] = 0;
        if (c == 0u) fs->sweeps = (int)(sw + 1);
    }
    return c != 0u;
}

// a = plus plane then minus plane (P words each), b the same; the fixed
// point ends in both
__global__ void __launch_bounds__(CC_THREADS) k_cc_flood_points_coop(const int32_t* __restrict__ faces, uint64_t* a,
                                                                      uint64_t* b, int64_t P, int64_t max_sweeps,
                                                                      FloodSync* fs) {
    unsigned gen = 0;
    for (int64_t sw = 0; sw < max_sweeps; ++sw) {
        const uint64_t* src = (sw & 1) ? b : a;
        uint64_t* dst = (sw & 1) ? a : b;
        bool changed = false;
        for (int64_t p = 2 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
             p += (int64_t)gridDim.x * blockDim.x)
            changed |= point_sweep_one<true>(faces, src, src + P, dst, dst + P, p);
        flag_if_any(changed, &fs->chg[sw % 3]);
        if (!grid_barrier(fs, gen)) return;
        if (!flood_continues(fs, sw)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&fs->err, 2);
}

// a = plus plane then minus plane (nw words each), b the same
__global__ void __launch_bounds__(CC_THREADS) k_cc_flood_words_coop(const uint32_t* __restrict__ open, uint32_t* a,
                                                                     uint32_t* b, int nwx, int ny, int nz,
                                                                     int64_t max_sweeps, FloodSync* fs) {
    const int64_t nw = (int64_t)nwx * ny * nz;
    unsigned gen = 0;
    for (int64_t sw = 0; sw < max_sweeps; ++sw) {
        const uint32_t* src = (sw & 1) ? b : a;
        uint32_t* dst = (sw & 1) ? a : b;
        bool changed = false;
        for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
            changed |= cell_sweep_one<true>(open, src, src + nw, dst, dst + nw, w, nwx, ny, nz);
        flag_if_any(changed, &fs->chg[sw % 3]);
        if (!grid_barrier(fs, gen)) return;
        if (!flood_continues(fs, sw)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&fs->err, 2);
}

// far cells take their label's far package; counts the moves
__global__ void __launch_bounds__(CC_THREADS) k_cc_far(int32_t* __restrict__ cell_pkg, const uint32_t* __restrict__ plus,
                                                        const uint32_t* __restrict__ minus, int nx, int nwx, int64_t nc,
                                                        unsigned long long* count) {
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = cell_pkg[e];
        if (p < 2) {
            const uint32_t u = (uint32_t)e, r = u / (uint32_t)nx, I = u - r * (uint32_t)nx;
            const int64_t w = (int64_t)r * nwx + (I >> 5);
            const uint32_t bit = 1u << (I & 31);
            const int l = (plus[w] & bit) ? 1 : ((minus[w] & bit) ? -1 : 0);
            if (l != 0) {
                const int32_t want = l < 0 ? 0 : 1;
                if (p != want) {
                    cell_pkg[e] = want;
                    ++c;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Jacobi sweeps in batches of CC_BATCH until one changes nothing; `a` ends
// on the fixed point and `sweeps` counts up to the first sweep that changed
// nothing.  Host-synchronising.
constexpr int CC_BATCH = 8;

template <class Sweep, class T>
cudaError_t flood(Sweep sweep, T*& a, T*& b, int* dflag, int* hflag, int64_t max_sweeps, int64_t& sweeps,
                  cudaStream_t s) {
    for (;;) {
        cudaError_t e = cudaMemsetAsync(dflag, 0, CC_BATCH * sizeof(int), s);
        for (int k = 0; k < CC_BATCH && e == cudaSuccess; ++k) {
            sweep(a, b, dflag + k);
            e = cudaGetLastError();
            T* t = a;
            a = b;
            b = t;
            ++sweeps;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, dflag, CC_BATCH * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (hflag[CC_BATCH - 1] == 0) {  // count up to the first sweep that changed nothing
            int k = 0;
            while (hflag[k] != 0) ++k;
            sweeps -= CC_BATCH - 1 - k;
            return cudaSuccess;
        }
        if (sweeps > max_sweeps) return cudaErrorLaunchTimeout;  // cannot happen: every sweep labels an entry
    }
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// words of one bit plane of the cell flood
int64_t plane_words(const int32_t dims[3]) { return (int64_t)((dims[0] + 31) / 32) * dims[1] * dims[2]; }

// CTAs of a cooperative launch of `kernel`: all resident at once, at most
// three per SM (fewer CTAs at each barrier; on the h = 0.002 torus 1, 2
// and 3 per SM took 1.63, 1.35 and 1.34 ms for the correction, 4 per SM
// 1.57 ms, and 1.46 ms with 100 ns between polls),
// no more than the entries need; 0 when the device cannot launch
// cooperatively
int coop_blocks(const void* kernel, int64_t n, int device) {
    int coop = 0, per_sm = 0, sms = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, CC_THREADS, 0) != cudaSuccess || per_sm < 1)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) return 0;
    const int64_t need = (n + CC_THREADS - 1) / CC_THREADS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::min(per_sm, 3) * sms));
}

// One persistent flood: reset the sync block, launch, read back its end
// state (host-synchronising).  Gives cudaErrorLaunchTimeout when a barrier
// wait gave up or no fixed point came within the sweep bound.
template <class... Args>
cudaError_t run_coop_flood(void (*kernel)(Args...), int blocks, FloodSync* fs, FloodSync* hfs, unsigned absent,
                           int64_t& sweeps, cudaStream_t s, Args... args) {
    *hfs = FloodSync{};  // pinned; free: the stream was synchronised after the last read-back
    hfs->absent = absent;
    cudaError_t e = cudaMemcpyAsync(fs, hfs, sizeof(FloodSync), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    void* argv[] = {(void*)&args...};
    e = cudaLaunchCooperativeKernel((const void*)kernel, dim3((unsigned)blocks), dim3(CC_THREADS), argv, 0, s);
    note_launch();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hfs, fs, sizeof(FloodSync), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (hfs->err != 0) return cudaErrorLaunchTimeout;
    sweeps = hfs->sweeps;
    return cudaSuccess;
}

}  // namespace

bool consistency_persistent(int device) {
    int coop = 0;
    return cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) == cudaSuccess && coop != 0;
}

size_t consistency_scratch_bytes(int64_t P, const int32_t dims[3]) {
    const size_t plane = (size_t)plane_words(dims) * sizeof(uint32_t);
    return 2 * al256(2 * (size_t)P * sizeof(uint64_t)) + al256(plane) + 2 * al256(2 * plane) + 256;
}

cudaError_t run_consistency(const GridFF& G, int64_t P, int64_t nc, int32_t* cell_pkg, const int32_t* pkg_cell,
                            const uint8_t* pkg_type, int32_t* nbr, int32_t* faces, float* phi, float tau,
                            void* scratch, void* host_pin, int64_t out[4], cudaStream_t s, unsigned debug) {
    const unsigned absent_pt = debug & SG_DEBUG_CC_ABSENT_POINTS ? 1u : 0u;
    const unsigned absent_cell = debug & SG_DEBUG_CC_ABSENT_CELLS ? 1u : 0u;
    const bool per_sweep = (debug & SG_DEBUG_CC_PER_SWEEP) != 0;
    char* sp = (char*)scratch;
    uint64_t* sa = (uint64_t*)sp;  // point planes: plus (P words), then minus (P words)
    sp += al256(2 * (size_t)P * sizeof(uint64_t));
    uint64_t* sb = (uint64_t*)sp;
    sp += al256(2 * (size_t)P * sizeof(uint64_t));
    const int nx = G.dims[0], ny = G.dims[1], nz = G.dims[2], nwx = (nx + 31) / 32;
    const int64_t nw = plane_words(G.dims);
    uint32_t* open = (uint32_t*)sp;
    sp += al256((size_t)nw * sizeof(uint32_t));
    uint32_t* la = (uint32_t*)sp;  // plus plane, then minus plane
    sp += al256(2 * (size_t)nw * sizeof(uint32_t));
    uint32_t* lb = (uint32_t*)sp;
    sp += al256(2 * (size_t)nw * sizeof(uint32_t));
    int* dflag = (int*)sp;                                               // CC_BATCH ints, or
    FloodSync* fs = (FloodSync*)sp;                                      // the persistent floods' sync block
    unsigned long long* cnt = (unsigned long long*)(sp + 64);            // 2 counters
    int* hflag = (int*)host_pin;                                         // the same on the host
    FloodSync* hfs = (FloodSync*)host_pin;
    unsigned long long* hcnt = (unsigned long long*)((char*)host_pin + 64);  // 2 counters
    static_assert(sizeof(FloodSync) <= 64 && CC_BATCH * sizeof(int) <= 64, "sync block and flags fit 64 bytes");
    int device = 0;
    cudaGetDevice(&device);
    const int64_t n_act = (P - 2) * PKG3;
    cudaError_t e;
    if ((e = cudaMemsetAsync(sa, 0, 2 * (size_t)P * sizeof(uint64_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sb, 0, 2 * (size_t)P * sizeof(uint64_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    int64_t sweeps_pt = 0, sweeps_cell = 0;
    if (n_act > 0) {
        k_cc_seed_points<<<cc_blocks(n_act), CC_THREADS, 0, s>>>(phi, (uint32_t*)sa, (uint32_t*)(sa + P), n_act, tau);
        note_launch();
        const int cbp = per_sweep ? 0 : coop_blocks((const void*)k_cc_flood_points_coop, P - 2, device);
        if (cbp > 0) {
            e = run_coop_flood(k_cc_flood_points_coop, cbp, fs, hfs, absent_pt, sweeps_pt, s, (const int32_t*)faces, sa, sb,
                               P, n_act + 1, fs);
        } else {
            const unsigned nb = cc_blocks(P - 2);
            e = flood(
                [&](const uint64_t* src, uint64_t* dst, int* flag) {
                    k_cc_flood_points<<<nb, CC_THREADS, 0, s>>>(faces, src, src + P, dst, dst + P, P, flag);
                    note_launch();
                },
                sa, sb, dflag, hflag, n_act + 1, sweeps_pt, s);
        }
        if (e != cudaSuccess) return e;
    }
    k_cc_seed_words<<<cc_blocks(32 * nw), CC_THREADS, 0, s>>>(cell_pkg, pkg_type, sa, sa + P, open, la, la + nw, nx, nwx,
                                                              32 * nw);
    note_launch();
    const int cbw = per_sweep ? 0 : coop_blocks((const void*)k_cc_flood_words_coop, nw, device);
    if (cbw > 0) {
        e = run_coop_flood(k_cc_flood_words_coop, cbw, fs, hfs, absent_cell, sweeps_cell, s, (const uint32_t*)open, la, lb,
                           nwx, ny, nz, nc + 1, fs);
    } else {
        const unsigned cb = cc_blocks(nw);
        e = flood(
            [&](const uint32_t* src, uint32_t* dst, int* flag) {
                k_cc_flood_words<<<cb, CC_THREADS, 0, s>>>(open, src, src + nw, dst, dst + nw, nwx, ny, nz, flag);
                note_launch();
            },
            la, lb, dflag, hflag, nc + 1, sweeps_cell, s);
    }
    if (e != cudaSuccess) return e;
    // both floods settled: only now are phi and the tables changed, so that a
    // flood that gives up leaves the grid as it was (the cell flood reads the
    // point labels, never phi)
    if (n_act > 0) {
        k_cc_apply<<<cc_blocks(n_act / 4), CC_THREADS, 0, s>>>(reinterpret_cast<float4*>(phi), (const uint32_t*)sa,
                                                                (const uint32_t*)(sa + P), n_act / 4, cnt);
        note_launch();
    }
    k_cc_far<<<cc_blocks(nc), CC_THREADS, 0, s>>>(cell_pkg, la, la + nw, nx, nwx, nc, cnt + 1);
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
