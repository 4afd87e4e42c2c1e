// sg_tag.cu -- band tagging, package numbering, neighbourhood table and
// initial level-set values ("Initialization Process", steps 1-5).
//
// One thread per background cell for the flags, one per (package, entry)
// for the table, one per data point for the level set.  All integer
// results are exact; the only floating-point decision (core or not) is
// taken on a float-float distance.
#include "sg_internal.cuh"

namespace sg {
namespace {

constexpr int TAG_THREADS = 256;

// Launch the instantiation of a shape-templated kernel for kind `kind` (the
// statement `launch` names it with template argument K).
#define SG_SHAPE_DISPATCH(kind, launch)                         \
    do {                                                        \
        switch (kind) {                                         \
        case SHAPE_SPHERE: { constexpr int K = SHAPE_SPHERE; launch; } break;           \
        case SHAPE_PLANE: { constexpr int K = SHAPE_PLANE; launch; } break;             \
        case SHAPE_TORUS: { constexpr int K = SHAPE_TORUS; launch; } break;             \
        case SHAPE_PRISM: { constexpr int K = SHAPE_PRISM; launch; } break;             \
        case SHAPE_ROUNDED_BOX: { constexpr int K = SHAPE_ROUNDED_BOX; launch; } break; \
        default: { constexpr int K = SHAPE_SHELL; launch; } break;                      \
        }                                                       \
    } while (0)

// Cell (I, J, K) of linear index c = I + nx (J + ny K).  Grids hold fewer
// than 2^31 cells, so two 32-bit divisions suffice.
__device__ __forceinline__ void cell_coords(int64_t c, const int* dims, int64_t& I, int64_t& J, int64_t& K) {
    const uint32_t u = (uint32_t)c, nx = (uint32_t)dims[0], ny = (uint32_t)dims[1];
    const uint32_t q = u / nx, k = q / ny;
    I = u - q * nx;
    J = q - k * ny;
    K = k;
}

// Step 1: core cells, |d(centre)| < T; far cells keep the sign of d.  The
// distance is first evaluated in float; when it is farther than `margin`
// from both T and 0 in magnitude, the float decision stands (the float error
// of these formulas is below 1e-6 (1 + |x|), the margin is 1.5e-4 (1 + |x|)),
// otherwise it is decided on the float-float distance.
template <int K>
__device__ __forceinline__ uint8_t classify_cell(const GridFF& G, const ShapeFF& S, const int64_t (&I)[3]) {
    const float Tf = G.T.hi;
    float xf[3];
    float xmax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xf[a] = G.lo[a].hi + G.h.hi * (float)(4 * (int)I[a] + 2);
        xmax = fmaxf(xmax, fabsf(xf[a]));
    }
    const float df = f_sdf_k<K>(S, xf);
    const float margin = 1.5e-4f * (1.0f + xmax);
    if (fabsf(fabsf(df) - Tf) > margin && fabsf(df) > margin) return fabsf(df) < Tf ? 2 : (df < 0.0f ? 0 : 1);
    ff x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = ff_add(G.lo[a], ff_mul_f(G.h, (float)(4 * (int)I[a] + 2)));
    const ff d = ff_sdf_k<K>(S, x);
    return ff_lt(ff_abs(d), G.T) ? 2 : (ff_neg_p(d) ? 0 : 1);
}

// Step 1 over all cells; bit i of core_bits[w] flags cell 32 w + i core.
// A warp classifies 32 consecutive cells (its first cell a multiple of 32).
template <int K>
__global__ void __launch_bounds__(TAG_THREADS) k_tag_flags(GridFF G, ShapeFF S, uint8_t* __restrict__ cell_type,
                                                            uint32_t* __restrict__ core_bits, int64_t nc) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < nc;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = base + lane;
        uint8_t t = 0;
        if (c < nc) {
            int64_t I[3];
            cell_coords(c, G.dims, I[0], I[1], I[2]);
            t = classify_cell<K>(G, S, I);
            cell_type[c] = t;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, c < nc && t == 2);
        if (lane == 0) core_bits[base >> 5] = m;
    }
}

// Step 1 of a finer layer ("Multi-resolution Level-set"): only the cells
// covered by a core cell of the coarser layer (same lo, half the dims, twice
// the spacing) evaluate their distance; every other cell is far, inside when
// its coarse cell is far inside or is an inner cell whose level set (data
// point 0) is negative.  A fine cell inside a coarse cell that is not core
// lies at least 1.13 fine cells from the surface, so it cannot be core.
template <int K>
__global__ void __launch_bounds__(TAG_THREADS) k_tag_flags_from(GridFF G, ShapeFF S, const int32_t* __restrict__ c_cell_pkg,
                                                                 const uint8_t* __restrict__ c_pkg_type,
                                                                 const float* __restrict__ c_phi, int cnx, int cny,
                                                                 uint8_t* __restrict__ cell_type,
                                                                 uint32_t* __restrict__ core_bits, int64_t nc,
                                                                 unsigned long long* __restrict__ evaluated) {
    unsigned long long ev = 0;
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < nc;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = base + lane;
        uint8_t t = 0;
        if (c < nc) {
            int64_t I[3];
            cell_coords(c, G.dims, I[0], I[1], I[2]);
            const int64_t pc = __ldg(c_cell_pkg + (I[0] >> 1) + cnx * ((I[1] >> 1) + (int64_t)cny * (I[2] >> 1)));
            if (pc >= 2 && __ldg(c_pkg_type + pc) == 2) {
                t = classify_cell<K>(G, S, I);
                ++ev;
            } else {
                t = (pc < 2 ? pc == 0 : __ldg(c_phi + pc * PKG3) < 0.0f) ? 0 : 1;
            }
            cell_type[c] = t;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, c < nc && t == 2);
        if (lane == 0) core_bits[base >> 5] = m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_down_sync(0xffffffffu, ev, o);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd(evaluated, ev);
}

// Bits of cells s .. s + 31 of a bit mask (zero outside its nw words).
__device__ __forceinline__ uint32_t bit_window(const uint32_t* __restrict__ bits, int64_t nw, int64_t s) {
    const int64_t q = s >> 5;  // floor division, also for s < 0
    const uint32_t lo = (q >= 0 && q < nw) ? bits[q] : 0u;
    const uint32_t hi = (q + 1 >= 0 && q + 1 < nw) ? bits[q + 1] : 0u;
    return __funnelshift_r(lo, hi, (int)(s & 31));
}

// Step 2: inner cells, not core and one of the 26 neighbours is core, on
// bit masks: a thread takes the 32 cells of word w, gathers the core bits
// of their 27-cell neighbourhoods as 27 shifted windows of the core mask
// (cell c + dx + nx dy + nx ny dz at bit i for cell c = 32 w + i), each
// window cleared where its move leaves the domain (cells in the first or
// last column, row or plane).  Writes the active mask (core or inner), its
// population per word and type 3 for the inner cells.
__global__ void __launch_bounds__(TAG_THREADS) k_tag_inner(GridFF G, uint8_t* __restrict__ cell_type,
                                                            const uint32_t* __restrict__ core,
                                                            uint32_t* __restrict__ act, uint32_t* __restrict__ count,
                                                            int64_t nc) {
    pdl_enter();
    const int nx = G.dims[0], ny = G.dims[1], nz = G.dims[2];
    const int64_t nw = (nc + 31) >> 5, plane = (int64_t)nx * ny;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c0 = w << 5;
        const int nvalid = (int)min((int64_t)32, nc - c0);
        int64_t I, J, K;
        cell_coords(c0, G.dims, I, J, K);
        int i = (int)I, j = (int)J, k = (int)K;
        uint32_t xl = 0, xh = 0, yl = 0, yh = 0, zl = 0, zh = 0;
        for (int b = 0; b < nvalid; ++b) {
            const uint32_t bit = 1u << b;
            xl |= i == 0 ? bit : 0u;
            xh |= i == nx - 1 ? bit : 0u;
            yl |= j == 0 ? bit : 0u;
            yh |= j == ny - 1 ? bit : 0u;
            zl |= k == 0 ? bit : 0u;
            zh |= k == nz - 1 ? bit : 0u;
            if (++i == nx) {
                i = 0;
                if (++j == ny) {
                    j = 0;
                    ++k;
                }
            }
        }
        uint32_t near = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const uint32_t mz = dz < 0 ? ~zl : (dz > 0 ? ~zh : ~0u);
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const uint32_t m = mz & (dy < 0 ? ~yl : (dy > 0 ? ~yh : ~0u));
                const int64_t s = c0 + dy * (int64_t)nx + dz * plane;
                near |= m & ((bit_window(core, nw, s - 1) & ~xl) | bit_window(core, nw, s) |
                             (bit_window(core, nw, s + 1) & ~xh));
            }
        }
        const uint32_t valid = nvalid == 32 ? 0xffffffffu : (1u << nvalid) - 1u;
        const uint32_t cw = core[w];
        const uint32_t inner = near & ~cw & valid;
        act[w] = cw | inner;
        count[w] = __popc(cw | inner);
        for (uint32_t m = inner; m; m &= m - 1) cell_type[c0 + __ffs(m) - 1] = 3;
    }
}

// Step 3: ids in increasing cell index = 2 + number of active cells before
// c: the scanned population of the words before c's word plus the active
// bits below c's bit.
__global__ void __launch_bounds__(TAG_THREADS) k_tag_scatter(const uint8_t* __restrict__ cell_type,
                                                              const uint32_t* __restrict__ act,
                                                              const uint32_t* __restrict__ prefix,
                                                              int32_t* __restrict__ cell_pkg,
                                                              int32_t* __restrict__ pkg_cell,
                                                              uint8_t* __restrict__ pkg_type, int64_t nc) {
    if (blockIdx.x == 0 && threadIdx.x < 2) {
        pkg_cell[threadIdx.x] = -1;
        pkg_type[threadIdx.x] = (uint8_t)threadIdx.x;
    }
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        uint8_t t = cell_type[c];
        if (t >= 2) {
            const int64_t w = c >> 5;
            const uint32_t below = act[w] & ((1u << (c & 31)) - 1u);
            const int32_t id = 2 + (int32_t)(prefix[w] + __popc(below));
            cell_pkg[c] = id;
            pkg_cell[id] = (int32_t)c;
            pkg_type[id] = t;
        } else {
            cell_pkg[c] = t;
        }
    }
}

// Step 5: neighbourhood; outside the domain -> package 1; far packages self.
// A thread takes one row (dy, dz) of three entries of a package: the
// package's cell coordinates once per row, the three x-neighbours from one
// stretch of cell_pkg, and 12 contiguous bytes of the table.
__global__ void __launch_bounds__(TAG_THREADS) k_fill_nbr(GridFF G, const int32_t* __restrict__ cell_pkg,
                                                           const int32_t* __restrict__ pkg_cell,
                                                           int32_t* __restrict__ nbr, int64_t P) {
    pdl_enter();
    const int nx = G.dims[0], ny = G.dims[1], nz = G.dims[2];
    const int64_t total = P * 9;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / 9;
        const int row = (int)(e - p * 9);  // row = (dy + 1) + 3 (dz + 1)
        int32_t* out = nbr + p * NB + 3 * row;
        if (p < 2) {
            out[0] = out[1] = out[2] = (int32_t)p;
            continue;
        }
        int64_t I, J, K;
        cell_coords(pkg_cell[p], G.dims, I, J, K);
        const int b = (int)J + row % 3 - 1, c = (int)K + row / 3 - 1;
        const bool in_yz = b >= 0 && c >= 0 && b < ny && c < nz;
        const int64_t base = (int64_t)nx * (b + (int64_t)ny * c);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int a = (int)I + dx;
            out[dx + 1] = in_yz && a >= 0 && a < nx ? cell_pkg[base + a] : 1;
        }
    }
}

// Compact face table: entries 12, 14, 10, 16, 4, 22 of each neighbourhood.
__global__ void __launch_bounds__(TAG_THREADS) k_fill_faces(const int32_t* __restrict__ nbr,
                                                             int32_t* __restrict__ faces, int64_t P) {
    pdl_enter();
    const int face_n[8] = {12, 14, 10, 16, 4, 22, -1, -1};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * 8;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(e & 7);
        faces[e] = face_n[f] < 0 ? 0 : nbr[(e >> 3) * NB + face_n[f]];
    }
}

// Table check: every id in range, far packages their own neighbours, each
// active package its own centre entry and its cell's package, every
// neighbour entry the package of that neighbour cell (1 outside the domain),
// the face rows copies of the neighbour rows, every cell's package in range
// and naming it back.  Every read is bounds-checked first; an inconsistency
// sets ERR_BAD_INDEX in *err.
__global__ void __launch_bounds__(TAG_THREADS) k_check_tables(GridFF G, const int32_t* __restrict__ cell_pkg,
                                                               const int32_t* __restrict__ pkg_cell,
                                                               const uint8_t* __restrict__ pkg_type,
                                                               const int32_t* __restrict__ nbr,
                                                               const int32_t* __restrict__ faces, int64_t P,
                                                               int64_t nc, int* err) {
    const int face_n[6] = {12, 14, 10, 16, 4, 22};
    const int64_t nx = G.dims[0], ny = G.dims[1], nz = G.dims[2];
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P + nc; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < P) {
            const int64_t p = e;
            const int32_t* row = nbr + p * NB;
            for (int n = 0; n < NB; ++n) bad |= row[n] < 0 || row[n] >= P || (p < 2 && row[n] != p);
            if (p >= 2) {
                bad |= row[13] != p || pkg_type[p] < 2 || pkg_type[p] > 3;
                const int64_t c = pkg_cell[p];
                if (c < 0 || c >= nc) {
                    bad = true;
                } else {
                    bad |= cell_pkg[c] != p;
                    const int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
                    for (int n = 0; n < NB; ++n) {
                        const int64_t a = I + n % 3 - 1, b = J + (n / 3) % 3 - 1, k = K + n / 9 - 1;
                        const bool in = a >= 0 && b >= 0 && k >= 0 && a < nx && b < ny && k < nz;
                        bad |= row[n] != (in ? cell_pkg[a + nx * (b + ny * k)] : 1);
                    }
                }
            }
            for (int f = 0; f < 6; ++f) bad |= faces[p * 8 + f] != row[face_n[f]];
            bad |= faces[p * 8 + 6] != 0 || faces[p * 8 + 7] != 0;
        } else {
            const int64_t c = e - P;
            const int64_t v = cell_pkg[c];
            if (v < 0 || v >= P)
                bad = true;
            else if (v >= 2)
                bad |= pkg_cell[v] != c;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_BAD_INDEX);
}

// Step 4: phi at cell-centred data points, float-float, rounded once.
// The fine lattice coordinates lo_a + (e + 1/2) h, e = 4 I + l in
// [0, 4 dims_a), of the three axes in float-float, one after the other:
// the data points' coordinates, tabulated once per call.
__global__ void __launch_bounds__(TAG_THREADS) k_coord_table(GridFF G, ff* __restrict__ tab) {
    pdl_enter();
    const int n0 = 4 * G.dims[0], n1 = 4 * G.dims[1], n = n0 + n1 + 4 * G.dims[2];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int a = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
        const int m = e - (a == 0 ? 0 : (a == 1 ? n0 : n0 + n1));
        tab[e] = ff_add(G.lo[a], ff_mul_f(G.h, (float)m + 0.5f));
    }
}

template <int K>
__global__ void __launch_bounds__(TAG_THREADS, K == SHAPE_PRISM ? 4 : 8) k_init_sdf(GridFF G, ShapeFF S, const int32_t* __restrict__ pkg_cell,
                                                           const ff* __restrict__ tab, float* __restrict__ phi,
                                                           int64_t P, float F) {
    write_far(phi, -F, F);
    const int64_t total = (P - 2) * PKG3;
    const int off[3] = {0, 4 * G.dims[0], 4 * (G.dims[0] + G.dims[1])};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = 2 + e / PKG3;
        int d = (int)(e & (PKG3 - 1));
        int64_t I[3];
        cell_coords(pkg_cell[p], G.dims, I[0], I[1], I[2]);
        const int l[3] = {d & 3, (d >> 2) & 3, d >> 4};
        ff x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float2 v = __ldg(reinterpret_cast<const float2*>(tab) + off[a] + 4 * (int)I[a] + l[a]);
            x[a] = ff{v.x, v.y};
        }
        phi[p * PKG3 + d] = ff_to_float(ff_sdf_k<K>(S, x));
    }
}

// Plain torus and prism (no rotation, centre at the origin): a thread per
// package column (i, j) forms the column part of the distance once and
// finishes it at the column's four points along z (the same operations per
// point as k_init_sdf).
template <int K>
__global__ void __launch_bounds__(TAG_THREADS, K == SHAPE_PRISM ? 4 : 8) k_init_sdf_col(GridFF G, ShapeFF S,
                                                               const int32_t* __restrict__ pkg_cell,
                                                               const ff* __restrict__ tab, float* __restrict__ phi,
                                                               int64_t P, float F) {
    pdl_enter();
    write_far(phi, -F, F);
    const int64_t total = (P - 2) * 16;
    const int off[3] = {0, 4 * G.dims[0], 4 * (G.dims[0] + G.dims[1])};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = 2 + e / 16;
        const int c = (int)(e & 15), i = c & 3, j = c >> 2;
        int64_t I[3];
        cell_coords(pkg_cell[p], G.dims, I[0], I[1], I[2]);
        const float2 vx = __ldg(reinterpret_cast<const float2*>(tab) + off[0] + 4 * (int)I[0] + i);
        const float2 vy = __ldg(reinterpret_cast<const float2*>(tab) + off[1] + 4 * (int)I[1] + j);
        const ff col = ff_column_k<K>(S, ff{vx.x, vx.y}, ff{vy.x, vy.y});
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 vz = __ldg(reinterpret_cast<const float2*>(tab) + off[2] + 4 * (int)I[2] + k);
            phi[p * PKG3 + i + 4 * j + 16 * k] = ff_to_float(ff_finish_k<K>(S, col, ff{vz.x, vz.y}));
        }
    }
}

unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;  // grid-stride beyond
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_tag_flags(const GridFF& G, const ShapeFF& S, uint8_t* cell_type, uint32_t* core_bits, int64_t nc,
                             cudaStream_t s) {
    SG_SHAPE_DISPATCH(S.kind, (k_tag_flags<K><<<grid_for(nc, TAG_THREADS), TAG_THREADS, 0, s>>>(G, S, cell_type, core_bits,
                                                                                                nc)));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tag_flags_from(const GridFF& G, const ShapeFF& S, const int32_t* c_cell_pkg,
                                  const uint8_t* c_pkg_type, const float* c_phi, int cnx, int cny, uint8_t* cell_type,
                                  uint32_t* core_bits, int64_t nc, unsigned long long* evaluated, cudaStream_t s) {
    SG_SHAPE_DISPATCH(S.kind, (k_tag_flags_from<K><<<grid_for(nc, TAG_THREADS), TAG_THREADS, 0, s>>>(
                                  G, S, c_cell_pkg, c_pkg_type, c_phi, cnx, cny, cell_type, core_bits, nc, evaluated)));
    note_launch();
    return cudaGetLastError();
}

// Morton package ids: cell centres of the active packages (linear ids), for
// the Morton sort; then every package moves to its rank in that order.
__global__ void __launch_bounds__(TAG_THREADS) k_cell_centres(GridF G, const int32_t* __restrict__ pkg_cell,
                                                               float* __restrict__ x, float* __restrict__ y,
                                                               float* __restrict__ z, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = pkg_cell[2 + r];
        const int64_t I = c % G.dims[0], J = (c / G.dims[0]) % G.dims[1], K = c / ((int64_t)G.dims[0] * G.dims[1]);
        x[r] = G.lo[0] + G.h * (float)(4 * I + 2);
        y[r] = G.lo[1] + G.h * (float)(4 * J + 2);
        z[r] = G.lo[2] + G.h * (float)(4 * K + 2);
    }
}

__global__ void __launch_bounds__(TAG_THREADS) k_renumber(const int32_t* __restrict__ order,
                                                           const int32_t* __restrict__ old_cell,
                                                           const uint8_t* __restrict__ old_type,
                                                           int32_t* __restrict__ pkg_cell, uint8_t* __restrict__ pkg_type,
                                                           int32_t* __restrict__ cell_pkg, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t was = 2 + order[r];
        const int32_t c = old_cell[was];
        pkg_cell[2 + r] = c;
        pkg_type[2 + r] = old_type[was];
        cell_pkg[c] = (int32_t)(2 + r);
    }
}

cudaError_t launch_check_tables(const GridFF& G, const int32_t* cell_pkg, const int32_t* pkg_cell,
                                const uint8_t* pkg_type, const int32_t* nbr, const int32_t* faces, int64_t P,
                                int64_t nc, int* err, cudaStream_t s) {
    k_check_tables<<<grid_for(P + nc, TAG_THREADS), TAG_THREADS, 0, s>>>(G, cell_pkg, pkg_cell, pkg_type, nbr, faces,
                                                                         P, nc, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_cell_centres(const GridF& G, const int32_t* pkg_cell, float* x, float* y, float* z, int64_t n,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cell_centres<<<grid_for(n, TAG_THREADS), TAG_THREADS, 0, s>>>(G, pkg_cell, x, y, z, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_renumber(const int32_t* order, const int32_t* old_cell, const uint8_t* old_type, int32_t* pkg_cell,
                            uint8_t* pkg_type, int32_t* cell_pkg, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_renumber<<<grid_for(n, TAG_THREADS), TAG_THREADS, 0, s>>>(order, old_cell, old_type, pkg_cell, pkg_type, cell_pkg,
                                                                n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tag_inner(const GridFF& G, uint8_t* cell_type, const uint32_t* core_bits, uint32_t* act_bits,
                             uint32_t* count, int64_t nc, cudaStream_t s) {
    const int64_t nw = (nc + 31) >> 5;
    return launch_pdl(k_tag_inner, grid_for(nw, TAG_THREADS), TAG_THREADS, 0, s, G, cell_type, core_bits, act_bits, count,
                      nc);
}

cudaError_t launch_tag_scatter(const uint8_t* cell_type, const uint32_t* act_bits, const uint32_t* prefix,
                               int32_t* cell_pkg, int32_t* pkg_cell, uint8_t* pkg_type, int64_t nc, cudaStream_t s) {
    k_tag_scatter<<<grid_for(nc, TAG_THREADS), TAG_THREADS, 0, s>>>(cell_type, act_bits, prefix, cell_pkg, pkg_cell,
                                                                     pkg_type, nc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill_nbr(const GridFF& G, const int32_t* cell_pkg, const int32_t* pkg_cell, int32_t* nbr,
                            int64_t P, cudaStream_t s) {
    return launch_pdl(k_fill_nbr, grid_for(P * 9, TAG_THREADS), TAG_THREADS, 0, s, G, cell_pkg, pkg_cell, nbr, P);
}

cudaError_t launch_fill_faces(const int32_t* nbr, int32_t* faces, int64_t P, cudaStream_t s) {
    return launch_pdl(k_fill_faces, grid_for(P * 8, TAG_THREADS), TAG_THREADS, 0, s, nbr, faces, P);
}

cudaError_t launch_init_sdf(const GridFF& G, const ShapeFF& S, const int32_t* pkg_cell, float* phi, float F,
                            int64_t P, void* table, cudaStream_t s) {
    if (P <= 2) return launch_set_far(phi, -F, F, s);  // otherwise the init kernel writes the far packages
    const int n = 4 * (G.dims[0] + G.dims[1] + G.dims[2]);
    cudaError_t e = launch_pdl(k_coord_table, (n + TAG_THREADS - 1) / TAG_THREADS, TAG_THREADS, 0, s, G, (ff*)table);
    if (e != cudaSuccess) return e;
    const ff* tab = (const ff*)table;
    if (S.plain && S.kind == SHAPE_TORUS)
        return launch_pdl(k_init_sdf_col<SHAPE_TORUS>, grid_for((P - 2) * 16, TAG_THREADS), TAG_THREADS, 0, s, G, S,
                          pkg_cell, tab, phi, P, F);
    if (S.plain && S.kind == SHAPE_PRISM)
        return launch_pdl(k_init_sdf_col<SHAPE_PRISM>, grid_for((P - 2) * 16, TAG_THREADS), TAG_THREADS, 0, s, G, S,
                          pkg_cell, tab, phi, P, F);
    else
        SG_SHAPE_DISPATCH(S.kind, (k_init_sdf<K><<<grid_for((P - 2) * PKG3, TAG_THREADS), TAG_THREADS, 0, s>>>(
                                      G, S, pkg_cell, tab, phi, P, F)));
    note_launch();
    return cudaGetLastError();
}

}  // namespace sg
