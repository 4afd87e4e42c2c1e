// sg_batch.cu -- many bodies in one launch per sweep.
//
// The packages of every body are concatenated into one global store: body b
// owns ids [base_b, base_b + P_b), its own far packages at base_b and
// base_b + 1, neighbour ids shifted by base_b, and a row of per-body
// constants (computed exactly as the single-grid launchers compute them, so
// a batched sweep equals the per-body sweeps bit for bit).  Each sweep is one
// persistent kernel: CTAs take work items of consecutive packages from an
// atomic counter until the store is exhausted, which balances bodies of very
// different sizes.  The whole sequence gradient -> smoothed sign -> reinit
// sweeps -> kernel integrals is captured once per plan into a CUDA graph and
// replayed.  The autotuner times every (packages per item, staging depth)
// pair and keeps the fastest.
//
// Relaxation ("Grid-Particle Coupling" as the surface force of particle
// relaxation): particles of all bodies, stored body after body, are probed
// and displaced by one kernel per step; the sweeps and every step are
// captured into one graph.
#include <cctype>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg_probe.cuh"
#include "sg_integrals.cuh"
#include "sg_mlp.cuh"
#include "sg_rows.cuh"

struct sg_batch_graph {
    sg_batch_plan plan;
    cudaGraphExec_t exec;
};

struct sg_relax_graph {
    sg_batch_plan plan;
    sg_relax r;
    std::vector<int64_t> offsets;
    cudaGraphExec_t exec = nullptr;
};

struct sg_batch {
    int n = 0;
    int64_t P = 0;  // packages of all bodies, far packages included
    std::vector<int64_t> base, npk, cell_base;
    std::vector<double> h, eps;
    std::vector<sg_grid_desc> desc;
    double R = 2.0;             // kernel support of every body, in units of its h
    bool default_kernel = true;  // every body has support 2h and eps = h (the surrogate's kernel)
    const sg_mlp* mlp = nullptr;  // surrogate of plans with integrals_mode 1
    sg_allocator alloc{};
    bool user_alloc = false;
    cudaStream_t stream = nullptr;   // caller's stream: graphs run here
    cudaStream_t capture = nullptr;  // private stream used only to capture
    int device = 0;
    sg::Buf phi, tmp, s0, phi0, f[8], nbr, faces, type, body, params, counters, cells, sur, relax, probe_tab;
    sg::Buf sur_work;  // list of network points of the surrogate integrals
    size_t n_counters = 0;
    float params_cfl = -1.0f;
    std::vector<sg_batch_graph> graphs;
    sg_relax_graph rx;
    std::string last_error;
};

namespace sg {
namespace {

// Per-body constants, in the form the single-grid launchers pass them.
struct BodyParams {
    float inv2h;    // 1 / (2h)
    float h2;       // h^2
    float cfl;      // dt / h with dt rounded to float first
    float dt;       // cfl h
    float inv_eps;  // 1 / h
    float F;        // far value
    float pad[2];
};

constexpr int BT = 256;       // threads per CTA
constexpr int BT_HW = BT / 16;  // half-warps (row kernels and integrals: packages per slot)

__device__ __forceinline__ int64_t next_item(unsigned* counter, int* s_item) {
    __syncthreads();
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_item;
}

// Gradient over the global store.  A work item is 16 * ppi consecutive
// packages; each half-warp handles ppi of them, DEPTH at a time.
template <int DEPTH>
__global__ void __launch_bounds__(BT) k_batch_gradient(const int32_t* __restrict__ faces, const uint8_t* __restrict__ type,
                                                       const int32_t* __restrict__ body,
                                                       const BodyParams* __restrict__ prm, const float* __restrict__ phi,
                                                       float* __restrict__ gx, float* __restrict__ gy,
                                                       float* __restrict__ gz, float* __restrict__ s0, int64_t P, int ppi,
                                                       unsigned* counter) {
    __shared__ int s_item;
    const int64_t per_item = (int64_t)BT_HW * ppi, items = (P + per_item - 1) / per_item;
    for (;;) {
        const int64_t item = next_item(counter, &s_item);
        if (item >= items) break;
        for (int k = 0; k < ppi; k += DEPTH) {
            RowSlot sl[DEPTH];
            Rows w[DEPTH];
            bool act[DEPTH];
            float inv2h[DEPTH], h2[DEPTH];
            // rows loaded for every package (as in the reinit sweep), stored for active ones
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) {
                const int64_t p = item * per_item + (int64_t)(k + d) * BT_HW + (threadIdx.x >> 4);
                const int64_t pc = p < P ? p : 0;
                sl[d] = make_slot(p, p < P && k + d < ppi);
                act[d] = sl[d].valid && __ldg(type + pc) >= 2;
                const BodyParams* bp = prm + __ldg(body + pc);
                inv2h[d] = __ldg(&bp->inv2h);
                h2[d] = __ldg(&bp->h2);
            }
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) w[d] = load_rows(phi, faces, sl[d]);
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) {
                if (!act[d]) continue;
                float4 ox, oy, oz;
                gradient_row(w[d], inv2h[d], ox, oy, oz);
                reinterpret_cast<float4*>(gx)[sl[d].q4] = ox;
                reinterpret_cast<float4*>(gy)[sl[d].q4] = oy;
                reinterpret_cast<float4*>(gz)[sl[d].q4] = oz;
                // the smoothed sign of the sweeps that follow, from the same row of phi
                float4 sg = w[d].c;
                sg.x = smoothed_sign(sg.x, h2[d]);
                sg.y = smoothed_sign(sg.y, h2[d]);
                sg.z = smoothed_sign(sg.z, h2[d]);
                sg.w = smoothed_sign(sg.w, h2[d]);
                reinterpret_cast<float4*>(s0)[sl[d].q4] = sg;
            }
        }
    }
}

// Reinit sweep over the global store: a work item is 16 * ppi packages, each
// half-warp takes ppi of them, DEPTH at a time; a package's body constants
// are read with its sign, ahead of the rows.  DEPTH 1 is bounded to 40
// registers (6 CTAs per SM), which it fits without spills.
template <int DEPTH>
__global__ void __launch_bounds__(BT, DEPTH == 1 ? 6 : 1) k_batch_reinit(const int32_t* __restrict__ faces, const uint8_t* __restrict__ type,
                                                     const int32_t* __restrict__ body,
                                                     const BodyParams* __restrict__ prm, const float* __restrict__ s0,
                                                     const float* __restrict__ phi_in, float* __restrict__ phi_out,
                                                     int64_t P, int ppi, unsigned* counter, int reverse) {
    __shared__ int s_item;
    const int64_t per_item = (int64_t)BT_HW * ppi, items = (P + per_item - 1) / per_item;
    for (;;) {
        int64_t item = next_item(counter, &s_item);
        if (item >= items) break;
        // every other sweep walks the store backwards (the first one, after the
        // forward gradient and smoothed-sign pass, among them), so that it starts on the
        // packages the previous pass left in L2 (the Jacobi results do not
        // depend on the order)
        if (reverse) item = items - 1 - item;
        for (int k = 0; k < ppi; k += DEPTH) {
            RowSlot sl[DEPTH];
            Rows w[DEPTH];
            float4 sg[DEPTH];
            float cfl[DEPTH], dtv[DEPTH];
            bool act[DEPTH];
            // the rows of every package in the store are loaded (a far package's
            // face rows name itself), so that the loads do not wait for the
            // package's type and body constants; only active packages store
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) {
                const int64_t p = item * per_item + (int64_t)(k + d) * BT_HW + (threadIdx.x >> 4);
                const int64_t pc = p < P ? p : 0;
                sl[d] = make_slot(p, p < P && k + d < ppi);
                act[d] = sl[d].valid && __ldg(type + pc) >= 2;
                const BodyParams* bp = prm + __ldg(body + pc);
                cfl[d] = __ldg(&bp->cfl);
                dtv[d] = __ldg(&bp->dt);
                sg[d] = sl[d].valid ? __ldg(reinterpret_cast<const float4*>(s0) + sl[d].q4)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) w[d] = load_rows(phi_in, faces, sl[d]);
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) {
                if (!act[d]) continue;
                reinterpret_cast<float4*>(phi_out)[sl[d].q4] = reinit_row(w[d], sg[d], cfl[d], dtv[d]);
            }
        }
    }
}

__global__ void k_batch_offset_nbr(const int32_t* __restrict__ src, int32_t* __restrict__ dst, int64_t n,
                                   int32_t offset) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e] + offset;
}

__global__ void k_batch_fill_body(int32_t* __restrict__ body, int64_t begin, int64_t n, int32_t b) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        body[begin + e] = b;
}

// far packages of every body: W = 1 inside, 0 outside
__global__ void k_batch_far_W(float* __restrict__ W, const int64_t* __restrict__ base, int n) {
    const int b = blockIdx.x;
    if (b >= n) return;
    W[base[b] * PKG3 + threadIdx.x] = threadIdx.x < PKG3 ? 1.0f : 0.0f;
}

// Per-body constants of the relaxation, in the form the single-grid probe
// uses them, plus the body's particle range and its first tile (CTA).
struct RelaxBody {
    ff lat_c[3];   // lattice constants of the probe (lo/h + 1/2, float-float)
    ff lat_ih;     // 1/h, float-float
    float inv_h;   // 1/h rounded to float once (the displacement's clip)
    int dims[3];
    float step_h;  // displacement scale times h, rounded to float once
    int64_t cells;    // offset of the body's cells in the global cell table
    int64_t first;    // first particle
    int64_t end;      // one past the last particle
    int64_t tile0;    // first tile
    int64_t far_out;  // global id of the body's far+ package
};

constexpr int RX_THREADS = 256;  // particles per tile
// Launch bounds of the relaxation kernel (each thread takes its particle
// through the steps of a launch): four CTAs per SM, 64 registers (a 4-byte
// spill in two instantiations).  50 steps of 10^8 particles on 64 bodies,
// point-interleaved table: 51.4 ms, against 52.3 ms at three CTAs (80
// registers, no spill).  With the scalar [P][8][64] table: three CTAs 53.4
// ms, four 54.1, five (spilling) 58.3, six (spilling) 65.4; one launch per
// step at six CTAs, 78.5 ms.
constexpr int RX_MIN_CTAS = 4;
constexpr int RX_TILES = 16;      // consecutive tiles a CTA walks (4: 54.0 ms at four CTAs per SM)
constexpr int RX_MAX_STEPS = 64;  // steps per launch

// `steps` relaxation steps for every particle: each step probes phi and g
// (and, in the last step with NFL = 8, the integrals) and moves the particle
// by -step h clip(phi / h, -1, 1) n.  The fields do not change during a call
// and particles do not interact, so a thread takes its particle through all
// the steps with the position in registers and writes it back once; every
// step's arithmetic is that of a step-by-step sweep over all particles, so
// the positions and outputs are bitwise the same.  A CTA walks RX_TILES
// consecutive 256-particle tiles (of one body or of consecutive bodies), so
// that a warp's successive particles are near each other in the Morton walk
// and hit the packages L1 holds; its first body is the last whose first tile
// is at most its first tile.
template <int NFL, bool OFF32>
__global__ void __launch_bounds__(RX_THREADS, RX_MIN_CTAS) k_batch_relax(const RelaxBody* __restrict__ rb, int nbody,
                                                            int64_t tiles, const int32_t* __restrict__ cells,
                                                            const int32_t* __restrict__ nbr,
                                                            const float4* __restrict__ tab, int64_t half,
                                                            float* __restrict__ x, float* __restrict__ y,
                                                            float* __restrict__ z, int steps, ProbeOut out) {
    const int64_t t0 = (int64_t)blockIdx.x * RX_TILES, t1 = min(tiles, t0 + RX_TILES);
    int lo = 0, hi = nbody - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&rb[mid].tile0) <= t0)
            lo = mid;
        else
            hi = mid - 1;
    }
    for (int64_t t = t0; t < t1; ++t) {
        while (lo + 1 < nbody && __ldg(&rb[lo + 1].tile0) <= t) ++lo;  // the body of tile t
        const RelaxBody B = rb[lo];
        const int64_t q = B.first + (t - B.tile0) * RX_THREADS + threadIdx.x;
        if (q >= B.end) continue;
        float pos[3] = {x[q], y[q], z[q]};
        float acc[8];
        // the steps before the last: phi and g, the move
        for (int k = 1; k < steps; ++k) {
            const ProbeAt A = probe_locate(B.lat_c, B.lat_ih, B.dims, cells + B.cells, B.far_out, pos);
            if (OFF32)
                probe_interp_quad32<4>(nbr, tab, 16u * (uint32_t)half, A, acc);
            else
                probe_interp_quad<4>(nbr, tab, half, A, acc);
            const float inv = probe_inv_norm(acc);
            const float m = B.step_h * fminf(fmaxf(acc[0] * B.inv_h, -1.0f), 1.0f);
            pos[0] = fmaf(-m, acc[1] * inv, pos[0]);
            pos[1] = fmaf(-m, acc[2] * inv, pos[1]);
            pos[2] = fmaf(-m, acc[3] * inv, pos[2]);
        }
        // the last step: also the outputs asked for
        const ProbeAt A = probe_locate(B.lat_c, B.lat_ih, B.dims, cells + B.cells, B.far_out, pos);
        if (OFF32)
            probe_interp_quad32<NFL>(nbr, tab, 16u * (uint32_t)half, A, acc);
        else
            probe_interp_quad<NFL>(nbr, tab, half, A, acc);
        const float inv = probe_inv_norm(acc);
        const float n0 = acc[1] * inv, n1 = acc[2] * inv, n2 = acc[3] * inv;
        const float m = B.step_h * fminf(fmaxf(acc[0] * B.inv_h, -1.0f), 1.0f);
        x[q] = fmaf(-m, n0, pos[0]);
        y[q] = fmaf(-m, n1, pos[1]);
        z[q] = fmaf(-m, n2, pos[2]);
        if (out.o[0]) out.o[0][q] = acc[0];
        if (out.o[1]) out.o[1][q] = n0;
        if (out.o[2]) out.o[2][q] = n1;
        if (out.o[3]) out.o[3][q] = n2;
        if (NFL == 8) {
#pragma unroll
            for (int f = 4; f < 8; ++f)
                if (out.o[f]) out.o[f][q] = acc[f];
        }
    }
}

unsigned flat_grid(int64_t n) {
    int64_t b = (n + BT - 1) / BT;
    if (b < 1) b = 1;
    if (b > 148 * 32) b = 148 * 32;
    return (unsigned)b;
}

void* b_alloc(sg_batch* b, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (b->user_alloc) {
        p = b->alloc.alloc(bytes, (void*)b->stream, b->alloc.ctx);
    } else if (cudaMallocAsync(&p, bytes, b->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void b_free(sg_batch* b, Buf& x) {
    if (x.p) {
        if (b->user_alloc)
            b->alloc.free(x.p, x.bytes, (void*)b->stream, b->alloc.ctx);
        else
            cudaFreeAsync(x.p, b->stream);
    }
    x.p = nullptr;
    x.bytes = 0;
}

bool b_ensure(sg_batch* b, Buf& x, size_t bytes) {
    if (x.p && x.bytes >= bytes) return true;
    b_free(b, x);
    x.p = b_alloc(b, bytes);
    if (!x.p) return false;
    x.bytes = bytes;
    return true;
}

sg_status b_fail(sg_batch* b, sg_status st, const std::string& msg) {
    if (b) b->last_error = msg;
    return st;
}

bool same_plan(const sg_batch_plan& a, const sg_batch_plan& b) {
    return a.pkgs_per_item == b.pkgs_per_item && a.depth == b.depth && a.reinit_iterations == b.reinit_iterations &&
           a.cfl == b.cfl && a.integrals_mode == b.integrals_mode;
}

bool valid_plan(const sg_batch* b, const sg_batch_plan* p) {
    const int ppi = p->pkgs_per_item;
    return (ppi == 1 || ppi == 2 || ppi == 4 || ppi == 8) && (p->depth == 1 || p->depth == 2) && p->depth <= ppi &&
           p->reinit_iterations >= 0 && p->cfl > 0.0f && std::isfinite(p->cfl) &&
           (p->integrals_mode == 0 || (p->integrals_mode == 1 && b->mlp && b->default_kernel));
}

int persistent_blocks(const void* kernel, int device) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BT, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (per_sm < 1) per_sm = 1;
    if (sms < 1) sms = 1;
    return per_sm * sms;
}

// Upload the per-body constants for a CFL number (stream-ordered).
cudaError_t upload_params(sg_batch* b, float cfl) {
    std::vector<BodyParams> hp(b->n);
    for (int i = 0; i < b->n; ++i) {
        const double h = b->h[i];
        BodyParams& q = hp[i];
        q.inv2h = (float)(1.0 / (2.0 * h));
        q.h2 = (float)(h * h);
        const float dt = (float)((double)cfl * h);
        q.dt = dt;
        q.cfl = (float)((double)dt / h);
        q.inv_eps = (float)(1.0 / b->eps[i]);
        q.F = 0.0f;
        q.pad[0] = q.pad[1] = 0.0f;
    }
    cudaError_t e = cudaMemcpyAsync(b->params.p, hp.data(), hp.size() * sizeof(BodyParams), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // the host vector goes out of scope
    if (e == cudaSuccess) b->params_cfl = cfl;
    return e;
}

// Record the sweep sequence of a plan on stream s.
cudaError_t record_run(sg_batch* b, const sg_batch_plan& plan, cudaStream_t s) {
    const int ppi = plan.pkgs_per_item, iters = plan.reinit_iterations;
    const int32_t* nbr = (const int32_t*)b->nbr.p;
    const int32_t* faces = (const int32_t*)b->faces.p;
    const uint8_t* type = (const uint8_t*)b->type.p;
    const int32_t* body = (const int32_t*)b->body.p;
    const BodyParams* prm = (const BodyParams*)b->params.p;
    float* phi = (float*)b->phi.p;
    float* tmp = (float*)b->tmp.p;
    float* s0 = (float*)b->s0.p;
    float* fo[8];
    for (int i = 0; i < 8; ++i) fo[i] = (float*)b->f[i].p;
    unsigned* ctr = (unsigned*)b->counters.p;
    cudaError_t e = cudaMemsetAsync(ctr, 0, b->n_counters * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int c = 0;
    if (plan.depth == 2) {
        const int nb = persistent_blocks((const void*)k_batch_gradient<2>, b->device);
        k_batch_gradient<2><<<nb, BT, 0, s>>>(faces, type, body, prm, phi, fo[1], fo[2], fo[3], s0, b->P, ppi,
                                              ctr + c++);
    } else {
        const int nb = persistent_blocks((const void*)k_batch_gradient<1>, b->device);
        k_batch_gradient<1><<<nb, BT, 0, s>>>(faces, type, body, prm, phi, fo[1], fo[2], fo[3], s0, b->P, ppi,
                                              ctr + c++);
    }
    note_launch();
    float* a = phi;
    float* o = tmp;
    const int nbr2 = persistent_blocks((const void*)k_batch_reinit<2>, b->device);
    const int nbr1 = persistent_blocks((const void*)k_batch_reinit<1>, b->device);
    for (int it = 0; it < iters; ++it) {
        if (plan.depth == 2)
            k_batch_reinit<2><<<nbr2, BT, 0, s>>>(faces, type, body, prm, s0, a, o, b->P, ppi, ctr + c++, (it & 1) ^ 1);
        else
            k_batch_reinit<1><<<nbr1, BT, 0, s>>>(faces, type, body, prm, s0, a, o, b->P, ppi, ctr + c++, (it & 1) ^ 1);
        note_launch();
        float* t = a;
        a = o;
        o = t;
    }
    if (a != phi) {
        if ((e = cudaMemcpyAsync(phi, a, (size_t)b->P * PKG3 * sizeof(float), cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
            return e;
    }
    if (plan.integrals_mode == 1)
        return launch_batch_surrogate_integrals(nbr, type, body, (const SurBody*)b->sur.p, phi, fo[4], fo[5], fo[6],
                                                fo[7], b->P, b->mlp, b->sur_work.p, mlp_err(b->mlp), b->device, s);
    // the single-grid kernel's warps on package pairs, with each body's Heaviside width
    static_assert(sizeof(BodyParams) % sizeof(float) == 0, "BodyParams as floats");
    return launch_batch_kernel_integrals(nbr, type, body,
                                         reinterpret_cast<const float*>(prm) + offsetof(BodyParams, inv_eps) / sizeof(float),
                                         (int)(sizeof(BodyParams) / sizeof(float)), phi, fo[4], fo[5], fo[6], fo[7],
                                         b->P, b->R, s);
}

// Record the packing of the probe table and `steps` relaxation steps on
// stream s (tables already uploaded, probe table allocated).
cudaError_t record_relax(sg_batch* b, const sg_relax& r, int64_t tiles, cudaStream_t s) {
    ProbeFields F;
    F.f[0] = (const float*)b->phi.p;
    for (int i = 1; i < 8; ++i) F.f[i] = (const float*)b->f[i].p;
    ProbeOut o;
    bool integ = false;
    for (int i = 0; i < 8; ++i) {
        o.o[i] = r.out[i];
        if (i >= 4 && r.out[i]) integ = true;
    }
    const RelaxBody* rb = (const RelaxBody*)b->relax.p;
    const int32_t* cells = (const int32_t*)b->cells.p;
    const int32_t* nbr = (const int32_t*)b->nbr.p;
    float4* tab = (float4*)b->probe_tab.p;
    const int64_t half = b->P * PKG3;  // the table's second half: W, G
    if (r.steps < 1 || tiles < 1) return cudaSuccess;
    cudaError_t e = launch_pack_probe(F, tab, b->P * PKG3, s);
    if (e != cudaSuccess) return e;
    const unsigned ctas = (unsigned)((tiles + RX_TILES - 1) / RX_TILES);
    // a launch takes every particle through up to RX_MAX_STEPS steps (a
    // launch of 10^8 particles then lasts at most about 70 ms, whatever the
    // call's step count); the last launch interpolates W, G as well when
    // they are asked for, and only it writes the outputs
    const bool off32 = b->P < ((int64_t)1 << 21) && !force_wide_offsets();  // table offsets in bytes fit 32 bits
    const ProbeOut none{};
    const dim3 grid(ctas), block(RX_THREADS);
    for (int64_t k0 = 0; k0 < r.steps; k0 += RX_MAX_STEPS) {
        const int n = (int)std::min<int64_t>(RX_MAX_STEPS, r.steps - k0);
        const bool last = k0 + n == r.steps;
        const ProbeOut& oo = last ? o : none;
        if (last && integ) {
            if (off32)
                k_batch_relax<8, true><<<grid, block, 0, s>>>(rb, b->n, tiles, cells, nbr, tab, half, r.x, r.y, r.z,
                                                              n, oo);
            else
                k_batch_relax<8, false><<<grid, block, 0, s>>>(rb, b->n, tiles, cells, nbr, tab, half, r.x, r.y, r.z,
                                                               n, oo);
        } else if (off32) {
            k_batch_relax<4, true><<<grid, block, 0, s>>>(rb, b->n, tiles, cells, nbr, tab, half, r.x, r.y, r.z, n,
                                                          oo);
        } else {
            k_batch_relax<4, false><<<grid, block, 0, s>>>(rb, b->n, tiles, cells, nbr, tab, half, r.x, r.y, r.z, n,
                                                           oo);
        }
        note_launch();
    }
    return cudaGetLastError();
}

bool same_relax(const sg_relax_graph& g, const sg_batch_plan& plan, const sg_relax& r, const int64_t* offsets,
                int n) {
    if (!g.exec || g.r.n != r.n || g.r.x != r.x || g.r.y != r.y || g.r.z != r.z || g.r.steps != r.steps ||
        g.r.step != r.step || g.r.sweeps != r.sweeps)
        return false;
    for (int i = 0; i < 8; ++i)
        if (g.r.out[i] != r.out[i]) return false;
    if (r.sweeps && !same_plan(g.plan, plan)) return false;
    if ((int)g.offsets.size() != n + 1) return false;
    for (int i = 0; i <= n; ++i)
        if (g.offsets[i] != offsets[i]) return false;
    return true;
}

void drop_graphs(sg_batch* b, bool surrogate_only) {
    std::vector<sg_batch_graph> keep;
    for (auto& gr : b->graphs) {
        if (!surrogate_only || gr.plan.integrals_mode == 1)
            cudaGraphExecDestroy(gr.exec);
        else
            keep.push_back(gr);
    }
    b->graphs.swap(keep);
    if (b->rx.exec && (!surrogate_only || (b->rx.r.sweeps && b->rx.plan.integrals_mode == 1))) {
        cudaGraphExecDestroy(b->rx.exec);
        b->rx.exec = nullptr;
    }
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" {

sg_status sg_batch_create(sg_grid* const* grids, int32_t n, void* stream, sg_batch** out) {
    SG_TRACE("sg_batch_create");
    if (!grids || n < 1 || !out) return SG_ERR_INVALID;
    *out = nullptr;
    int64_t P = 0;
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return SG_ERR_INVALID;
        if (grids[i]->state < 2) return SG_ERR_STATE;
        if (grids[i]->device != grids[0]->device) return SG_ERR_INVALID;
        // one tap table for all bodies: the same support in units of h, at most 2h
        const double R = support_h(grids[i]->desc), R0 = support_h(grids[0]->desc);
        if (R > 2.0 || std::fabs(R - R0) > 1e-12 * R0) return SG_ERR_INVALID;
        P += grids[i]->P;
    }
    if (P >= (1LL << 31) / NB) return SG_ERR_CAPACITY;
    int64_t n_cells = 0;
    for (int i = 0; i < n; ++i) n_cells += grids[i]->nc;
    sg_batch* b = new (std::nothrow) sg_batch();
    if (!b) return SG_ERR_OOM;
    b->n = n;
    b->P = P;
    b->R = support_h(grids[0]->desc);
    b->stream = (cudaStream_t)stream;
    b->alloc = grids[0]->alloc;
    b->user_alloc = grids[0]->user_alloc;
    b->device = grids[0]->device;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    sg_status st = SG_OK;
    const size_t fb = (size_t)P * PKG3 * sizeof(float);
    bool ok = b_ensure(b, b->phi, fb) && b_ensure(b, b->tmp, fb) && b_ensure(b, b->s0, fb) && b_ensure(b, b->phi0, fb) &&
              b_ensure(b, b->nbr, (size_t)P * NB * 4) && b_ensure(b, b->faces, (size_t)P * 8 * 4) &&
              b_ensure(b, b->type, (size_t)P) &&
              b_ensure(b, b->body, (size_t)P * 4) && b_ensure(b, b->params, (size_t)n * sizeof(BodyParams)) &&
              b_ensure(b, b->counters, 4096) && b_ensure(b, b->cells, (size_t)n_cells * 4) &&
              b_ensure(b, b->sur, (size_t)n * sizeof(SurBody));
    for (int i = 1; ok && i < 8; ++i) ok = b_ensure(b, b->f[i], fb);
    b->f[0] = Buf{};  // slot 0 (phi) is b->phi
    cudaError_t e = cudaSuccess;
    std::vector<int64_t> bases(n);
    if (!ok) {
        st = SG_ERR_OOM;
    } else {
        b->n_counters = 4096 / sizeof(unsigned);
        int64_t off = 0, coff = 0;
        std::vector<SurBody> sb(n);
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            sg_grid* g = grids[i];
            bases[i] = off;
            b->base.push_back(off);
            b->cell_base.push_back(coff);
            b->npk.push_back(g->P);
            b->h.push_back(g->desc.h);
            b->eps.push_back(heaviside_eps(g->desc));
            b->desc.push_back(g->desc);
            b->default_kernel &= default_kernel(g->desc);
            sb[i] = sur_body(g->desc.h);
            // background cells -> global package ids
            k_batch_offset_nbr<<<flat_grid(g->nc), BT, 0, b->stream>>>((const int32_t*)g->cell_pkg.p,
                                                                       (int32_t*)b->cells.p + coff, g->nc,
                                                                       (int32_t)off);
            note_launch();
            coff += g->nc;
            e = cudaMemcpyAsync((float*)b->phi0.p + off * PKG3, g->field[SG_FIELD_PHI].p,
                                (size_t)g->P * PKG3 * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((uint8_t*)b->type.p + off, g->pkg_type.p, (size_t)g->P, cudaMemcpyDeviceToDevice,
                                    b->stream);
            if (e == cudaSuccess) {
                k_batch_offset_nbr<<<flat_grid(g->P * NB), BT, 0, b->stream>>>(
                    (const int32_t*)g->nbr.p, (int32_t*)b->nbr.p + off * NB, g->P * NB, (int32_t)off);
                k_batch_fill_body<<<flat_grid(g->P), BT, 0, b->stream>>>((int32_t*)b->body.p, off, g->P, i);
                note_launch(2);
                e = cudaGetLastError();
            }
            off += g->P;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->sur.p, sb.data(), (size_t)n * sizeof(SurBody), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = launch_fill_faces((const int32_t*)b->nbr.p, (int32_t*)b->faces.p, P, b->stream);
        for (int i = 1; i < 8 && e == cudaSuccess; ++i) e = cudaMemsetAsync(b->f[i].p, 0, fb, b->stream);
        if (e == cudaSuccess) {
            Buf tmpbase;
            tmpbase.p = b_alloc(b, (size_t)n * sizeof(int64_t));
            if (!tmpbase.p) {
                st = SG_ERR_OOM;
            } else {
                tmpbase.bytes = (size_t)n * sizeof(int64_t);
                e = cudaMemcpyAsync(tmpbase.p, bases.data(), (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice,
                                    b->stream);
                if (e == cudaSuccess) {
                    k_batch_far_W<<<n, 2 * PKG3, 0, b->stream>>>((float*)b->f[4].p, (const int64_t*)tmpbase.p, n);
                    note_launch();
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // bases lives on this stack
                b_free(b, tmpbase);
            }
        }
        if (e == cudaSuccess && st == SG_OK)
            e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
        if (e == cudaSuccess && st == SG_OK) e = upload_params(b, 0.5f);
        if (e != cudaSuccess) st = SG_ERR_CUDA;
    }
    if (st == SG_OK) {
        // phi and the ping-pong buffer start from the grids' phi (far values included)
        e = cudaMemcpyAsync(b->phi.p, b->phi0.p, fb, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->tmp.p, b->phi0.p, fb, cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) st = SG_ERR_CUDA;
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    if (st != SG_OK) {
        cudaGetLastError();
        sg_batch_destroy(b);
        return st;
    }
    *out = b;
    return SG_OK;
}

sg_status sg_batch_destroy(sg_batch* b) {
    if (!b) return SG_ERR_INVALID;
    drop_graphs(b, false);
    Buf* bufs[] = {&b->phi,  &b->tmp,    &b->s0,       &b->phi0,  &b->nbr, &b->faces, &b->type,
                   &b->body, &b->params, &b->counters, &b->cells, &b->sur, &b->relax, &b->probe_tab, &b->sur_work};
    for (Buf* x : bufs) b_free(b, *x);
    for (int i = 1; i < 8; ++i) b_free(b, b->f[i]);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
    return SG_OK;
}

int64_t sg_batch_n_packages(const sg_batch* b) { return b ? b->P : 0; }

const char* sg_batch_last_error(const sg_batch* b) { return b ? b->last_error.c_str() : "null batch"; }

sg_status sg_batch_reset(sg_batch* b) {
    SG_TRACE("sg_batch_reset");
    if (!b) return SG_ERR_INVALID;
    const size_t fb = (size_t)b->P * PKG3 * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(b->phi.p, b->phi0.p, fb, cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess) return b_fail(b, SG_ERR_CUDA, std::string("reset: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_batch_run(sg_batch* b, const sg_batch_plan* plan) {
    SG_TRACE("sg_batch_run");
    if (!b || !plan) return SG_ERR_INVALID;
    if (!valid_plan(b, plan)) return b_fail(b, SG_ERR_INVALID, "sg_batch_run: bad plan");
    if (plan->integrals_mode == 1 && b->P >= SUR_MAX_PACKAGES)
        return b_fail(b, SG_ERR_CAPACITY, "sg_batch_run: the surrogate takes fewer than 2^24 packages");
    if ((size_t)plan->reinit_iterations + 4 > b->n_counters)
        return b_fail(b, SG_ERR_CAPACITY, "sg_batch_run: too many reinit iterations");
    cudaError_t e;
    if (plan->cfl != b->params_cfl) {
        // the graphs read the constants from device memory at replay
        if ((e = upload_params(b, plan->cfl)) != cudaSuccess)
            return b_fail(b, SG_ERR_CUDA, std::string("params: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    for (auto& gr : b->graphs)
        if (same_plan(gr.plan, *plan)) exec = gr.exec;
    if (!exec) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t er = record_run(b, *plan, b->capture);
            e = cudaStreamEndCapture(b->capture, &graph);
            if (er != cudaSuccess) e = er;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return b_fail(b, SG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        }
        b->graphs.push_back(sg_batch_graph{*plan, exec});
    }
    e = cudaGraphLaunch(exec, b->stream);
    if (e != cudaSuccess) return b_fail(b, SG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_batch_autotune(sg_batch* b, sg_batch_plan* plan, int32_t reps, float* times_ms) {
    SG_TRACE("sg_batch_autotune");
    if (!b || !plan || reps < 1) return SG_ERR_INVALID;
    static const int cand[8][2] = {{1, 1}, {2, 1}, {2, 2}, {4, 1}, {4, 2}, {8, 1}, {8, 2}, {1, 1}};
    float best = INFINITY;
    sg_batch_plan best_plan = *plan;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return b_fail(b, SG_ERR_CUDA, "autotune: events");
    sg_status st = SG_OK;
    for (int c = 0; c < 7 && st == SG_OK; ++c) {
        sg_batch_plan p = *plan;
        p.pkgs_per_item = cand[c][0];
        p.depth = cand[c][1];
        if ((st = sg_batch_reset(b)) != SG_OK || (st = sg_batch_run(b, &p)) != SG_OK) break;  // capture + warm
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && st == SG_OK; ++r) {
            st = sg_batch_reset(b);
            if (st == SG_OK) st = sg_batch_run(b, &p);
        }
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = b_fail(b, SG_ERR_CUDA, "autotune: sync");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (times_ms) times_ms[c] = ms;
        if (ms < best) {
            best = ms;
            best_plan = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SG_OK) return st;
    *plan = best_plan;
    return sg_batch_reset(b);
}

// Autotuner cache: a text file of lines "<key> <pkgs_per_item> <depth>";
// the last line of a key wins, lines that do not parse or name no candidate
// are skipped.
sg_status sg_autotune_cache_lookup(const char* path, const char* key, int32_t* pkgs_per_item, int32_t* depth,
                                   int32_t* found) {
    if (!path || !key || !pkgs_per_item || !depth || !found) return SG_ERR_INVALID;
    *found = 0;
    FILE* f = std::fopen(path, "r");
    if (!f) return SG_OK;  // no cache yet
    char line[512], k[400];
    int ppi = 0, dep = 0;
    while (std::fgets(line, sizeof line, f)) {
        if (std::sscanf(line, "%399s %d %d", k, &ppi, &dep) != 3 || std::strcmp(k, key) != 0) continue;
        const bool ok = (ppi == 1 || ppi == 2 || ppi == 4 || ppi == 8) && (dep == 1 || dep == 2) && dep <= ppi;
        if (!ok) continue;
        *pkgs_per_item = ppi;
        *depth = dep;
        *found = 1;
    }
    std::fclose(f);
    return SG_OK;
}

sg_status sg_autotune_cache_store(const char* path, const char* key, int32_t pkgs_per_item, int32_t depth) {
    if (!path || !key || !*key || std::strlen(key) >= 400) return SG_ERR_INVALID;
    for (const char* c = key; *c; ++c)
        if (*c == ' ' || *c == '\t' || *c == '\n' || *c == '\r') return SG_ERR_INVALID;
    if (!(pkgs_per_item == 1 || pkgs_per_item == 2 || pkgs_per_item == 4 || pkgs_per_item == 8) ||
        !(depth == 1 || depth == 2) || depth > pkgs_per_item)
        return SG_ERR_INVALID;
    FILE* f = std::fopen(path, "a");  // one short line per append
    if (!f) return SG_ERR_IO;
    const int w = std::fprintf(f, "%s %d %d\n", key, (int)pkgs_per_item, (int)depth);
    const int c = std::fclose(f);
    return (w < 0 || c != 0) ? SG_ERR_IO : SG_OK;
}

sg_status sg_batch_autotune_key(const sg_batch* b, const sg_batch_plan* plan, char* key, int32_t cap) {
    if (!b || !plan || !key || cap < 1) return SG_ERR_INVALID;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) {
        cudaGetLastError();
        return SG_ERR_CUDA;
    }
    std::string name(prop.name);
    for (char& ch : name)
        if (!(std::isalnum((unsigned char)ch) || ch == '-' || ch == '.')) ch = '_';
    int bucket = 0;
    while (bucket < 62 && ((int64_t)1 << (bucket + 1)) <= b->P) ++bucket;
    const int n = std::snprintf(key, (size_t)cap, "gpu=%s;sm=%d;cc=%d.%d;sweeps=%d;integrals=%d;packages=2^%d",
                                name.c_str(), prop.multiProcessorCount, prop.major, prop.minor,
                                (int)plan->reinit_iterations, (int)plan->integrals_mode, bucket);
    return (n < 0 || n >= cap) ? SG_ERR_CAPACITY : SG_OK;
}

sg_status sg_batch_autotune_cached(sg_batch* b, sg_batch_plan* plan, int32_t reps, const char* path, int32_t* hit) {
    SG_TRACE("sg_batch_autotune_cached");
    if (!b || !plan || !path || reps < 1) return SG_ERR_INVALID;
    if (hit) *hit = 0;
    char key[400];
    sg_status st = sg_batch_autotune_key(b, plan, key, (int32_t)sizeof key);
    if (st != SG_OK) return b_fail(b, st, "autotune: cache key");
    int32_t ppi = 0, dep = 0, found = 0;
    if ((st = sg_autotune_cache_lookup(path, key, &ppi, &dep, &found)) != SG_OK) return st;
    if (found) {
        plan->pkgs_per_item = ppi;
        plan->depth = dep;
        if (hit) *hit = 1;
        return SG_OK;
    }
    if ((st = sg_batch_autotune(b, plan, reps, nullptr)) != SG_OK) return st;
    st = sg_autotune_cache_store(path, key, plan->pkgs_per_item, plan->depth);
    return st == SG_OK ? SG_OK : b_fail(b, st, std::string("autotune: cannot write the cache file ") + path);
}

sg_status sg_batch_get_field(sg_batch* b, int32_t body, int32_t field, void** dev_ptr, int64_t* n_elems) {
    if (!b || !dev_ptr || !n_elems || body < 0 || body >= b->n) return SG_ERR_INVALID;
    const int64_t off = b->base[body], np = b->npk[body];
    float* base = nullptr;
    switch (field) {
    case SG_FIELD_PHI: base = (float*)b->phi.p; break;
    case SG_FIELD_GX: case SG_FIELD_GY: case SG_FIELD_GZ:
    case SG_FIELD_W: case SG_FIELD_GWX: case SG_FIELD_GWY: case SG_FIELD_GWZ:
        base = (float*)b->f[field].p;
        break;
    case SG_FIELD_S0: base = (float*)b->s0.p; break;
    case SG_FIELD_NBR:
        *dev_ptr = (int32_t*)b->nbr.p + off * NB;
        *n_elems = np * NB;
        return SG_OK;
    case SG_FIELD_CELL_PKG: {
        const sg_grid_desc& d = b->desc[body];
        *dev_ptr = (int32_t*)b->cells.p + b->cell_base[body];
        *n_elems = (int64_t)d.dims[0] * d.dims[1] * d.dims[2];
        return SG_OK;
    }
    default:
        return b_fail(b, SG_ERR_INVALID, "sg_batch_get_field: unknown field");
    }
    *dev_ptr = base + off * PKG3;
    *n_elems = np * PKG3;
    return SG_OK;
}

sg_status sg_batch_set_surrogate(sg_batch* b, const sg_mlp* m) {
    if (!b) return SG_ERR_INVALID;
    if (m != b->mlp) {
        // captured surrogate graphs name the old network's weights
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess && m) {
            int prev = -1;
            cudaGetDevice(&prev);
            if (prev != b->device) cudaSetDevice(b->device);
            e = setup_batch_surrogate();
            if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
        }
        if (e != cudaSuccess) return b_fail(b, SG_ERR_CUDA, std::string("set surrogate: ") + cudaGetErrorString(e));
        if (m && !b_ensure(b, b->sur_work, sur_work_bytes(b->P)))
            return b_fail(b, SG_ERR_OOM, "set surrogate: out of memory");
        drop_graphs(b, true);
        b->mlp = m;
    }
    return SG_OK;
}

sg_status sg_batch_relax(sg_batch* b, const sg_batch_plan* plan, const sg_relax* r) {
    SG_TRACE("sg_batch_relax");
    if (!b || !r || !r->offsets || r->n < 0 || r->steps < 0 || !std::isfinite(r->step) || (r->sweeps && !plan))
        return SG_ERR_INVALID;
    if (r->n > 0 && (!r->x || !r->y || !r->z)) return SG_ERR_INVALID;
    if (r->offsets[0] != 0 || r->offsets[b->n] != r->n)
        return b_fail(b, SG_ERR_INVALID, "sg_batch_relax: offsets must run from 0 to n");
    int64_t tiles = 0;
    for (int i = 0; i < b->n; ++i) {
        const int64_t c = r->offsets[i + 1] - r->offsets[i];
        if (c < 0) return b_fail(b, SG_ERR_INVALID, "sg_batch_relax: offsets decrease");
        tiles += (c + RX_THREADS - 1) / RX_THREADS;
    }
    if (tiles >= (1LL << 31)) return b_fail(b, SG_ERR_CAPACITY, "sg_batch_relax: too many particles");
    if (r->sweeps) {
        if (!valid_plan(b, plan)) return b_fail(b, SG_ERR_INVALID, "sg_batch_relax: bad plan");
        if (plan->integrals_mode == 1 && b->P >= SUR_MAX_PACKAGES)
            return b_fail(b, SG_ERR_CAPACITY, "sg_batch_relax: the surrogate takes fewer than 2^24 packages");
        if ((size_t)plan->reinit_iterations + 4 > b->n_counters)
            return b_fail(b, SG_ERR_CAPACITY, "sg_batch_relax: too many reinit iterations");
    }
    cudaError_t e;
    if (r->sweeps && plan->cfl != b->params_cfl) {
        if ((e = upload_params(b, plan->cfl)) != cudaSuccess)
            return b_fail(b, SG_ERR_CUDA, std::string("params: ") + cudaGetErrorString(e));
    }
    const sg_batch_plan none{};
    const sg_batch_plan& pl = r->sweeps ? *plan : none;
    if (!same_relax(b->rx, pl, *r, r->offsets, b->n)) {
        if (b->rx.exec) {
            cudaGraphExecDestroy(b->rx.exec);
            b->rx.exec = nullptr;
        }
        std::vector<RelaxBody> hb(b->n);
        int64_t t0 = 0;
        for (int i = 0; i < b->n; ++i) {
            const sg_grid_desc& d = b->desc[i];
            RelaxBody& q = hb[i];
            for (int a = 0; a < 3; ++a) q.dims[a] = d.dims[a];
            set_lattice(q.lat_c, q.lat_ih, d.lo, d.h);
            q.inv_h = (float)(1.0 / d.h);
            q.step_h = (float)((double)r->step * d.h);
            q.cells = b->cell_base[i];
            q.first = r->offsets[i];
            q.end = r->offsets[i + 1];
            q.tile0 = t0;
            q.far_out = b->base[i] + 1;
            t0 += (q.end - q.first + RX_THREADS - 1) / RX_THREADS;
        }
        if (!b_ensure(b, b->relax, (size_t)b->n * sizeof(RelaxBody)) ||
            !b_ensure(b, b->probe_tab, (size_t)b->P * PKG3 * 32))
            return b_fail(b, SG_ERR_OOM, "sg_batch_relax: out of memory");
        e = cudaMemcpyAsync(b->relax.p, hb.data(), hb.size() * sizeof(RelaxBody), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // hb goes out of scope
        if (e != cudaSuccess) return b_fail(b, SG_ERR_CUDA, std::string("relax table: ") + cudaGetErrorString(e));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t er = r->sweeps ? record_run(b, pl, b->capture) : cudaSuccess;
            if (er == cudaSuccess) er = record_relax(b, *r, tiles, b->capture);
            e = cudaStreamEndCapture(b->capture, &graph);
            if (er != cudaSuccess) e = er;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return b_fail(b, SG_ERR_CUDA, std::string("relax capture: ") + cudaGetErrorString(e));
        }
        b->rx.plan = pl;
        b->rx.r = *r;
        b->rx.r.offsets = nullptr;
        b->rx.offsets.assign(r->offsets, r->offsets + b->n + 1);
        b->rx.exec = exec;
    }
    e = cudaGraphLaunch(b->rx.exec, b->stream);
    if (e != cudaSuccess) return b_fail(b, SG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return SG_OK;
}

}  // extern "C"
