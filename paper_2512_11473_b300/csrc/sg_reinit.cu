// sg_reinit.cu -- the Godunov reinitialisation of one grid: the smoothed
// sign of the level set at call entry and one Jacobi sweep over the active
// packages (a half-warp per package, a float4 row per lane, the row code of
// sg_rows.cuh shared with the batched sweeps).
#include "sg_rows.cuh"

namespace sg {
namespace {

constexpr int SW_THREADS = 256;

unsigned flat_blocks(int64_t n) {
    int64_t b = (n + SW_THREADS - 1) / SW_THREADS;
    if (b < 1) b = 1;
    if (b > 148 * 64) b = 148 * 64;
    return (unsigned)b;
}

__global__ void __launch_bounds__(SW_THREADS) k_reinit_s0(const float* __restrict__ phi, float* __restrict__ s0,
                                                           int64_t n_act, float h2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_act; e += (int64_t)gridDim.x * blockDim.x)
        s0[2 * PKG3 + e] = smoothed_sign(phi[2 * PKG3 + e], h2);
}

// One sweep; the first of a call (FIRST) reads phi at call entry, so it
// forms the smoothed sign S0 of its own row there and stores it for the
// sweeps that follow (a separate instantiation, so that the other sweeps
// keep their 32 registers without spills).
template <bool FIRST>
__global__ void __launch_bounds__(ROW_THREADS, 8) k_reinit_step(const int32_t* __restrict__ faces, float* s0,
                                                              const float* phi_in, float* __restrict__ phi_out,
                                                              int64_t P, float cfl, float dt, float h2, int reverse) {
    // Sweeps are launched as programmatic dependents of the previous sweep:
    // wait until it has completed (its phi is our input, and we overwrite its
    // input), then let the next sweep's CTAs launch as this one drains.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (FIRST) {  // far packages of S0 (the sign) and of the output (phi's far values)
        write_far(s0, -1.0f, 1.0f);
        if (blockIdx.x == 0 && threadIdx.x < 2 * PKG3) phi_out[threadIdx.x] = __ldca(phi_in + threadIdx.x);
    }
    const RowSlot s = row_slot_dir(P, reverse);
    const Rows w = load_rows_t<true>(phi_in, faces, s);
    float4 sg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s.valid) {
        if (FIRST) {
            sg = make_float4(smoothed_sign(w.c.x, h2), smoothed_sign(w.c.y, h2), smoothed_sign(w.c.z, h2),
                             smoothed_sign(w.c.w, h2));
            reinterpret_cast<float4*>(s0)[s.q4] = sg;
        } else {
            sg = __ldca(reinterpret_cast<const float4*>(s0) + s.q4);
        }
    }
    if (!s.valid) return;
    reinterpret_cast<float4*>(phi_out)[s.q4] = reinit_row(w, sg, cfl, dt);
}

}  // namespace

cudaError_t launch_reinit_s0(const GridF& G, const float* phi, float* s0, int64_t P, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    int64_t n = (P - 2) * PKG3;
    k_reinit_s0<<<flat_blocks(n), SW_THREADS, 0, s>>>(phi, s0, n, (float)(G.h_d * G.h_d));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_reinit_step(const GridF& G, const int32_t* faces, float* s0, const float* phi_in,
                               float* phi_out, float dt, int64_t P, int reverse, int first, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    // dt sqrt(G) = (dt / h) sqrt(h^2 G) and dt / h is the CFL number
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(row_blocks(P));
    cfg.blockDim = dim3(ROW_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const float cfl = (float)(dt / G.h_d), h2 = (float)(G.h_d * G.h_d);
    const cudaError_t e = first ? cudaLaunchKernelEx(&cfg, k_reinit_step<true>, faces, s0, phi_in, phi_out, P, cfl,
                                                     dt, h2, reverse)
                                : cudaLaunchKernelEx(&cfg, k_reinit_step<false>, faces, s0, phi_in, phi_out, P, cfl,
                                                     dt, h2, reverse);
    note_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sg
