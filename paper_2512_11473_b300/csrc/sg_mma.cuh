// sg_mma.cuh -- warp-level BF16 tensor-core tiles (mma.sync m16n8k16, FP32
// accumulation) for the surrogate's small dense layers.
//
// Fragment ownership (PTX ISA, mma.m16n8k16 with .bf16 operands), with
// g = lane / 4 and t = lane % 4:
//   A 16x16 row-major:  a[0] = A[g][2t..2t+1],   a[1] = A[g+8][2t..2t+1],
//                       a[2] = A[g][2t+8..+9],   a[3] = A[g+8][2t+8..+9]
//   B 16x8  (k, n):     b[0] = B[2t..2t+1][g],   b[1] = B[2t+8..+9][g]
//   C 16x8  f32:        c[0..1] = C[g][2t..2t+1], c[2..3] = C[g+8][2t..2t+1]
// Two consecutive bf16 share one 32-bit register, lower index in the low half.
// B is kept in shared memory as Bt[n][k] (k contiguous), so each b register
// is one aligned 32-bit load.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace sg {
namespace {

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragment of rows r0..r0+15 and columns k0..k0+15 of a row-major tile.
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* s, int stride, int r0, int k0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* p = s + (r0 + g) * stride + k0 + 2 * t;
    a[0] = ld32(p);
    a[1] = ld32(p + 8 * stride);
    a[2] = ld32(p + 8);
    a[3] = ld32(p + 8 * stride + 8);
}

// B fragment of columns n0..n0+7 and rows k0..k0+15, from Bt[n][k].
__device__ __forceinline__ void frag_b(uint32_t (&b)[2], const __nv_bfloat16* s, int stride, int n0, int k0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* p = s + (n0 + g) * stride + k0 + 2 * t;
    b[0] = ld32(p);
    b[1] = ld32(p + 8);
}

// acc[nt] (16 x 8N) += A (16 x K) * B, B given as Bt[n][k]; K multiple of 16.
template <int K, int NT>
__device__ __forceinline__ void warp_gemm(float (&acc)[NT][4], const __nv_bfloat16* A, int sa, int r0,
                                          const __nv_bfloat16* Bt, int sb, int n_base) {
#pragma unroll
    for (int kk = 0; kk < K; kk += 16) {
        uint32_t a[4];
        frag_a(a, A, sa, r0, kk);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            uint32_t b[2];
            frag_b(b, Bt, sb, n_base + 8 * nt, kk);
            mma_16816(acc[nt], a, b);
        }
    }
}

__device__ __forceinline__ float tanh_approx(float x) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// logistic sigmoid through the hardware tanh: 1 / (1 + e^-z) = (1 + tanh(z/2)) / 2
__device__ __forceinline__ float sigmoidf_(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }
// SiLU z sigmoid(z) = h + h tanh(h) with h = z/2
__device__ __forceinline__ float silu_(float z) {
    const float h = 0.5f * z;
    return fmaf(h, tanh_approx(h), h);
}

}  // namespace
}  // namespace sg
