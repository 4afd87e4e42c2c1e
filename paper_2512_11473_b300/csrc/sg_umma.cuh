// sg_umma.cuh -- fifth-generation tensor cores (tcgen05) for the surrogate's
// dense layers on sm_103a: shared-memory operand descriptors, the instruction
// descriptor of a BF16 x BF16 -> FP32 product, tensor-memory (TMEM)
// allocation, MMA issue and completion through an mbarrier (waits bounded),
// and TMEM loads.  Written from the PTX ISA's description of the tcgen05
// instructions.
//
// Operands live in shared memory in the no-swizzle K-major layout: "core
// matrices" of 8 rows x 16 bytes (8 bf16 along K) stored as 128 contiguous
// bytes, row r of the core matrix at byte 16 r.  For an R x K operand the K/8
// core matrices of an 8-row group sit side by side (128 bytes apart: the
// leading byte offset) and the 8-row groups follow each other (16 K bytes
// apart: the stride byte offset):
//   byte(r, k) = (r / 8) 16 K + (k / 8) 128 + (r % 8) 16 + (k % 8) 2.
// A K = 16 slice starting at column k0 is the same layout from byte
// 16 k0 on, so one descriptor per slice walks the K dimension.
//
// The accumulator of an M = 128 product sits in TMEM with row i in lane i and
// column j in column (base + j); warp w of the CTA reads lanes 32 w .. 32 w + 31.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sg {
namespace umma {

__host__ __device__ constexpr uint32_t kmajor_byte(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (16 * K) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 64-bit shared-memory matrix descriptor: start address / 16 (bits 0-13),
// leading byte offset / 16 (16-29), stride byte offset / 16 (32-45), the
// descriptor version 1 (46-47), base offset 0, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Descriptor of the K = 16 slice k0 of a K-major operand with K columns at
// shared address base.
__device__ __forceinline__ uint64_t kslice_desc(uint32_t base, int K, int k0) {
    return smem_desc(base + 16u * (uint32_t)k0, 128u, 16u * (uint32_t)K);
}

// 32-bit instruction descriptor of kind::f16 with FP32 accumulation (bits 4-5
// = 1), A and B in BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16
// = 0), N / 8 in bits 17-22 and M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM columns for this CTA, allocated by one whole warp; the address is
// written to *slot (shared memory).  The CTA allocates once, so it gives
// up its permit to allocate again at once.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Free the columns again (the warp that allocated them).
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A B^T (+ D when accumulate), issued by one thread.
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                    uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier receives one arrival when every MMA this thread issued before
// has completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the phase with the given parity has completed; false when
// max_polls polls (each a bounded hardware wait) found it still open.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_polls) {
    const uint32_t a = smem_u32(mbar);
    for (uint32_t i = 0; i < max_polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Ordering of tensor-core work against thread synchronisation, and of
// ordinary shared-memory stores against the tensor core's reads.
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape):
// thread t of warp w reads lane 32 w + t, columns col .. col + 15 of taddr.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// TMEM address of this warp's lane quarter at column col.
__device__ __forceinline__ uint32_t tmem_lane_addr(uint32_t base, int warp, int col) {
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col;
}

// Eight bf16 (from eight floats, round to nearest) as one 16-byte word.
__device__ __forceinline__ uint4 pack8_bf16(const float* f) {
    uint4 u;
    __nv_bfloat162 p;
    p = __floats2bfloat162_rn(f[0], f[1]);
    u.x = *reinterpret_cast<uint32_t*>(&p);
    p = __floats2bfloat162_rn(f[2], f[3]);
    u.y = *reinterpret_cast<uint32_t*>(&p);
    p = __floats2bfloat162_rn(f[4], f[5]);
    u.z = *reinterpret_cast<uint32_t*>(&p);
    p = __floats2bfloat162_rn(f[6], f[7]);
    u.w = *reinterpret_cast<uint32_t*>(&p);
    return u;
}

}  // namespace umma
}  // namespace sg
