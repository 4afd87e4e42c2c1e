// sg_mlp.cu -- the kernel-integral surrogate network: 27 inputs -> 64 -> 64 ->
// 4 outputs, SiLU hidden activations, BF16 weights and activations, FP32
// accumulation on the tensor cores (sg_mma.cuh), FP32 master weights and Adam
// (Kingma & Ba 2015).  Not in the paper: the learned stand-in for the kernel
// integral of "Integral with SPH Smoothing Kernel and Grid-Particle Coupling".
//
// Canonical parameter vector (FP32, shared with the host):
//   W1[64][27], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]   (6212 values)
// Packed device copy (what the kernels stage in shared memory), BF16 with
// padded rows so that fragment loads hit distinct banks:
//   W1t[64][40]  W1 with inputs padded to 32     (B operand of layer 1)
//   W2 [64][72]                                  (B operand of layer 2)
//   W3 [8][72]   rows 4..7 zero                  (B operand of layer 3)
//   W2T[64][72]  transpose of W2                 (B operand of dh1 = dz2 W2)
//   W3T[64][24]  transpose of W3, outputs padded (B operand of dh2 = dy W3)
//   then b1[64], b2[64], b3[8] in FP32.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg_mlp.cuh"
#include "sg_mma.cuh"
#include "sg_integrals.cuh"
#include "sg_rows.cuh"

struct sg_mlp {
    cudaStream_t stream = nullptr;
    int device = 0;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    unsigned char* packed = nullptr;
    int64_t step = 0;
    std::string last_error;
};

namespace sg {
namespace {

constexpr int TR_WARPS = 4;
constexpr int TR_ROWS = 16 * TR_WARPS;  // samples per CTA of the training kernel
constexpr int SX = MLP_KIN + 8;         // row stride of input tiles (40)
constexpr int SY = 24;                  // row stride of output-gradient tiles

// canonical index -> packed placement
__global__ void k_mlp_pack(const float* __restrict__ master, unsigned char* __restrict__ packed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(packed);
    float* bias = reinterpret_cast<float*>(packed + MLP_PACK_BIAS_BYTE);
    const float v = master[k];
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    if (k < MLP_OFF_B1) {
        const int o = k / MLP_IN, i = k % MLP_IN;
        w[MLP_PK_W1T + o * MLP_S1 + i] = b;
    } else if (k < MLP_OFF_W2) {
        bias[k - MLP_OFF_B1] = v;
    } else if (k < MLP_OFF_B2) {
        const int o = (k - MLP_OFF_W2) / MLP_H, i = (k - MLP_OFF_W2) % MLP_H;
        w[MLP_PK_W2 + o * MLP_S2 + i] = b;
        w[MLP_PK_W2T + i * MLP_S2 + o] = b;
    } else if (k < MLP_OFF_W3) {
        bias[MLP_H + k - MLP_OFF_B2] = v;
    } else if (k < MLP_OFF_B3) {
        const int o = (k - MLP_OFF_W3) / MLP_H, i = (k - MLP_OFF_W3) % MLP_H;
        w[MLP_PK_W3 + o * MLP_S2 + i] = b;
        w[MLP_PK_W3T + i * MLP_S3T + o] = b;
    } else {
        bias[2 * MLP_H + k - MLP_OFF_B3] = v;
    }
}

__global__ void k_adam(float* __restrict__ master, float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    const float g = grad[k];
    const float mk = beta1 * m[k] + (1.0f - beta1) * g;
    const float vk = beta2 * v[k] + (1.0f - beta2) * g * g;
    m[k] = mk;
    v[k] = vk;
    master[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    grad[k] = 0.0f;
}

// Copy the packed weights (bytes, multiple of 16) into shared memory.
__device__ __forceinline__ void stage_weights(unsigned char* dst, const unsigned char* __restrict__ src, int bytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// Rows of a 16-row input tile: lane pairs load one 64-byte row (27 values
// plus zero padding, bf16).  Rows past n are zero.
__device__ __forceinline__ void load_x_tile(__nv_bfloat16* X, const __nv_bfloat16* __restrict__ x,
                                            const int32_t* __restrict__ idx, int64_t row0, int64_t n) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = lane + 32 * h;  // 64 quarter-rows of 16 bytes
        const int r = q >> 2, c = q & 3;
        const int64_t row = row0 + r;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < n) {
            const int64_t src = idx ? (int64_t)__ldg(idx + row) : row;
            v = __ldg(reinterpret_cast<const uint4*>(x + src * MLP_KIN) + c);
        }
        *reinterpret_cast<uint4*>(X + r * SX + 8 * c) = v;
    }
    __syncwarp();
}

// Forward of one 16-row tile through the three layers; y = output tile
// values in fragment layout (cols 2t, 2t+1 of rows g, g+8 of n-tile 0).
// SiLU of the accumulators of n-tiles 2m and 2m + 1 (columns 16m..16m+15),
// packed as the A fragment of k-tile m of the next layer: the C layout of
// two adjacent 16x8 tiles is the A layout of one 16x16 tile, so hidden
// activations never leave the registers.
__device__ __forceinline__ void silu_to_a(const float (&c0)[4], const float (&c1)[4], uint32_t (&a)[4]) {
    __nv_bfloat162 v;
    v = __floats2bfloat162_rn(silu_(c0[0]), silu_(c0[1]));
    a[0] = *reinterpret_cast<uint32_t*>(&v);
    v = __floats2bfloat162_rn(silu_(c0[2]), silu_(c0[3]));
    a[1] = *reinterpret_cast<uint32_t*>(&v);
    v = __floats2bfloat162_rn(silu_(c1[0]), silu_(c1[1]));
    a[2] = *reinterpret_cast<uint32_t*>(&v);
    v = __floats2bfloat162_rn(silu_(c1[2]), silu_(c1[3]));
    a[3] = *reinterpret_cast<uint32_t*>(&v);
}

// One 16-row tile through the network: X [16][SX] bf16 inputs in shared
// memory (27 values, zero padding to 32), weights W and biases as packed;
// y = the lane's accumulator fragment of the 4 outputs (columns 2t, 2t+1 of
// rows g and g + 8; columns >= 4 are padding).
__device__ __forceinline__ void forward_tile(const __nv_bfloat16* W, const float* bias, const __nv_bfloat16* X,
                                             float (&y)[4]) {
    const int lane = threadIdx.x & 31, t = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
        acc[nt][0] = b0, acc[nt][1] = b1, acc[nt][2] = b0, acc[nt][3] = b1;
    }
    warp_gemm<MLP_KIN, 8>(acc, X, SX, 0, W + MLP_PK_W1T, MLP_S1, 0);
    uint32_t a[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m) silu_to_a(acc[2 * m], acc[2 * m + 1], a[m]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[MLP_H + 8 * nt + 2 * t], b1 = bias[MLP_H + 8 * nt + 2 * t + 1];
        acc[nt][0] = b0, acc[nt][1] = b1, acc[nt][2] = b0, acc[nt][3] = b1;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t b[2];
            frag_b(b, W + MLP_PK_W2, MLP_S2, 8 * nt, 16 * m);
            mma_16816(acc[nt], a[m], b);
        }
#pragma unroll
    for (int m = 0; m < 4; ++m) silu_to_a(acc[2 * m], acc[2 * m + 1], a[m]);
    const float c0 = 2 * t < MLP_OUT ? bias[2 * MLP_H + 2 * t] : 0.0f;
    const float c1 = 2 * t + 1 < MLP_OUT ? bias[2 * MLP_H + 2 * t + 1] : 0.0f;
    y[0] = c0, y[1] = c1, y[2] = c0, y[3] = c1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        uint32_t b[2];
        frag_b(b, W + MLP_PK_W3, MLP_S2, 0, 16 * m);
        mma_16816(y, a[m], b);
    }
}

// y[n][4] = MLP(x[n][32]); one warp per 16-row tile.
__global__ void __launch_bounds__(128) k_mlp_forward(const unsigned char* __restrict__ packed, int64_t n,
                                                      const __nv_bfloat16* __restrict__ x, float* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(smem);
    const float* bias = reinterpret_cast<const float*>(smem + MLP_PACK_BIAS_BYTE);
    stage_weights(smem, packed, MLP_PACK_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(smem + MLP_PACK_BYTES) + warp * 16 * SX;
    __syncthreads();
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        load_x_tile(X, x, nullptr, tile * 16, n);
        float o[4];
        forward_tile(W, bias, X, o);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = tile * 16 + g + 8 * (i >> 1);
            const int col = 2 * t + (i & 1);
            if (row < n && col < MLP_OUT) y[row * MLP_OUT + col] = o[i];
        }
        __syncwarp();
    }
}

// Shared-memory plan of the training kernel (bytes).
constexpr int TR_W = MLP_PACK_BYTES;                                   // weights + biases
constexpr int TR_WARP_BF16 = 16 * SX + 4 * 16 * MLP_S2 + 16 * SY;      // X, A1, A2, DZ2, (spare), DY
constexpr int TR_WARP_F32 = 2 * 16 * MLP_H;                            // SiLU'(z1), SiLU'(z2)
constexpr int TR_T_ROWS = MLP_KIN + 3 * MLP_H + 16 + MLP_H;            // XT, A1T, A2T, DZ2T, DYT, DZ1T rows
constexpr int TR_TS = TR_ROWS + 8;                                     // transposed row stride (72)
constexpr int TR_BYTES = TR_W + TR_WARPS * (TR_WARP_BF16 * 2 + TR_WARP_F32 * 4) + TR_T_ROWS * TR_TS * 2 + 64;

// Gradient of the mean squared error of one batch (rows idx[0..n) or 0..n)
// with respect to every canonical parameter, added into grad; the loss is
// added into *loss.  A CTA takes 64 samples (one 16-row tile per warp), runs
// forward and backward per tile on the tensor cores, then forms the weight
// gradients as K = 64 products of the transposed tiles.
__global__ void __launch_bounds__(TR_WARPS * 32) k_mlp_train(const unsigned char* __restrict__ packed, int64_t n,
                                                            const __nv_bfloat16* __restrict__ x,
                                                            const float* __restrict__ tgt,
                                                            const int32_t* __restrict__ idx, float scale,
                                                            float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(smem);
    const float* bias = reinterpret_cast<const float*>(smem + MLP_PACK_BIAS_BYTE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(smem + TR_W) + warp * TR_WARP_BF16;
    __nv_bfloat16* X = wb;
    __nv_bfloat16* A1 = X + 16 * SX;
    __nv_bfloat16* A2 = A1 + 16 * MLP_S2;
    __nv_bfloat16* DZ2 = A2 + 16 * MLP_S2;
    __nv_bfloat16* DY = DZ2 + 2 * 16 * MLP_S2;
    float* D1 = reinterpret_cast<float*>(smem + TR_W + TR_WARPS * TR_WARP_BF16 * 2) + warp * TR_WARP_F32;
    float* D2 = D1 + 16 * MLP_H;
    __nv_bfloat16* T0 =
        reinterpret_cast<__nv_bfloat16*>(smem + TR_W + TR_WARPS * (TR_WARP_BF16 * 2 + TR_WARP_F32 * 4));
    __nv_bfloat16* XT = T0;                           // [32][72]
    __nv_bfloat16* A1T = XT + MLP_KIN * TR_TS;        // [64][72]
    __nv_bfloat16* A2T = A1T + MLP_H * TR_TS;         // [64][72]
    __nv_bfloat16* DZ2T = A2T + MLP_H * TR_TS;        // [64][72]
    __nv_bfloat16* DYT = DZ2T + MLP_H * TR_TS;        // [16][72]
    __nv_bfloat16* DZ1T = DYT + 16 * TR_TS;           // [64][72]

    stage_weights(smem, packed, MLP_PACK_BYTES);
    // zero the padded output-gradient tiles (cols 4..15 must stay zero)
    for (int i = lane; i < 16 * SY; i += 32) DY[i] = __float2bfloat16_rn(0.0f);
    for (int i = threadIdx.x; i < 16 * TR_TS; i += blockDim.x) DYT[i] = __float2bfloat16_rn(0.0f);
    __syncthreads();

    const int64_t row0 = (int64_t)blockIdx.x * TR_ROWS + 16 * warp;
    const int col0 = 16 * warp;  // this warp's sample columns in the transposed tiles
    load_x_tile(X, x, idx, row0, n);
    for (int i = lane; i < 16 * MLP_KIN; i += 32) {
        const int r = i / MLP_KIN, c = i % MLP_KIN;
        XT[c * TR_TS + col0 + r] = X[r * SX + c];
    }
    // ---- forward, keeping SiLU'(z) ----
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
        acc[nt][0] = b0, acc[nt][1] = b1, acc[nt][2] = b0, acc[nt][3] = b1;
    }
    warp_gemm<MLP_KIN, 8>(acc, X, SX, 0, W + MLP_PK_W1T, MLP_S1, 0);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g + 8 * (i >> 1), c = 8 * nt + 2 * t + (i & 1);
            const float z = acc[nt][i], s = sigmoidf_(z);
            const __nv_bfloat16 a = __float2bfloat16_rn(z * s);
            A1[r * MLP_S2 + c] = a;
            A1T[c * TR_TS + col0 + r] = a;
            D1[r * MLP_H + c] = s * (1.0f + z * (1.0f - s));
        }
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[MLP_H + 8 * nt + 2 * t], b1 = bias[MLP_H + 8 * nt + 2 * t + 1];
        acc[nt][0] = b0, acc[nt][1] = b1, acc[nt][2] = b0, acc[nt][3] = b1;
    }
    warp_gemm<MLP_H, 8>(acc, A1, MLP_S2, 0, W + MLP_PK_W2, MLP_S2, 0);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g + 8 * (i >> 1), c = 8 * nt + 2 * t + (i & 1);
            const float z = acc[nt][i], s = sigmoidf_(z);
            const __nv_bfloat16 a = __float2bfloat16_rn(z * s);
            A2[r * MLP_S2 + c] = a;
            A2T[c * TR_TS + col0 + r] = a;
            D2[r * MLP_H + c] = s * (1.0f + z * (1.0f - s));
        }
    __syncwarp();
    float o[1][4];
    {
        const float c0 = 2 * t < MLP_OUT ? bias[2 * MLP_H + 2 * t] : 0.0f;
        const float c1 = 2 * t + 1 < MLP_OUT ? bias[2 * MLP_H + 2 * t + 1] : 0.0f;
        o[0][0] = c0, o[0][1] = c1, o[0][2] = c0, o[0][3] = c1;
    }
    warp_gemm<MLP_H, 1>(o, A2, MLP_S2, 0, W + MLP_PK_W3, MLP_S2, 0);
    // ---- loss and dL/dy ----
    float lsum = 0.0f;
    float dys[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = g + 8 * (i >> 1), c = 2 * t + (i & 1);
        const int64_t row = row0 + r;
        float dy = 0.0f;
        if (row < n && c < MLP_OUT) {
            const int64_t src = idx ? (int64_t)__ldg(idx + row) : row;
            const float e = o[0][i] - __ldg(tgt + src * MLP_OUT + c);
            lsum += e * e * scale;
            dy = 2.0f * e * scale;
        }
        dys[i] = dy;
        const __nv_bfloat16 b = __float2bfloat16_rn(dy);
        DY[r * SY + c] = b;
        DYT[c * TR_TS + col0 + r] = b;
    }
    __syncwarp();
    // bias gradient of layer 3: column sums of dy (over g, i.e. lane bits 2..4)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        float s = dys[j] + dys[j + 2];
        for (int off = 4; off < 32; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (g == 0 && 2 * t + j < MLP_OUT) atomicAdd(grad + MLP_OFF_B3 + 2 * t + j, s);
    }
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0 && loss) atomicAdd(loss, lsum);
    // ---- dh2 = dy W3, dz2 = dh2 SiLU'(z2) ----
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    warp_gemm<16, 8>(acc, DY, SY, 0, W + MLP_PK_W3T, MLP_S3T, 0);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float bs[2] = {0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g + 8 * (i >> 1), c = 8 * nt + 2 * t + (i & 1);
            const float dz = acc[nt][i] * D2[r * MLP_H + c];
            bs[i & 1] += dz;
            const __nv_bfloat16 b = __float2bfloat16_rn(dz);
            DZ2[r * MLP_S2 + c] = b;
            DZ2T[c * TR_TS + col0 + r] = b;
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float s = bs[j];
            for (int off = 4; off < 32; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (g == 0) atomicAdd(grad + MLP_OFF_B2 + 8 * nt + 2 * t + j, s);
        }
    }
    __syncwarp();
    // ---- dh1 = dz2 W2, dz1 = dh1 SiLU'(z1) ----
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    warp_gemm<MLP_H, 8>(acc, DZ2, MLP_S2, 0, W + MLP_PK_W2T, MLP_S2, 0);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float bs[2] = {0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g + 8 * (i >> 1), c = 8 * nt + 2 * t + (i & 1);
            const float dz = acc[nt][i] * D1[r * MLP_H + c];
            bs[i & 1] += dz;
            DZ1T[c * TR_TS + col0 + r] = __float2bfloat16_rn(dz);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float s = bs[j];
            for (int off = 4; off < 32; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (g == 0) atomicAdd(grad + MLP_OFF_B1 + 8 * nt + 2 * t + j, s);
        }
    }
    __syncthreads();
    // ---- weight gradients over the CTA's 64 samples (K = 64) ----
    // dW1[o][i] = sum_s dz1[s][o] x[s][i]; dW2[o][i] = sum_s dz2[s][o] a1[s][i]
    {
        float a4[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) a4[nt][0] = a4[nt][1] = a4[nt][2] = a4[nt][3] = 0.0f;
        warp_gemm<TR_ROWS, 4>(a4, DZ1T, TR_TS, 16 * warp, XT, TR_TS, 0);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int o_ = 16 * warp + g + 8 * (i >> 1), in = 8 * nt + 2 * t + (i & 1);
                if (in < MLP_IN) atomicAdd(grad + MLP_OFF_W1 + o_ * MLP_IN + in, a4[nt][i]);
            }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    warp_gemm<TR_ROWS, 8>(acc, DZ2T, TR_TS, 16 * warp, A1T, TR_TS, 0);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o_ = 16 * warp + g + 8 * (i >> 1), in = 8 * nt + 2 * t + (i & 1);
            atomicAdd(grad + MLP_OFF_W2 + o_ * MLP_H + in, acc[nt][i]);
        }
    // dW3[o][i] = sum_s dy[s][o] a2[s][i] (rows o < 4 of a 16-row tile), split by warps over i
    {
        float a2[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) a2[nt][0] = a2[nt][1] = a2[nt][2] = a2[nt][3] = 0.0f;
        warp_gemm<TR_ROWS, 2>(a2, DYT, TR_TS, 0, A2T, TR_TS, 16 * warp);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int o_ = g + 8 * (i >> 1), in = 16 * warp + 8 * nt + 2 * t + (i & 1);
                if (o_ < MLP_OUT) atomicAdd(grad + MLP_OFF_W3 + o_ * MLP_H + in, a2[nt][i]);
            }
    }
}

// ---------------------------------------------------------------------------
// Surrogate kernel integrals.  Per data point, from the 6^3 tile of phi around
// its package (float, the same rounding on host and device):
//   inputs   v_n = clip(phi_s / h, -1, 1)                   (27 offsets s)
//   trivial  every tap saturates the Heaviside on one side: W = 1 or 0, G = 0
//   fallback |phi / h| < 1, or |kappa| h > 0.1 with kappa the 7-point
//            Laplacian: the exact 27-tap sum (bit-identical to mode 0)
//   network  everything else: the tensor-core MLP
// ---------------------------------------------------------------------------

// |kappa| h > 0.1 with kappa the 7-point Laplacian (sum of the six face
// neighbours - 6 phi) / h^2, i.e. |a| > 0.1 h for the numerator a, decided
// as on the real values: the float sum a is within 7 roundings, 2^-21 S, of
// the exact one (S the float sum of the terms' magnitudes); only when |a|
// falls within 2^-19 S of the bound is the numerator re-formed in
// float-float (error about 2^-44 S).
__device__ __forceinline__ bool curvature_exceeds(float xp, float xm, float yp, float ym, float zp, float zm, float c,
                                                  const SurConst& C) {
    const float a = __fadd_rn(__fadd_rn(__fadd_rn(xp, xm), __fadd_rn(yp, ym)),
                              __fsub_rn(__fadd_rn(zp, zm), __fmul_rn(6.0f, c)));
    const float S = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(xp), fabsf(xm)), __fadd_rn(fabsf(yp), fabsf(ym))),
                              __fadd_rn(__fadd_rn(fabsf(zp), fabsf(zm)), __fmul_rn(6.0f, fabsf(c))));
    const float d = __fsub_rn(fabsf(a), C.kap_thr);
    if (fabsf(d) > __fmul_rn(0x1p-19f, S) + __fmul_rn(0x1p-22f, C.kap_thr)) return d > 0.0f;
    ff s = ff_add(two_sum(xp, xm), two_sum(yp, ym));
    s = ff_add(s, two_sum(zp, zm));
    s = ff_add(s, two_prod(-6.0f, c));  // -6 phi exactly
    if (s.hi < 0.0f) s = ff_neg(s);
    return ff_gt(s, C.kap_thr_ff);
}

// Class of a data point from the 6^3 phi tile around its package, on the
// real values of the float phi (the same decisions as an exact evaluation):
// trivial where every tap has |phi_s| >= h on one side (the Heaviside
// saturates), fallback where |phi| < h or |kappa| h > 0.1, network else.
// v receives the inputs clip(phi_s / h, -1, 1).
__device__ __forceinline__ int sur_classify(const float* tile, int d, const SurConst& C, float (&v)[MLP_IN]) {
    const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
    const int e0 = (i + 1) + TILE_Y * (j + 1) + TILE_Z * (k + 1);
    bool all_in = true, all_out = true;
#pragma unroll
    for (int n = 0; n < MLP_IN; ++n) {
        const int sx = n % 3 - 1, sy = (n / 3) % 3 - 1, sz = n / 9 - 1;
        const float f = tile[e0 + sx + TILE_Y * sy + TILE_Z * sz];
        all_in &= -f >= C.h_up;
        all_out &= f >= C.h_up;
        v[n] = fminf(fmaxf(__fmul_rn(f, C.inv_h), -1.0f), 1.0f);
    }
    if (all_in) return SG_SUR_TRIVIAL_IN;
    if (all_out) return SG_SUR_TRIVIAL_OUT;
    const float c = tile[e0];
    if (fabsf(c) < C.h_up) return SG_SUR_FALLBACK;
    if (curvature_exceeds(tile[e0 + 1], tile[e0 - 1], tile[e0 + TILE_Y], tile[e0 - TILE_Y], tile[e0 + TILE_Z],
                          tile[e0 - TILE_Z], c, C))
        return SG_SUR_FALLBACK;
    return SG_SUR_NETWORK;
}

constexpr int SU_THREADS = 256;
constexpr int SU_PK = SU_THREADS / PKG3;  // packages per round
constexpr int SU_QROWS = SU_PK * PKG3;    // queue rows (all points of a round)
constexpr int SU_WARPS = SU_THREADS / 32;
// dynamic shared memory: weights | phi tiles | H tiles | queue rows | queue ids (hidden activations stay in
// registers, see forward_tile)
constexpr int SU_OFF_PHI = MLP_PACK_BYTES;
constexpr int SU_OFF_H = SU_OFF_PHI + SU_PK * TILE_N * 4;
constexpr int SU_OFF_QX = SU_OFF_H + SU_PK * TILE_N * 4;
constexpr int SU_OFF_QI = SU_OFF_QX + SU_QROWS * SX * 2;
constexpr int SU_BYTES = SU_OFF_QI + SU_QROWS * 8;
static_assert(SU_OFF_H % 16 == 0 && SU_OFF_QX % 16 == 0 && SU_OFF_QI % 16 == 0, "16-byte aligned regions");

// Stage the phi tile (and optionally the Heaviside tile) of package p.
__device__ __forceinline__ void stage_tile(const int* nb27, const float* __restrict__ phi, float inv_eps, int d,
                                           float* tphi, float* tH) {
    stage_rows(nb27, phi, inv_eps, d, tphi, tH);
}

// BATCH: packages of many bodies in one store; far packages (type < 2) are
// skipped and each package takes its body's constants.
template <bool BATCH>
__global__ void __launch_bounds__(SU_THREADS) k_sur_integrals(const int32_t* __restrict__ nbr,
                                                              const float* __restrict__ phi, float* __restrict__ W,
                                                              float* __restrict__ gx, float* __restrict__ gy,
                                                              float* __restrict__ gz, int64_t P, KernelCoef K,
                                                              float inv_eps0, SurConst C0,
                                                              const unsigned char* __restrict__ packed,
                                                              unsigned long long* __restrict__ stats,
                                                              const uint8_t* __restrict__ type,
                                                              const int32_t* __restrict__ body,
                                                              const SurBody* __restrict__ sb) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_nb[SU_PK][NB];
    __shared__ int s_qn;
    __shared__ unsigned s_cnt[4];
    const __nv_bfloat16* Wt = reinterpret_cast<const __nv_bfloat16*>(smem);
    const float* bias = reinterpret_cast<const float*>(smem + MLP_PACK_BIAS_BYTE);
    float* s_phi = reinterpret_cast<float*>(smem + SU_OFF_PHI);
    float* s_H = reinterpret_cast<float*>(smem + SU_OFF_H);
    __nv_bfloat16* s_qx = reinterpret_cast<__nv_bfloat16*>(smem + SU_OFF_QX);
    int64_t* s_qi = reinterpret_cast<int64_t*>(smem + SU_OFF_QI);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    stage_weights(smem, packed, MLP_PACK_BYTES);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    float* outs[4] = {W, gx, gy, gz};
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t rounds = (P - 2 + SU_PK - 1) / SU_PK;
    for (int64_t rd = blockIdx.x; rd < rounds; rd += gridDim.x) {
        const int64_t p = 2 + rd * SU_PK + lp;
        const bool valid = p < P && (!BATCH || __ldg(type + (p < P ? p : 0)) >= 2);
        SurConst C = C0;
        float inv_eps = inv_eps0;
        if (BATCH && valid) {
            const SurBody q = sb[__ldg(body + p)];
            C = q.C;
            inv_eps = q.inv_eps;
        }
        if (threadIdx.x == 0) s_qn = 0;
        if (valid && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
        __syncthreads();
        if (valid) stage_tile(s_nb[lp], phi, inv_eps, d, s_phi + lp * TILE_N, s_H + lp * TILE_N);
        __syncthreads();
        if (valid) {
            float v[MLP_IN];
            const int cls = sur_classify(s_phi + lp * TILE_N, d, C, v);
            atomicAdd(&s_cnt[cls], 1u);
            const int64_t at = p * PKG3 + d;
            if (cls == SG_SUR_NETWORK) {
                const int q = atomicAdd(&s_qn, 1);
                __nv_bfloat16* row = s_qx + q * SX;
#pragma unroll
                for (int n = 0; n < MLP_KIN; ++n) row[n] = __float2bfloat16_rn(n < MLP_IN ? v[n] : 0.0f);
                s_qi[q] = at;
            } else if (cls == SG_SUR_FALLBACK) {
                float w, ax, ay, az;
                integrals_point(s_H + lp * TILE_N, d, K, w, ax, ay, az);
                W[at] = w;
                gx[at] = ax;
                gy[at] = ay;
                gz[at] = az;
            } else {
                W[at] = cls == SG_SUR_TRIVIAL_IN ? 1.0f : 0.0f;
                gx[at] = 0.0f;
                gy[at] = 0.0f;
                gz[at] = 0.0f;
            }
        }
        __syncthreads();
        const int qn = s_qn;
        for (int tile = warp; tile * 16 < qn; tile += SU_WARPS) {
            __nv_bfloat16* X = s_qx + tile * 16 * SX;
            // rows past the queue end are zeroed so that the tile is defined
            for (int r = qn - tile * 16 + (lane >> 2); r < 16; r += 8)
                if (r >= 0)
                    for (int c = 8 * (lane & 3); c < 8 * (lane & 3) + 8; ++c) X[r * SX + c] = __float2bfloat16_rn(0.0f);
            __syncwarp();
            float y[4];
            forward_tile(Wt, bias, X, y);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = tile * 16 + g + 8 * (i >> 1), col = 2 * t + (i & 1);
                if (r < qn && col < MLP_OUT) outs[col][s_qi[r]] = y[i];
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (stats && threadIdx.x < 4) atomicAdd(stats + threadIdx.x, (unsigned long long)s_cnt[threadIdx.x]);
}

// class of every data point (255 for far packages)
__global__ void __launch_bounds__(SU_THREADS) k_sur_classify(const int32_t* __restrict__ nbr,
                                                             const float* __restrict__ phi, int64_t P, SurConst C,
                                                             uint8_t* __restrict__ cls) {
    __shared__ int s_nb[SU_PK][NB];
    __shared__ float s_phi[SU_PK][TILE_N];
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t p = (int64_t)blockIdx.x * SU_PK + lp;
    const bool act = p >= 2 && p < P;
    if (act && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
    __syncthreads();
    if (act) stage_tile(s_nb[lp], phi, 0.0f, d, s_phi[lp], nullptr);
    __syncthreads();
    if (p < P) {
        float v[MLP_IN];
        cls[p * PKG3 + d] = act ? (uint8_t)sur_classify(s_phi[lp], d, C, v) : (uint8_t)255;
    }
}

__device__ __forceinline__ bool keep_sample(uint64_t seed, int64_t pt, uint32_t keep24) {
    // SplitMix64 of (seed + point index); keep when its top 24 bits < keep24
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(pt + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z >> 40) < keep24;
}

// Training samples: network-class points kept by the hash, in point order.
// Pass 1 (offsets == nullptr) counts per package; pass 2 writes the rows.
__global__ void __launch_bounds__(SU_THREADS) k_sur_samples(const int32_t* __restrict__ nbr,
                                                            const float* __restrict__ phi, int64_t P, SurConst C,
                                                            uint64_t seed, uint32_t keep24,
                                                            uint32_t* __restrict__ counts,
                                                            const uint32_t* __restrict__ offsets, int64_t cap,
                                                            const float* __restrict__ W, const float* __restrict__ gx,
                                                            const float* __restrict__ gy, const float* __restrict__ gz,
                                                            __nv_bfloat16* __restrict__ xo, float* __restrict__ to) {
    __shared__ int s_nb[SU_PK][NB];
    __shared__ float s_phi[SU_PK][TILE_N];
    __shared__ unsigned s_ball[SU_PK][2];
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * SU_PK + lp;
    const bool act = p >= 2 && p < P;
    if (act && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
    __syncthreads();
    if (act) stage_tile(s_nb[lp], phi, 0.0f, d, s_phi[lp], nullptr);
    __syncthreads();
    float v[MLP_IN];
    const int64_t pt = p * PKG3 + d;
    const bool take = act && sur_classify(s_phi[lp], d, C, v) == SG_SUR_NETWORK && keep_sample(seed, pt, keep24);
    const unsigned ball = __ballot_sync(0xffffffffu, take);
    if (lane == 0) s_ball[lp][d >> 5] = ball;
    __syncthreads();
    if (!offsets) {
        if (act && d == 0) counts[p] = __popc(s_ball[lp][0]) + __popc(s_ball[lp][1]);
        return;
    }
    if (!take) return;
    const int rank = __popc(ball & ((1u << lane) - 1u)) + (d >= 32 ? __popc(s_ball[lp][0]) : 0);
    const int64_t row = (int64_t)offsets[p] + rank;
    if (row >= cap) return;
#pragma unroll
    for (int n = 0; n < MLP_KIN; ++n) xo[row * MLP_KIN + n] = __float2bfloat16_rn(n < MLP_IN ? v[n] : 0.0f);
    to[row * 4 + 0] = W[pt];
    to[row * 4 + 1] = gx[pt];
    to[row * 4 + 2] = gy[pt];
    to[row * 4 + 3] = gz[pt];
}

// The fallback's curvature bound |kappa| h > 0.1.
constexpr double SUR_KAPPA_H_MAX = 0.1;

SurConst sur_const_h(double h) {
    SurConst C;
    C.inv_h = (float)(1.0 / h);
    float up = (float)h;
    if ((double)up < h) up = std::nextafter(up, INFINITY);
    C.h_up = up;
    C.kap_thr = (float)(SUR_KAPPA_H_MAX * h);
    C.kap_thr_ff = split_ff(SUR_KAPPA_H_MAX * h);
    return C;
}

SurConst sur_const(const sg_grid* g) { return sur_const_h(g->desc.h); }

unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

sg_status m_fail(sg_mlp* m, sg_status st, const std::string& msg) {
    if (m) m->last_error = msg;
    return st;
}

}  // namespace

const unsigned char* mlp_packed(const sg_mlp* m) { return m->packed; }

}  // namespace sg

using namespace sg;

extern "C" {

sg_status sg_mlp_create(const float* params, void* stream, sg_mlp** out) {
    if (!params || !out) return SG_ERR_INVALID;
    *out = nullptr;
    sg_mlp* m = new (std::nothrow) sg_mlp();
    if (!m) return SG_ERR_OOM;
    m->stream = (cudaStream_t)stream;
    cudaGetDevice(&m->device);
    const size_t pb = MLP_NPARAM * sizeof(float);
    cudaError_t e = cudaMalloc(&m->master, 4 * pb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return SG_ERR_OOM;
    }
    m->m = m->master + MLP_NPARAM;
    m->v = m->m + MLP_NPARAM;
    m->grad = m->v + MLP_NPARAM;
    e = cudaMalloc(&m->packed, MLP_PACK_BYTES);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(m->master);
        delete m;
        return SG_ERR_OOM;
    }
    sg_status st = sg_mlp_set_params(m, params);
    if (st != SG_OK) {
        sg_mlp_destroy(m);
        return st;
    }
    *out = m;
    return SG_OK;
}

sg_status sg_mlp_destroy(sg_mlp* m) {
    if (!m) return SG_ERR_INVALID;
    if (m->master) cudaFree(m->master);
    if (m->packed) cudaFree(m->packed);
    delete m;
    return SG_OK;
}

sg_status sg_mlp_set_params(sg_mlp* m, const float* params) {
    if (!m || !params) return SG_ERR_INVALID;
    const size_t pb = MLP_NPARAM * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(m->master, params, pb, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, 3 * pb, m->stream);  // moments and gradient
    if (e == cudaSuccess) e = cudaMemsetAsync(m->packed, 0, MLP_PACK_BYTES, m->stream);
    if (e == cudaSuccess) {
        k_mlp_pack<<<cdiv(MLP_NPARAM, 256), 256, 0, m->stream>>>(m->master, m->packed);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);  // params may be a temporary host buffer
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("set_params: ") + cudaGetErrorString(e));
    m->step = 0;
    return SG_OK;
}

sg_status sg_mlp_get_params(sg_mlp* m, float* params) {
    if (!m || !params) return SG_ERR_INVALID;
    cudaError_t e = cudaMemcpyAsync(params, m->master, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("get_params: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_mlp_forward(sg_mlp* m, int64_t n, const void* x, float* y) {
    if (!m || n < 0 || (n > 0 && (!x || !y))) return SG_ERR_INVALID;
    if (n == 0) return SG_OK;
    const int smem = MLP_PACK_BYTES + 4 * 16 * SX * 2;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        unsigned blocks = cdiv(n, 64);
        if (blocks > 148 * 8) blocks = 148 * 8;
        k_mlp_forward<<<blocks, 128, smem, m->stream>>>(m->packed, n, (const __nv_bfloat16*)x, y);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_mlp_loss_grad(sg_mlp* m, int64_t n, const void* x, const float* t, const int32_t* idx, float* grad,
                           float* loss) {
    if (!m || n < 1 || !x || !t || !grad) return SG_ERR_INVALID;
    cudaError_t e = cudaMemsetAsync(grad, 0, MLP_NPARAM * sizeof(float), m->stream);
    if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_BYTES);
    if (e == cudaSuccess) {
        k_mlp_train<<<cdiv(n, TR_ROWS), TR_WARPS * 32, TR_BYTES, m->stream>>>(
            m->packed, n, (const __nv_bfloat16*)x, t, idx, 1.0f / (float)(n * MLP_OUT), grad, loss);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("loss_grad: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_mlp_train_step(sg_mlp* m, int64_t batch, const void* x, const float* t, const int32_t* idx, float lr,
                            float* loss) {
    if (!m || batch < 1 || !x || !t || !(lr >= 0.0f)) return SG_ERR_INVALID;
    cudaError_t e = cudaSuccess;
    if (loss) e = cudaMemsetAsync(loss, 0, sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_BYTES);
    if (e == cudaSuccess) {
        // the gradient buffer is zero here: k_adam clears it after every step
        k_mlp_train<<<cdiv(batch, TR_ROWS), TR_WARPS * 32, TR_BYTES, m->stream>>>(
            m->packed, batch, (const __nv_bfloat16*)x, t, idx, 1.0f / (float)(batch * MLP_OUT), m->grad, loss);
        m->step += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 - std::pow(b1, (double)m->step)), c2 = (float)(1.0 - std::pow(b2, (double)m->step));
        k_adam<<<cdiv(MLP_NPARAM, 256), 256, 0, m->stream>>>(m->master, m->grad, m->m, m->v, lr, (float)b1, (float)b2,
                                                             1e-8f, c1, c2);
        k_mlp_pack<<<cdiv(MLP_NPARAM, 256), 256, 0, m->stream>>>(m->master, m->packed);
        note_launch(3);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("train_step: ") + cudaGetErrorString(e));
    return SG_OK;
}

const char* sg_mlp_last_error(const sg_mlp* m) { return m ? m->last_error.c_str() : "null mlp"; }

sg_status sg_surrogate_classify(sg_grid* g, uint8_t* cls) {
    if (!g || !cls) return SG_ERR_INVALID;
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_surrogate_classify: phi not initialised");
    k_sur_classify<<<cdiv(g->P, SU_PK), SU_THREADS, 0, g->stream>>>((const int32_t*)g->nbr.p,
                                                                     (const float*)g->field[SG_FIELD_PHI].p, g->P,
                                                                     sur_const(g), cls);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "surrogate classify");
    return SG_OK;
}

sg_status sg_surrogate_samples(sg_grid* g, uint64_t seed, float keep, int64_t cap, void* x_bf16, float* t,
                               int64_t* count) {
    if (!g || !count || cap < 0 || !(keep >= 0.0f && keep <= 1.0f) || (cap > 0 && (!x_bf16 || !t)))
        return SG_ERR_INVALID;
    if (g->state < 2) return fail(g, SG_ERR_STATE, "sg_surrogate_samples: phi not initialised");
    if (field_fresh(g, SG_FIELD_W)) return fail(g, SG_ERR_STATE, "sg_surrogate_samples: no exact integrals");
    const int64_t P = g->P;
    const size_t cb = ((size_t)P * 4 + 255) & ~(size_t)255;
    if (!ensure(g, g->scratch, 2 * cb + scan_scratch_bytes(P) + 256))
        return fail(g, SG_ERR_OOM, "sg_surrogate_samples: out of memory");
    uint32_t* counts = (uint32_t*)g->scratch.p;
    uint32_t* offsets = (uint32_t*)((char*)g->scratch.p + cb);
    uint32_t* total = (uint32_t*)((char*)g->scratch.p + 2 * cb);
    void* scan_scratch = (char*)g->scratch.p + 2 * cb + 256;
    const SurConst C = sur_const(g);
    const uint32_t keep24 = keep >= 1.0f ? (1u << 24) : (uint32_t)(keep * 16777216.0f);
    const int32_t* nbr = (const int32_t*)g->nbr.p;
    const float* phi = (const float*)g->field[SG_FIELD_PHI].p;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)P * 4, g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "samples");
    k_sur_samples<<<cdiv(P, SU_PK), SU_THREADS, 0, g->stream>>>(nbr, phi, P, C, seed, keep24, counts, nullptr, 0,
                                                                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    note_launch();
    if ((e = exclusive_scan_u32(counts, offsets, P, total, scan_scratch, g->stream)) != cudaSuccess)
        return cuda_fail(g, e, "samples scan");
    if (cap > 0) {
        k_sur_samples<<<cdiv(P, SU_PK), SU_THREADS, 0, g->stream>>>(
            nbr, phi, P, C, seed, keep24, counts, offsets, cap, (const float*)g->field[SG_FIELD_W].p,
            (const float*)g->field[SG_FIELD_GWX].p, (const float*)g->field[SG_FIELD_GWY].p,
            (const float*)g->field[SG_FIELD_GWZ].p, (__nv_bfloat16*)x_bf16, t);
        note_launch();
    }
    if ((e = cudaMemcpyAsync(g->host_pin.p, total, 4, cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(g->stream)) != cudaSuccess)
        return cuda_fail(g, e, "samples count");
    *count = (int64_t)*(uint32_t*)g->host_pin.p;
    return SG_OK;
}

sg_status sg_surrogate_stats(sg_grid* g, int64_t* counts) {
    if (!g || !counts) return SG_ERR_INVALID;
    if (!g->stats.p) {
        for (int i = 0; i < 4; ++i) counts[i] = 0;
        return SG_OK;
    }
    unsigned long long h[4];
    cudaError_t e = cudaMemcpyAsync(h, g->stats.p, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "stats");
    for (int i = 0; i < 4; ++i) counts[i] = (int64_t)h[i];
    return SG_OK;
}

}  // extern "C"

namespace sg {

cudaError_t launch_surrogate_integrals(sg_grid* g, const sg_mlp* m, float* W, float* gx, float* gy, float* gz) {
    cudaError_t e;
    if ((e = launch_set_far(W, 1.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = launch_set_far(gx, 0.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = launch_set_far(gy, 0.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = launch_set_far(gz, 0.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g->stats.p, 0, 4 * sizeof(unsigned long long), g->stream)) != cudaSuccess) return e;
    if (g->P <= 2) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(k_sur_integrals<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SU_BYTES)) !=
        cudaSuccess)
        return e;
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sur_integrals<false>, SU_THREADS, SU_BYTES);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const int64_t rounds = (g->P - 2 + SU_PK - 1) / SU_PK;
    int64_t blocks = (int64_t)(per_sm < 1 ? 1 : per_sm) * (sms < 1 ? 1 : sms);
    if (blocks > rounds) blocks = rounds;
    k_sur_integrals<false><<<(unsigned)blocks, SU_THREADS, SU_BYTES, g->stream>>>(
        (const int32_t*)g->nbr.p, (const float*)g->field[SG_FIELD_PHI].p, W, gx, gy, gz, g->P, kernel_coef(),
        (float)(1.0 / g->desc.h), sur_const(g), m->packed, (unsigned long long*)g->stats.p, nullptr, nullptr,
        nullptr);
    note_launch();
    return cudaGetLastError();
}

SurBody sur_body(double h) {
    SurBody q;
    q.C = sur_const_h(h);
    q.inv_eps = (float)(1.0 / h);
    return q;
}

cudaError_t setup_batch_surrogate() {
    return cudaFuncSetAttribute(k_sur_integrals<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SU_BYTES);
}

cudaError_t launch_batch_surrogate_integrals(const int32_t* nbr, const uint8_t* type, const int32_t* body,
                                             const SurBody* sb, const float* phi, float* W, float* gx, float* gy,
                                             float* gz, int64_t P, const sg_mlp* m, int device, cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sur_integrals<true>, SU_THREADS, SU_BYTES);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int64_t rounds = (P - 2 + SU_PK - 1) / SU_PK;
    int64_t blocks = (int64_t)(per_sm < 1 ? 1 : per_sm) * (sms < 1 ? 1 : sms);
    if (blocks > rounds) blocks = rounds;
    k_sur_integrals<true><<<(unsigned)blocks, SU_THREADS, SU_BYTES, s>>>(nbr, phi, W, gx, gy, gz, P, kernel_coef(),
                                                                         0.0f, SurConst{}, m->packed, nullptr, type,
                                                                         body, sb);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sg
