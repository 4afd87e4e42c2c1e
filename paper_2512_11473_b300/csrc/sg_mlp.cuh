// sg_mlp.cuh -- layout constants of the surrogate network shared by the
// training kernels (sg_mlp.cu) and the fused integral kernel (sg_surrogate.cu).
#pragma once
#include "sg_internal.cuh"

namespace sg {

constexpr int MLP_IN = 27, MLP_KIN = 32, MLP_H = 64, MLP_OUT = 4;

// canonical parameter vector: W1[64][27], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_OUT * MLP_H;
constexpr int MLP_NPARAM = MLP_OFF_B3 + MLP_OUT;
static_assert(MLP_NPARAM == SG_MLP_NPARAM, "parameter count");

// packed device copy: bf16 row strides and offsets (elements), then FP32 biases
constexpr int MLP_S1 = MLP_KIN + 8, MLP_S2 = MLP_H + 8, MLP_S3T = 24;
constexpr int MLP_PK_W1T = 0;
constexpr int MLP_PK_W2 = MLP_PK_W1T + MLP_H * MLP_S1;
constexpr int MLP_PK_W3 = MLP_PK_W2 + MLP_H * MLP_S2;
constexpr int MLP_PK_W2T = MLP_PK_W3 + 8 * MLP_S2;
constexpr int MLP_PK_W3T = MLP_PK_W2T + MLP_H * MLP_S2;
constexpr int MLP_PK_BF16 = MLP_PK_W3T + MLP_H * MLP_S3T;
constexpr int MLP_PACK_BIAS_BYTE = MLP_PK_BF16 * 2;
constexpr int MLP_PACK_BYTES = MLP_PACK_BIAS_BYTE + (2 * MLP_H + 8) * 4;
static_assert(MLP_PACK_BIAS_BYTE % 16 == 0 && MLP_PACK_BYTES % 16 == 0, "packed layout alignment");

const unsigned char* mlp_packed(const sg_mlp* m);

}  // namespace sg
