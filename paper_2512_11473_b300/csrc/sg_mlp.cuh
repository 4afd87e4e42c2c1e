// sg_mlp.cuh -- layout of the surrogate network's parameters: the canonical
// FP32 vector shared with the host, and the packed device copy the tcgen05
// kernels stage in shared memory.
#pragma once
#include "sg_internal.cuh"

namespace sg {

constexpr int MLP_IN = 27, MLP_H = 64, MLP_OUT = 4;
constexpr int MLP_K1 = SG_MLP_ROW;  // layer-1 operand width: the input row (inputs, zero padding)
// Inputs as BF16 high and low parts (columns 27..53 carry v - bf16(v), met by
// the same weights) or as BF16 values alone.
constexpr bool MLP_SPLIT = MLP_K1 >= 2 * MLP_IN + 1;
constexpr int MLP_N3 = 16;          // layer-3 rows of the product (4 outputs, zero padded)
static_assert(MLP_K1 % 16 == 0 && MLP_K1 >= MLP_IN, "input row");

// canonical parameter vector: W1[64][27], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_OUT * MLP_H;
constexpr int MLP_NPARAM = MLP_OFF_B3 + MLP_OUT;
static_assert(MLP_NPARAM == SG_MLP_NPARAM, "parameter count");

// Packed device copy (bytes).  Each matrix is a K-major tensor-core operand
// in the no-swizzle core-matrix layout of sg_umma.cuh (rows = the product's
// N dimension); BF16.
//   W1 [64][K1]   layer 1, B operand (input columns >= 27 zero)
//   W2 [64][64]   layer 2, B operand
//   W3 [16][64]   layer 3, B operand (rows 4..15 zero)
//   b1[64], b2[64], b3[16] FP32                      -- the forward part ends here
//   W2T[64][64]   W2 transposed: B operand of dA1 = dZ2 W2
//   W3T[64][16]   W3 transposed (columns 4..15 zero): B operand of dA2 = dY W3
constexpr int PK_W1 = 0;
constexpr int PK_W2 = PK_W1 + MLP_H * MLP_K1 * 2;
constexpr int PK_W3 = PK_W2 + MLP_H * MLP_H * 2;
constexpr int PK_BIAS = PK_W3 + MLP_N3 * MLP_H * 2;
constexpr int PK_FWD_BYTES = (PK_BIAS + (2 * MLP_H + MLP_N3) * 4 + 127) / 128 * 128;
constexpr int PK_W2T = PK_FWD_BYTES;
constexpr int PK_W3T = PK_W2T + MLP_H * MLP_H * 2;
constexpr int PK_BYTES = PK_W3T + MLP_H * MLP_N3 * 2;
static_assert(PK_W2 % 128 == 0 && PK_W3 % 128 == 0 && PK_BIAS % 16 == 0 && PK_FWD_BYTES % 128 == 0 &&
                  PK_W3T % 128 == 0 && PK_BYTES % 16 == 0,
              "packed layout alignment");

const unsigned char* mlp_packed(const sg_mlp* m);
int* mlp_err(const sg_mlp* m);

}  // namespace sg
