// sg_mlp.cu -- the kernel-integral surrogate network on the fifth-generation
// tensor cores: 27 inputs -> 64 -> 64 -> 4 outputs, SiLU hidden activations,
// BF16 weights and activations, FP32 accumulation in tensor memory, FP32
// master weights and Adam (Kingma & Ba 2015).  Not in the paper: the learned
// stand-in for the kernel integral of "Integral with SPH Smoothing Kernel and
// Grid-Particle Coupling".
//
// Every product is a tcgen05.mma of M = 128 rows (one row per thread of a
// 128-thread CTA), operands K-major in shared memory (sg_umma.cuh), issued by
// one thread, completion signalled through an mbarrier:
//   forward   Z1 = X W1^T, Z2 = A1 W2^T, Y = A2 W3^T           (N = 64, 64, 16)
//   backward  dA2 = dY W3, dA1 = dZ2 W2                         (N = 64)
//   gradients [dZ1^T; dZ2^T] [X | A1] (one product, K = the 128 rows): the
//             diagonal blocks are dW1 and dW2, and a column of ones among X's
//             padding columns yields the bias gradients db1 and db2.
// Each CTA writes its partial gradient; a second kernel sums the partials in
// CTA order (training is reproducible), takes the Adam step and repacks the
// BF16 weights.
//
// Surrogate integrals (sg_kernel_integrals mode 1) run in two passes: pass A
// stages each package's tiles, classifies every data point, writes the
// trivial constants and the exact fallback sums (the code of mode 0) and
// appends network points to a list; pass B takes the list in 128-row tiles,
// gathers and canonicalises the inputs (sg_sur.cuh) and runs the network.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg_sur.cuh"

struct sg_mlp {
    cudaStream_t stream = nullptr;
    int device = 0;
    float *master = nullptr, *m = nullptr, *v = nullptr;
    unsigned char* packed = nullptr;
    float* part = nullptr;  // per-CTA partial gradients [ctas][MLP_NPARAM] and losses [ctas]
    int64_t part_ctas = 0;
    int* err = nullptr;  // device error word (ERR_TIMEOUT)
    int64_t step = 0;
    bool train_smem_set = false;  // the training kernel's shared-memory limit raised on this device
    std::string last_error;
};

namespace sg {
namespace {

constexpr int TC_ROWS = 128;               // rows of a tile = threads of a tensor-core CTA
constexpr uint32_t WAIT_POLLS = 1u << 20;  // bounded waits for a product (each poll is itself bounded)

// ---------------------------------------------------------------------------
// Parameters: canonical vector <-> packed operands
// ---------------------------------------------------------------------------

// Place canonical parameter k (value v) in the packed copy.
__device__ __forceinline__ void pack_param(int k, float v, unsigned char* __restrict__ packed) {
    using umma::kmajor_byte;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    float* bias = reinterpret_cast<float*>(packed + PK_BIAS);
    auto put = [&](int off, uint32_t byte) { *reinterpret_cast<__nv_bfloat16*>(packed + off + byte) = b; };
    if (k < MLP_OFF_B1) {
        const int o = k / MLP_IN, i = k % MLP_IN;
        put(PK_W1, kmajor_byte(o, i, MLP_K1));
        if (MLP_SPLIT) put(PK_W1, kmajor_byte(o, MLP_IN + i, MLP_K1));  // the low parts meet the same weight
    } else if (k < MLP_OFF_W2) {
        bias[k - MLP_OFF_B1] = v;
    } else if (k < MLP_OFF_B2) {
        const int o = (k - MLP_OFF_W2) / MLP_H, i = (k - MLP_OFF_W2) % MLP_H;
        put(PK_W2, kmajor_byte(o, i, MLP_H));
        put(PK_W2T, kmajor_byte(i, o, MLP_H));
    } else if (k < MLP_OFF_W3) {
        bias[MLP_H + k - MLP_OFF_B2] = v;
    } else if (k < MLP_OFF_B3) {
        const int o = (k - MLP_OFF_W3) / MLP_H, i = (k - MLP_OFF_W3) % MLP_H;
        put(PK_W3, kmajor_byte(o, i, MLP_H));
        put(PK_W3T, kmajor_byte(i, o, MLP_N3));
    } else {
        bias[2 * MLP_H + k - MLP_OFF_B3] = v;
    }
}

__global__ void k_mlp_pack(const float* __restrict__ master, unsigned char* __restrict__ packed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < MLP_NPARAM) pack_param(k, master[k], packed);
}

// Sums of the per-CTA partials in CTA order: the gradient (and loss) of the
// whole batch, independent of scheduling.
//
// Sum over c = 0 .. n-1 of a[c * stride], added in order of c, by the four
// lanes of an aligned lane quad: for each block of 128 terms, lane j of the
// quad loads terms 32 j .. 32 j + 31 (all 32 in flight at once), then lane 0
// adds its terms to the running sum, hands it to lane 1 by a shuffle, and so
// on: the same additions in the same order as one thread walking c = 0 .. n-1,
// with one memory latency per 128 terms.  Every lane of the warp must call it
// (with `active` false for quads without a sum); every lane of a quad gets
// the sum.
__device__ __forceinline__ float ordered_sum_quad(const float* __restrict__ a, int n, int64_t stride, bool active) {
    const int lane = threadIdx.x & 31, j = lane & 3, base = lane & ~3;
    float s = 0.0f;
    for (int c0 = 0; c0 < n; c0 += 128) {
        float q[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int c = c0 + 32 * j + u;
            q[u] = (active && c < n) ? a[(int64_t)c * stride] : 0.0f;
        }
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            if (j == st) {
#pragma unroll
                for (int u = 0; u < 32; ++u)
                    if (c0 + 32 * st + u < n) s += q[u];
            }
            s = __shfl_sync(0xffffffffu, s, base + st);
        }
    }
    return s;
}

// Threads of the partial-sum kernels: a lane quad per parameter.
constexpr int SUM_THREADS = 256;
inline unsigned sum_blocks() { return (unsigned)((4 * MLP_NPARAM + SUM_THREADS - 1) / SUM_THREADS); }

// The loss: the CTAs' loss shares in CTA order, by warp 0 of CTA 0.
__device__ __forceinline__ void sum_loss(const float* __restrict__ part, int ctas, float* __restrict__ loss) {
    if (loss && blockIdx.x == 0 && threadIdx.x < 32) {
        const float l = ordered_sum_quad(part + (int64_t)ctas * MLP_NPARAM, ctas, 1, true);
        if (threadIdx.x == 0) *loss = l;
    }
}

// The gradient and loss of the batch (sg_mlp_loss_grad).
__global__ void __launch_bounds__(SUM_THREADS) k_mlp_grad_sum(const float* __restrict__ part, int ctas,
                                                              float* __restrict__ grad, float* __restrict__ loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, k = e >> 2;
    const bool act = k < MLP_NPARAM;
    const float g = ordered_sum_quad(part + (act ? k : 0), ctas, MLP_NPARAM, act);
    if (act && (e & 3) == 0) grad[k] = g;
    sum_loss(part, ctas, loss);
}

// Ordered sum of the partials, bias-corrected Adam step on the master
// weights, repacking of the BF16 copy.
__global__ void __launch_bounds__(SUM_THREADS) k_mlp_adam(const float* __restrict__ part, int ctas,
                                                          float* __restrict__ master, float* __restrict__ m,
                                                          float* __restrict__ v, unsigned char* __restrict__ packed,
                                                          float lr, float beta1, float beta2, float eps, float c1,
                                                          float c2, float* __restrict__ loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, k = e >> 2;
    const bool act = k < MLP_NPARAM;
    const float g = ordered_sum_quad(part + (act ? k : 0), ctas, MLP_NPARAM, act);
    if (act && (e & 3) == 0) {
        const float mk = beta1 * m[k] + (1.0f - beta1) * g;
        const float vk = beta2 * v[k] + (1.0f - beta2) * g * g;
        m[k] = mk;
        v[k] = vk;
        const float w = master[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        master[k] = w;
        pack_param(k, w, packed);
    }
    sum_loss(part, ctas, loss);
}

// ---------------------------------------------------------------------------
// Tensor-core tile machinery
// ---------------------------------------------------------------------------
// The threads that work one tile: the whole CTA of 128 threads (group 0,
// synchronised by __syncthreads), or one of the 128-thread warpgroups of a
// larger CTA (group g >= 0 with named barrier 1 + g).
struct Tc {
    uint32_t tmem;   // TMEM address of the group's columns
    uint64_t* bar;   // completion barrier of the group's products
    uint32_t phase;  // parity of the next completion
    bool ok;         // every wait so far completed (uniform over the group)
    int group;       // -1: the whole CTA; else the warpgroup, named barrier 1 + group
};

__device__ __forceinline__ int tc_row() { return threadIdx.x & (TC_ROWS - 1); }

// The thread that issues the group's products: the group's first thread, or
// thread 0 when the whole CTA (of one or more warpgroups on the same rows)
// works one tile.
__device__ __forceinline__ bool tc_issuer(const Tc& t) { return t.group < 0 ? threadIdx.x == 0 : tc_row() == 0; }

__device__ __forceinline__ void tc_sync(const Tc& t) {
    if (t.group < 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + t.group), "r"(TC_ROWS) : "memory");
}

__device__ __forceinline__ bool tc_sync_and(const Tc& t, bool v) {
    if (t.group < 0) return __syncthreads_and(v) != 0;
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(1 + t.group), "r"(TC_ROWS)
        : "memory");
    return r != 0;
}

// Warp 0 allocates ncols TMEM columns for the whole CTA and thread 0
// initialises one barrier per group (bars[0 .. groups)); group g (or the
// whole CTA, groups = 0) then uses columns [g ncols / groups, ...).
__device__ __forceinline__ Tc tc_begin(uint64_t* bars, uint32_t* slot, uint32_t ncols, int groups = 0) {
    if (threadIdx.x < 32) umma::tmem_alloc(slot, ncols);
    if (threadIdx.x == 0)
        for (int g = 0; g < (groups > 0 ? groups : 1); ++g) umma::mbar_init(bars + g, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    Tc t;
    t.group = groups > 0 ? (int)(threadIdx.x / TC_ROWS) : -1;
    const int g = t.group < 0 ? 0 : t.group;
    t.tmem = *slot + (uint32_t)(groups > 0 ? g * (int)(ncols / groups) : 0);
    t.bar = bars + g;
    t.phase = 0;
    t.ok = true;
    return t;
}

// Make this thread's shared-memory operand stores visible to the tensor
// core and order its TMEM reads before the next product.
__device__ __forceinline__ void tc_publish(const Tc& t) {
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    tc_sync(t);
}

// D (TMEM columns from tcol) = A B^T, A and B K-major with K columns, N
// columns of D; the group's first thread issues the K / 16 products and
// commits.
__device__ __forceinline__ void tc_gemm(const Tc& t, uint32_t tcol, const unsigned char* A, const unsigned char* B,
                                        int K, int N) {
    if (tc_issuer(t)) {
        umma::fence_after_sync();
        const uint32_t id = umma::idesc_bf16(TC_ROWS, N), sa = umma::smem_u32(A), sb = umma::smem_u32(B);
        for (int k = 0; k < K; k += 16)
            umma::mma(t.tmem + tcol, umma::kslice_desc(sa, K, k), umma::kslice_desc(sb, K, k), id, k > 0 ? 1u : 0u);
        umma::commit(t.bar);
    }
}

// Every thread of the group waits for the products committed last.
__device__ __forceinline__ bool tc_wait(Tc& t) {
    const bool done = umma::mbar_wait(t.bar, t.phase, WAIT_POLLS);
    t.ok = tc_sync_and(t, done);
    if (t.ok) t.phase ^= 1u;
    umma::fence_after_sync();
    return t.ok;
}

// Free the CTA's TMEM columns (every group done); after a wait that gave up,
// first wait (bounded) for the group's product still in flight and raise
// ERR_TIMEOUT.
__device__ __forceinline__ void tc_end(Tc& t, uint32_t slot_base, uint32_t ncols, int* err) {
    if (!t.ok && tc_issuer(t)) {
        umma::mbar_wait(t.bar, t.phase, WAIT_POLLS);
        if (err) atomicOr(err, ERR_TIMEOUT);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (threadIdx.x < 32) umma::tmem_dealloc(slot_base, ncols);
}

__device__ __forceinline__ uint32_t lane_col(const Tc& t, int col) {
    return umma::tmem_lane_addr(t.tmem, threadIdx.x >> 5, col);
}

// 32 consecutive accumulator columns of this thread's row.
__device__ __forceinline__ void tc_ld32(const Tc& t, int col, float (&v)[32]) {
    float a[16], b[16];
    umma::tmem_ld16(lane_col(t, col), a);
    umma::tmem_ld16(lane_col(t, col + 16), b);
    umma::tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = a[i], v[16 + i] = b[i];
}

// Hidden layer out of TMEM: row r of the 32 columns of half h at tcol, plus
// bias, SiLU, rounded to BF16 into the K-major operand A ([128][64]).
__device__ __forceinline__ void tc_hidden_half(const Tc& t, int tcol, const float* bias, unsigned char* A, int h) {
    const int r = tc_row();
    float v[32];
    tc_ld32(t, tcol + 32 * h, v);
    silu32_bias(v, bias + 32 * h);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(A + umma::kmajor_byte(r, 32 * h + 8 * q, MLP_H)) = umma::pack8_bf16(v + 8 * q);
}

// Both halves (the 64 columns) by this thread.
__device__ __forceinline__ void tc_hidden(const Tc& t, int tcol, const float* bias, unsigned char* A) {
#pragma unroll
    for (int h = 0; h < 2; ++h) tc_hidden_half(t, tcol, bias, A, h);
}

// The three layers of one 128-row tile: T holds the K-major input rows
// ([128][K1]) and is reused for the hidden activations ([128][64]); y gets
// this thread's four outputs.  W is the packed forward part in shared memory.
__device__ __forceinline__ void tc_forward(Tc& t, const unsigned char* W, unsigned char* T, float (&y)[4]) {
    const float* bias = reinterpret_cast<const float*>(W + PK_BIAS);
    tc_publish(t);
    tc_gemm(t, 0, T, W + PK_W1, MLP_K1, MLP_H);
    if (!tc_wait(t)) return;
    tc_hidden(t, 0, bias, T);  // layer 1 has read the inputs
    tc_publish(t);
    tc_gemm(t, 0, T, W + PK_W2, MLP_H, MLP_H);
    if (!tc_wait(t)) return;
    tc_hidden(t, 0, bias + MLP_H, T);
    tc_publish(t);
    tc_gemm(t, 0, T, W + PK_W3, MLP_H, MLP_N3);
    if (!tc_wait(t)) return;
    float v[16];
    umma::tmem_ld16(lane_col(t, 0), v);
    umma::tmem_wait_ld();
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) y[o] = v[o] + bias[2 * MLP_H + o];
}

__device__ __forceinline__ void stage_bytes(unsigned char* dst, const unsigned char* __restrict__ src, int bytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

constexpr int FWD_T = PK_FWD_BYTES;               // tile operand after the forward weights
constexpr int FWD_BYTES = FWD_T + TC_ROWS * MLP_H * 2;  // (input rows need at most as much as A)
static_assert(MLP_K1 <= MLP_H, "the input tile fits the activation tile");

// y[n][4] = network(x[n][K1]) on raw input rows.
__global__ void __launch_bounds__(TC_ROWS) k_mlp_forward(const unsigned char* __restrict__ packed, int64_t n,
                                                          const __nv_bfloat16* __restrict__ x, float* __restrict__ y,
                                                          int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    stage_bytes(smem, packed, PK_FWD_BYTES);
    unsigned char* T = smem + FWD_T;
    Tc t = tc_begin(&bar, &slot, 64);
    const uint32_t tbase = t.tmem;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    for (int64_t tile = blockIdx.x; tile < tiles && t.ok; tile += gridDim.x) {
        const int64_t row = tile * TC_ROWS + threadIdx.x;
#pragma unroll
        for (int c = 0; c < MLP_K1 / 8; ++c) {
            const uint4 v = row < n ? __ldg(reinterpret_cast<const uint4*>(x + row * MLP_K1) + c) : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(T + umma::kmajor_byte(threadIdx.x, 8 * c, MLP_K1)) = v;
        }
        float o[4];
        tc_forward(t, smem, T, o);
        if (t.ok && row < n) *reinterpret_cast<float4*>(y + row * MLP_OUT) = make_float4(o[0], o[1], o[2], o[3]);
    }
    tc_end(t, tbase, 64, err);
}

// ---------------------------------------------------------------------------
// Training: forward, backward and the partial gradient of 128 rows per CTA.
// ---------------------------------------------------------------------------
constexpr int NG = MLP_K1 + MLP_H;  // rows of the gradient product's B operand: X^T then A1^T
constexpr int ONES = MLP_K1 - 1;    // a padding input column: its B row holds ones (bias gradients)
static_assert(NG % 16 == 0 && NG <= 256, "gradient product width");
constexpr int TR_X = (PK_BYTES + 127) / 128 * 128;
constexpr int TR_A1 = TR_X + TC_ROWS * MLP_K1 * 2;
constexpr int TR_A2 = TR_A1 + TC_ROWS * MLP_H * 2;
constexpr int TR_DY = TR_A2 + TC_ROWS * MLP_H * 2;
constexpr int TR_DZ2 = TR_DY + TC_ROWS * MLP_N3 * 2;
constexpr int TR_AG = TR_DZ2 + TC_ROWS * MLP_H * 2;  // [128 features][128 rows]: dZ1^T then dZ2^T
constexpr int TR_BG = TR_AG + 128 * TC_ROWS * 2;     // [NG][128 rows]
constexpr int TR_RED = TR_BG + NG * TC_ROWS * 2;
constexpr int TR_BYTES = TR_RED + TC_ROWS * 4;
// TMEM columns of the training kernel
constexpr int TM_Z1 = 0, TM_Z2 = 64, TM_Y = 128, TM_DA = 192, TM_G = 0;

__device__ __forceinline__ void put_bf16(unsigned char* base, uint32_t byte, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + byte) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ float get_bf16(const unsigned char* base, uint32_t byte) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + byte));
}

// The threads of the training kernel: TR_GROUPS warpgroups work the same 128
// rows (thread r of each: row r, in the TMEM lane quarter of its warp).
// Every epilogue over 64 columns is split between the groups, group g
// taking columns TR_CW g .. TR_CW g + TR_CW - 1, so each thread's serial chain
// of TMEM loads, SiLU and operand stores is 1 / TR_GROUPS as long as with one
// thread per row.  Every value is formed by the same operations whatever the
// split.
constexpr int TR_GROUPS = 4;  // (two groups: 18.7 us per batch of 16384 against 18.4 us)
constexpr int TR_THREADS = TR_GROUPS * TC_ROWS;
constexpr int TR_CW = MLP_H / TR_GROUPS;
static_assert(TR_GROUPS >= 2 && TR_CW % 16 == 0, "column split of the training epilogues");

// N consecutive accumulator columns of this thread's row (N a multiple of 16).
template <int N>
__device__ __forceinline__ void tc_ldn(const Tc& t, int col, float (&v)[N]) {
#pragma unroll
    for (int c = 0; c < N; c += 16) {
        float a[16];
        umma::tmem_ld16(lane_col(t, col + c), a);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[c + i] = a[i];
    }
    umma::tmem_wait_ld();
}

// v[i] = silu_(v[i] + bias[i]) for N consecutive columns (the pairs of
// silu32_bias: the same bits)
template <int N>
__device__ __forceinline__ void silu_bias_n(float (&v)[N], const float* bias) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        const float2 s = silu2_bias(make_float2(v[i], v[i + 1]), *reinterpret_cast<const float2*>(bias + i));
        v[i] = s.x;
        v[i + 1] = s.y;
    }
}

// Copy `bytes` (a multiple of 16) from global to shared memory with up to
// eight 16-byte loads per thread in flight.
__device__ __forceinline__ void stage_bytes_ahead(unsigned char* dst, const unsigned char* __restrict__ src, int bytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    const int n = bytes / 16;
    for (int b = threadIdx.x; b < n; b += 8 * blockDim.x) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = b + u * (int)blockDim.x;
            if (i < n) v[u] = __ldg(s + i);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = b + u * (int)blockDim.x;
            if (i < n) d[i] = v[u];
        }
    }
}

// The gradient product's output rows (hidden units) m against columns
// C0 .. C0 + 15: row m < 64 is unit m of layer 1 (columns: the inputs, the
// ones column for the bias), row m >= 64 unit m - 64 of layer 2 (columns
// K1 .. K1 + 63: the layer-1 activations).
template <int C0>
__device__ __forceinline__ void grad_chunk(const Tc& t, int m, float* __restrict__ pg) {
    float v[16];
    tc_ldn<16>(t, TM_G + C0, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int c = C0 + i;
        if (m < MLP_H) {
            if (c < MLP_IN) pg[MLP_OFF_W1 + m * MLP_IN + c] = v[i];
            if (c == ONES) pg[MLP_OFF_B1 + m] = v[i];
        } else {
            if (c >= MLP_K1) pg[MLP_OFF_W2 + (m - MLP_H) * MLP_H + (c - MLP_K1)] = v[i];
            if (c == ONES) pg[MLP_OFF_B2 + (m - MLP_H)] = v[i];
        }
    }
    if (MLP_SPLIT && m < MLP_H) {
        // columns 27..53 carry the low parts of the same inputs
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = C0 + i;
            if (c >= MLP_IN && c < 2 * MLP_IN) pg[MLP_OFF_W1 + m * MLP_IN + (c - MLP_IN)] += v[i];
        }
    }
}

// Chunk q (columns 16 q .. 16 q + 15) of the gradient product.
__device__ __forceinline__ void grad_chunk_q(const Tc& t, int q, int m, float* __restrict__ pg) {
    static_assert(NG == 96, "six 16-column chunks of the gradient product");
    switch (q) {
        case 0: grad_chunk<0>(t, m, pg); break;
        case 1: grad_chunk<16>(t, m, pg); break;
        case 2: grad_chunk<32>(t, m, pg); break;
        case 3: grad_chunk<48>(t, m, pg); break;
        case 4: grad_chunk<64>(t, m, pg); break;
        default: grad_chunk<80>(t, m, pg); break;
    }
}

// Gradient of L = scale * sum over rows and outputs of (y - t)^2 for rows
// idx[0..n) (or 0..n): CTA c writes part[c][MLP_NPARAM] and its loss share
// part[gridDim.x * MLP_NPARAM + c].
__global__ void __launch_bounds__(TR_THREADS, 1) k_mlp_train(const unsigned char* __restrict__ packed, int64_t n,
                                                              const __nv_bfloat16* __restrict__ x,
                                                              const float* __restrict__ tgt,
                                                              const int32_t* __restrict__ idx, float scale,
                                                              float* __restrict__ part, int* err) {
    using umma::kmajor_byte;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const unsigned char* W = smem;
    const float* bias = reinterpret_cast<const float*>(smem + PK_BIAS);
    unsigned char *X = smem + TR_X, *A1 = smem + TR_A1, *A2 = smem + TR_A2, *DY = smem + TR_DY,
                  *DZ2 = smem + TR_DZ2, *AG = smem + TR_AG, *BG = smem + TR_BG;
    float* red = reinterpret_cast<float*>(smem + TR_RED);
    const int r = tc_row();
    const int g = threadIdx.x / TC_ROWS;  // warpgroup: columns TR_CW g ..
    const int cg = TR_CW * g;
    const int64_t row = (int64_t)blockIdx.x * TC_ROWS + r;
    const bool valid = row < n;
    const int64_t src = valid ? (idx ? (int64_t)__ldg(idx + row) : row) : 0;
    // the row's targets, read ahead for the loss (group 0)
    float tv[MLP_OUT];
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) tv[o] = (g == 0 && valid) ? __ldg(tgt + src * MLP_OUT + o) : 0.0f;
    // the row's inputs, read ahead of the weights
    uint4 xv[MLP_K1 / 8];
#pragma unroll
    for (int c = 0; c < MLP_K1 / 8; ++c)
        xv[c] = valid ? __ldg(reinterpret_cast<const uint4*>(x + src * MLP_K1) + c) : make_uint4(0, 0, 0, 0);
    stage_bytes_ahead(smem, packed, PK_BYTES);
    // inputs: X (K-major rows, group 0) and X^T (rows 0..K1-1 of the gradient
    // product's B, shared by the other groups; row ONES = 1)
    {
        __align__(16) __nv_bfloat16 xr[MLP_K1];
#pragma unroll
        for (int c = 0; c < MLP_K1 / 8; ++c) {
            const uint4 v = xv[c];
            if (g == 0)
                *reinterpret_cast<uint4*>(X + kmajor_byte(r, 8 * c, MLP_K1)) = v;
            else
                *reinterpret_cast<uint4*>(xr + 8 * c) = v;
        }
        if (g > 0) {
#pragma unroll
            for (int c = 0; c < MLP_K1; ++c)
                if (c % (TR_GROUPS - 1) == g - 1)
                    *reinterpret_cast<__nv_bfloat16*>(BG + kmajor_byte(c, r, TC_ROWS)) =
                        c == ONES ? __float2bfloat16_rn(1.0f) : xr[c];
        }
    }
    Tc t = tc_begin(&bar, &slot, 256);
    const uint32_t tbase = t.tmem;
    float* pg = part + (int64_t)blockIdx.x * MLP_NPARAM;
    float s3 = 0.0f;  // this thread's dW3 / db3 sum (the last thread: the loss share)
    static_assert(TR_THREADS > MLP_OUT * (MLP_H + 1), "one dW3 / db3 sum per thread, and a thread for the loss");
    do {
        // layer 1
        tc_publish(t);
        tc_gemm(t, TM_Z1, X, W + PK_W1, MLP_K1, MLP_H);
        if (!tc_wait(t)) break;
        {
            float v[TR_CW];
            tc_ldn<TR_CW>(t, TM_Z1 + cg, v);
            silu_bias_n<TR_CW>(v, bias + cg);
#pragma unroll
            for (int q = 0; q < TR_CW / 8; ++q)
                *reinterpret_cast<uint4*>(A1 + kmajor_byte(r, cg + 8 * q, MLP_H)) = umma::pack8_bf16(v + 8 * q);
#pragma unroll
            for (int i = 0; i < TR_CW; ++i) put_bf16(BG, kmajor_byte(MLP_K1 + cg + i, r, TC_ROWS), v[i]);
        }
        // layer 2
        tc_publish(t);
        tc_gemm(t, TM_Z2, A1, W + PK_W2, MLP_H, MLP_H);
        if (!tc_wait(t)) break;
        {
            float v[TR_CW];
            tc_ldn<TR_CW>(t, TM_Z2 + cg, v);
            silu_bias_n<TR_CW>(v, bias + MLP_H + cg);
#pragma unroll
            for (int q = 0; q < TR_CW / 8; ++q)
                *reinterpret_cast<uint4*>(A2 + kmajor_byte(r, cg + 8 * q, MLP_H)) = umma::pack8_bf16(v + 8 * q);
        }
        // layer 3, loss, dY (group 0: the 16 output columns)
        tc_publish(t);
        tc_gemm(t, TM_Y, A2, W + PK_W3, MLP_H, MLP_N3);
        if (!tc_wait(t)) break;
        if (g == 0) {
            float v[16], dy[16];
            umma::tmem_ld16(lane_col(t, TM_Y), v);
            umma::tmem_wait_ld();
            float l = 0.0f;
#pragma unroll
            for (int o = 0; o < 16; ++o) dy[o] = 0.0f;
#pragma unroll
            for (int o = 0; o < MLP_OUT; ++o) {
                if (valid) {
                    const float e = v[o] + bias[2 * MLP_H + o] - tv[o];
                    l += e * e * scale;
                    dy[o] = 2.0f * e * scale;
                }
            }
            red[r] = l;
#pragma unroll
            for (int q = 0; q < 2; ++q)
                *reinterpret_cast<uint4*>(DY + kmajor_byte(r, 8 * q, MLP_N3)) = umma::pack8_bf16(dy + 8 * q);
        }
        // dA2 = dY W3, dZ2 = dA2 SiLU'(z2)
        tc_publish(t);
        tc_gemm(t, TM_DA, DY, W + PK_W3T, MLP_N3, MLP_H);
        if (!tc_wait(t)) break;
        {
            float da[TR_CW], z[TR_CW];
            tc_ldn<TR_CW>(t, TM_DA + cg, da);
            tc_ldn<TR_CW>(t, TM_Z2 + cg, z);
#pragma unroll
            for (int i = 0; i < TR_CW; ++i) {
                const float zz = z[i] + bias[MLP_H + cg + i], s = sigmoidf_(zz);
                da[i] *= s * (1.0f + zz * (1.0f - s));
            }
#pragma unroll
            for (int q = 0; q < TR_CW / 8; ++q)
                *reinterpret_cast<uint4*>(DZ2 + kmajor_byte(r, cg + 8 * q, MLP_H)) = umma::pack8_bf16(da + 8 * q);
#pragma unroll
            for (int i = 0; i < TR_CW; ++i) put_bf16(AG, kmajor_byte(MLP_H + cg + i, r, TC_ROWS), da[i]);
        }
        // dA1 = dZ2 W2, dZ1 = dA1 SiLU'(z1)
        tc_publish(t);
        tc_gemm(t, TM_DA, DZ2, W + PK_W2T, MLP_H, MLP_H);
        if (!tc_wait(t)) break;
        {
            float da[TR_CW], z[TR_CW];
            tc_ldn<TR_CW>(t, TM_DA + cg, da);
            tc_ldn<TR_CW>(t, TM_Z1 + cg, z);
#pragma unroll
            for (int i = 0; i < TR_CW; ++i) {
                const float zz = z[i] + bias[cg + i], s = sigmoidf_(zz);
                put_bf16(AG, kmajor_byte(cg + i, r, TC_ROWS), da[i] * (s * (1.0f + zz * (1.0f - s))));
            }
        }
        // [dZ1^T; dZ2^T] [X | A1]: dW1, db1 (rows 0..63), dW2, db2 (rows 64..127)
        tc_publish(t);
        tc_gemm(t, TM_G, AG, BG, TC_ROWS, NG);
        // while that product runs: dW3 = dY^T A2 and db3 on the CUDA cores
        // (4 x 65 sums over the rows in row order, one per thread; stored
        // below once the product has completed)
        if (threadIdx.x < MLP_OUT * (MLP_H + 1)) {
            const int o = threadIdx.x / (MLP_H + 1), i = threadIdx.x % (MLP_H + 1), ia = i < MLP_H ? i : 0;
#pragma unroll 1
            for (int k0 = 0; k0 < TC_ROWS; k0 += 16) {
                float dyv[16], av[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    dyv[u] = get_bf16(DY, kmajor_byte(k0 + u, o, MLP_N3));
                    av[u] = get_bf16(A2, kmajor_byte(k0 + u, ia, MLP_H));
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) s3 += i < MLP_H ? dyv[u] * av[u] : dyv[u];
            }
        } else if (threadIdx.x == TR_THREADS - 1) {
            // and the CTA's loss share, in row order
#pragma unroll 16
            for (int k = 0; k < TC_ROWS; ++k) s3 += red[k];
        }
        if (!tc_wait(t)) break;
        if (MLP_SPLIT) {
            // the low-part columns add into entries of several chunks: one thread per row
            if (g == 0)
                for (int q = 0; q < NG / 16; ++q) grad_chunk_q(t, q, r, pg);
        } else {
            for (int q = g; q < NG / 16; q += TR_GROUPS) grad_chunk_q(t, q, r, pg);
        }
    } while (false);
    __syncthreads();
    if (t.ok) {
        if (threadIdx.x < MLP_OUT * (MLP_H + 1)) {
            const int o = threadIdx.x / (MLP_H + 1), i = threadIdx.x % (MLP_H + 1);
            if (i < MLP_H)
                pg[MLP_OFF_W3 + o * MLP_H + i] = s3;
            else
                pg[MLP_OFF_B3 + o] = s3;
        }
        if (threadIdx.x == TR_THREADS - 1) part[(int64_t)gridDim.x * MLP_NPARAM + blockIdx.x] = s3;
    }
    tc_end(t, tbase, 256, err);
}

// ---------------------------------------------------------------------------
// Surrogate integrals, pass A: classes, trivial constants, exact fallback,
// list of network points.
// ---------------------------------------------------------------------------
constexpr int SA_WARPS = 8;  // warps per CTA
#ifndef SG_SA_MIN_CTAS
#define SG_SA_MIN_CTAS 4
#endif

// The structure of the exact kernel (k_kernel_integrals): each warp takes
// pairs of packages in turn and stages their Heaviside tiles by x-rows; it
// also keeps the phi tiles (for the curvature) and a row mask per tile row
// (bit i of the low byte: value i >= h, of the high byte: -value >= h, the
// exact comparisons of sur_class_at).  A package whose whole tile lies at
// |phi| >= h on one side is trivial without per-point work; otherwise each
// lane classifies its row of four points from the AND of the 3 x 3 masks
// around it and the fallback test.  Trivial points get the exact constants,
// fallback points the exact sums exactly as mode 0 forms them, and network
// points (written 0 here) go on the list, one reservation per warp.  With
// BATCH, packages of type < 2 are skipped and every package takes its body's
// constants.
template <bool BATCH>
__global__ void __launch_bounds__(SA_WARPS * 32, SG_SA_MIN_CTAS)
    k_sur_a(const int32_t* __restrict__ nbr, const float* __restrict__ phi, float* __restrict__ W,
            float* __restrict__ gx, float* __restrict__ gy, float* __restrict__ gz, int64_t P, KernelCoef K,
            SurBody B0, const uint8_t* __restrict__ type, const int32_t* __restrict__ body,
            const SurBody* __restrict__ sb, int32_t* __restrict__ list, unsigned* __restrict__ count,
            unsigned long long* __restrict__ stats) {
    __shared__ __align__(16) float s_H[SA_WARPS][2][TILE_N];
    __shared__ __align__(16) float s_phi[SA_WARPS][2][TILE_N];
    __shared__ uint16_t s_mask[SA_WARPS][2][36];
    __shared__ int s_nb[SA_WARPS][2][32];
    __shared__ SurBody s_B[SA_WARPS][2];
    __shared__ unsigned s_cnt[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    float(*tH)[TILE_N] = s_H[warp];
    float(*tP)[TILE_N] = s_phi[warp];
    uint16_t(*tM)[36] = s_mask[warp];
    int(*tnb)[32] = s_nb[warp];
    // staging rows of this lane: e = lane, lane + 32, lane + 64 (< 72):
    // package e / 36, row e % 36; each row's indices packed in one word
    // (package + 1: 2 bits, row: 6, neighbour slot: 5, first element in the
    // package: 6, tile offset: 8)
    unsigned r_w[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = lane + 32 * q, rr = e % 36;
        const int y = rr % 6 - 1, z = rr / 6 - 1;
        const int oy = ((y + 4) >> 2) - 1, oz = ((z + 4) >> 2) - 1;
        const unsigned pk1 = e < 72 ? (unsigned)(e / 36 + 1) : 0u;
        const unsigned nbs = (unsigned)(3 * (oy + 1) + 9 * (oz + 1));
        const unsigned d0 = (unsigned)(4 * (y - 4 * oy) + 16 * (z - 4 * oz));
        const unsigned e0 = (unsigned)(TILE_Y * (y + 1) + TILE_Z * (z + 1));
        r_w[q] = pk1 | (unsigned)rr << 2 | nbs << 8 | d0 << 13 | e0 << 19;
    }
    const int half = lane >> 4, r = lane & 15;
    const int j = r & 3, k = r >> 2;
    const int64_t pairs = (P - 2 + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * SA_WARPS;
    unsigned cnt[4] = {0, 0, 0, 0};
    int nb_next[2] = {0, 0};
    int64_t pr = (int64_t)blockIdx.x * SA_WARPS + warp;
    if (pr < pairs && lane < NB) {
        nb_next[0] = __ldg(nbr + (2 + 2 * pr) * NB + lane);
        if (3 + 2 * pr < P) nb_next[1] = __ldg(nbr + (3 + 2 * pr) * NB + lane);
    }
    for (; pr < pairs; pr += stride) {
        const int64_t p0 = 2 + 2 * pr;
        const bool two = p0 + 1 < P;
        bool ok = lane < 2 && (lane == 0 || two);
        if (lane < 2) {
            SurBody b = B0;
            if (BATCH && ok) {
                ok = __ldg(type + p0 + lane) >= 2;
                if (ok) b = sb[__ldg(body + p0 + lane)];
            }
            s_B[warp][lane] = b;
        }
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        if (lane < NB) {
            tnb[0][lane] = nb_next[0];
            tnb[1][lane] = nb_next[1];
        }
        __syncwarp();
        const int64_t pn = pr + stride;
        if (pn < pairs && lane < NB) {
            nb_next[0] = __ldg(nbr + (2 + 2 * pn) * NB + lane);
            if (3 + 2 * pn < P) nb_next[1] = __ldg(nbr + (3 + 2 * pn) * NB + lane);
        }
        unsigned bits[2] = {0u, 0u}, keep[2] = {3u, 3u};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const unsigned wq = r_w[q];
            const int pk = (int)(wq & 3u) - 1, rr = (int)((wq >> 2) & 63u), nbs = (int)((wq >> 8) & 31u);
            const int d0 = (int)((wq >> 13) & 63u), e0 = (int)(wq >> 19);
            if (pk < 0 || !((okm >> pk) & 1u)) continue;
            const int* nb = tnb[pk];
            // 32-bit byte offsets (stores of fewer than 2^24 packages)
            const char* pb = reinterpret_cast<const char*>(phi) + 4u * (uint32_t)d0;
            const float4 v = __ldg(reinterpret_cast<const float4*>(pb + 4u * PKG3 * (uint32_t)nb[nbs + 1]));
            const float vm = __ldg(reinterpret_cast<const float*>(pb + 4u * (PKG3 * (uint32_t)nb[nbs] + 3u)));
            const float vp = __ldg(reinterpret_cast<const float*>(pb + 4u * PKG3 * (uint32_t)nb[nbs + 2]));
            const float f[6] = {vm, v.x, v.y, v.z, v.w, vp};
            const float ie = s_B[warp][pk].inv_eps, hu = s_B[warp][pk].C.h_up;
            float2* t = reinterpret_cast<float2*>(tH[pk] + e0);  // rows start on 8-byte boundaries
            float2* tp = reinterpret_cast<float2*>(tP[pk] + e0);
            unsigned b = 0, mo = 0, mi = 0;
#pragma unroll
            for (int i = 0; i < 6; i += 2) {
                const float h0 = heaviside_neg(f[i], ie), h1 = heaviside_neg(f[i + 1], ie);
                t[i / 2] = make_float2(h0, h1);
                tp[i / 2] = make_float2(f[i], f[i + 1]);
                b |= (h0 != 0.0f ? 1u : 0u) | (h0 != 1.0f ? 2u : 0u) | (h1 != 0.0f ? 1u : 0u) | (h1 != 1.0f ? 2u : 0u);
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                mo |= (f[i] >= hu ? 1u : 0u) << i;
                mi |= (-f[i] >= hu ? 1u : 0u) << i;
            }
            tM[pk][rr] = (uint16_t)(mo | (mi << 8));
            bits[pk] |= b;
            keep[pk] &= (mo == 0x3Fu ? 1u : 0u) | (mi == 0x3Fu ? 2u : 0u);
        }
        bits[0] = __reduce_or_sync(0xffffffffu, bits[0]);
        bits[1] = __reduce_or_sync(0xffffffffu, bits[1]);
        keep[0] = __reduce_and_sync(0xffffffffu, keep[0]);
        keep[1] = __reduce_and_sync(0xffffffffu, keep[1]);
        __syncwarp();
        unsigned net = 0;
        const int64_t pt0 = (p0 + half) * PKG3 + 4 * r;
        if ((okm >> half) & 1u) {
            const unsigned triv = keep[half];
            // classes of the row's four points as bit masks (bit i: point i)
            unsigned tin = 0, fb = 0;
            if (triv) {
                tin = (triv & 2u) ? 0xFu : 0u;
            } else {
                // the 27-tap trivial tests from the 3 x 3 tile rows around
                // the row: point i is trivially outside (inside) when bits
                // i .. i + 2 of the AND of those masks are set; |phi| < h at
                // the point itself when neither bit i + 1 of its own row is
                const SurConst C = s_B[warp][half].C;
                unsigned m = 0xFFFFu, mc = 0;
#pragma unroll
                for (int sz = 0; sz < 3; ++sz)
#pragma unroll
                    for (int sy = 0; sy < 3; ++sy) {
                        const unsigned v = tM[half][(j + sy) + 6 * (k + sz)];
                        m &= v;
                        if (sz == 1 && sy == 1) mc = v;
                    }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (((m >> (8 + i)) & 7u) == 7u) {
                        tin |= 1u << i;
                    } else if (((m >> i) & 7u) != 7u) {
                        const int e0 = tile_e0(4 * r + i);
                        const float* tl = tP[half];
                        const bool f = !((mc >> (i + 1)) & 0x101u) ||
                                       curvature_exceeds(tl[e0 + 1], tl[e0 - 1], tl[e0 + TILE_Y], tl[e0 - TILE_Y],
                                                         tl[e0 + TILE_Z], tl[e0 - TILE_Z], tl[e0], C);
                        if (f)
                            fb |= 1u << i;
                        else
                            net |= 1u << i;
                    }
                }
            }
            cnt[SG_SUR_TRIVIAL_IN] += __popc(tin);
            cnt[SG_SUR_TRIVIAL_OUT] += 4 - __popc(tin | fb | net);
            cnt[SG_SUR_FALLBACK] += __popc(fb);
            cnt[SG_SUR_NETWORK] += __popc(net);
            float w[4], ax[4], ay[4], az[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                w[i] = (tin >> i) & 1u ? 1.0f : 0.0f;
                ax[i] = ay[i] = az[i] = 0.0f;
            }
            if (fb) {  // the exact sums exactly as mode 0 forms them
                float sw, sx, sy, sz;
                if (integrals_saturated(bits[half], sw, sx, sy, sz)) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if ((fb >> i) & 1u) w[i] = sw, ax[i] = sx, ay[i] = sy, az[i] = sz;
                } else {
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        if (!((fb >> (2 * pp)) & 3u)) continue;
                        float2 w2, x2, y2, z2;
                        integrals_point2(tH[half], 4 * r + 2 * pp, K, w2, x2, y2, z2);
                        if ((fb >> (2 * pp)) & 1u) w[2 * pp] = w2.x, ax[2 * pp] = x2.x, ay[2 * pp] = y2.x, az[2 * pp] = z2.x;
                        if ((fb >> (2 * pp + 1)) & 1u)
                            w[2 * pp + 1] = w2.y, ax[2 * pp + 1] = x2.y, ay[2 * pp + 1] = y2.y, az[2 * pp + 1] = z2.y;
                    }
                }
            }
            const uint32_t ob = 4u * (uint32_t)pt0;
            auto row = [ob](float* a) { return reinterpret_cast<float4*>(reinterpret_cast<char*>(a) + ob); };
            *row(W) = make_float4(w[0], w[1], w[2], w[3]);
            *row(gx) = make_float4(ax[0], ax[1], ax[2], ax[3]);
            *row(gy) = make_float4(ay[0], ay[1], ay[2], ay[3]);
            *row(gz) = make_float4(az[0], az[1], az[2], az[3]);
        }
        // network points: one list reservation per warp
        const unsigned c = __popc(net);
        unsigned incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            unsigned base = 0;
            if (lane == 31) base = atomicAdd(count, total);
            base = __shfl_sync(0xffffffffu, base, 31);
            unsigned at = base + incl - c;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((net >> i) & 1u) list[at++] = (int32_t)(pt0 + i);
        }
        __syncwarp();  // the next pair's staging overwrites the tiles
    }
    // class counts: a shared atomic per warp and class, one global atomic per CTA and class
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const unsigned v = __reduce_add_sync(0xffffffffu, cnt[c]);
        if (lane == 0 && v) atomicAdd(&s_cnt[c], v);
    }
    __syncthreads();
    if (stats && threadIdx.x < 4 && s_cnt[threadIdx.x])
        atomicAdd(stats + threadIdx.x, (unsigned long long)s_cnt[threadIdx.x]);
}

// Persistent grid of pass A: the CTAs that fit on all SMs at once.
template <bool BATCH>
unsigned sur_a_grid(int64_t P, int device) {
    static int per_sm = 0, sms = 0;  // per instantiation, on the first device asked (all alike here)
    if (!sms) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sur_a<BATCH>, SA_WARPS * 32, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    }
    const int64_t pairs = (P - 2 + 1) / 2;
    int64_t b = (int64_t)std::max(per_sm, 1) * std::max(sms, 1);
    const int64_t need = (pairs + SA_WARPS - 1) / SA_WARPS;
    if (b > need) b = need;
    return (unsigned)std::max<int64_t>(b, 1);
}

// ---------------------------------------------------------------------------
// Surrogate integrals, pass B: the network over the list, 128 rows a tile.
// ---------------------------------------------------------------------------
// 128-row tile streams (warpgroups) per CTA: two, sharing one copy of the
// weights, measured 347 against 334 us for one on the h = 0.002 torus (at
// the 64 registers that four CTAs of two groups allow, the kernel spills)
constexpr int SB_GROUPS = 1;
constexpr int SB_T = PK_FWD_BYTES;                     // tile operands, one per group
constexpr int SB_BYTES = SB_T + SB_GROUPS * TC_ROWS * MLP_H * 2;
static_assert(SB_T % 128 == 0, "tile alignment");

// The 27 phi values around data point q = 64 p + d, through the index
// shift of package p.
__device__ __forceinline__ void gather27(const int32_t* __restrict__ nbr, const float* __restrict__ phi, int64_t q,
                                         float (&f)[MLP_IN]) {
    const int64_t p = q >> 6;
    const int d = (int)(q & 63), i = d & 3, j = (d >> 2) & 3, k = d >> 4;
#pragma unroll
    for (int n = 0; n < MLP_IN; ++n) {
        const int ii = i + n % 3 - 1, jj = j + (n / 3) % 3 - 1, kk = k + n / 9 - 1;
        const int ox = ((ii + 4) >> 2) - 1, oy = ((jj + 4) >> 2) - 1, oz = ((kk + 4) >> 2) - 1;
        const int slot = 13 + ox + 3 * oy + 9 * oz;
        const uint32_t pk = slot == 13 ? (uint32_t)p : (uint32_t)__ldg(nbr + p * NB + slot);
        // 32-bit byte offsets: the store holds fewer than 2^24 packages (checked at launch)
        const uint32_t off = 4u * (pk * PKG3 + (uint32_t)((ii - 4 * ox) + PKG * (jj - 4 * oy) + PKG * PKG * (kk - 4 * oz)));
        f[n] = __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(phi) + off));
    }
}

// In-register moves of a row of 27 values indexed n = x + 3 y + 9 z (slots
// 27.. untouched).  With `on`, v[m] becomes v[t(m)] for a digit map t that
// is an involution, so the pairs (m, t(m)) swap; selects, so that v stays
// in registers.
__host__ __device__ constexpr int pow3(int a) { return a == 0 ? 1 : 3 * pow3(a - 1); }

// t: digit A -> 2 - digit A (the reflection of axis A)
template <int A>
__device__ __forceinline__ void cond_reflect(float (&v)[32], bool on) {
#pragma unroll
    for (int m = 0; m < MLP_IN; ++m) {
        if ((m / pow3(A)) % 3 != 0) continue;
        const int m2 = m + 2 * pow3(A);
        const float a = v[m], b = v[m2];
        v[m] = on ? b : a;
        v[m2] = on ? a : b;
    }
}

// t: digits A and B exchanged
template <int A, int B>
__device__ __forceinline__ void cond_swap_axes(float (&v)[32], bool on) {
#pragma unroll
    for (int m = 0; m < MLP_IN; ++m) {
        const int da = (m / pow3(A)) % 3, db = (m / pow3(B)) % 3;
        if (da >= db) continue;
        const int m2 = m + (db - da) * (pow3(A) - pow3(B));
        const float a = v[m], b = v[m2];
        v[m] = on ? b : a;
        v[m2] = on ? a : b;
    }
}

// Which of the conditional axis exchanges (0 1), then (1 2), then (0 1)
// carry the reflected row to canonical order under each of the six
// permutations (3 bits per permutation, first exchange in the low bit).
constexpr uint32_t PERM_EXCHANGES = 0u | 2u << 3 | 4u << 6 | 3u << 9 | 6u << 12 | 7u << 15;

// Canonical input row of a point into the tile operand T (row r); returns
// the transform code.  The row is put in canonical order in registers (the
// value of original input n goes to column canon_pos(n, reflections, perm):
// the reflections, then the permutation as up to three axis exchanges) and
// written as four 16-byte stores of eight BF16 values (columns 27.. zero).
static_assert(!MLP_SPLIT && MLP_K1 == 32, "canon_row writes 27 BF16 inputs and 5 zero columns");
__device__ __forceinline__ int canon_row(const float (&f)[MLP_IN], float inv_h, unsigned char* T, int r) {
    const int code = canon_code(f[13], f[14], f[12], f[16], f[10], f[22], f[4]);
    const float sgn = (code & 1) ? -1.0f : 1.0f;
    float v[MLP_K1];
#pragma unroll
    for (int n = 0; n < MLP_IN; ++n) v[n] = fminf(fmaxf(__fmul_rn(sgn * f[n], inv_h), -1.0f), 1.0f);
#pragma unroll
    for (int n = MLP_IN; n < MLP_K1; ++n) v[n] = 0.0f;
    cond_reflect<0>(v, (code >> 1) & 1);
    cond_reflect<1>(v, (code >> 2) & 1);
    cond_reflect<2>(v, (code >> 3) & 1);
    const uint32_t ex = PERM_EXCHANGES >> (3 * (code >> 4));
    cond_swap_axes<0, 1>(v, ex & 1u);
    cond_swap_axes<1, 2>(v, ex & 2u);
    cond_swap_axes<0, 1>(v, ex & 4u);
#pragma unroll
    for (int q = 0; q < MLP_K1 / 8; ++q)
        *reinterpret_cast<uint4*>(T + umma::kmajor_byte(r, 8 * q, MLP_K1)) = umma::pack8_bf16(v + 8 * q);
    return code;
}

// Canonical positions of the 27 inputs under each of the 48 (reflection,
// permutation) pairs: pos[(rb | perm << 3) * 27 + n].
__device__ __forceinline__ void build_pos(uint8_t* pos) {
    for (int e = threadIdx.x; e < 48 * MLP_IN; e += blockDim.x) {
        const int combo = e / MLP_IN, n = e % MLP_IN;
        pos[e] = (uint8_t)canon_pos(n, combo & 7, combo >> 3);
    }
}

// SB_GROUPS warpgroups per CTA, each a stream of 128-row tiles with its own
// tensor-memory columns, barrier and tile operand, sharing one copy of the
// weights.
template <bool BATCH>
__global__ void __launch_bounds__(SB_GROUPS * TC_ROWS) k_sur_b(const int32_t* __restrict__ nbr,
                                                               const float* __restrict__ phi, float* __restrict__ W,
                                                               float* __restrict__ gx, float* __restrict__ gy,
                                                               float* __restrict__ gz, float inv_h0,
                                                               const int32_t* __restrict__ body,
                                                               const SurBody* __restrict__ sb,
                                                               const int32_t* __restrict__ list,
                                                               const unsigned* __restrict__ count,
                                                               const unsigned char* __restrict__ packed, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[SB_GROUPS];
    __shared__ uint32_t slot;
    stage_bytes(smem, packed, PK_FWD_BYTES);
    Tc t = tc_begin(bars, &slot, 64 * SB_GROUPS, SB_GROUPS > 1 ? SB_GROUPS : 0);  // one group: the whole CTA
    const uint32_t tbase = slot;
    unsigned char* T = smem + SB_T + (t.group > 0 ? t.group : 0) * TC_ROWS * MLP_H * 2;
    const int r = tc_row();
    const int64_t n = (int64_t)*count;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    for (int64_t tile = (int64_t)blockIdx.x * SB_GROUPS + (t.group > 0 ? t.group : 0); tile < tiles && t.ok;
         tile += (int64_t)gridDim.x * SB_GROUPS) {
        const int64_t row = tile * TC_ROWS + r;
        const bool valid = row < n;
        int64_t q = 0;
        int code = 0;
        if (valid) {
            q = (int64_t)__ldg(list + row);
            float f[MLP_IN];
            gather27(nbr, phi, q, f);
            const float inv_h = BATCH ? sb[__ldg(body + (q >> 6))].C.inv_h : inv_h0;
            code = canon_row(f, inv_h, T, r);
        } else {
#pragma unroll
            for (int c = 0; c < MLP_K1 / 8; ++c)
                *reinterpret_cast<uint4*>(T + umma::kmajor_byte(r, 8 * c, MLP_K1)) = make_uint4(0, 0, 0, 0);
        }
        float y[4], o[4];
        tc_forward(t, smem, T, y);
        if (t.ok && valid) {
            uncanon_outputs(code, y, o);
            W[q] = o[0];
            gx[q] = o[1];
            gy[q] = o[2];
            gz[q] = o[3];
        }
    }
    tc_end(t, tbase, 64 * SB_GROUPS, err);
}

// ---------------------------------------------------------------------------
// Classes and training samples
// ---------------------------------------------------------------------------
constexpr int SU_THREADS = 256;
constexpr int SU_PK = SU_THREADS / PKG3;  // packages per CTA

// class of every data point (255 for far packages)
__global__ void __launch_bounds__(SU_THREADS) k_sur_classify(const int32_t* __restrict__ nbr,
                                                             const float* __restrict__ phi, int64_t P, SurConst C,
                                                             uint8_t* __restrict__ cls) {
    __shared__ int s_nb[SU_PK][NB];
    __shared__ __align__(16) float s_phi[SU_PK][TILE_N];
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63;
    const int64_t p = (int64_t)blockIdx.x * SU_PK + lp;
    const bool act = p >= 2 && p < P;
    if (act && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
    __syncthreads();
    if (act) stage_rows(s_nb[lp], phi, 0.0f, d, s_phi[lp], nullptr);
    __syncthreads();
    if (p < P) cls[p * PKG3 + d] = act ? (uint8_t)sur_class_at(s_phi[lp], tile_e0(d), C) : (uint8_t)255;
}

__device__ __forceinline__ bool keep_sample(uint64_t seed, int64_t pt, uint32_t keep24) {
    // SplitMix64 of (seed + point index); keep when its top 24 bits < keep24
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(pt + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z >> 40) < keep24;
}

// Training samples: network-class points kept by the hash, in point order,
// as canonical input rows and canonical targets (the exact W, G^ carried
// into the point's canonical frame).  Pass 1 (offsets == nullptr) counts per
// package; pass 2 writes the rows.
__global__ void __launch_bounds__(SU_THREADS) k_sur_samples(const int32_t* __restrict__ nbr,
                                                            const float* __restrict__ phi, int64_t P, SurConst C,
                                                            uint64_t seed, uint32_t keep24,
                                                            uint32_t* __restrict__ counts,
                                                            const uint32_t* __restrict__ offsets, int64_t cap,
                                                            const float* __restrict__ W, const float* __restrict__ gx,
                                                            const float* __restrict__ gy, const float* __restrict__ gz,
                                                            __nv_bfloat16* __restrict__ xo, float* __restrict__ to) {
    __shared__ int s_nb[SU_PK][NB];
    __shared__ __align__(16) float s_phi[SU_PK][TILE_N];
    __shared__ unsigned s_ball[SU_PK][2];
    __shared__ uint8_t s_pos[48 * MLP_IN];
    const int lp = threadIdx.x >> 6, d = threadIdx.x & 63, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * SU_PK + lp;
    const bool act = p >= 2 && p < P;
    if (act && d < NB) s_nb[lp][d] = __ldg(nbr + p * NB + d);
    if (offsets) build_pos(s_pos);
    __syncthreads();
    if (act) stage_rows(s_nb[lp], phi, 0.0f, d, s_phi[lp], nullptr);
    __syncthreads();
    const int e0 = tile_e0(d);
    const int64_t pt = p * PKG3 + d;
    const bool take = act && sur_class_at(s_phi[lp], e0, C) == SG_SUR_NETWORK && keep_sample(seed, pt, keep24);
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
    const float* tl = s_phi[lp];
    float f[MLP_IN];
#pragma unroll
    for (int n = 0; n < MLP_IN; ++n) f[n] = tl[e0 + (n % 3 - 1) + TILE_Y * ((n / 3) % 3 - 1) + TILE_Z * (n / 9 - 1)];
    const int code = canon_code(f[13], f[14], f[12], f[16], f[10], f[22], f[4]);
    const float sgn = (code & 1) ? -1.0f : 1.0f;
    const uint8_t* ps = s_pos + (code >> 1) * MLP_IN;
    float xr[MLP_K1];
#pragma unroll
    for (int c = 0; c < MLP_K1; ++c) xr[c] = 0.0f;
#pragma unroll
    for (int n = 0; n < MLP_IN; ++n) {
        const float v = fminf(fmaxf(__fmul_rn(sgn * f[n], C.inv_h), -1.0f), 1.0f);
        const int c = ps[n];
        xr[c] = v;  // dynamic index: a local-memory row, written once per sample
    }
#pragma unroll
    for (int c = 0; c < MLP_IN; ++c) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(xr[c]);
        xo[row * MLP_K1 + c] = hi;
        if (MLP_SPLIT) xo[row * MLP_K1 + MLP_IN + c] = __float2bfloat16_rn(xr[c] - __bfloat162float(hi));
    }
#pragma unroll
    for (int c = MLP_SPLIT ? 2 * MLP_IN : MLP_IN; c < MLP_K1; ++c) xo[row * MLP_K1 + c] = __float2bfloat16_rn(0.0f);
    const float ex[4] = {W[pt], gx[pt], gy[pt], gz[pt]};
    float tc[4];
    canon_targets(code, ex, tc);
    *reinterpret_cast<float4*>(to + row * 4) = make_float4(tc[0], tc[1], tc[2], tc[3]);
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

// Persistent grid of a tensor-core kernel: the CTAs that fit on every SM
// at once by registers, shared memory, threads and the 512 TMEM columns
// (ncols per CTA), so that no CTA waits for another's columns.
unsigned tc_grid(const void* fn, int smem, uint32_t ncols, int device, int64_t tiles, int threads = TC_ROWS) {
    cudaFuncAttributes fa{};
    int sms = 0, smem_sm = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) cudaGetLastError();
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device);
    int per_sm = (int)(512 / ncols);
    per_sm = std::min(per_sm, 2048 / threads);
    const int regs = (std::max(fa.numRegs, 1) + 7) / 8 * 8;
    if (regs_sm > 0) per_sm = std::min(per_sm, regs_sm / (regs * threads));
    if (smem_sm > 0) per_sm = std::min(per_sm, smem_sm / (smem + (int)fa.sharedSizeBytes + 1024));
    int64_t b = (int64_t)std::max(per_sm, 1) * std::max(sms, 1);
    if (tiles > 0 && b > tiles) b = tiles;
    return (unsigned)std::max<int64_t>(b, 1);
}

// Partial-gradient buffer for `ctas` CTAs.
bool ensure_part(sg_mlp* m, int64_t ctas) {
    if (m->part && m->part_ctas >= ctas) return true;
    if (m->part) cudaFree(m->part);
    m->part = nullptr;
    m->part_ctas = 0;
    if (cudaMalloc(&m->part, (size_t)ctas * (MLP_NPARAM + 1) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        m->part = nullptr;
        return false;
    }
    m->part_ctas = ctas;
    return true;
}

cudaError_t launch_train(sg_mlp* m, int64_t n, const void* x, const float* t, const int32_t* idx) {
    if (!m->train_smem_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_BYTES);
        if (e != cudaSuccess) return e;
        m->train_smem_set = true;
    }
    k_mlp_train<<<cdiv(n, TC_ROWS), TR_THREADS, TR_BYTES, m->stream>>>(m->packed, n, (const __nv_bfloat16*)x, t, idx,
                                                                       1.0f / (float)(n * MLP_OUT), m->part, m->err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

const unsigned char* mlp_packed(const sg_mlp* m) { return m->packed; }
int* mlp_err(const sg_mlp* m) { return m->err; }

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
    if (cudaMalloc(&m->master, 3 * pb + 256) != cudaSuccess || cudaMalloc(&m->packed, PK_BYTES) != cudaSuccess) {
        cudaGetLastError();
        sg_mlp_destroy(m);
        return SG_ERR_OOM;
    }
    m->m = m->master + MLP_NPARAM;
    m->v = m->m + MLP_NPARAM;
    m->err = reinterpret_cast<int*>(m->v + MLP_NPARAM);
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
    if (m->part) cudaFree(m->part);
    delete m;
    return SG_OK;
}

sg_status sg_mlp_set_params(sg_mlp* m, const float* params) {
    if (!m || !params) return SG_ERR_INVALID;
    const size_t pb = MLP_NPARAM * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(m->master, params, pb, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, 2 * pb + sizeof(int), m->stream);  // moments, error word
    if (e == cudaSuccess) e = cudaMemsetAsync(m->packed, 0, PK_BYTES, m->stream);         // padding stays zero
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
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(params, m->master, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("get_params: ") + cudaGetErrorString(e));
    if (err) return m_fail(m, SG_ERR_TIMEOUT, "a tensor-core product did not complete in time");
    return SG_OK;
}

sg_status sg_mlp_forward(sg_mlp* m, int64_t n, const void* x, float* y) {
    SG_TRACE("sg_mlp_forward");
    if (!m || n < 0 || (n > 0 && (!x || !y))) return SG_ERR_INVALID;
    if (n == 0) return SG_OK;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_BYTES);
    if (e == cudaSuccess) {
        k_mlp_forward<<<tc_grid((const void*)k_mlp_forward, FWD_BYTES, 64, m->device, tiles), TC_ROWS, FWD_BYTES,
                        m->stream>>>(m->packed, n, (const __nv_bfloat16*)x, y, m->err);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_mlp_loss_grad(sg_mlp* m, int64_t n, const void* x, const float* t, const int32_t* idx, float* grad,
                           float* loss) {
    SG_TRACE("sg_mlp_loss_grad");
    if (!m || n < 1 || !x || !t || !grad) return SG_ERR_INVALID;
    const int64_t ctas = (n + TC_ROWS - 1) / TC_ROWS;
    if (!ensure_part(m, ctas)) return m_fail(m, SG_ERR_OOM, "loss_grad: out of memory");
    cudaError_t e = launch_train(m, n, x, t, idx);
    if (e == cudaSuccess) {
        k_mlp_grad_sum<<<sum_blocks(), SUM_THREADS, 0, m->stream>>>(m->part, (int)ctas, grad, loss);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("loss_grad: ") + cudaGetErrorString(e));
    return SG_OK;
}

sg_status sg_mlp_train_step(sg_mlp* m, int64_t batch, const void* x, const float* t, const int32_t* idx, float lr,
                            float* loss) {
    SG_TRACE("sg_mlp_train_step");
    if (!m || batch < 1 || !x || !t || !(lr >= 0.0f)) return SG_ERR_INVALID;
    const int64_t ctas = (batch + TC_ROWS - 1) / TC_ROWS;
    if (!ensure_part(m, ctas)) return m_fail(m, SG_ERR_OOM, "train_step: out of memory");
    cudaError_t e = launch_train(m, batch, x, t, idx);
    if (e == cudaSuccess) {
        m->step += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 - std::pow(b1, (double)m->step)), c2 = (float)(1.0 - std::pow(b2, (double)m->step));
        k_mlp_adam<<<sum_blocks(), SUM_THREADS, 0, m->stream>>>(m->part, (int)ctas, m->master, m->m, m->v, m->packed,
                                                                lr, (float)b1, (float)b2, 1e-8f, c1, c2, loss);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return m_fail(m, SG_ERR_CUDA, std::string("train_step: ") + cudaGetErrorString(e));
    return SG_OK;
}

const char* sg_mlp_last_error(const sg_mlp* m) { return m ? m->last_error.c_str() : "null mlp"; }

sg_status sg_surrogate_classify(sg_grid* g, uint8_t* cls) {
    SG_TRACE("sg_surrogate_classify");
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
    SG_TRACE("sg_surrogate_samples");
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
    SG_TRACE("sg_surrogate_stats");
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

size_t sur_work_bytes(int64_t P) { return 256 + ((size_t)(P > 2 ? P - 2 : 0) * PKG3 * 4 + 255) / 256 * 256; }

cudaError_t launch_surrogate_integrals(sg_grid* g, const sg_mlp* m, void* work, float* W, float* gx, float* gy,
                                       float* gz) {
    cudaError_t e;
    if ((e = launch_set_far(W, 1.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = launch_set_far(gx, 0.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = launch_set_far(gy, 0.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = launch_set_far(gz, 0.0f, 0.0f, g->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g->stats.p, 0, 4 * sizeof(unsigned long long), g->stream)) != cudaSuccess) return e;
    if (g->P <= 2) return cudaSuccess;
    unsigned* count = (unsigned*)work;
    int32_t* list = (int32_t*)((char*)work + 256);
    if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned), g->stream)) != cudaSuccess) return e;
    const int32_t* nbr = (const int32_t*)g->nbr.p;
    const float* phi = (const float*)g->field[SG_FIELD_PHI].p;
    k_sur_a<false><<<sur_a_grid<false>(g->P, g->device), SA_WARPS * 32, 0, g->stream>>>(
        nbr, phi, W, gx, gy, gz, g->P, kernel_coef(), sur_body(g->desc.h), nullptr, nullptr, nullptr, list, count,
        (unsigned long long*)g->stats.p);
    if ((e = cudaFuncSetAttribute(k_sur_b<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SB_BYTES)) !=
        cudaSuccess)
        return e;
    k_sur_b<false><<<tc_grid((const void*)k_sur_b<false>, SB_BYTES, 64 * SB_GROUPS, g->device, 0, SB_GROUPS * TC_ROWS),
                     SB_GROUPS * TC_ROWS, SB_BYTES, g->stream>>>(
        nbr, phi, W, gx, gy, gz, (float)(1.0 / g->desc.h), nullptr, nullptr, list, count, m->packed,
        (int*)g->err.p);
    note_launch(2);
    return cudaGetLastError();
}

SurBody sur_body(double h) {
    SurBody q;
    q.C = sur_const_h(h);
    q.inv_eps = (float)(1.0 / h);
    return q;
}

cudaError_t setup_batch_surrogate() {
    return cudaFuncSetAttribute(k_sur_b<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SB_BYTES);
}

cudaError_t launch_batch_surrogate_integrals(const int32_t* nbr, const uint8_t* type, const int32_t* body,
                                             const SurBody* sb, const float* phi, float* W, float* gx, float* gy,
                                             float* gz, int64_t P, const sg_mlp* m, void* work, int* err, int device,
                                             cudaStream_t s) {
    if (P <= 2) return cudaSuccess;
    unsigned* count = (unsigned*)work;
    int32_t* list = (int32_t*)((char*)work + 256);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_sur_a<true><<<sur_a_grid<true>(P, device), SA_WARPS * 32, 0, s>>>(
        nbr, phi, W, gx, gy, gz, P, kernel_coef(), SurBody{}, type, body, sb, list, count, nullptr);
    k_sur_b<true><<<tc_grid((const void*)k_sur_b<true>, SB_BYTES, 64 * SB_GROUPS, device, 0, SB_GROUPS * TC_ROWS),
                    SB_GROUPS * TC_ROWS, SB_BYTES, s>>>(
        nbr, phi, W, gx, gy, gz, 0.0f, body, sb, list, count, m->packed, err);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace sg
