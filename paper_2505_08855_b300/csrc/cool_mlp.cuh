// cool_mlp.cuh -- the surrogate object and the MLP parameter layout.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "cool_internal.cuh"

namespace cool {

// FP32 parameter vector (master copy, gradients and Adam moments share it):
//   W1 [128][16] (columns 0..3: the four coordinates, column 4: the side of
//   the K2 switch, columns 5..15 stay zero), b1 [128],
//   W2 [128 out][128 in], b2 [128], w3 [128], b3 [1].
//
// Network input row (16 bf16 columns, one MMA K step): each normalised
// coordinate x_d in [-1, 1] enters as two bf16 parts, hi = bf16(x_d) in
// column d and lo = bf16(x_d - hi) in column 4 + d, so the input carries
// 16 bits of x_d instead of 8; column 8 is s = +1 above the K2 switch
// temperature and -1 at or below it (the synchrotron channel jumps there,
// which a smooth network cannot follow).  The bf16 first-layer operand
// repeats W1's coordinate columns for the lo parts:
//   W1op[:, d] = W1op[:, 4 + d] = bf16(W1[:, d]) (d < 4), W1op[:, 8] = bf16(W1[:, 4]).
constexpr int kP_W1 = 0;
constexpr int kP_b1 = kP_W1 + 128 * 16;
constexpr int kP_W2 = kP_b1 + 128;
constexpr int kP_b2 = kP_W2 + 128 * 128;
constexpr int kP_w3 = kP_b2 + 128;
constexpr int kP_b3 = kP_w3 + 128;
constexpr int kP_n = kP_b3 + 1;
constexpr int kP_alloc = (kP_n + 63) & ~63;

struct MlpDev {
    const __nv_bfloat16* W1b;    // [128][16]  bf16 copy of W1
    const __nv_bfloat16* W2b;    // [128][128] bf16 copy of W2 ([out][in])
    const __nv_bfloat16* W2Tb;   // [128][128] bf16 copy of W2^T ([in][out])
    const float* p;              // FP32 parameters (layout above)
    float mean, std;             // output standardisation: log2 value = mean + std * net
    float l0[4], span[4];        // input normalisation: x = 2 (l - l0)/span - 1
    float xs;                    // normalised log2 of the K2 switch temperature
};

// Operand column of W1's master column c (c < 5), and of its repeat.
__host__ __device__ constexpr int w1_op_col(int c) { return c < 4 ? c : 8; }

// The 16-column input row described above.
__device__ __forceinline__ void input_row(const float (&x)[4], float xs, __nv_bfloat16 (&row)[16]) {
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(x[d]);
        row[d] = hi;
        row[4 + d] = __float2bfloat16_rn(x[d] - __bfloat162float(hi));
    }
    row[8] = __float2bfloat16_rn(x[3] > xs ? 1.f : -1.f);
#pragma unroll
    for (int k = 9; k < 16; ++k) row[k] = __float2bfloat16_rn(0.f);
}

}  // namespace cool

struct cool_surrogate {
    uint32_t magic;
    int device;
    int channel;
    cool_table_spec spec;       // of the table it was fitted to
    double l0[4], span[4];
    double x_switch;            // normalised log2 of the K2 switch temperature
    double mean, std;
    float* d_p;                 // parameters
    float* d_g;                 // gradient accumulators
    float* d_m;                 // Adam first moments
    float* d_v;                 // Adam second moments
    __nv_bfloat16* d_W1b;
    __nv_bfloat16* d_W2b;
    __nv_bfloat16* d_W2Tb;
    unsigned* d_err;
    uint32_t* d_mask;           // fallback bit per 4-D table cell
    long long mask_bits;
    long long mask_set;         // cells flagged
    double final_loss;
    long long steps;
};

constexpr uint32_t kSurrogateMagic = 0x5C0DE5A1u;
