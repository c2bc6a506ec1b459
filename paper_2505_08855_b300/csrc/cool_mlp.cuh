// cool_mlp.cuh -- the surrogate object and the MLP parameter layout.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "cool_internal.cuh"

namespace cool {

// FP32 parameter vector (master copy, gradients and Adam moments share it):
//   W1 [128][16] (input columns 4..15 stay zero), b1 [128],
//   W2 [128 out][128 in], b2 [128], w3 [128], b3 [1].
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
};

}  // namespace cool

struct cool_surrogate {
    uint32_t magic;
    int device;
    int channel;
    cool_table_spec spec;       // of the table it was fitted to
    double l0[4], span[4];
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
