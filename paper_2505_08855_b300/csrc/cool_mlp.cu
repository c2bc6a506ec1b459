// cool_mlp.cu -- the learned surrogate of the synchrotron table channel (not
// in the paper): an MLP 4 -> 128 -> 128 -> 1 with SiLU, BF16 weights and
// activations as tensor-core operands, FP32 accumulation in tensor memory.
// Every matrix product -- the two forward layers and the three backward
// products (dW2 = dZ2^T H1, dH1 = dZ2 W2, dW1 = dZ1^T X) -- is a hand-issued
// tcgen05.mma; the output layer (128 -> 1), the activations, the loss and
// Adam run on the CUDA cores.
//
// A tile is 128 samples (one per thread; 4 warps = the 128 TMEM lanes).
// Input width 4 is padded to 16 (one MMA K step).  Operands use the K-major
// core-matrix layout of cool_mma.cuh.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "cool_internal.cuh"
#include "cool_mlp.cuh"
#include "cool_mma.cuh"

namespace cool {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kT = 128;     // tile rows = threads
constexpr int kHid = 128;
constexpr int kIn = 16;

// ---- training kernel shared memory (bytes) ----------------------------------
constexpr int kOffW1 = 0;                          // W1  [128 f1][16 in]    B of layer 1
constexpr int kOffW2 = kOffW1 + kHid * kIn * 2;    // W2  [128 f2][128 f1]   B of layer 2
constexpr int kOffW2T = kOffW2 + kHid * kHid * 2;  // W2^T [128 f1][128 f2] B of dH1
constexpr int kOffX = kOffW2T + kHid * kHid * 2;   // X   [128 s][16]        A of layer 1
constexpr int kOffXT = kOffX + kT * kIn * 2;       // X^T [16][128 s]        B of dW1
constexpr int kOffH1 = kOffXT + kIn * kT * 2;      // H1  [128 s][128 f1]    A of layer 2; then dZ1^T
constexpr int kOffH1T = kOffH1 + kT * kHid * 2;    // H1^T [128 f1][128 s]   B of dW2
constexpr int kOffDZ2 = kOffH1T + kHid * kT * 2;   // dZ2 [128 s][128 f2]    A of dH1
constexpr int kOffDZ2T = kOffDZ2 + kT * kHid * 2;  // dZ2^T [128 f2][128 s]  A of dW2
constexpr int kOffRed = kOffDZ2T + kHid * kT * 2;  // gb1, gb2, gw3 [128], gb3, loss (fp32)
constexpr int kRedN = 3 * kHid + 8;
constexpr int kOffBar = kOffRed + kRedN * 4;
constexpr int kSmemTrain = kOffBar + 16;

// TMEM columns of the training kernel (512 = one CTA per SM).
constexpr uint32_t kColZ1 = 0, kColZ2 = 128, kColDW2 = 256, kColDH1 = 384, kColDW1 = 0;

// ---- evaluation kernel shared memory ----------------------------------------
constexpr int kEOffW1 = 0;
constexpr int kEOffW2 = kEOffW1 + kHid * kIn * 2;
constexpr int kEOffX = kEOffW2 + kHid * kHid * 2;
constexpr int kEOffH1 = kEOffX + kT * kIn * 2;
constexpr int kEOffBar = kEOffH1 + kT * kHid * 2;
constexpr int kSmemEval = kEOffBar + 16;

using mma::sigm;
using mma::st_row32;
using mma::st_bf16;
using mma::load_kmajor;
using mma::issue;
using mma::operands_ready;
using mma::mma_done;

// One training tile of 128 samples: forward, MSE against y (standardised
// targets), backward; the gradients (of the batch mean, inv_batch = 1/B) are
// added into g (parameter layout of cool_mlp.cuh), the loss into g[kP_n].
__global__ void __launch_bounds__(kT, 1) k_mlp_train_tile(MlpDev w, const float* __restrict__ x,
                                                         const float* __restrict__ y, long long first,
                                                         float inv_batch, float* __restrict__ g, unsigned* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float* red = reinterpret_cast<float*>(sm + kOffRed);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffBar + 8);
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const long long row = first + (long long)blockIdx.x * kT + t;
    const float* P = w.p;
    load_kmajor(sm + kOffW1, w.W1b, kHid, kIn);
    load_kmajor(sm + kOffW2, w.W2b, kHid, kHid);
    load_kmajor(sm + kOffW2T, w.W2Tb, kHid, kHid);
    for (int i = t; i < kRedN; i += kT) red[i] = 0.f;
    {
        float xv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = x[4 * row + k];
        // X row t (16 columns: two 16-byte chunks) and X^T column t
        __align__(16) bf16 tmp[16];
        input_row(xv, w.xs, tmp);
#pragma unroll
        for (int c = 0; c < kIn; c += 8)
            *reinterpret_cast<uint4*>(sm + kOffX + mma::kmajor_offset(t, c, kIn)) =
                *reinterpret_cast<const uint4*>(tmp + c);
#pragma unroll
        for (int k = 0; k < kIn; ++k)
            *reinterpret_cast<bf16*>(sm + kOffXT + mma::kmajor_offset(k, t, kT)) = tmp[k];
    }
    const float target = y[row];
    if (t == 0) {
        mma::mbar_init(mma::smem_addr(mbar), 1);
        mma::fence_mbar_init();
    }
    if (warp == 0) mma::tmem_alloc(mma::smem_addr(tslot), 512);
    operands_ready();
    const uint32_t tm = *tslot;
    const uint32_t mb = mma::smem_addr(mbar);
    // ---- layer 1: Z1 = X W1^T ----
    if (t == 0) {
        issue(tm + kColZ1, sm + kOffX, sm + kOffW1, kIn, kHid);
        mma::commit(mb);
    }
    mma_done(mb, 0, err);
    // ---- H1 = SiLU(Z1 + b1) ----
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 32) {
        float z[32];
        mma::tmem_ld32(tm + lane_off + kColZ1 + c0, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float zz = z[j] + P[kP_b1 + c0 + j];
            z[j] = zz * sigm(zz);
            st_bf16(sm + kOffH1T, c0 + j, t, kT, z[j]);
        }
        st_row32(sm + kOffH1, t, c0, kHid, z);
    }
    operands_ready();
    // ---- layer 2: Z2 = H1 W2^T ----
    if (t == 0) {
        issue(tm + kColZ2, sm + kOffH1, sm + kOffW2, kHid, kHid);
        mma::commit(mb);
    }
    mma_done(mb, 1, err);
    // ---- output layer, loss, dZ2 ----
    float yh = P[kP_b3];
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 32) {
        float z[32];
        mma::tmem_ld32(tm + lane_off + kColZ2 + c0, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float zz = z[j] + P[kP_b2 + c0 + j];
            yh = fmaf(zz * sigm(zz), P[kP_w3 + c0 + j], yh);
        }
    }
    const float r = yh - target;
    const float dy = 2.f * r * inv_batch;
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 32) {
        float z[32];
        mma::tmem_ld32(tm + lane_off + kColZ2 + c0, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float zz = z[j] + P[kP_b2 + c0 + j];
            const float s = sigm(zz);
            const float h2 = zz * s;
            const float dz = dy * P[kP_w3 + c0 + j] * s * (1.f + zz * (1.f - s));
            atomicAdd(&red[kHid + c0 + j], dz);          // gb2
            atomicAdd(&red[2 * kHid + c0 + j], dy * h2);  // gw3
            st_bf16(sm + kOffDZ2T, c0 + j, t, kT, dz);
            z[j] = dz;
        }
        st_row32(sm + kOffDZ2, t, c0, kHid, z);
    }
    atomicAdd(&red[3 * kHid], dy);                     // gb3
    atomicAdd(&red[3 * kHid + 1], r * r * inv_batch);  // loss
    operands_ready();
    // ---- dW2 = dZ2^T H1 and dH1 = dZ2 W2 (one commit) ----
    if (t == 0) {
        issue(tm + kColDW2, sm + kOffDZ2T, sm + kOffH1T, kT, kHid);
        issue(tm + kColDH1, sm + kOffDZ2, sm + kOffW2T, kHid, kHid);
        mma::commit(mb);
    }
    mma_done(mb, 0, err);
    // ---- dZ1 = dH1 . SiLU'(Z1 + b1), written as dZ1^T over the H1 region ----
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 32) {
        float dh[32], z[32];
        mma::tmem_ld32(tm + lane_off + kColDH1 + c0, dh);
        mma::tmem_ld32(tm + lane_off + kColZ1 + c0, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float zz = z[j] + P[kP_b1 + c0 + j];
            const float s = sigm(zz);
            const float d = dh[j] * s * (1.f + zz * (1.f - s));
            atomicAdd(&red[c0 + j], d);  // gb1
            st_bf16(sm + kOffH1, c0 + j, t, kT, d);
        }
    }
    operands_ready();
    // ---- dW1 = dZ1^T X ----
    if (t == 0) {
        issue(tm + kColDW1, sm + kOffH1, sm + kOffXT, kT, kIn);
        mma::commit(mb);
    }
    const bool ok = mma_done(mb, 1, err);
    // ---- weight gradients: thread t owns output feature t ----
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            mma::tmem_ld32(tm + lane_off + kColDW2 + c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) atomicAdd(&g[kP_W2 + t * kHid + c0 + j], v[j]);
        }
        float v[32];
        mma::tmem_ld32(tm + lane_off + kColDW1, v);
        // fold the operand columns back onto W1's master columns
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(&g[kP_W1 + t * kIn + k], v[k] + v[4 + k]);
        atomicAdd(&g[kP_W1 + t * kIn + 4], v[8]);
    }
    mma::fence_before_sync();
    __syncthreads();
    atomicAdd(&g[kP_b1 + t], red[t]);
    atomicAdd(&g[kP_b2 + t], red[kHid + t]);
    atomicAdd(&g[kP_w3 + t], red[2 * kHid + t]);
    if (t == 0) {
        atomicAdd(&g[kP_b3], red[3 * kHid]);
        atomicAdd(&g[kP_n], red[3 * kHid + 1]);
    }
    if (warp == 0) mma::tmem_dealloc(tm, 512);
}

// Adam on the FP32 parameters, then the BF16 operand copies; gradients are
// zeroed for the next batch.
__global__ void k_adam(float* p, float* g, float* m, float* v, float lr, float b1, float b2, float eps, float bc1,
                       float bc2, bf16* W1b, bf16* W2b, bf16* W2Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP_n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    g[i] = 0.f;
    float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    if (i < kP_b1 && (i % kIn) >= 5) pi = 0.f;  // unused input columns
    p[i] = pi;
    if (i < kP_b1) {
        const int r = i / kIn, c = i % kIn;
        if (c < 4) W1b[r * kIn + 4 + c] = __float2bfloat16_rn(pi);
        if (c < 5) W1b[r * kIn + w1_op_col(c)] = __float2bfloat16_rn(pi);
    } else if (i >= kP_W2 && i < kP_b2) {
        const int j = i - kP_W2;
        W2b[j] = __float2bfloat16_rn(pi);
        W2Tb[(j % kHid) * kHid + j / kHid] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_refresh_bf16(const float* p, bf16* W1b, bf16* W2b, bf16* W2Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kP_b1) {
        const int r = i / kIn, c = i % kIn;
        const float v = c < 4 ? p[r * kIn + c] : c < 8 ? p[r * kIn + c - 4] : c == 8 ? p[r * kIn + 4] : 0.f;
        W1b[i] = __float2bfloat16_rn(v);
    }
    if (i >= kP_W2 && i < kP_b2) {
        const int j = i - kP_W2;
        W2b[j] = __float2bfloat16_rn(p[i]);
        W2Tb[(j % kHid) * kHid + j / kHid] = __float2bfloat16_rn(p[i]);
    }
}

// ---- forward-only evaluation ---------------------------------------------------
// mode 0: points x [n][4] (normalised) -> out[i] = log2 value.
// mode 1: the table's nodes (index i, natural layout): compare with the FP64
//         table and flag every 4-D cell touching a node whose relative error
//         |2^(l_mlp - l_tab) - 1| exceeds tol.
// mode 2: cell centres (index i over (nH-1)(nB-1)(nN-1)(nT-1)): compare with
//         the table's multilinear value there (mean of the 16 corners).
__global__ void __launch_bounds__(kT) k_mlp_eval(MlpDev w, int mode, const float* __restrict__ x, float* out,
                                                long long n, DevTable tab, uint32_t* mask, float tol, unsigned* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kEOffBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kEOffBar + 8);
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const float* P = w.p;
    load_kmajor(sm + kEOffW1, w.W1b, kHid, kIn);
    load_kmajor(sm + kEOffW2, w.W2b, kHid, kHid);
    if (t == 0) {
        mma::mbar_init(mma::smem_addr(mbar), 1);
        mma::fence_mbar_init();
    }
    if (warp == 0) mma::tmem_alloc(mma::smem_addr(tslot), 256);
    operands_ready();
    const uint32_t tm = *tslot;
    const uint32_t mb = mma::smem_addr(mbar);
    const int nH = tab.n[0], nB = tab.n[1], nN = tab.n[2], nT = tab.n[3];
    uint32_t phase = 0;
    const long long ntiles = (n + kT - 1) / kT;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long i = tile * kT + t;
        const bool live = i < n;
        float xv[4] = {0.f, 0.f, 0.f, 0.f};
        int idx[4] = {0, 0, 0, 0};
        if (live) {
            if (mode == 0) {
#pragma unroll
                for (int d = 0; d < 4; ++d) xv[d] = x[4 * i + d];
            } else {
                long long r = i;
                const int dims[4] = {mode == 1 ? nH : nH - 1, mode == 1 ? nB : nB - 1, mode == 1 ? nN : nN - 1,
                                     mode == 1 ? nT : nT - 1};
                for (int d = 3; d >= 0; --d) {
                    idx[d] = (int)(r % dims[d]);
                    r /= dims[d];
                }
                const int nd[4] = {nH, nB, nN, nT};
#pragma unroll
                for (int d = 0; d < 4; ++d)
                    xv[d] = 2.f * ((float)idx[d] + (mode == 2 ? 0.5f : 0.f)) / (float)(nd[d] - 1) - 1.f;
            }
        }
        {
            __align__(16) bf16 tmp[16];
            input_row(xv, w.xs, tmp);
            *reinterpret_cast<uint4*>(sm + kEOffX + mma::kmajor_offset(t, 0, kIn)) = *reinterpret_cast<const uint4*>(tmp);
            *reinterpret_cast<uint4*>(sm + kEOffX + mma::kmajor_offset(t, 8, kIn)) =
                *reinterpret_cast<const uint4*>(tmp + 8);
        }
        operands_ready();
        if (t == 0) {
            issue(tm, sm + kEOffX, sm + kEOffW1, kIn, kHid);
            mma::commit(mb);
        }
        mma_done(mb, phase, err);
        phase ^= 1u;
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float z[32];
            mma::tmem_ld32(tm + lane_off + c0, z);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float zz = z[j] + P[kP_b1 + c0 + j];
                z[j] = zz * sigm(zz);
            }
            st_row32(sm + kEOffH1, t, c0, kHid, z);
        }
        operands_ready();
        if (t == 0) {
            issue(tm + 128, sm + kEOffH1, sm + kEOffW2, kHid, kHid);
            mma::commit(mb);
        }
        mma_done(mb, phase, err);
        phase ^= 1u;
        float yh = P[kP_b3];
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float z[32];
            mma::tmem_ld32(tm + lane_off + 128 + c0, z);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float zz = z[j] + P[kP_b2 + c0 + j];
                yh = fmaf(zz * sigm(zz), P[kP_w3 + c0 + j], yh);
            }
        }
        const float lv = fmaf(w.std, yh, w.mean);
        if (live) {
            if (mode == 0) {
                out[i] = lv;
            } else {
                double ref;
                if (mode == 1) {
                    ref = tab.ls64[i];
                } else {
                    ref = 0.0;
                    for (int c = 0; c < 16; ++c) {
                        const long long e = (((long long)(idx[0] + (c & 1)) * nB + idx[1] + ((c >> 1) & 1)) * nN +
                                             idx[2] + ((c >> 2) & 1)) * nT + idx[3] + ((c >> 3) & 1);
                        ref += tab.ls64[e];
                    }
                    ref *= 1.0 / 16.0;
                }
                const double rel = fabs(exp2((double)lv - ref) - 1.0);
                if (!(rel <= (double)tol)) {
                    for (int c = 0; c < 16; ++c) {
                        const int d0 = mode == 1 ? (c & 1) : 0, d1 = mode == 1 ? ((c >> 1) & 1) : 0;
                        const int d2 = mode == 1 ? ((c >> 2) & 1) : 0, d3 = mode == 1 ? ((c >> 3) & 1) : 0;
                        if (mode == 2 && c > 0) break;
                        const int h = idx[0] - d0, b = idx[1] - d1, nn = idx[2] - d2, tt = idx[3] - d3;
                        if (h < 0 || b < 0 || nn < 0 || tt < 0 || h >= nH - 1 || b >= nB - 1 || nn >= nN - 1 ||
                            tt >= nT - 1)
                            continue;
                        const long long cell = (((long long)h * (nB - 1) + b) * (nN - 1) + nn) * (nT - 1) + tt;
                        atomicOr(&mask[cell >> 5], 1u << (cell & 31));
                    }
                }
            }
        }
        __syncthreads();   // the next tile rewrites X and H1
    }
    mma::fence_before_sync();
    __syncthreads();
    if (warp == 0) mma::tmem_dealloc(tm, 256);
}

// ---- host side --------------------------------------------------------------------
std::mutex g_sur_mu;
std::unordered_set<const cool_surrogate*>& live_surrogates() {
    static std::unordered_set<const cool_surrogate*> s;
    return s;
}

bool sur_ok(const cool_surrogate* s) {
    if (!s) return false;
    std::lock_guard<std::mutex> g(g_sur_mu);
    return live_surrogates().count(s) == 1 && s->magic == kSurrogateMagic;
}

MlpDev mlp_dev(const cool_surrogate* s) {
    MlpDev w;
    w.W1b = s->d_W1b;
    w.W2b = s->d_W2b;
    w.W2Tb = s->d_W2Tb;
    w.p = s->d_p;
    w.mean = (float)s->mean;
    w.std = (float)s->std;
    for (int d = 0; d < 4; ++d) {
        w.l0[d] = (float)s->l0[d];
        w.span[d] = (float)s->span[d];
    }
    w.xs = (float)s->x_switch;
    return w;
}

void sur_free_memory(cool_surrogate* s) {
    void* ptrs[] = {s->d_p, s->d_g, s->d_m, s->d_v, s->d_W1b, s->d_W2b, s->d_W2Tb, s->d_err, s->d_mask};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// SplitMix64 on the host for the initial weights.
uint64_t sm64(uint64_t& st) {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double host_uniform(uint64_t& st) { return (double)(sm64(st) >> 11) * (1.0 / 9007199254740992.0); }

__global__ void k_standardise(const double* y64, float* y32, long long n, double mean, double inv_std) {
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y32[i] = (float)((y64[i] - mean) * inv_std);
}

__global__ void k_moments(const double* y, long long n, double* acc) {
    double s = 0.0, s2 = 0.0;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        s += y[i];
        s2 += y[i] * y[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], s);
        atomicAdd(&acc[1], s2);
    }
}

int sm_count_here() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cool_status launch_train_tiles(cool_surrogate* s, const float* x, const float* y, long long first, int ntiles,
                               float inv_batch, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTrain);
    if (e != cudaSuccess) return set_cuda_error(e);
    k_mlp_train_tile<<<ntiles, kT, kSmemTrain, st>>>(mlp_dev(s), x, y, first, inv_batch, s->d_g, s->d_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

cool_status launch_eval(const cool_surrogate* s, const cool_table* t, int mode, const float* x, float* out,
                        long long n, uint32_t* mask, float tol, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemEval);
    if (e != cudaSuccess) return set_cuda_error(e);
    long long tiles = (n + kT - 1) / kT;
    long long cap = (long long)sm_count_here() * 2;   // two CTAs (2 x 256 TMEM columns) per SM
    long long blocks = tiles < cap ? tiles : cap;
    DevTable dt;
    memset(&dt, 0, sizeof(dt));
    if (t) dt = t->dev;
    k_mlp_eval<<<(int)blocks, kT, kSmemEval, st>>>(mlp_dev(s), mode, x, out, n, dt, mask, tol, s->d_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

}  // namespace
}  // namespace cool

using namespace cool;

extern "C" {

cool_status cool_fit_spec_default(cool_fit_spec* f) {
    if (!f) return COOL_ENULL;
    memset(f, 0, sizeof(*f));
    f->channel = 1;
    f->n_samples = 1LL << 24;
    f->batch = 16384;
    f->epochs = 16;
    f->lr = 2e-3;
    f->lr_final = 2e-5;
    f->seed = 20250513ull;
    f->fallback_tol = 1e-3;
    return COOL_OK;
}

cool_status cool_surrogate_fit(const cool_table* t, const cool_fit_spec* f, void* stream, cool_surrogate** out) {
    if (!t || !f || !out) return COOL_ENULL;
    *out = nullptr;
    if (!table_ok(t)) return COOL_ESTATE;
    if (f->channel != 1) return COOL_EUNSUPPORTED;
    if (f->batch < kT || f->batch % kT || f->n_samples < f->batch || f->n_samples % f->batch || f->epochs < 0 ||
        !(f->lr >= 0.0) || !(f->lr_final >= 0.0) || !(f->fallback_tol > 0.0))
        return COOL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cool_surrogate* s = new (std::nothrow) cool_surrogate;
    if (!s) return COOL_ENOMEM;
    memset(s, 0, sizeof(*s));
    s->magic = kSurrogateMagic;
    cudaGetDevice(&s->device);
    s->channel = f->channel;
    s->spec = t->spec;
    const double lo[4] = {t->spec.H_min, t->spec.B_min, t->spec.ne_min, t->spec.T_min};
    const double hi[4] = {t->spec.H_max, t->spec.B_max, t->spec.ne_max, t->spec.T_max};
    for (int d = 0; d < 4; ++d) {
        s->l0[d] = log2(lo[d]);
        s->span[d] = log2(hi[d]) - s->l0[d];
    }
    s->x_switch = 2.0 * (log2(t->spec.k2_switch_T) - s->l0[3]) / s->span[3] - 1.0;
    const int cells = 1;
    (void)cells;
    const long long nc = (long long)(t->spec.n_H - 1) * (t->spec.n_B - 1) * (t->spec.n_ne - 1) * (t->spec.n_Te - 1);
    s->mask_bits = nc;
    cudaError_t e = cudaSuccess;
    const size_t pb = sizeof(float) * kP_alloc;
    if (e == cudaSuccess) e = cudaMalloc(&s->d_p, pb);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_g, pb);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_W1b, sizeof(bf16) * kHid * kIn);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_W2b, sizeof(bf16) * kHid * kHid);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_W2Tb, sizeof(bf16) * kHid * kHid);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_mask, sizeof(uint32_t) * ((nc + 31) / 32));
    float* d_x = nullptr;
    double* d_y64 = nullptr;
    float* d_y = nullptr;
    double* d_acc = nullptr;
    const long long n = f->n_samples;
    if (e == cudaSuccess && f->epochs > 0) e = cudaMalloc(&d_x, sizeof(float) * 4 * n);
    if (e == cudaSuccess && f->epochs > 0) e = cudaMalloc(&d_y64, sizeof(double) * n);
    if (e == cudaSuccess && f->epochs > 0) e = cudaMalloc(&d_y, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_acc, sizeof(double) * 2);
    auto fail = [&](cool_status stt) {
        if (d_x) cudaFree(d_x);
        if (d_y64) cudaFree(d_y64);
        if (d_y) cudaFree(d_y);
        if (d_acc) cudaFree(d_acc);
        sur_free_memory(s);
        delete s;
        return stt;
    };
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? COOL_ENOMEM : set_cuda_error(e));
    // initial parameters: uniform(-a, a) with a = sqrt(6 / fan_in) (fan_in 5, 128), w3 small
    std::vector<float> hp(kP_alloc, 0.f);
    uint64_t rs = f->seed;
    for (int o = 0; o < kHid; ++o)
        for (int k = 0; k < 5; ++k) hp[kP_W1 + o * kIn + k] = (float)((2.0 * host_uniform(rs) - 1.0) * sqrt(6.0 / 5.0));
    for (int i = 0; i < kHid * kHid; ++i) hp[kP_W2 + i] = (float)((2.0 * host_uniform(rs) - 1.0) * sqrt(6.0 / 128.0));
    for (int i = 0; i < kHid; ++i) hp[kP_w3 + i] = (float)((2.0 * host_uniform(rs) - 1.0) * sqrt(1.0 / 128.0));
    e = cudaMemcpyAsync(s->d_p, hp.data(), pb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_g, 0, pb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_m, 0, pb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_v, 0, pb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_mask, 0, sizeof(uint32_t) * ((nc + 31) / 32), st);
    if (e != cudaSuccess) return fail(set_cuda_error(e));
    k_refresh_bf16<<<(kP_n + 255) / 256, 256, 0, st>>>(s->d_p, s->d_W1b, s->d_W2b, s->d_W2Tb);
    s->mean = 0.0;
    s->std = 1.0;
    if (f->epochs > 0) {
        cool_status cs = fit_samples_fp64(t->spec, n, f->seed, d_x, d_y64, st);
        if (cs != COOL_OK) return fail(cs);
        cudaMemsetAsync(d_acc, 0, sizeof(double) * 2, st);
        k_moments<<<sm_count_here() * 4, 256, 0, st>>>(d_y64, n, d_acc);
        double acc[2];
        e = cudaMemcpyAsync(acc, d_acc, sizeof(acc), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(set_cuda_error(e));
        s->mean = acc[0] / n;
        s->std = sqrt(fmax(acc[1] / n - s->mean * s->mean, 1e-30));
        k_standardise<<<sm_count_here() * 8, 256, 0, st>>>(d_y64, d_y, n, s->mean, 1.0 / s->std);
        const long long batches = n / f->batch;
        const long long total = batches * f->epochs;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        double bc1 = 1.0, bc2 = 1.0;
        for (long long stp = 0; stp < total; ++stp) {
            const long long first = (stp % batches) * f->batch;
            cs = launch_train_tiles(s, d_x, d_y, first, f->batch / kT, 1.f / f->batch, st);
            if (cs != COOL_OK) return fail(cs);
            bc1 *= b1;
            bc2 *= b2;
            const double frac = total > 1 ? (double)stp / (double)(total - 1) : 1.0;
            const double lr = f->lr_final + 0.5 * (f->lr - f->lr_final) * (1.0 + cos(3.141592653589793 * frac));
            if (stp == total - 1) {
                float loss = 0.f;
                e = cudaMemcpyAsync(&loss, s->d_g + kP_n, sizeof(float), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return fail(set_cuda_error(e));
                s->final_loss = loss;
            }
            cudaMemsetAsync(s->d_g + kP_n, 0, sizeof(float), st);
            k_adam<<<(kP_n + 255) / 256, 256, 0, st>>>(s->d_p, s->d_g, s->d_m, s->d_v, (float)lr, b1, b2, eps,
                                                       (float)(1.0 - bc1), (float)(1.0 - bc2), s->d_W1b, s->d_W2b,
                                                       s->d_W2Tb);
        }
        s->steps = total;
    }
    cudaFree(d_x);
    cudaFree(d_y64);
    cudaFree(d_y);
    d_x = nullptr; d_y64 = nullptr; d_y = nullptr;
    // error map over the table cells: nodes, then cell centres
    cool_status cs = launch_eval(s, t, 1, nullptr, nullptr,
                                 (long long)t->spec.n_H * t->spec.n_B * t->spec.n_ne * t->spec.n_Te, s->d_mask,
                                 (float)f->fallback_tol, st);
    if (cs == COOL_OK) cs = launch_eval(s, t, 2, nullptr, nullptr, nc, s->d_mask, (float)f->fallback_tol, st);
    if (cs != COOL_OK) return fail(cs);
    std::vector<uint32_t> hm((nc + 31) / 32);
    unsigned herr = 0;
    e = cudaMemcpyAsync(hm.data(), s->d_mask, sizeof(uint32_t) * hm.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(set_cuda_error(e));
    if (herr) return fail(COOL_ECUDA);
    long long set = 0;
    for (uint32_t wv : hm) set += __builtin_popcount(wv);
    s->mask_set = set;
    cudaFree(d_acc);
    d_acc = nullptr;
    {
        std::lock_guard<std::mutex> g(g_sur_mu);
        live_surrogates().insert(s);
    }
    *out = s;
    return COOL_OK;
}

cool_status cool_surrogate_free(cool_surrogate* s) {
    if (!s) return COOL_OK;
    {
        std::lock_guard<std::mutex> g(g_sur_mu);
        if (live_surrogates().erase(s) != 1) return COOL_ESTATE;
    }
    s->magic = 0;
    sur_free_memory(s);
    delete s;
    return COOL_OK;
}

cool_status cool_surrogate_info(const cool_surrogate* s, cool_surrogate_stats* out) {
    if (!s || !out) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    out->final_loss = s->final_loss;
    out->steps = s->steps;
    out->mask_cells = s->mask_bits;
    out->fallback_cells = s->mask_set;
    out->param_bytes_bf16 = (long long)(kHid * 5 + kHid * kHid) * 2 + (long long)(3 * kHid + 1) * 4;
    out->mean = s->mean;
    out->std = s->std;
    out->x_switch = s->x_switch;
    return COOL_OK;
}

cool_status cool_surrogate_get_params(const cool_surrogate* s, float* host, int n) {
    if (!s || !host) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    if (n != kP_n) return COOL_EINVAL;
    cudaError_t e = cudaMemcpy(host, s->d_p, sizeof(float) * kP_n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

cool_status cool_surrogate_set_params(cool_surrogate* s, const float* host, int n) {
    if (!s || !host) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    if (n != kP_n) return COOL_EINVAL;
    cudaError_t e = cudaMemcpy(s->d_p, host, sizeof(float) * kP_n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_cuda_error(e);
    k_refresh_bf16<<<(kP_n + 255) / 256, 256>>>(s->d_p, s->d_W1b, s->d_W2b, s->d_W2Tb);
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

cool_status cool_surrogate_grads(cool_surrogate* s, long long n, const float* x4, const float* y_std,
                                 float* grads_host, float* loss_host, void* stream) {
    if (!s || !x4 || !y_std || !grads_host) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    if (n < kT || n % kT) return COOL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(s->d_g, 0, sizeof(float) * kP_alloc, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    cool_status cs = launch_train_tiles(s, x4, y_std, 0, (int)(n / kT), 1.f / (float)n, st);
    if (cs != COOL_OK) return cs;
    std::vector<float> g(kP_alloc);
    e = cudaMemcpyAsync(g.data(), s->d_g, sizeof(float) * kP_alloc, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(e);
    memcpy(grads_host, g.data(), sizeof(float) * kP_n);
    if (loss_host) *loss_host = g[kP_n];
    cudaMemsetAsync(s->d_g, 0, sizeof(float) * kP_alloc, st);
    return COOL_OK;
}

cool_status cool_surrogate_eval(const cool_surrogate* s, long long n, const float* x4, float* y, void* stream) {
    if (!s || (n > 0 && (!x4 || !y))) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    if (n < 0) return COOL_EINVAL;
    return launch_eval(s, nullptr, 0, x4, y, n, nullptr, 0.f, (cudaStream_t)stream);
}

cool_status cool_surrogate_mask(const cool_surrogate* s, uint32_t* host_bits, long long words) {
    if (!s || !host_bits) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    if (words != (s->mask_bits + 31) / 32) return COOL_EINVAL;
    cudaError_t e = cudaMemcpy(host_bits, s->d_mask, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

cool_status cool_surrogate_set_mask(cool_surrogate* s, const uint32_t* host_bits, long long words) {
    if (!s || !host_bits) return COOL_ENULL;
    if (!sur_ok(s)) return COOL_ESTATE;
    if (words != (s->mask_bits + 31) / 32) return COOL_EINVAL;
    std::vector<uint32_t> hm(host_bits, host_bits + words);
    const long long tail = s->mask_bits & 31;
    if (tail) hm[words - 1] &= (1u << tail) - 1u;   // bits past the last cell stay clear
    long long set = 0;
    for (uint32_t w : hm) set += __builtin_popcount(w);
    cudaError_t e = cudaMemcpy(s->d_mask, hm.data(), sizeof(uint32_t) * words, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_cuda_error(e);
    s->mask_set = set;
    return COOL_OK;
}

cool_status cool_surrogate_infer(const cool_surrogate* s, const cool_table* t, const cool_params* p, long long n_cells,
                                 const float* rho, const float* B, const float* H, const float* u_e_in,
                                 const float* u_i_in, float* u_e_out, float* u_i_out, float* q_cool_out,
                                 float* q_cc_out, cool_counters* counters, void* stream) {
    if (!s || !t || !p) return COOL_ENULL;
    if (!sur_ok(s) || !table_ok(t)) return COOL_ESTATE;
    cool_status cs = validate_params(p);
    if (cs != COOL_OK) return cs;
    if (n_cells < 0) return COOL_EINVAL;
    const cool_table_spec& a = s->spec;
    const cool_table_spec& b = t->spec;
    if (a.n_H != b.n_H || a.n_B != b.n_B || a.n_ne != b.n_ne || a.n_Te != b.n_Te || a.H_min != b.H_min ||
        a.H_max != b.H_max || a.B_min != b.B_min || a.B_max != b.B_max || a.ne_min != b.ne_min ||
        a.ne_max != b.ne_max || a.T_min != b.T_min || a.T_max != b.T_max)
        return COOL_EINVAL;   // fitted to another table box
    if (b.dtype != COOL_F32 || p->mode != COOL_EXPLICIT_LIMITED || p->fp64_critical || p->path != COOL_PATH_L2WINDOW)
        return COOL_EUNSUPPORTED;
    if (n_cells == 0) return COOL_OK;
    if (!rho || !B || !H || !u_e_in || !u_i_in || !u_e_out || !u_i_out) return COOL_ENULL;
    const void* ptrs[] = {rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, q_cool_out, q_cc_out};
    for (const void* q : ptrs)
        if ((uintptr_t)q % 4 != 0) return COOL_EALIGN;
    if ((uintptr_t)counters % 8 != 0) return COOL_EALIGN;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device || dev != s->device) return COOL_ESTATE;
    return launch_step_surrogate(s, t, p, n_cells, rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, q_cool_out,
                                 q_cc_out, counters, (cudaStream_t)stream);
}

}  // extern "C"
