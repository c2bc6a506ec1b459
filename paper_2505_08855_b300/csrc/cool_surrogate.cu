// cool_surrogate.cu -- the learned surrogate of the rate table (not in the
// paper): a per-channel MLP 4 -> 128 -> 128 -> 1 (SiLU) on hand-written
// tcgen05 GEMMs.  This file starts with the GEMM primitive and its check
// entry point.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cool_internal.cuh"
#include "cool_mma.cuh"

namespace cool {
namespace {

constexpr int kGemmThreads = 128;          // 4 warps: TMEM lanes 0..127 = tile rows
constexpr int kGemmRegion = 64 * 1024;     // bytes per operand region (>= 2x the operand)
constexpr uint32_t kGemmTmemCols = 256;    // >= N

// C[M x N] = A[M x K] B[N x K]^T, bf16 in, fp32 out; one CTA per 128-row tile.
// Requires M % 128 == 0, N % 16 == 0, 16 <= N <= 128, K % 16 == 0, 16 <= K <= 128.
__global__ void __launch_bounds__(kGemmThreads, 1)
k_gemm_bf16_tc(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B, float* __restrict__ C,
               int M, int N, int K, unsigned* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + kGemmRegion;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kGemmRegion);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kGemmRegion + 8);
    const int t = threadIdx.x, warp = t >> 5;
    const int row0 = blockIdx.x * 128;
    const int kc = K >> 3;  // 16-byte chunks per row
    // operands into the core-matrix layout (16-byte chunks)
    for (int i = t; i < 128 * kc; i += kGemmThreads) {
        const int r = i / kc, c = i % kc;
        const uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)(row0 + r) * K + c * 8);
        *reinterpret_cast<uint4*>(sA + mma::kmajor_offset(r, c * 8, K)) = v;
    }
    for (int i = t; i < N * kc; i += kGemmThreads) {
        const int r = i / kc, c = i % kc;
        const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + c * 8);
        *reinterpret_cast<uint4*>(sB + mma::kmajor_offset(r, c * 8, K)) = v;
    }
    if (t == 0) {
        mma::mbar_init(mma::smem_addr(mbar), 1);
        mma::fence_mbar_init();
    }
    if (warp == 0) mma::tmem_alloc(mma::smem_addr(tslot), kGemmTmemCols);
    mma::fence_async_smem();
    mma::fence_before_sync();
    __syncthreads();
    mma::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (t == 0) {
        const uint32_t idesc = mma::idesc_bf16_f32(128, N);
        const uint32_t sbo = (uint32_t)kc * 128;
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = mma::sdesc(mma::smem_addr(sA) + s * 256, 128, sbo);
            const uint64_t bd = mma::sdesc(mma::smem_addr(sB) + s * 256, 128, sbo);
            mma::mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        mma::commit(mma::smem_addr(mbar));
    }
    bool ok = mma::mbar_wait(mma::smem_addr(mbar), 0, 1 << 20);
    if (!ok) {
        // no completion signal: report, wait once more (bounded) for the MMAs
        // in flight, then free the TMEM and return without reading it
        if (err) atomicOr(err, 1u);
        mma::mbar_wait(mma::smem_addr(mbar), 0, 1 << 16);
    }
    mma::fence_after_sync();
    for (int c0 = 0; ok && c0 < N; c0 += 32) {
        float v[32];
        mma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
        float* out = C + (size_t)(row0 + t) * N + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (c0 + j < N) out[j] = v[j];
    }
    mma::fence_before_sync();
    __syncthreads();
    if (warp == 0) mma::tmem_dealloc(tmem, kGemmTmemCols);
}

// The failure path of the bounded waits: one thread polls the first phase of
// an mbarrier that nothing arrives on, `polls` times, then reports and
// invalidates the barrier.  No copy or product is in flight, so nothing else
// needs to be waited for or freed.
__global__ void k_wait_timeout(int polls, unsigned* err) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x != 0) return;
    const uint32_t a = mma::smem_addr(&mbar);
    mma::mbar_init(a, 1);
    mma::fence_mbar_init();
    if (!mma::mbar_wait(a, 0, polls)) atomicOr(err, 1u);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" : : "r"(a) : "memory");
}

}  // namespace
}  // namespace cool

extern "C" cool_status cool_debug_wait_timeout(int polls, unsigned* err, void* stream) {
    using namespace cool;
    if (!err) return COOL_ENULL;
    if (polls < 1 || polls > (1 << 20)) return COOL_EINVAL;
    k_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(polls, err);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

extern "C" cool_status cool_debug_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K,
                                            unsigned* err, void* stream) {
    using namespace cool;
    if (!A || !B || !C) return COOL_ENULL;
    if (M <= 0 || M % 128 || N < 16 || N > 128 || N % 16 || K < 16 || K > 128 || K % 16) return COOL_EINVAL;
    if (((uintptr_t)A | (uintptr_t)B) % 16 || (uintptr_t)C % 4) return COOL_EALIGN;
    const size_t smem = 2 * kGemmRegion + 16;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    k_gemm_bf16_tc<<<M / 128, kGemmThreads, smem, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)A, (const __nv_bfloat16*)B, C, M, N, K, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}
