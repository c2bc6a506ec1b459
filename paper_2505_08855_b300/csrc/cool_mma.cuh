// cool_mma.cuh -- tcgen05 (5th-generation tensor core) building blocks for
// sm_103a, written from the PTX ISA: TMEM allocation, shared-memory matrix
// descriptors, the kind::f16 instruction descriptor, MMA issue and commit to
// an mbarrier, bounded mbarrier waits, and TMEM -> register loads.
//
// Operand layout used throughout (PTX "canonical layout", K-major, no
// swizzle): a matrix of R rows and K bf16 columns is stored as 8x8 core
// matrices of 128 contiguous bytes (8 rows of 16 bytes); core matrix
// (row group g, column chunk c) starts at byte (g * (K/8) + c) * 128.  Hence
// the descriptor's leading-dimension byte offset (between core matrices
// along K) is 128 and its stride-dimension byte offset (between row groups)
// is K/8 * 128.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace cool {
namespace mma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of an R x K K-major operand in the core-matrix layout.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int K) {
    return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (64 bit): start address >> 4 in bits 0-13,
// leading-dimension byte offset >> 4 in bits 16-29, stride-dimension byte
// offset >> 4 in bits 32-45, the fixed value 1 in bits 46-48, base offset 0,
// relative leading-dimension mode, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: dense, D = F32 (bits
// 4-5 = 1), A = B = BF16 (bits 7-9 = 1, bits 10-12 = 1), no negation, both
// operands K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 slice; issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on an mbarrier once every prior tcgen05.mma of this thread completes.
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
}

// Make generic-proxy writes to shared memory visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
}

// Bounded wait for the completion of the mbarrier phase `parity`: returns
// false after `limit` unsuccessful polls (each poll is itself time-bounded).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// TMEM allocation by one full warp; the base address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t slot_saddr, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :
                 : "r"(slot_saddr), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" : : : "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32 w .. 32 w + 31; taddr carries lane << 16 | column).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" : : : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Logistic sigmoid 1 / (1 + e^-z) from the hardware exp2 and reciprocal
// approximations (a few ulp); e^-z = inf for z < -88 gives 0.
__device__ __forceinline__ float sigm(float z) {
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z * -1.4426950408889634f));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.f + e));
    return r;
}

// 32 values into row r, columns k0..k0+31, of an R x K K-major operand.
__device__ __forceinline__ void st_row32(unsigned char* base, int r, int k0, int K, const float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 32; c += 8) {
        __align__(16) __nv_bfloat16 tmp[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) tmp[j] = __float2bfloat16_rn(v[c + j]);
        *reinterpret_cast<uint4*>(base + kmajor_offset(r, k0 + c, K)) = *reinterpret_cast<const uint4*>(tmp);
    }
}

__device__ __forceinline__ void st_bf16(unsigned char* base, int r, int k, int K, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + kmajor_offset(r, k, K)) = __float2bfloat16_rn(v);
}

// Row-major [R][K] bf16 in global memory -> the K-major layout.
__device__ __forceinline__ void load_kmajor(unsigned char* dst, const __nv_bfloat16* src, int R, int K) {
    const int kc = K >> 3;
    for (int i = threadIdx.x; i < R * kc; i += blockDim.x) {
        const int r = i / kc, c = i % kc;
        *reinterpret_cast<uint4*>(dst + kmajor_offset(r, c * 8, K)) =
            *reinterpret_cast<const uint4*>(src + (size_t)r * K + c * 8);
    }
}

// D (+)= A B^T over K (multiple of 16); issued by one thread, not committed.
__device__ __forceinline__ void issue(uint32_t d_tmem, const unsigned char* A, const unsigned char* B, int K, int N) {
    const uint32_t idesc = mma::idesc_bf16_f32(128, N);
    const uint32_t sbo = (uint32_t)(K >> 3) * 128;
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t ad = sdesc(smem_addr(A) + s * 256, 128, sbo);
        const uint64_t bd = sdesc(smem_addr(B) + s * 256, 128, sbo);
        mma::mma_bf16(d_tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
}

// Make shared-memory operand writes of all threads visible to the tensor core.
__device__ __forceinline__ void operands_ready() {
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// Wait for one committed MMA group (phase parity); on timeout report, wait
// once more (bounded) and continue.
__device__ __forceinline__ bool mma_done(uint32_t mbar, uint32_t parity, unsigned* err) {
    bool ok = mbar_wait(mbar, parity, 1 << 20);
    if (!ok) {
        if (err) atomicOr(err, 2u);
        mbar_wait(mbar, parity, 1 << 16);
    }
    fence_after_sync();
    return ok;
}

}  // namespace mma
}  // namespace cool
