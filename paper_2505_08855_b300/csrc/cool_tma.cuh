// cool_tma.cuh -- bulk asynchronous copies (the TMA engine, non-tensor
// form) global -> shared memory with completion on an mbarrier, written from
// the PTX ISA: the mbarrier's transaction count is armed by one thread, the
// copies complete it; waits are bounded.
#pragma once

#include <stdint.h>

#include "cool_mma.cuh"

namespace cool {
namespace tma {

// One arrival that also expects `bytes` of transactions on the mbarrier.
__device__ __forceinline__ void arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 :
                 : "r"(mbar), "r"(bytes)
                 : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to this CTA's shared memory; completion is counted on mbar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :
                 : "r"(dst_smem), "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

}  // namespace tma
}  // namespace cool
