// cool_step_f16.cu -- the FP32 step kernel k_step_f32 for the plain BF16 (1) and FP16 (2) table
// formats (the launcher is launch_step_f32 in cool_step.cu).
#include "cool_step_kernel.cuh"

namespace cool {

// Kernel of table format fmt (1 or 2), vector or scalar path, variant
// var = implicit | fp64_critical << 1 | counters << 2; nullptr for any other
// format.
const void* step_kernel_f16(int fmt, bool vec, int var) {
#define COOL_KV(V, F) k_step_f32<V, F, 0>, k_step_f32<V, F, 1>, k_step_f32<V, F, 2>, k_step_f32<V, F, 3>, \
                      k_step_f32<V, F, 8>, k_step_f32<V, F, 9>, k_step_f32<V, F, 10>, k_step_f32<V, F, 11>
    static const StepKernelFn table_v[2][8] = {{COOL_KV(true, 1)}, {COOL_KV(true, 2)}};
    static const StepKernelFn table_s[2][8] = {{COOL_KV(false, 1)}, {COOL_KV(false, 2)}};
#undef COOL_KV
    if (fmt < 1 || fmt > 2 || var < 0 || var > 7) return nullptr;
    return (const void*)(vec ? table_v[fmt - 1][var] : table_s[fmt - 1][var]);
}

}  // namespace cool
