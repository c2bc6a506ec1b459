// cool_bridge.cuh -- the cooling energy of one sub-cycle from the two
// channel values, for the step variants that read the synchrotron channel
// another way (the surrogate network, the texture paths).
#pragma once

#include "cool_step_common.cuh"

namespace cool {
namespace {

// The bridge of cool_energy, from the two channel values (log2, code units
// per sub-cycle) and log2 T_e.
__device__ __forceinline__ float bridge_energy(const CellC& c, float Ls, float Lb, float lT) {
    const float M = fmaxf(Ls, Lb);
    const float A = M + lg2a(1.f + ex2a(fminf(Ls, Lb) - M));
    const float Bb = fmaf(4.f, lT, c.lbb_off);
    const float lt = A - Bb;
    float lq;
    if (lt <= 60.f) {
        const float tau = ex2a(lt);
        const float D = fmaf(tau, fmaf(1.5f, tau + c.tau_sca, 1.7320508f), 1.f);
        lq = A - lg2a(D);
    } else {
        lq = Bb - 0.5849625f - (lt + lg2a(1.f + c.tau_sca * ex2a(-lt)));
    }
    return ex2a(fminf(lq, 126.f));
}

}  // namespace
}  // namespace cool
