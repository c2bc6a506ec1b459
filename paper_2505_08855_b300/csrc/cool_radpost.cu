// cool_radpost.cu -- the radiation-pressure correction of the electron
// temperature (Sec. 5.2): in cells whose local scattering depth tau_sca =
// n_e sigma_T H exceeds tau_crit, the simulation's thermal pressure is read
// as gas plus radiation, P = a T_e^4 + n k (T_e + T_i), and T_e recomputed.
// With hydrogen (n = n_e = n_i) and P = n k (T_e,sim + T_i) the ion terms
// cancel:  a T^4 + n k T = n k T_e,sim.
//
// Scaled, T = s y with s = (n k T_e,sim / a)^(1/4) the radiation-dominated
// root and beta = s / T_e,sim:  g(y) = y^4 + beta y - 1 = 0 on (0, 1].  g is
// increasing and convex there, so Newton's iteration
//   y <- (3 y^4 + 1) / (4 y^3 + beta)
// from the upper bound y0 = min(1, 1/beta) decreases monotonically to the
// root; five steps reach FP32 precision for every beta (one or two where a
// single pressure term dominates).  Everything is in FP32: s comes from
// nested square roots, so a T^4 (up to ~1e45 in cgs) never forms.
//
// One pass over the fields: read rho, H, u_e (12 B), write T_e (4 B) and
// optionally a thick flag (1 B) per cell; 16-byte aligned arrays move with
// 128-bit streaming accesses, four cells per thread.
#include <math.h>

#include "cool_internal.cuh"

namespace cool {
namespace {

struct RadK {
    float s_n;        // n_e per unit rho (rho_scale / m_p)
    float s_Te;       // T_e,sim per unit u_e / rho
    float s_tau;      // tau_sca per unit rho H  (rho_scale/m_p sigma_T r_g)
    float tau_crit;
    float sqrt_k_a;   // sqrt(k_B / a)
};

__device__ __forceinline__ float rad_te(const RadK& k, float rho, float H, float ue, unsigned char& thick) {
    thick = 0;
    if (!(isfinite(rho) && isfinite(H) && isfinite(ue)) || !(rho > 0.f) || !(ue > 0.f) || H < 0.f)
        return __int_as_float(0x7fc00000);   // NaN: invalid cell
    const float te = __fdividef(k.s_Te * ue, rho);
    const float tau = k.s_tau * rho * H;
    if (!(tau > k.tau_crit)) return te;
    thick = 1;
    // s = (n k T_e / a)^(1/4) as nested square roots (no FP32 overflow for
    // n <= 1e30 cm^-3, T_e <= 1e30 K), beta = s / T_e
    const float s = sqrtf(sqrtf(k.s_n * rho) * sqrtf(te) * k.sqrt_k_a);
    const float beta = __fdividef(s, te);
    if (beta > 0x1p40f) return te;                // radiation negligible: T = T_e (1 - O(beta^-4))
    if (beta < 0x1p-40f) return s;                // gas pressure negligible: T = s (1 - O(beta))
    float y = fminf(1.f, __fdividef(1.f, beta));
#pragma unroll
    for (int it = 0; it < 5; ++it) {
        const float y3 = y * y * y;
        y = __fdividef(fmaf(3.f * y3, y, 1.f), fmaf(4.f, y3, beta));
    }
    return s * y;
}

__global__ void __launch_bounds__(256) k_radiation_te(RadK k, long long n, const float* __restrict__ rho,
                                                      const float* __restrict__ H, const float* __restrict__ ue,
                                                      float* __restrict__ te_out, unsigned char* thick_out,
                                                      bool vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long start = 0;
    if (vec) {
        const long long n4 = n / 4;
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
            const float4 r = __ldcs(reinterpret_cast<const float4*>(rho) + q);
            const float4 h = __ldcs(reinterpret_cast<const float4*>(H) + q);
            const float4 u = __ldcs(reinterpret_cast<const float4*>(ue) + q);
            unsigned char t0, t1, t2, t3;
            float4 o;
            o.x = rad_te(k, r.x, h.x, u.x, t0);
            o.y = rad_te(k, r.y, h.y, u.y, t1);
            o.z = rad_te(k, r.z, h.z, u.z, t2);
            o.w = rad_te(k, r.w, h.w, u.w, t3);
            __stcs(reinterpret_cast<float4*>(te_out) + q, o);
            if (thick_out)
                reinterpret_cast<uchar4*>(thick_out)[q] = make_uchar4(t0, t1, t2, t3);
        }
        start = n4 * 4;
    }
    for (long long i = start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned char t;
        te_out[i] = rad_te(k, rho[i], H[i], ue[i], t);
        if (thick_out) thick_out[i] = t;
    }
}

}  // namespace
}  // namespace cool

using namespace cool;

extern "C" cool_status cool_radiation_te(const cool_params* p, double tau_crit, double a_rad, long long n_cells,
                                         const float* rho, const float* H, const float* u_e, float* te_out,
                                         unsigned char* thick_out, void* stream) {
    if (!p) return COOL_ENULL;
    if (!(p->rho_scale > 0.0) || !isfinite(p->rho_scale) || !(p->M_bh_msun > 0.0) || !(p->gamma_e > 1.0) ||
        !(a_rad > 0.0) || !isfinite(a_rad) || !(tau_crit >= 0.0) || !isfinite(tau_crit))
        return COOL_EINVAL;
    if (n_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    if (!rho || !H || !u_e || !te_out) return COOL_ENULL;
    const uintptr_t al = (uintptr_t)rho | (uintptr_t)H | (uintptr_t)u_e | (uintptr_t)te_out;
    if (al % 4) return COOL_EALIGN;
    const bool vec = al % 16 == 0 && (!thick_out || (uintptr_t)thick_out % 4 == 0);
    const double rg = (kG * (p->M_bh_msun * kMsun)) / (kC * kC);
    RadK k;
    k.s_n = (float)(p->rho_scale / kMP);
    k.s_Te = (float)((p->gamma_e - 1.0) * kMP * kC * kC / kKB);
    k.s_tau = (float)(p->rho_scale / kMP * kSigT * rg);
    k.tau_crit = (float)tau_crit;
    k.sqrt_k_a = (float)sqrt(kKB / a_rad);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long work = vec ? (n_cells / 4 + 255) / 256 : (n_cells + 255) / 256;
    long long blocks = work < sms * 8LL ? work : sms * 8LL;
    if (blocks < 1) blocks = 1;
    k_radiation_te<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(k, n_cells, rho, H, u_e, te_out, thick_out, vec);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}
