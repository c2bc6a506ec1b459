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
// 128-bit streaming accesses, eight cells per thread (two float4 per field,
// both loaded before any arithmetic: 52 us against 62 us with one).
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

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The thin/thick split of one cell.  Returns T_e,sim (or NaN for an invalid
// cell) and sets *thick when the quartic must be solved; then s and beta
// are its scale and parameter (see the header comment).
__device__ __forceinline__ float rad_split(const RadK& k, float rho, float H, float ue, bool& thick, float& s,
                                           float& beta) {
    thick = false;
    if (!(isfinite(rho) && isfinite(H) && isfinite(ue)) || !(rho > 0.f) || !(ue > 0.f) || H < 0.f)
        return __int_as_float(0x7fc00000);   // NaN: invalid cell
    const float te = __fdividef(k.s_Te * ue, rho);
    const float tau = k.s_tau * rho * H;
    if (!(tau > k.tau_crit)) return te;
    thick = true;
    // s = (n k T_e / a)^(1/4) as nested square roots (no FP32 overflow for
    // n <= 1e30 cm^-3, T_e <= 1e30 K), beta = s / T_e
    s = sqrt_approx(sqrt_approx(k.s_n * rho) * sqrt_approx(te) * k.sqrt_k_a);
    beta = __fdividef(s, te);
    return te;
}

// The corrected temperature s y of a thick cell (T_e,sim given).
__device__ __forceinline__ float rad_solve(float te, float s, float beta) {
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

constexpr int kRadThreads = 256;
constexpr int kRadWarps = kRadThreads / 32;
constexpr int kWarpRad = 256;   // cells per warp and round (two float4 per lane)

// Each warp takes rounds of 256 consecutive cells (lane l holds cells
// 4l..4l+3 and 128+4l..128+4l+3).  Thin cells are finished at once; the
// thick ones (about one in ten on the benchmark cells, scattered) go to the
// warp's queue in shared memory and are solved by consecutive lanes, so the
// Newton iterations run on full lanes instead of on the one or two lanes
// per float4 slot that need them.  Outputs are staged in shared memory and
// leave as 128-bit stores.  Warps synchronise only with themselves.
__global__ void __launch_bounds__(kRadThreads) k_radiation_te(RadK k, long long n, const float* __restrict__ rho,
                                                              const float* __restrict__ H,
                                                              const float* __restrict__ ue,
                                                              float* __restrict__ te_out, unsigned char* thick_out,
                                                              bool vec) {
    __shared__ float s_te[kRadWarps][kWarpRad];
    __shared__ float s_s[kRadWarps][kWarpRad];
    __shared__ float s_b[kRadWarps][kWarpRad];
    __shared__ unsigned char s_q[kRadWarps][kWarpRad];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float* te_w = s_te[w];
    float* s_w = s_s[w];
    float* b_w = s_b[w];
    unsigned char* q_w = s_q[w];
    const long long rounds = (n + kWarpRad - 1) / kWarpRad;
    for (long long rd = (long long)blockIdx.x * kRadWarps + w; rd < rounds; rd += (long long)gridDim.x * kRadWarps) {
        float rv[8], hv[8], uv[8];
        const long long base = rd * kWarpRad;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const long long c0 = base + hf * 128 + 4 * lane;
            if (vec && c0 + 3 < n) {
                const float4 r = __ldcs(reinterpret_cast<const float4*>(rho + c0));
                const float4 h = __ldcs(reinterpret_cast<const float4*>(H + c0));
                const float4 u = __ldcs(reinterpret_cast<const float4*>(ue + c0));
                rv[4 * hf] = r.x; rv[4 * hf + 1] = r.y; rv[4 * hf + 2] = r.z; rv[4 * hf + 3] = r.w;
                hv[4 * hf] = h.x; hv[4 * hf + 1] = h.y; hv[4 * hf + 2] = h.z; hv[4 * hf + 3] = h.w;
                uv[4 * hf] = u.x; uv[4 * hf + 1] = u.y; uv[4 * hf + 2] = u.z; uv[4 * hf + 3] = u.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool in = c0 + e < n;
                    rv[4 * hf + e] = in ? rho[c0 + e] : 1.f;
                    hv[4 * hf + e] = in ? H[c0 + e] : 0.f;
                    uv[4 * hf + e] = in ? ue[c0 + e] : 1.f;
                }
            }
        }
        unsigned char th[8];
        int nq = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            bool tk;
            float sc = 0.f, be = 0.f;
            const int slot = (e >> 2) * 128 + 4 * lane + (e & 3);
            te_w[slot] = rad_split(k, rv[e], hv[e], uv[e], tk, sc, be);
            th[e] = tk ? 1 : 0;
            const unsigned m = __ballot_sync(0xffffffffu, tk);
            if (tk) {
                const int pos = nq + __popc(m & lt);
                s_w[slot] = sc;
                b_w[slot] = be;
                q_w[pos] = (unsigned char)slot;
            }
            nq += __popc(m);
        }
        __syncwarp();
        for (int q = lane; q < nq; q += 32) {
            const int slot = q_w[q];
            te_w[slot] = rad_solve(te_w[slot], s_w[slot], b_w[slot]);
        }
        __syncwarp();
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const long long c0 = base + hf * 128 + 4 * lane;
            const int s0 = hf * 128 + 4 * lane;
            if (vec && c0 + 3 < n) {
                __stcs(reinterpret_cast<float4*>(te_out + c0),
                       make_float4(te_w[s0], te_w[s0 + 1], te_w[s0 + 2], te_w[s0 + 3]));
                if (thick_out)
                    *reinterpret_cast<uchar4*>(thick_out + c0) =
                        make_uchar4(th[4 * hf], th[4 * hf + 1], th[4 * hf + 2], th[4 * hf + 3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (c0 + e < n) {
                        te_out[c0 + e] = te_w[s0 + e];
                        if (thick_out) thick_out[c0 + e] = th[4 * hf + e];
                    }
            }
        }
        __syncwarp();
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
    const long long work = (n_cells + kRadWarps * kWarpRad - 1) / (kRadWarps * kWarpRad);   // block rounds
    long long blocks = work < sms * 8LL ? work : sms * 8LL;
    if (blocks < 1) blocks = 1;
    k_radiation_te<<<(int)blocks, kRadThreads, 0, (cudaStream_t)stream>>>(k, n_cells, rho, H, u_e, te_out,
                                                                           thick_out, vec);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}
