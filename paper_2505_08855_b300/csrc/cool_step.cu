// cool_step.cu -- the per-cell two-temperature cooling step on sm_103a.
//
// Per cell (paper Sec. 3.2, tables of Sec. 2.6 / 2.8):
//   keys      n_e = rho rho_scale/m_p, B_G = |b| sqrt(4 pi rho_scale) c,
//             H_cm = H r_g, T_s = (gamma_s - 1) m_p c^2 (u_s/rho)/k_B
//   N_sub sub-cycles of h = dt t_g / N_sub, Lie-split in this order:
//   (i)  Coulomb exchange X = h n_e^2 C(T_i, T_e) (T_i - T_e) / e_scale
//        (Eq. 16), clamped so it does not cross T_e = T_i; FP64 inside the
//        band |T_e/T_i - 1| <= eq_band where T_i - T_e cancels;
//   (ii) radiative cooling: Q_thin = n_e^2 2^{lb(T_e)} + 2^{ls(H,B,n_e,T_e)}
//        (Eq. 10 from the table), bridge Q = Q_thin/(1 + tau_abs (sqrt 3 +
//        1.5 (tau_abs + tau_sca))) (Eqs. 11-12, the printed form multiplied
//        through by tau_abs), energy q = h Q / e_scale removed from u_e:
//        explicitly as min(q, limiter u_e) (Sec. 3.2.1 (i)), or in mode
//        IMPLICIT for stiff cells (q > limiter u_e) by backward Euler
//        u' = u_e - q(u'), bisection in log2 u (Sec. 3.2.1 (ii)).
//
// FP32 path design (B300):
//   - fields are SoA; 16-byte aligned arrays are read and written with
//     128-bit accesses, four cells per thread;
//   - node arrays, the 1-D bremsstrahlung and the 2-D Coulomb channels live
//     in shared memory (loaded once per persistent block);
//   - the 4-D synchrotron channel stays in global memory (L2-resident): the
//     step-invariant H, B, n_e axes are collapsed once per visited T_e
//     interval (8 corners x 2 adjacent T_e values, T_e fastest in memory),
//     so a sub-cycle that stays in its T_e interval reads no table memory;
//   - the bridge is evaluated in log2 space so that no intermediate
//     over/underflows FP32 over the table's 60-decade range.
#include <math.h>

#include "cool_internal.cuh"

namespace cool {
namespace {

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2a(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct StepK {
    DevTable tab;
    float s_n, s_B, s_H, s_Te, s_Ti;  // FP32 key scales (rounded once from FP64)
    float ce, ci, inv_cec;            // gamma - 1, 1/(ce + ci)
    double ce64, ci64, inv_cec64;
    float s_K;                        // m_p c^2 / k_B  (T_s = (gamma_s - 1) s_K u_s / rho)
    int band_fp64;
    float l_hs_e;                     // log2(h / e_scale)
    float l_bb;                       // log2(4 sigma_SB h / e_scale)
    float two_sigT;                   // 2 sigma_T
    float limiter, eq_band, clamp;
    int n_sub, mode, iters;
    int smem_floats;                  // floats of axes + lb + lc in shared memory
    int axes_floats;
};

// Shared-memory view of the small table parts.
struct Smem {
    const float* ax;   // concatenated axes (x, rx, lx per axis)
    const float* lb;
    const float* lc;
};

struct Sel {
    int j;
    float r;   // log2(key / x_j), unclamped
};

// Index selection on an axis (x, rx, lx arrays of n floats at `a`): the
// largest j in [0, n-2] with x[j] <= key (exact FP32 comparisons; a guess
// from log2 is corrected by walking), j = 0 below the first node.
__device__ __forceinline__ Sel select_axis(const float* a, int n, float inv_dl, float key,
                                           unsigned& clamp) {
    const float* x = a;
    const float* rx = a + n;
    const float* lx = a + 2 * n;
    Sel s;
    if (!(key >= x[0])) {
        clamp = 1u;
        s.j = 0;
    } else {
        int j = __float2int_rz((lg2a(key) - lx[0]) * inv_dl);
        j = min(max(j, 0), n - 2);
        while (j < n - 2 && x[j + 1] <= key) ++j;
        while (j > 0 && x[j] > key) --j;
        if (key > x[n - 1]) clamp = 1u;
        s.j = j;
    }
    s.r = lg2a(key * rx[s.j]);
    return s;
}

// Same, starting the walk from a previous index (keys that move little).
__device__ __forceinline__ Sel select_from(const float* a, int n, int j, float key,
                                           unsigned& clamp) {
    const float* x = a;
    const float* rx = a + n;
    Sel s;
    if (!(key >= x[0])) {
        clamp = 1u;
        j = 0;
    } else {
        while (j < n - 2 && x[j + 1] <= key) ++j;
        while (j > 0 && x[j] > key) --j;
        if (key > x[n - 1]) clamp = 1u;
    }
    s.j = j;
    s.r = lg2a(key * rx[j]);
    return s;
}

// Per-cell, step-invariant part of the 4-D lookup and the cooling constants.
struct CellC {
    const float* lsp;   // &ls[((jh nB + jb) nN + jn) nT]
    int oH, oB, oN;     // strides of the H, B, n_e corners
    float wh, wb, wn;
    float lb_off;       // log2(h n_e^2 / e_scale)
    float ls_off;       // log2(h / e_scale)
    float lbb_off;      // log2(4 sigma_SB h / (H_cm e_scale))
    float tau_sca;      // 2 n_e sigma_T H_cm
    float inv_e;        // s_Te / rho
};

struct Cache {
    int jt;             // T_e interval whose collapsed values are held
    float s0, s1;       // synchrotron channel at T_e nodes jt, jt+1 (collapsed)
    float b0, b1;       // bremsstrahlung channel at jt, jt+1
};

__device__ __forceinline__ float lerpf(float a, float b, float w) { return fmaf(w, b - a, a); }

__device__ __forceinline__ void gather(const CellC& c, const float* lb, int jt, Cache& cc) {
    const float* p = c.lsp + jt;
    float v000 = __ldg(p), v000b = __ldg(p + 1);
    float v001 = __ldg(p + c.oN), v001b = __ldg(p + c.oN + 1);
    float v010 = __ldg(p + c.oB), v010b = __ldg(p + c.oB + 1);
    float v011 = __ldg(p + c.oB + c.oN), v011b = __ldg(p + c.oB + c.oN + 1);
    const float* q = p + c.oH;
    float v100 = __ldg(q), v100b = __ldg(q + 1);
    float v101 = __ldg(q + c.oN), v101b = __ldg(q + c.oN + 1);
    float v110 = __ldg(q + c.oB), v110b = __ldg(q + c.oB + 1);
    float v111 = __ldg(q + c.oB + c.oN), v111b = __ldg(q + c.oB + c.oN + 1);
    float a0 = lerpf(lerpf(v000, v001, c.wn), lerpf(v010, v011, c.wn), c.wb);
    float a1 = lerpf(lerpf(v100, v101, c.wn), lerpf(v110, v111, c.wn), c.wb);
    float b0 = lerpf(lerpf(v000b, v001b, c.wn), lerpf(v010b, v011b, c.wn), c.wb);
    float b1 = lerpf(lerpf(v100b, v101b, c.wn), lerpf(v110b, v111b, c.wn), c.wb);
    cc.s0 = lerpf(a0, a1, c.wh);
    cc.s1 = lerpf(b0, b1, c.wh);
    cc.b0 = lb[jt];
    cc.b1 = lb[jt + 1];
    cc.jt = jt;
}

// Energy (code units) that cooling removes in one sub-cycle at T_e, with
// the bridge of Eq. 11 evaluated in log2 space:
//   A = log2 q_thin, B = log2 q_bb (q_bb = h 4 sigma T^4/(H e_scale)),
//   tau_abs = 2^(A - B), q = q_thin / (1 + tau_abs (sqrt3 + 1.5 (tau_abs + tau_sca))).
__device__ __forceinline__ float cool_energy(const StepK& k, const Smem& S, const CellC& c,
                                             Cache& cc, float Te, bool walk, unsigned& clamp) {
    const int nT = k.tab.n[3];
    const float* axT = S.ax + k.tab.axis_off[3];
    Sel s = walk && cc.jt >= 0 ? select_from(axT, nT, cc.jt, Te, clamp)
                               : select_axis(axT, nT, k.tab.inv_dl[3], Te, clamp);
    if (s.j != cc.jt) gather(c, S.lb, s.j, cc);
    float w = __saturatef(s.r * k.tab.inv_dl[3]);
    float Ls = lerpf(cc.s0, cc.s1, w) + c.ls_off;
    float Lb = lerpf(cc.b0, cc.b1, w) + c.lb_off;
    float lT = axT[2 * nT + s.j] + s.r;
    float M = fmaxf(Ls, Lb), d = fminf(Ls, Lb) - M;
    float A = d > -40.f ? M + lg2a(1.f + ex2a(d)) : M;
    float Bb = fmaf(4.f, lT, c.lbb_off);
    float lt = A - Bb;  // log2 tau_abs
    float lq;
    if (lt < -40.f) {
        lq = A;
    } else if (lt > 40.f) {
        // tau_abs > 2^40: q = q_bb / (1.5 (tau_abs + tau_sca)) to 2^-39
        lq = Bb - 0.5849625f - (lt + lg2a(1.f + c.tau_sca * ex2a(-lt)));
    } else {
        float tau = ex2a(lt);
        float D = fmaf(tau, fmaf(1.5f, tau + c.tau_sca, 1.7320508f), 1.f);
        lq = A - lg2a(D);
    }
    return ex2a(fminf(lq, 126.f));
}

struct Out {
    float ue, ui, qc, qx;
    unsigned flags;  // bit 0 clamped, 1 invalid, 2 stiff, 3 fp64 Coulomb, 4 implicit fail
};

__device__ Out step_cell(const StepK& k, const Smem& S, float rho, float B, float H, float ue,
                         float ui) {
    Out o;
    if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
        !(rho > 0.f) || !(ue > 0.f) || !(ui > 0.f) || B < 0.f || H < 0.f) {
        o.ue = ue; o.ui = ui; o.qc = 0.f; o.qx = 0.f; o.flags = 2u;
        return o;
    }
    unsigned clamp = 0u, stiff = 0u, band = 0u, fail = 0u;
    const DevTable& T = k.tab;
    const float ne = rho * k.s_n;
    const float Bg = B * k.s_B;
    const float Hc = H * k.s_H;
    const float inv_e = k.s_Te / rho;   // IEEE division
    const float inv_i = k.s_Ti / rho;
    const float kr = k.s_K / rho;
    CellC c;
    {
        Sel sh = select_axis(S.ax + T.axis_off[0], T.n[0], T.inv_dl[0], Hc, clamp);
        Sel sb = select_axis(S.ax + T.axis_off[1], T.n[1], T.inv_dl[1], Bg, clamp);
        Sel sn = select_axis(S.ax + T.axis_off[2], T.n[2], T.inv_dl[2], ne, clamp);
        c.oN = T.n[3];
        c.oB = T.n[2] * T.n[3];
        c.oH = T.n[1] * c.oB;
        c.lsp = T.ls + ((long long)(sh.j * T.n[1] + sb.j) * T.n[2] + sn.j) * T.n[3];
        c.wh = __saturatef(sh.r * T.inv_dl[0]);
        c.wb = __saturatef(sb.r * T.inv_dl[1]);
        c.wn = __saturatef(sn.r * T.inv_dl[2]);
        const float lne = lg2a(ne);
        c.ls_off = k.l_hs_e;
        c.lb_off = fmaf(2.f, lne, k.l_hs_e);
        c.lbb_off = k.l_bb - lg2a(Hc);
        c.tau_sca = k.two_sigT * ne * Hc;
        c.inv_e = inv_e;
    }
    const float lcc_off = c.lb_off;  // log2(h n_e^2 / e_scale)
    const int nC = T.n[4];
    const float* axC = S.ax + T.axis_off[4];
    Cache cc;
    cc.jt = -1;
    int jCe = -1, jCi = -1;
    float sum_q = 0.f, sum_x = 0.f;
    for (int sub = 0; sub < k.n_sub; ++sub) {
        // ---- (i) Coulomb exchange --------------------------------------------
        float Te = ue * inv_e;
        float Ti = ui * inv_i;
        Sel se = jCe >= 0 ? select_from(axC, nC, jCe, Te, clamp)
                          : select_axis(axC, nC, T.inv_dl[4], Te, clamp);
        Sel si = jCi >= 0 ? select_from(axC, nC, jCi, Ti, clamp)
                          : select_axis(axC, nC, T.inv_dl[4], Ti, clamp);
        jCe = se.j;
        jCi = si.j;
        float we = __saturatef(se.r * T.inv_dl[4]);
        float wi = __saturatef(si.r * T.inv_dl[4]);
        const float* row = S.lc + si.j * nC + se.j;
        float lC = lerpf(lerpf(row[0], row[1], we), lerpf(row[nC], row[nC + 1], we), wi);
        float rate = ex2a(fminf(lC + lcc_off, 126.f));
        // D = (gamma_i - 1) u_i - (gamma_e - 1) u_e; T_i - T_e = (s_K/rho) D and
        // the equilibrium point is X_eq = D / (ce + ci).  D cancels as T_e -> T_i:
        // it is formed by an error-free transformation of the product ce*u_e
        // (p + e = ce*u_e exactly), so D carries ~1 ulp of its own size.
        const bool in_band = fabsf(Te - Ti) <= k.eq_band * Ti;
        band |= in_band ? 1u : 0u;
        float X;
        if (k.band_fp64 && in_band) {
            // literal FP64 evaluation inside the band
            double D = k.ci64 * (double)ui - k.ce64 * (double)ue;
            double Xd = (double)rate * ((double)kr * D);
            double lim = (double)k.clamp * fabs(D * k.inv_cec64);
            if (fabs(Xd) > lim) Xd = copysign(lim, Xd);
            ue = (float)((double)ue + Xd);
            ui = (float)((double)ui - Xd);
            X = (float)Xd;
        } else {
            float pe = k.ce * ue;
            float ee = fmaf(k.ce, ue, -pe);
            float D = fmaf(k.ci, ui, -pe) - ee;
            X = rate * (kr * D);
            float lim = k.clamp * fabsf(D * k.inv_cec);
            if (fabsf(X) > lim) X = copysignf(lim, X);
            ue += X;
            ui -= X;
        }
        sum_x += X;
        // ---- (ii) radiative cooling ----------------------------------------
        float q = cool_energy(k, S, c, cc, ue * inv_e, true, clamp);
        float du;
        if (k.mode == 1 && q > k.limiter * ue) {
            stiff = 1u;
            const float u0 = ue;
            float b = lg2a(u0);
            float a = b - 60.f;
            float ua = ex2a(a);
            unsigned trial = 0u;  // trial points of the solve do not count as clamped keys
            float ga = ua - u0 + cool_energy(k, S, c, cc, ua * inv_e, false, trial);
            if (!(ga < 0.f)) {
                fail = 1u;
                du = k.limiter * u0;
            } else {
                for (int it = 0; it < k.iters; ++it) {
                    float m = 0.5f * (a + b);
                    if (m == a || m == b) break;
                    float um = ex2a(m);
                    float g = um - u0 + cool_energy(k, S, c, cc, um * inv_e, false, trial);
                    if (g > 0.f) b = m; else a = m;
                }
                du = u0 - ex2a(0.5f * (a + b));
            }
        } else {
            du = fminf(q, k.limiter * ue);
        }
        ue -= du;
        sum_q += du;
    }
    o.ue = ue; o.ui = ui; o.qc = sum_q; o.qx = sum_x;
    o.flags = clamp | (stiff << 2) | (band << 3) | (fail << 4);
    return o;
}

__device__ __forceinline__ void load_smem(const StepK& k, float* sm) {
    const int na = k.axes_floats;
    for (int i = threadIdx.x; i < na; i += blockDim.x) sm[i] = k.tab.axes[i];
    const int nT = k.tab.n[3];
    for (int i = threadIdx.x; i < nT; i += blockDim.x) sm[na + i] = k.tab.lb[i];
    const int nC2 = k.tab.n[4] * k.tab.n[4];
    for (int i = threadIdx.x; i < nC2; i += blockDim.x) sm[na + nT + i] = k.tab.lc[i];
    __syncthreads();
}

__device__ __forceinline__ void count_flags(unsigned f, cool_counters* cnt) {
    // warp-aggregated counter updates
    const unsigned full = __activemask();
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        unsigned m = __ballot_sync(full, (f >> b) & 1u);
        if (m && (threadIdx.x & 31) == (__ffs(full) - 1)) {
            unsigned long long* dst = nullptr;
            switch (b) {
            case 0: dst = &cnt->n_clamped; break;
            case 1: dst = &cnt->n_nonfinite; break;
            case 2: dst = &cnt->n_stiff; break;
            case 3: dst = &cnt->n_fp64_coulomb; break;
            default: dst = &cnt->n_implicit_fail; break;
            }
            atomicAdd(dst, (unsigned long long)__popc(m));
        }
    }
}

constexpr int kThreads = 256;
constexpr int kTile = 4 * kThreads;  // cells per tile: one float4 per thread per field

// VEC: fields are 16-byte aligned.  Each block walks tiles of kTile cells:
// the five input fields are read with 128-bit streaming loads into shared
// memory, each thread then steps cells t, t+256, t+512, t+768 (conflict-free
// shared-memory access, one cell's state in registers at a time), and the
// outputs leave through shared memory with 128-bit streaming stores.  The
// remainder (and unaligned arrays) take a scalar grid-stride loop.
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_step_f32(StepK k, long long n, const float* __restrict__ rho,
                                                      const float* __restrict__ Bf, const float* __restrict__ Hf,
                                                      const float* ue_in, const float* ui_in, float* ue_out,
                                                      float* ui_out, float* qc_out, float* qx_out,
                                                      cool_counters* cnt) {
    extern __shared__ float sm[];
    load_smem(k, sm);
    Smem S;
    S.ax = sm;
    S.lb = sm + k.axes_floats;
    S.lc = sm + k.axes_floats + k.tab.n[3];
    const int t = threadIdx.x;
    long long scalar_start = 0;
    if (VEC) {
        float* tile = sm + ((k.smem_floats + 3) & ~3);   // 16-byte aligned
        float4* t4 = reinterpret_cast<float4*>(tile);    // 7 fields x kThreads float4
        const long long ntiles = n / kTile;
        for (long long tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
            const long long q = tb * kThreads + t;       // float4 index
            t4[0 * kThreads + t] = __ldcs(reinterpret_cast<const float4*>(rho) + q);
            t4[1 * kThreads + t] = __ldcs(reinterpret_cast<const float4*>(Bf) + q);
            t4[2 * kThreads + t] = __ldcs(reinterpret_cast<const float4*>(Hf) + q);
            t4[3 * kThreads + t] = __ldcs(reinterpret_cast<const float4*>(ue_in) + q);
            t4[4 * kThreads + t] = __ldcs(reinterpret_cast<const float4*>(ui_in) + q);
            __syncthreads();
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int j = c * kThreads + t;
                Out o = step_cell(k, S, tile[j], tile[kTile + j], tile[2 * kTile + j], tile[3 * kTile + j],
                                  tile[4 * kTile + j]);
                tile[3 * kTile + j] = o.ue;
                tile[4 * kTile + j] = o.ui;
                tile[5 * kTile + j] = o.qc;
                tile[6 * kTile + j] = o.qx;
                if (cnt) count_flags(o.flags, cnt);
            }
            __syncthreads();
            __stcs(reinterpret_cast<float4*>(ue_out) + q, t4[3 * kThreads + t]);
            __stcs(reinterpret_cast<float4*>(ui_out) + q, t4[4 * kThreads + t]);
            if (qc_out) __stcs(reinterpret_cast<float4*>(qc_out) + q, t4[5 * kThreads + t]);
            if (qx_out) __stcs(reinterpret_cast<float4*>(qx_out) + q, t4[6 * kThreads + t]);
            __syncthreads();
        }
        scalar_start = ntiles * kTile;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = scalar_start + (long long)blockIdx.x * blockDim.x + t; i < n; i += stride) {
        Out o = step_cell(k, S, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i]);
        ue_out[i] = o.ue;
        ui_out[i] = o.ui;
        if (qc_out) qc_out[i] = o.qc;
        if (qx_out) qx_out[i] = o.qx;
        if (cnt) count_flags(o.flags, cnt);
    }
}

// ---------------------------------------------------------------------------
// FP64 instantiation: all arithmetic in FP64 on the FP64 table channels
// (the same algorithm; index selection compares the FP64 key with the FP32
// nodes, weights from FP64 log2).
// ---------------------------------------------------------------------------
struct StepK64 {
    DevTable tab;
    double s_n, s_B, s_H, s_Te, s_Ti, ce, ci, hs, escale;
    double limiter, eq_band, clamp;
    int n_sub, mode, iters;
};

__device__ int select64(const DevTable& T, int a, double key, double& w, unsigned& clamp) {
    const int n = T.n[a];
    const float* x = T.axes + T.axis_off[a];
    int j = 0;
    if (!(key >= (double)x[0])) {
        clamp = 1u;
    } else {
        int lo = 0, hi = n - 2;  // largest j in [0, n-2] with x[j] <= key
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if ((double)x[mid] <= key) lo = mid; else hi = mid - 1;
        }
        j = lo;
        if (key > (double)x[n - 1]) clamp = 1u;
    }
    double wl = key > 0.0 ? (log2(key) - (T.l0_64[a] + j * T.dl64[a])) / T.dl64[a] : 0.0;
    w = fmin(fmax(wl, 0.0), 1.0);
    return j;
}

struct Cell64 {
    int jh, jb, jn;
    double wh, wb, wn, ne, Hc;
};

__device__ double cool_q64(const StepK64& k, const Cell64& c, double ue, double rho, unsigned& clamp) {
    const DevTable& T = k.tab;
    double Te = k.s_Te * ue / rho;
    double wt;
    int jt = select64(T, 3, Te, wt, clamp);
    const int nB = T.n[1], nN = T.n[2], nT = T.n[3];
    double ls = 0.0;
    for (int cidx = 0; cidx < 16; ++cidx) {
        int bh = cidx & 1, bb = (cidx >> 1) & 1, bn = (cidx >> 2) & 1, bt = (cidx >> 3) & 1;
        double wgt = (bh ? c.wh : 1.0 - c.wh) * (bb ? c.wb : 1.0 - c.wb) * (bn ? c.wn : 1.0 - c.wn) *
                     (bt ? wt : 1.0 - wt);
        long long idx = (((long long)(c.jh + bh) * nB + (c.jb + bb)) * nN + (c.jn + bn)) * nT + jt + bt;
        ls += wgt * T.ls64[idx];
    }
    double lb = (1.0 - wt) * T.lb64[jt] + wt * T.lb64[jt + 1];
    double qthin = c.ne * c.ne * exp2(lb) + exp2(ls);
    double bb4 = 4.0 * kSigSB * Te * Te * Te * Te;
    double tau_sca = 2.0 * c.ne * kSigT * c.Hc;
    double tau_abs = c.Hc * qthin / bb4;
    double Q = qthin / (1.0 + tau_abs * (sqrt(3.0) + 1.5 * (tau_abs + tau_sca)));
    return k.hs * Q / k.escale;
}

__global__ void k_step_f64(StepK64 k, long long n, const double* rho, const double* Bf,
                           const double* Hf, const double* ue_in, const double* ui_in, double* ue_out,
                           double* ui_out, double* qc_out, double* qx_out, cool_counters* cnt) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double r = rho[i], B = Bf[i], H = Hf[i], ue = ue_in[i], ui = ui_in[i];
        unsigned clamp = 0u, stiff = 0u, band = 0u, fail = 0u, invalid = 0u;
        double sum_q = 0.0, sum_x = 0.0;
        if (!(isfinite(r) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
            !(r > 0.0) || !(ue > 0.0) || !(ui > 0.0) || B < 0.0 || H < 0.0) {
            invalid = 1u;
        } else {
            const DevTable& T = k.tab;
            Cell64 c;
            c.ne = r * k.s_n;
            c.Hc = H * k.s_H;
            c.jh = select64(T, 0, c.Hc, c.wh, clamp);
            c.jb = select64(T, 1, B * k.s_B, c.wb, clamp);
            c.jn = select64(T, 2, c.ne, c.wn, clamp);
            const int nC = T.n[4];
            for (int sub = 0; sub < k.n_sub; ++sub) {
                double Te = k.s_Te * ue / r, Ti = k.s_Ti * ui / r;
                if (fabs(Te / Ti - 1.0) <= k.eq_band) band = 1u;
                double we, wi;
                int je = select64(T, 4, Te, we, clamp);
                int ji = select64(T, 4, Ti, wi, clamp);
                const double* lc = T.lc64;
                double lC = (1.0 - wi) * (1.0 - we) * lc[ji * nC + je] + (1.0 - wi) * we * lc[ji * nC + je + 1] +
                            wi * (1.0 - we) * lc[(ji + 1) * nC + je] + wi * we * lc[(ji + 1) * nC + je + 1];
                double X = k.hs * c.ne * c.ne * exp2(lC) * (Ti - Te) / k.escale;
                double Xeq = (k.ci * ui - k.ce * ue) / (k.ce + k.ci);
                double lim = k.clamp * fabs(Xeq);
                if (fabs(X) > lim) X = copysign(lim, X);
                ue += X;
                ui -= X;
                sum_x += X;
                double q = cool_q64(k, c, ue, r, clamp);
                double du;
                if (k.mode == 1 && q > k.limiter * ue) {
                    stiff = 1u;
                    double a = log2(ue) - 60.0, b = log2(ue);
                    unsigned dummy = 0u;
                    double ga = exp2(a) - ue + cool_q64(k, c, exp2(a), r, dummy);
                    if (!(ga < 0.0)) {
                        fail = 1u;
                        du = k.limiter * ue;
                    } else {
                        for (int it = 0; it < k.iters; ++it) {
                            double m = 0.5 * (a + b);
                            double um = exp2(m);
                            if (um - ue + cool_q64(k, c, um, r, dummy) > 0.0) b = m; else a = m;
                        }
                        du = ue - exp2(0.5 * (a + b));
                    }
                } else {
                    du = q < k.limiter * ue ? q : k.limiter * ue;
                }
                ue -= du;
                sum_q += du;
            }
        }
        ue_out[i] = ue;
        ui_out[i] = ui;
        if (qc_out) qc_out[i] = sum_q;
        if (qx_out) qx_out[i] = sum_x;
        if (cnt) count_flags(clamp | (invalid << 1) | (stiff << 2) | (band << 3) | (fail << 4), cnt);
    }
}

__global__ void k_debug_lookup(DevTable T, int axis, long long n, const float* keys, int* idx, float* w) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned clamp = 0u;
        Sel s = select_axis(T.axes + T.axis_off[axis], T.n[axis], T.inv_dl[axis], keys[i], clamp);
        idx[i] = s.j;
        w[i] = __saturatef(s.r * T.inv_dl[axis]);
    }
}

void fill_common(const cool_table* t, const cool_params* p, double& rg, double& hs, double& escale) {
    rg = (kG * (p->M_bh_msun * kMsun)) / (kC * kC);
    double tg = rg / kC;
    hs = p->dt * tg / p->n_sub;
    escale = p->rho_scale * kC * kC;
    (void)t;
}

int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

cool_status launch_step_f32(const cool_table* t, const cool_params* p, long long n,
                            const float* rho, const float* B, const float* H,
                            const float* ue, const float* ui, float* ue_o, float* ui_o,
                            float* qc, float* qx, cool_counters* cnt, cudaStream_t st) {
    StepK k;
    k.tab = t->dev;
    double rg, hs, escale;
    fill_common(t, p, rg, hs, escale);
    k.s_n = (float)(p->rho_scale / kMP);
    k.s_B = (float)(sqrt(4.0 * kPi * p->rho_scale) * kC);
    k.s_H = (float)rg;
    k.s_Te = (float)((p->gamma_e - 1.0) * kMP * kC * kC / kKB);
    k.s_Ti = (float)((p->gamma_i - 1.0) * kMP * kC * kC / kKB);
    k.ce64 = p->gamma_e - 1.0;
    k.ci64 = p->gamma_i - 1.0;
    k.inv_cec64 = 1.0 / (k.ce64 + k.ci64);
    k.ce = (float)k.ce64;
    k.ci = (float)k.ci64;
    k.inv_cec = (float)k.inv_cec64;
    k.s_K = (float)(kMP * kC * kC / kKB);
    k.band_fp64 = p->band_fp64;
    k.l_hs_e = (float)log2(hs / escale);
    k.l_bb = (float)log2(4.0 * kSigSB * hs / escale);
    k.two_sigT = (float)(2.0 * kSigT);
    k.limiter = (float)p->limiter_frac;
    k.eq_band = (float)p->eq_band;
    k.clamp = (float)p->coulomb_clamp;
    k.n_sub = p->n_sub;
    k.mode = (int)p->mode;
    k.iters = p->implicit_iters;
    int na = 0;
    for (int a = 0; a < 5; ++a) na += 3 * t->dev.n[a];
    k.axes_floats = na;
    k.smem_floats = na + t->dev.n[3] + t->dev.n[4] * t->dev.n[4];
    if (n == 0) return COOL_OK;
    bool vec = ((uintptr_t)rho | (uintptr_t)B | (uintptr_t)H | (uintptr_t)ue | (uintptr_t)ui |
                (uintptr_t)ue_o | (uintptr_t)ui_o | (uintptr_t)qc | (uintptr_t)qx) % 16 == 0;
    size_t smem = (size_t)((k.smem_floats + 3) & ~3) * sizeof(float);
    if (vec) smem += (size_t)7 * kTile * sizeof(float);
    auto fn = vec ? k_step_f32<true> : k_step_f32<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (per_sm < 1) per_sm = 1;
    long long work = vec ? (n + kTile - 1) / kTile : (n + kThreads - 1) / kThreads;
    long long cap = (long long)sm_count() * per_sm;  // one resident wave, persistent blocks
    long long blocks = work < cap ? work : cap;
    if (blocks < 1) blocks = 1;
    fn<<<(int)blocks, kThreads, smem, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

cool_status launch_step_f64(const cool_table* t, const cool_params* p, long long n,
                            const double* rho, const double* B, const double* H,
                            const double* ue, const double* ui, double* ue_o, double* ui_o,
                            double* qc, double* qx, cool_counters* cnt, cudaStream_t st) {
    StepK64 k;
    k.tab = t->dev;
    double rg, hs, escale;
    fill_common(t, p, rg, hs, escale);
    k.s_n = p->rho_scale / kMP;
    k.s_B = sqrt(4.0 * kPi * p->rho_scale) * kC;
    k.s_H = rg;
    k.ce = p->gamma_e - 1.0;
    k.ci = p->gamma_i - 1.0;
    k.s_Te = k.ce * kMP * kC * kC / kKB;
    k.s_Ti = k.ci * kMP * kC * kC / kKB;
    k.hs = hs;
    k.escale = escale;
    k.limiter = p->limiter_frac;
    k.eq_band = p->eq_band;
    k.clamp = p->coulomb_clamp;
    k.n_sub = p->n_sub;
    k.mode = (int)p->mode;
    k.iters = p->implicit_iters;
    if (n == 0) return COOL_OK;
    long long blocks = (n + 127) / 128;
    long long cap = (long long)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    k_step_f64<<<(int)blocks, 128, 0, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

cool_status launch_debug_lookup(const cool_table* t, int axis, long long n, const float* keys,
                                int* idx, float* w, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_debug_lookup<<<(int)blocks, 256, 0, st>>>(t->dev, axis, n, keys, idx, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

}  // namespace cool
