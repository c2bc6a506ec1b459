// cool_step_cell.cuh -- the per-cell step of the FP32 kernels (the Coulomb
// exchange, the cooling with the bridge, the limiter or the implicit
// solve, the disk geometry), the shared-memory loader and the counter
// aggregation, used by the forward kernels (cool_step.cu, the TMA-staged
// cool_step_tma.cu) and the adjoint (cool_step_bwd.cu).
#pragma once

#include "cool_step_common.cuh"

namespace cool {
namespace {
struct Out {
    float ue, ui, qc, qx;
    unsigned flags;  // bit 0 clamped, 1 invalid, 2 stiff, 3 equilibrium band, 4 implicit fail, 6 floored
    unsigned near;   // a key fell near a node: redo the cell with EXACT
};

// VAR: bit 5 = the flagging pass of an fp64_critical kernel (a stiff cell
// is flagged and takes the limited step: its result is discarded),
// bit 0 = implicit mode compiled in, bit 1 = fp64_critical compiled in,
// bit 2 = disk geometry (radius r per cell: H_th from the state and the
// temperature floor; Sec. 2.7, Sec. 3.2.3), bit 4 = the paper's table layout
// (COOL_PATH_QTOTAL: explicit, FP32 table, no geometry).  The explicit FP32 kernel carries
// no solver code, no FP64 code and no geometry.  EXACT: every index by the
// exact rule (select_sub<A, true>: node compares where the lg2 guess is in
// doubt); otherwise o.near asks for that when some key fell near a node.
template <int FMT, int VAR, bool EXACT>
__device__ __forceinline__ Out step_cell(const StepK& k, const Smem& S, float* win, float rho, float B,
                                         float H, float ue, float ui, float r) {
    Out o;
    o.near = 0u;
    float t_floor = -1.f;   // gas temperature P/rho below which a sub-cycle does not cool
    if (VAR & 4) {
        if (k.h_from_state && isfinite(r) && r > 0.f && rho > 0.f && ue > 0.f && ui > 0.f) {
            // H_th = c_s / Omega_K, c_s^2 = gamma P / (rho + u + P), gamma = 1 + P/u,
            // Omega_K = 1 / (r^1.5 + a)
            const float P = fmaf(k.ce, ue, k.ci * ui);
            const float u = ue + ui;
            const float cs2 = (1.f + P / u) * P / (rho + u + P);
            H = sqrtf(cs2) * fmaf(r, sqrtf(r), k.spin);
        }
        if (k.h_floor > 0.f) {
            const float v = k.h_floor * r / fmaf(r, sqrtf(r), k.spin);
            t_floor = 1.5707963f * v * v;
        }
    }
    if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
        !(rho > 0.f) || !(ue > 0.f) || !(ui > 0.f) || B < 0.f || H < 0.f ||
        ((VAR & 4) && !(isfinite(r) && r > 0.f))) {
        o.ue = ue; o.ui = ui; o.qc = 0.f; o.qx = 0.f; o.flags = 2u;
        return o;
    }
    unsigned clamp = 0u, stiff = 0u, band = 0u, fail = 0u, floored = 0u;
    const DevTable& T = k.tab;
    Cache cc;
    cc.base = -8;
    cc.win = win;
    cc.near = 0u;
    const float ne = rho * k.s_n;
    const float Bg = B * k.s_B;
    const float Hc = H * k.s_H;
    const float inv_e = k.s_Te / rho;   // IEEE division (the key sequence of the interface)
    const float inv_i = k.s_Ti / rho;
    const float kr = k.s_K / rho;
    CellC c;
    {
        const SelW sh = select_sub<0, EXACT>(k, S.ax + T.axis_off[0] + T.n[0], T.n[0], T.inv_dl[0], Hc, clamp,
                                             cc.near);
        const SelW sb = select_sub<1, EXACT>(k, S.ax + T.axis_off[1] + T.n[1], T.n[1], T.inv_dl[1], Bg, clamp,
                                             cc.near);
        const SelW sn = select_sub<2, EXACT>(k, S.ax + T.axis_off[2] + T.n[2], T.n[2], T.inv_dl[2], ne, clamp,
                                             cc.near);
        const int rowf = 8 * T.nblk;                       // floats per n_e row
        c.oN = rowf;
        c.oB = rowf * T.n[2];
        c.oH = c.oB * T.n[1];
        c.row = ((VAR & 16) ? T.lst : T.lsb) + (long long)((sh.j * T.n[1] + sb.j) * T.n[2] + sn.j) * rowf;
        c.wh = sh.w;
        c.wb = sb.w;
        c.wn = sn.w;
        const float lne = lg2a(ne);
        c.ls_off = k.l_hs_e;
        c.lb_off = fmaf(2.f, lne, k.l_hs_e);
        c.lbb_off = k.l_bb - lg2a(Hc);
        c.tau_sca = k.two_sigT * ne * Hc;
    }
    const float lcc_off = c.lb_off;  // log2(h n_e^2 / e_scale)
    Cell64 c64;                      // fp64_critical implicit: the cell's FP64 selections, made when first stiff
    c64.jt = -2;
    const int nC = T.n[4];
    const float* axC = S.ax + T.axis_off[4];
    float sum_q = 0.f, sum_x = 0.f;
    for (int sub = 0; sub < k.n_sub; ++sub) {
        // ---- (i) Coulomb exchange --------------------------------------------
        const float Te = ue * inv_e;
        const float Ti = ui * inv_i;
        const SelW se = select_sub<4, EXACT>(k, axC + nC, nC, T.inv_dl[4], Te, clamp, cc.near);
        const SelW si = select_sub<4, EXACT>(k, axC + nC, nC, T.inv_dl[4], Ti, clamp, cc.near);
        const float we = se.w;
        const float wi = si.w;
        const int ls = k.lc_stride;
        const float* row = S.lc + si.j * ls + se.j;
        const float lC = lerpf(lerpf(row[0], row[1], we), lerpf(row[ls], row[ls + 1], we), wi);
        const float rate = ex2a(fminf(lC + lcc_off, 126.f));
        // D = (gamma_i - 1) u_i - (gamma_e - 1) u_e; T_i - T_e = (s_K/rho) D and
        // the equilibrium point is X_eq = D / (ce + ci).  D cancels as T_e -> T_i:
        // it is formed by an error-free transformation of the product ce*u_e
        // (p + e = ce*u_e exactly), so D carries ~1 ulp of its own size.
        const bool in_band = fabsf(Te - Ti) <= k.eq_band * Ti;
        band |= in_band ? 1u : 0u;
        float X;
        if ((VAR & 2) && in_band) {
            // literal FP64 evaluation inside the band
            double D = k.ci64 * (double)ui - k.ce64 * (double)ue;
            double Xd = (double)rate * ((double)kr * D);
            double lim = (double)k.clamp * fabs(D * k.inv_cec64);
            if (fabs(Xd) > lim) Xd = copysign(lim, Xd);
            ue = (float)((double)ue + Xd);
            ui = (float)((double)ui - Xd);
            X = (float)Xd;
        } else {
            const float pe = k.ce * ue;
            const float ee = fmaf(k.ce, ue, -pe);
            const float D = fmaf(k.ci, ui, -pe) - ee;
            X = rate * (kr * D);
            const float lim = k.clamp * fabsf(D * k.inv_cec);
            X = fabsf(X) > lim ? copysignf(lim, X) : X;
            ue += X;
            ui -= X;
        }
        sum_x += X;
        // ---- temperature floor: no cooling below T_floor -----------------------
        if ((VAR & 4) && fmaf(k.ce, ue, k.ci * ui) < t_floor * rho) {
            floored = 1u;
            continue;
        }
        // ---- (ii) radiative cooling ----------------------------------------
        const float q = (VAR & 16) ? cool_energy_total<EXACT>(k, S, c, cc, ue * inv_e, clamp)
                                   : cool_energy<FMT, EXACT>(k, S, c, cc, ue * inv_e, clamp);
        float du = fminf(q, k.limiter * ue);
        if ((VAR & 1) && q > k.limiter * ue) {
            stiff = 1u;
            if (!(VAR & 32)) {   // bit 5: flagged only, the cell is stepped again with the solve
                float u1;
                bool ok;
                if (VAR & 2) {
                    // the FP32 root, refined in FP64 (Newton from it, else a
                    // bracketed solve around it or over the whole bracket)
                    float u32 = 0.f;
                    if (!implicit_fp32<FMT, EXACT>(k, S, c, cc, inv_e, ue, q, u32)) u32 = 0.f;
                    ok = implicit_fp64_cell(k, T, rho, B, H, ue, u1, u32, c64);
                } else {
                    ok = implicit_fp32<FMT, EXACT>(k, S, c, cc, inv_e, ue, q, u1);
                }
                if (ok) du = ue - u1;
                else fail = 1u;
            }
        }
        ue -= du;
        sum_q += du;
    }
    o.ue = ue; o.ui = ui; o.qc = sum_q; o.qx = sum_x;
    o.flags = clamp | (stiff << 2) | (band << 3) | (fail << 4) | (floored << 6);
    o.near = EXACT ? 0u : cc.near;
    return o;
}

__device__ __forceinline__ void load_smem(const StepK& k, float* sm) {
    const int na = k.axes_floats;
    for (int i = threadIdx.x; i < na; i += blockDim.x) sm[i] = k.tab.axes[i];
    const int nT = k.tab.n[3];
    for (int i = threadIdx.x; i < nT; i += blockDim.x) sm[na + i] = k.tab.lb[i];
    const int nC = k.tab.n[4];
    for (int i = threadIdx.x; i < nC * nC; i += blockDim.x) {
        const int r = i / nC;
        sm[na + nT + r * k.lc_stride + (i - r * nC)] = k.tab.lc[i];
    }
    // the T_e interval records read by cool_energy
    const float* axT = k.tab.axes + k.tab.axis_off[3];
    float4* tn = reinterpret_cast<float4*>(sm + k.tn_off);
    for (int j = threadIdx.x; j < nT - 1; j += blockDim.x)
        tn[j] = make_float4(axT[nT + j], axT[2 * nT + j], k.tab.lb[j], k.tab.lb[j + 1]);
    __syncthreads();
}

__device__ __forceinline__ Smem smem_view(const StepK& k, const float* sm) {
    Smem S;
    S.ax = sm;
    S.lb = sm + k.axes_floats;
    S.lc = sm + k.axes_floats + k.tab.n[3];
    S.tn = reinterpret_cast<const float4*>(sm + k.tn_off);
    return S;
}

// count_flags bit 7: the cell was stepped again with the exact index rule
constexpr unsigned kFlagRedo = 1u << 7;

__device__ __forceinline__ void count_flags(unsigned f, cool_counters* cnt) {
    // warp-aggregated counter updates
    const unsigned full = __activemask();
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b == 5) continue;   // surrogate fallback: not set by this kernel
        unsigned m = __ballot_sync(full, (f >> b) & 1u);
        if (m && (threadIdx.x & 31) == (__ffs(full) - 1)) {
            unsigned long long* dst = nullptr;
            switch (b) {
            case 0: dst = &cnt->n_clamped; break;
            case 1: dst = &cnt->n_nonfinite; break;
            case 2: dst = &cnt->n_stiff; break;
            case 3: dst = &cnt->n_fp64_coulomb; break;
            case 4: dst = &cnt->n_implicit_fail; break;
            case 6: dst = &cnt->n_floor; break;
            default: dst = &cnt->n_exact_redo; break;
            }
            atomicAdd(dst, (unsigned long long)__popc(m));
        }
    }
}

constexpr int kWarpCells = 128;          // cells per warp tile: one float4 per lane per field
constexpr int kWarps = kThreads / 32;

// Shared memory of one block: the small table parts (axes, brems, Coulomb),
// then the per-thread synchrotron windows (8 x kThreads floats), then, for
// the vector path, one staging tile of 5 x kWarpCells floats per warp.
__host__ __device__ __forceinline__ int smem_table_floats(const StepK& k) { return (k.smem_floats + 3) & ~3; }

#ifndef COOL_MINB
#define COOL_MINB 3
#endif

}  // namespace
}  // namespace cool
