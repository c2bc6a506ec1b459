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
#include "cool_step_common.cuh"
#include "cool_tma.cuh"

namespace cool {
namespace {
struct Out {
    float ue, ui, qc, qx;
    unsigned flags;  // bit 0 clamped, 1 invalid, 2 stiff, 3 equilibrium band, 4 implicit fail, 6 floored
};

// VAR: bit 0 = implicit mode compiled in, bit 1 = fp64_critical compiled in,
// bit 2 = disk geometry (radius r per cell: H_th from the state and the
// temperature floor; Sec. 2.7, Sec. 3.2.3).  The explicit FP32 kernel carries
// no solver code, no FP64 code and no geometry.
template <int FMT, int VAR>
__device__ __forceinline__ Out step_cell(const StepK& k, const Smem& S, float* win, float rho, float B,
                                         float H, float ue, float ui, float r) {
    Out o;
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
    const float ne = rho * k.s_n;
    const float Bg = B * k.s_B;
    const float Hc = H * k.s_H;
    const float inv_e = k.s_Te / rho;   // IEEE division (the key sequence of the interface)
    const float inv_i = k.s_Ti / rho;
    const float kr = k.s_K / rho;
    CellC c;
    {
        Sel sh = select_axis(S.ax + T.axis_off[0], T.n[0], T.inv_dl[0], Hc, clamp);
        Sel sb = select_axis(S.ax + T.axis_off[1], T.n[1], T.inv_dl[1], Bg, clamp);
        Sel sn = select_axis(S.ax + T.axis_off[2], T.n[2], T.inv_dl[2], ne, clamp);
        const int rowf = 8 * T.nblk;                       // floats per n_e row
        c.oN = rowf;
        c.oB = rowf * T.n[2];
        c.oH = c.oB * T.n[1];
        c.row = T.lsb + (long long)((sh.j * T.n[1] + sb.j) * T.n[2] + sn.j) * rowf;
        c.wh = __saturatef(sh.r * T.inv_dl[0]);
        c.wb = __saturatef(sb.r * T.inv_dl[1]);
        c.wn = __saturatef(sn.r * T.inv_dl[2]);
        const float lne = lg2a(ne);
        c.ls_off = k.l_hs_e;
        c.lb_off = fmaf(2.f, lne, k.l_hs_e);
        c.lbb_off = k.l_bb - lg2a(Hc);
        c.tau_sca = k.two_sigT * ne * Hc;
    }
    const float lcc_off = c.lb_off;  // log2(h n_e^2 / e_scale)
    const int nC = T.n[4];
    const float* axC = S.ax + T.axis_off[4];
    Cache cc;
    cc.base = -8;
    cc.win = win;
    float sum_q = 0.f, sum_x = 0.f;
    for (int sub = 0; sub < k.n_sub; ++sub) {
        // ---- (i) Coulomb exchange --------------------------------------------
        const float Te = ue * inv_e;
        const float Ti = ui * inv_i;
        const Sel se = select_axis(axC, nC, T.inv_dl[4], Te, clamp);
        const Sel si = select_axis(axC, nC, T.inv_dl[4], Ti, clamp);
        const float we = __saturatef(se.r * T.inv_dl[4]);
        const float wi = __saturatef(si.r * T.inv_dl[4]);
        const float* row = S.lc + si.j * nC + se.j;
        const float lC = lerpf(lerpf(row[0], row[1], we), lerpf(row[nC], row[nC + 1], we), wi);
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
        const float q = cool_energy<FMT>(k, S, c, cc, ue * inv_e, clamp);
        float du = fminf(q, k.limiter * ue);
        if ((VAR & 1) && q > k.limiter * ue) {
            stiff = 1u;
            float u1;
            const bool ok = (VAR & 2) ? implicit_fp64_cell(k, T, rho, B, H, ue, u1)
                                      : implicit_fp32<FMT>(k, S, c, cc, inv_e, ue, q, u1);
            if (ok) du = ue - u1;
            else fail = 1u;
        }
        ue -= du;
        sum_q += du;
    }
    o.ue = ue; o.ui = ui; o.qc = sum_q; o.qx = sum_x;
    o.flags = clamp | (stiff << 2) | (band << 3) | (fail << 4) | (floored << 6);
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
    for (int b = 0; b < 7; ++b) {
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
            default: dst = &cnt->n_floor; break;
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

// VEC: all arrays 16-byte aligned.  Each warp walks its own tiles of 128
// cells: the five input fields arrive by 128-bit streaming loads into the
// warp's staging area, each lane steps cells lane, lane+32, lane+64, lane+96
// (one cell's state in registers at a time), the outputs overwrite the
// staging area and leave by 128-bit streaming stores.  Warps synchronise
// only with themselves (__syncwarp), so a slow cell delays one warp, not the
// block.  The remainder (and unaligned arrays) take a scalar loop.
template <bool VEC, int FMT, int VAR>
#ifndef COOL_MINB
#define COOL_MINB 3
#endif
__global__ void __launch_bounds__(kThreads, COOL_MINB) k_step_f32(StepK k, long long n, const float* __restrict__ rho,
                                                         const float* __restrict__ Bf, const float* __restrict__ Hf,
                                                         const float* ue_in, const float* ui_in, float* ue_out,
                                                         float* ui_out, float* qc_out, float* qx_out,
                                                         cool_counters* cnt, const float* __restrict__ rr) {
    constexpr int NF = (VAR & 4) ? 6 : 5;   // staged input fields
    extern __shared__ float sm[];
    load_smem(k, sm);
    Smem S;
    S.ax = sm;
    S.lb = sm + k.axes_floats;
    S.lc = sm + k.axes_floats + k.tab.n[3];
    float* win = sm + smem_table_floats(k) + threadIdx.x;   // kMaxW x kThreads window
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    long long scalar_start = 0;
    if (VEC) {
        float* tile = sm + smem_table_floats(k) + kMaxW * kThreads + warp * NF * kWarpCells;
        float4* t4 = reinterpret_cast<float4*>(tile);
        const long long ntiles = n / kWarpCells;
        for (long long tw = (long long)blockIdx.x * kWarps + warp; tw < ntiles; tw += (long long)gridDim.x * kWarps) {
            const long long q = tw * 32 + lane;  // float4 index of this lane
            t4[0 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(rho) + q);
            t4[1 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(Bf) + q);
            t4[2 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(Hf) + q);
            t4[3 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(ue_in) + q);
            t4[4 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(ui_in) + q);
            if (VAR & 4) t4[5 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(rr) + q);
            __syncwarp();
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int j = c * 32 + lane;
                Out o = step_cell<FMT, VAR>(k, S, win, tile[j], tile[kWarpCells + j], tile[2 * kWarpCells + j],
                                            tile[3 * kWarpCells + j], tile[4 * kWarpCells + j],
                                            (VAR & 4) ? tile[5 * kWarpCells + j] : 0.f);
                // inputs of cell j are consumed: outputs reuse its slots
                tile[3 * kWarpCells + j] = o.ue;
                tile[4 * kWarpCells + j] = o.ui;
                tile[0 * kWarpCells + j] = o.qc;
                tile[1 * kWarpCells + j] = o.qx;
                if (cnt) count_flags(o.flags, cnt);
            }
            __syncwarp();
            __stcs(reinterpret_cast<float4*>(ue_out) + q, t4[3 * 32 + lane]);
            __stcs(reinterpret_cast<float4*>(ui_out) + q, t4[4 * 32 + lane]);
            if (qc_out) __stcs(reinterpret_cast<float4*>(qc_out) + q, t4[0 * 32 + lane]);
            if (qx_out) __stcs(reinterpret_cast<float4*>(qx_out) + q, t4[1 * 32 + lane]);
            __syncwarp();
        }
        scalar_start = ntiles * kWarpCells;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = scalar_start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Out o = step_cell<FMT, VAR>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], (VAR & 4) ? rr[i] : 0.f);
        ue_out[i] = o.ue;
        ui_out[i] = o.ui;
        if (qc_out) qc_out[i] = o.qc;
        if (qx_out) qx_out[i] = o.qx;
        if (cnt) count_flags(o.flags, cnt);
    }
}

// COOL_PATH_TMA_SMEM: the vector kernel with its field staging done by the
// TMA engine.  Each warp owns two staging buffers (5 fields x 128 cells) and
// two mbarriers; while the warp steps tile i from one buffer, lane 0 has the
// bulk copies of tile i + 1 (five 512-byte copies) landing in the other, so
// the fields of the next tile need no load instructions and no wait at the
// start of the tile.  Outputs overwrite the inputs of their cell in the
// buffer and leave by 128-bit streaming stores, as in k_step_f32.  The
// window holds only the W nodes of the table format's block.  Waits are
// bounded: a copy that does not complete sets *err bit 0 (the tile's
// outputs are then not written).
__device__ unsigned g_tma_err;

template <int FMT, int VAR>
__global__ void __launch_bounds__(kThreads, COOL_MINB) k_step_tma(StepK k, long long n, const float* __restrict__ rho,
                                                         const float* __restrict__ Bf, const float* __restrict__ Hf,
                                                         const float* ue_in, const float* ui_in, float* ue_out,
                                                         float* ui_out, float* qc_out, float* qx_out,
                                                         cool_counters* cnt) {
    constexpr int W = Fmt<FMT>::W;
    constexpr int TILE = 5 * kWarpCells;     // floats per buffer
    extern __shared__ __align__(16) float smt[];
    load_smem(k, smt);
    Smem S;
    S.ax = smt;
    S.lb = smt + k.axes_floats;
    S.lc = smt + k.axes_floats + k.tab.n[3];
    float* win = smt + smem_table_floats(k) + threadIdx.x;   // W x kThreads window
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* bufs = smt + smem_table_floats(k) + W * kThreads + warp * 2 * TILE;
    uint64_t* mb = reinterpret_cast<uint64_t*>(smt + smem_table_floats(k) + W * kThreads + kWarps * 2 * TILE) +
                   warp * 2;
    const uint32_t mbar[2] = {mma::smem_addr(mb), mma::smem_addr(mb + 1)};
    if (lane == 0) {
        mma::mbar_init(mbar[0], 1);
        mma::mbar_init(mbar[1], 1);
        mma::fence_mbar_init();
    }
    __syncwarp();
    const float* src[5] = {rho, Bf, Hf, ue_in, ui_in};
    const long long ntiles = n / kWarpCells;
    const long long step = (long long)gridDim.x * kWarps;
    auto issue = [&](long long tw, int b) {   // lane 0
        tma::arrive_expect_tx(mbar[b], 5 * kWarpCells * sizeof(float));
#pragma unroll
        for (int f = 0; f < 5; ++f)
            tma::bulk_g2s(mma::smem_addr(bufs + b * TILE + f * kWarpCells), src[f] + tw * kWarpCells,
                          kWarpCells * sizeof(float), mbar[b]);
    };
    long long tw = (long long)blockIdx.x * kWarps + warp;
    if (lane == 0 && tw < ntiles) issue(tw, 0);
    uint32_t phase[2] = {0u, 0u};
    int b = 0;
    for (; tw < ntiles; tw += step) {
        const long long nx = tw + step;
        if (lane == 0 && nx < ntiles) {
            mma::fence_async_smem();   // the other buffer's generic reads and writes are done (warp-synchronised)
            issue(nx, b ^ 1);
        }
        const bool ok = mma::mbar_wait(mbar[b], phase[b], 1 << 22);
        phase[b] ^= 1u;
        if (!ok) {
            if (lane == 0) atomicOr(&g_tma_err, 1u);
            mma::mbar_wait(mbar[b], phase[b] ^ 1u, 1 << 16);
        }
        float* tile = bufs + b * TILE;
        float4* t4 = reinterpret_cast<float4*>(tile);
        const long long q = tw * 32 + lane;
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int j = c * 32 + lane;
                Out o = step_cell<FMT, VAR>(k, S, win, tile[j], tile[kWarpCells + j], tile[2 * kWarpCells + j],
                                            tile[3 * kWarpCells + j], tile[4 * kWarpCells + j], 0.f);
                tile[3 * kWarpCells + j] = o.ue;
                tile[4 * kWarpCells + j] = o.ui;
                tile[0 * kWarpCells + j] = o.qc;
                tile[1 * kWarpCells + j] = o.qx;
                if (cnt) count_flags(o.flags, cnt);
            }
            __syncwarp();
            __stcs(reinterpret_cast<float4*>(ue_out) + q, t4[3 * 32 + lane]);
            __stcs(reinterpret_cast<float4*>(ui_out) + q, t4[4 * 32 + lane]);
            if (qc_out) __stcs(reinterpret_cast<float4*>(qc_out) + q, t4[0 * 32 + lane]);
            if (qx_out) __stcs(reinterpret_cast<float4*>(qx_out) + q, t4[1 * 32 + lane]);
        }
        __syncwarp();
        b ^= 1;
    }
    const long long scalar_start = ntiles * kWarpCells;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = scalar_start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Out o = step_cell<FMT, VAR>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], 0.f);
        ue_out[i] = o.ue;
        ui_out[i] = o.ui;
        if (qc_out) qc_out[i] = o.qc;
        if (qx_out) qx_out[i] = o.qx;
        if (cnt) count_flags(o.flags, cnt);
    }
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


// ---------------------------------------------------------------------------
// Adjoint (cool_step_bwd).  Per cell: the forward sub-cycles are recomputed
// with the forward kernel's own functions (same trajectory, same branches),
// keeping each sub-cycle's state; then a reverse sweep applies, per
// sub-cycle, the hand-derived partial derivatives of the cooling energy q
// and of the Coulomb transfer X (below), the limiter's branch, and for an
// implicit sub-cycle the implicit-function theorem at the root
// (du*/du1 = 1/(1 + dq/du), du*/dtheta = -dq/dtheta / (1 + dq/du)).
// Table adjoints go to the natural layouts: synchrotron [nH nB nN nT] with
// global atomics, brems and Coulomb through shared-memory partial sums.
// ---------------------------------------------------------------------------
constexpr int kMaxSub = 64;
constexpr float kLn2 = 0.69314718056f;

// Cooling energy q(u) and d ln q / d ln x for x = u, rho, B, H, plus
// dq/dLs and dq/dLb for the table scatter (FP32 octet layout).
struct QGrad {
    float q, du, drho, dB, dH;   // d ln q / d ln x
    float Gs, Gb;                // dq/dLs, dq/dLb
    int jt;
    float wt;
    float S0, S1;
};

struct CellD {                   // per-cell derivative constants
    float cH, cB, cN;            // d w_{h,b,n} / d ln(H, B, rho) (0 where clamped)
};

// The 4-D channel collapsed over (H, B, n_e) at the two T_e nodes of
// interval j, with its derivatives along H, B and n_e: kept while the
// cell's reverse sweep stays in that interval (the common case), so the 16
// corner values are read once per visited interval instead of once per
// sub-cycle.
struct GCache {
    int j;                       // interval held, -1 if none
    float Sv[2], dSh[2], dSb[2], dSn[2];
};

__device__ __forceinline__ void grad_corners(const CellC& c, int j, GCache& gc) {
    const float* p = reinterpret_cast<const float*>(c.row) + (j / 7) * 8 + (j % 7);
    const float* q1 = p + c.oH;
    const float* base[8] = {p, p + c.oN, p + c.oB, p + c.oB + c.oN, q1, q1 + c.oN, q1 + c.oB, q1 + c.oB + c.oN};
    float v[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i][0] = __ldg(base[i]);
        v[i][1] = __ldg(base[i] + 1);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        // corner order: (h, b, n) = 000, 001, 010, 011, 100, 101, 110, 111
        const float q00 = lerpf(v[0][t], v[1][t], c.wn), q01 = lerpf(v[2][t], v[3][t], c.wn);
        const float q10 = lerpf(v[4][t], v[5][t], c.wn), q11 = lerpf(v[6][t], v[7][t], c.wn);
        const float P0 = lerpf(q00, q01, c.wb), P1 = lerpf(q10, q11, c.wb);
        gc.Sv[t] = lerpf(P0, P1, c.wh);
        gc.dSh[t] = P1 - P0;
        gc.dSb[t] = lerpf(q01 - q00, q11 - q10, c.wh);
        const float n00 = v[1][t] - v[0][t], n01 = v[3][t] - v[2][t], n10 = v[5][t] - v[4][t], n11 = v[7][t] - v[6][t];
        gc.dSn[t] = lerpf(lerpf(n00, n01, c.wb), lerpf(n10, n11, c.wb), c.wh);
    }
    gc.j = j;
}

__device__ __forceinline__ QGrad cool_grad(const StepK& k, const Smem& S, const CellC& c, const CellD& cd,
                                           GCache& gc, float u, float inv_e) {
    QGrad g;
    const DevTable& T = k.tab;
    const int nT = T.n[3];
    const float* axT = S.ax + T.axis_off[3];
    unsigned dummy = 0u;
    const float Te = u * inv_e;
    const Sel s = select_axis(axT, nT, T.inv_dl[3], Te, dummy);
    const int j = s.j;
    const float wraw = s.r * T.inv_dl[3];
    const float wt = __saturatef(wraw);
    const float cT = (wraw > 0.f && wraw < 1.f) ? T.inv_dl[3] / kLn2 : 0.f;   // dwt / d ln Te
    // corner values at nodes j, j+1 (octet layout: block j/7, offset j%7)
    if (gc.j != j) grad_corners(c, j, gc);
    const float* Sv = gc.Sv;
    const float* dSh = gc.dSh;
    const float* dSb = gc.dSb;
    const float* dSn = gc.dSn;
    const float b0 = S.lb[j], b1 = S.lb[j + 1];
    const float Ls = lerpf(Sv[0], Sv[1], wt) + c.ls_off;
    const float Lb = lerpf(b0, b1, wt) + c.lb_off;
    const float lT = axT[2 * nT + j] + s.r;
    const float M = fmaxf(Ls, Lb);
    const float A = M + lg2a(1.f + ex2a(fminf(Ls, Lb) - M));
    const float sig_s = ex2a(Ls - A);
    const float Bb = fmaf(4.f, lT, c.lbb_off);
    const float lt = A - Bb;
    float lq, kap, ctau;
    if (lt <= 60.f) {
        const float tau = ex2a(lt);
        const float D = fmaf(tau, fmaf(1.5f, tau + c.tau_sca, 1.7320508f), 1.f);
        lq = A - lg2a(D);
        kap = tau * (1.7320508f + 3.f * tau + 1.5f * c.tau_sca) / D;
        ctau = 1.5f * tau / (D * kLn2);
    } else {
        const float tau = ex2a(fminf(lt, 126.f));
        lq = Bb - 0.5849625f - (lt + lg2a(1.f + c.tau_sca * ex2a(-lt)));
        const float fr = 1.f / (1.f + c.tau_sca * ex2a(-lt));   // tau / (tau + tau_sca)
        kap = 1.f + fr;
        ctau = fr / (tau * kLn2);
    }
    g.q = ex2a(fminf(lq, 126.f));
    const float live = lq < 126.f ? 1.f : 0.f;
    // derivatives of Ls, Lb, Bb, tau_sca with respect to ln u, ln rho, ln B, ln H
    const float dLs_u = (Sv[1] - Sv[0]) * cT;
    const float dLs_rho = -dLs_u + lerpf(dSn[0], dSn[1], wt) * cd.cN;
    const float dLs_B = lerpf(dSb[0], dSb[1], wt) * cd.cB;
    const float dLs_H = lerpf(dSh[0], dSh[1], wt) * cd.cH;
    const float dLb_u = (b1 - b0) * cT;
    const float dLb_rho = -dLb_u + 2.f / kLn2;
    const float dA_u = sig_s * dLs_u + (1.f - sig_s) * dLb_u;
    const float dA_rho = sig_s * dLs_rho + (1.f - sig_s) * dLb_rho;
    const float dA_B = sig_s * dLs_B;
    const float dA_H = sig_s * dLs_H;
    const float w1 = (1.f - kap) * kLn2 * live, w2 = kap * kLn2 * live, w3 = ctau * kLn2 * live;
    g.du = w1 * dA_u + w2 * (4.f / kLn2);
    g.drho = w1 * dA_rho + w2 * (-4.f / kLn2) - w3 * c.tau_sca;
    g.dB = w1 * dA_B;
    g.dH = w1 * dA_H + w2 * (-1.f / kLn2) - w3 * c.tau_sca;
    g.Gs = g.q * w1 * sig_s;
    g.Gb = g.q * w1 * (1.f - sig_s);
    g.jt = j;
    g.wt = wt;
    g.S0 = Sv[0];
    g.S1 = Sv[1];
    return g;
}

// Coulomb transfer X(u_e, u_i) of one sub-cycle (the forward's FP32 form)
// and its partial derivatives.
struct XGrad {
    float X, due, dui, drho;
    bool clamped;
    int ji, je;
    float wi, we;
};

__device__ __forceinline__ XGrad coulomb_grad(const StepK& k, const Smem& S, float ue, float ui, float rho,
                                              float inv_e, float inv_i, float kr, float lcc_off) {
    XGrad x;
    const DevTable& T = k.tab;
    const int nC = T.n[4];
    const float* axC = S.ax + T.axis_off[4];
    unsigned dummy = 0u;
    const Sel se = select_axis(axC, nC, T.inv_dl[4], ue * inv_e, dummy);
    const Sel si = select_axis(axC, nC, T.inv_dl[4], ui * inv_i, dummy);
    const float re = se.r * T.inv_dl[4], ri = si.r * T.inv_dl[4];
    const float we = __saturatef(re), wi = __saturatef(ri);
    const float ce_w = (re > 0.f && re < 1.f) ? T.inv_dl[4] / kLn2 : 0.f;
    const float ci_w = (ri > 0.f && ri < 1.f) ? T.inv_dl[4] / kLn2 : 0.f;
    const float* row = S.lc + si.j * nC + se.j;
    const float c00 = row[0], c01 = row[1], c10 = row[nC], c11 = row[nC + 1];
    const float lC = lerpf(lerpf(c00, c01, we), lerpf(c10, c11, we), wi);
    const float rate = ex2a(fminf(lC + lcc_off, 126.f));
    const float pe = k.ce * ue;
    const float ee = fmaf(k.ce, ue, -pe);
    const float D = fmaf(k.ci, ui, -pe) - ee;
    float X = rate * (kr * D);
    const float lim = k.clamp * fabsf(D * k.inv_cec);
    x.clamped = fabsf(X) > lim;
    if (x.clamped) {
        const float sg = (X >= 0.f ? 1.f : -1.f) * (D >= 0.f ? 1.f : -1.f);
        X = copysignf(lim, X);
        x.due = -sg * k.clamp * k.inv_cec * k.ce;
        x.dui = sg * k.clamp * k.inv_cec * k.ci;
        x.drho = 0.f;
    } else {
        const float dlC_we = lerpf(c01 - c00, c11 - c10, wi);
        const float dlC_wi = lerpf(c10 - c00, c11 - c01, we);
        const float live = (lC + lcc_off) < 126.f ? 1.f : 0.f;
        x.due = X * kLn2 * dlC_we * ce_w * live / ue - rate * kr * k.ce;
        x.dui = X * kLn2 * dlC_wi * ci_w * live / ui + rate * kr * k.ci;
        // d ln X / d ln rho = ln2 dlC/d ln rho + 2 (n_e^2) - 1 (s_K/rho); a saturated
        // rate keeps only the -1
        x.drho = live > 0.f ? X * (1.f - kLn2 * (dlC_we * ce_w + dlC_wi * ci_w)) / rho : -X / rho;
    }
    x.X = X;
    x.ji = si.j;
    x.je = se.j;
    x.wi = wi;
    x.we = we;
    return x;
}

// SMS: the per-sub-cycle state lives in shared memory (n_sub <= kSmemSub,
// column layout, conflict-free) instead of thread-local arrays.
constexpr int kSmemSub = 8;

template <bool SMS>
__global__ void __launch_bounds__(kThreads) k_step_bwd_f32(
    StepK k, long long n, const float* __restrict__ rho_in, const float* __restrict__ B_in,
    const float* __restrict__ H_in, const float* __restrict__ ue_in, const float* __restrict__ ui_in,
    const float* __restrict__ gue_out, const float* __restrict__ gui_out, float* g_rho, float* g_B, float* g_H,
    float* g_ue, float* g_ui, float* g_lb, float* g_ls, float* g_lc) {
    extern __shared__ float sm[];
    load_smem(k, sm);
    Smem S;
    S.ax = sm;
    S.lb = sm + k.axes_floats;
    S.lc = sm + k.axes_floats + k.tab.n[3];
    float* win = sm + smem_table_floats(k) + threadIdx.x;
    float* glb_s = sm + smem_table_floats(k) + kMaxW * kThreads;   // partial brems adjoints
    float* glc_s = glb_s + k.tab.n[3];                             // partial Coulomb adjoints
    const DevTable& T = k.tab;
    const int nT = T.n[3], nC = T.n[4];
    for (int i = threadIdx.x; i < nT + nC * nC; i += blockDim.x) glb_s[i] = 0.f;
    __syncthreads();
    // per-sub-cycle state: u_e, u_i before the exchange, u_e after it, the
    // implicit root, and the branch taken (0 free, 1 limited, 2 implicit)
    float* sst = glc_s + ((nC * nC + 3) & ~3);
    unsigned char* sbr = reinterpret_cast<unsigned char*>(sst + 4 * kSmemSub * kThreads);
    float l_ue[SMS ? 1 : kMaxSub], l_ui[SMS ? 1 : kMaxSub], l_u1[SMS ? 1 : kMaxSub], l_us[SMS ? 1 : kMaxSub];
    unsigned char l_br[SMS ? 1 : kMaxSub];
#define ST_UE(sub) (*(SMS ? &sst[(4 * (sub) + 0) * kThreads + threadIdx.x] : &l_ue[(sub)]))
#define ST_UI(sub) (*(SMS ? &sst[(4 * (sub) + 1) * kThreads + threadIdx.x] : &l_ui[(sub)]))
#define ST_U1(sub) (*(SMS ? &sst[(4 * (sub) + 2) * kThreads + threadIdx.x] : &l_u1[(sub)]))
#define ST_US(sub) (*(SMS ? &sst[(4 * (sub) + 3) * kThreads + threadIdx.x] : &l_us[(sub)]))
#define ST_BR(sub) (*(SMS ? &sbr[(sub) * kThreads + threadIdx.x] : &l_br[(sub)]))
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float rho = rho_in[i], B = B_in[i], H = H_in[i];
        float ue = ue_in[i], ui = ui_in[i];
        const float ge_out = gue_out[i], gi_out = gui_out[i];
        if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
            !(rho > 0.f) || !(ue > 0.f) || !(ui > 0.f) || B < 0.f || H < 0.f) {
            g_rho[i] = 0.f; g_B[i] = 0.f; g_H[i] = 0.f; g_ue[i] = ge_out; g_ui[i] = gi_out;
            continue;
        }
        unsigned clamp = 0u;
        const float ne = rho * k.s_n, Bg = B * k.s_B, Hc = H * k.s_H;
        const float inv_e = k.s_Te / rho, inv_i = k.s_Ti / rho, kr = k.s_K / rho;
        CellC c;
        CellD cd;
        {
            Sel sh = select_axis(S.ax + T.axis_off[0], T.n[0], T.inv_dl[0], Hc, clamp);
            Sel sb = select_axis(S.ax + T.axis_off[1], T.n[1], T.inv_dl[1], Bg, clamp);
            Sel sn = select_axis(S.ax + T.axis_off[2], T.n[2], T.inv_dl[2], ne, clamp);
            const int rowf = 8 * T.nblk;
            c.oN = rowf;
            c.oB = rowf * T.n[2];
            c.oH = c.oB * T.n[1];
            c.row = T.lsb + (long long)((sh.j * T.n[1] + sb.j) * T.n[2] + sn.j) * rowf;
            const float rh = sh.r * T.inv_dl[0], rb = sb.r * T.inv_dl[1], rn = sn.r * T.inv_dl[2];
            c.wh = __saturatef(rh);
            c.wb = __saturatef(rb);
            c.wn = __saturatef(rn);
            cd.cH = (rh > 0.f && rh < 1.f) ? T.inv_dl[0] / kLn2 : 0.f;
            cd.cB = (rb > 0.f && rb < 1.f) ? T.inv_dl[1] / kLn2 : 0.f;
            cd.cN = (rn > 0.f && rn < 1.f) ? T.inv_dl[2] / kLn2 : 0.f;
            c.ls_off = k.l_hs_e;
            c.lb_off = fmaf(2.f, lg2a(ne), k.l_hs_e);
            c.lbb_off = k.l_bb - lg2a(Hc);
            c.tau_sca = k.two_sigT * ne * Hc;
        }
        const float lcc_off = c.lb_off;
        Cache cc;
        cc.base = -8;
        cc.win = win;
        // ---- forward, recorded (the forward kernel's arithmetic) ----
        for (int sub = 0; sub < k.n_sub; ++sub) {
            ST_UE(sub) = ue;
            ST_UI(sub) = ui;
            const XGrad xg = coulomb_grad(k, S, ue, ui, rho, inv_e, inv_i, kr, lcc_off);
            ue += xg.X;
            ui -= xg.X;
            ST_U1(sub) = ue;
            const float q = cool_energy<0>(k, S, c, cc, ue * inv_e, clamp);
            float du = fminf(q, k.limiter * ue);
            unsigned char br = q < k.limiter * ue ? 0 : 1;
            if (k.mode == 1 && q > k.limiter * ue) {
                float u1;
                if (implicit_fp32<0>(k, S, c, cc, inv_e, ue, q, u1)) {
                    du = ue - u1;
                    br = 2;
                    ST_US(sub) = u1;
                }
            }
            ST_BR(sub) = br;
            ue -= du;
        }
        // ---- reverse sweep ----
        float ge = ge_out, gi = gi_out, grho = 0.f, gB = 0.f, gH = 0.f;
        GCache gc;
        gc.j = -1;
        for (int sub = k.n_sub - 1; sub >= 0; --sub) {
            float ge1;
            const unsigned char br = ST_BR(sub);
            if (br == 1) {
                ge1 = (1.f - k.limiter) * ge;
            } else {
                const float u = br == 2 ? ST_US(sub) : ST_U1(sub);
                const QGrad g = cool_grad(k, S, c, cd, gc, u, inv_e);
                const float qu = g.q * g.du / u;
                float sc;
                if (br == 2) {
                    const float den = 1.f + qu;
                    ge1 = ge / den;
                    sc = -ge / den;
                } else {
                    ge1 = ge * (1.f - qu);
                    sc = -ge;
                }
                grho += sc * g.q * g.drho / rho;
                if (g.dB != 0.f) gB += sc * g.q * g.dB / B;
                if (g.dH != 0.f) gH += sc * g.q * g.dH / H;
                if (g_ls) {
                    const float gs = sc * g.Gs;
                    const float wts[2] = {1.f - g.wt, g.wt};
                    const long long rowT = nT;
                    // natural-layout row of corner (jh, jb, jn): rebuilt from the packed row offset
                    const long long r0 = (long long)(c.row - T.lsb) / (8 * T.nblk);
                    const long long rows[8] = {r0, r0 + 1, r0 + T.n[2], r0 + T.n[2] + 1,
                                               r0 + (long long)T.n[1] * T.n[2], r0 + (long long)T.n[1] * T.n[2] + 1,
                                               r0 + (long long)T.n[1] * T.n[2] + T.n[2],
                                               r0 + (long long)T.n[1] * T.n[2] + T.n[2] + 1};
                    const float wh[2] = {1.f - c.wh, c.wh}, wb[2] = {1.f - c.wb, c.wb}, wn[2] = {1.f - c.wn, c.wn};
#pragma unroll
                    for (int cidx = 0; cidx < 8; ++cidx) {
                        const float wc = wh[cidx >> 2] * wb[(cidx >> 1) & 1] * wn[cidx & 1];
#pragma unroll
                        for (int t = 0; t < 2; ++t)
                            atomicAdd(&g_ls[rows[cidx] * rowT + g.jt + t], gs * wc * wts[t]);
                    }
                }
                if (g_lb) {
                    atomicAdd(&glb_s[g.jt], sc * g.Gb * (1.f - g.wt));
                    atomicAdd(&glb_s[g.jt + 1], sc * g.Gb * g.wt);
                }
            }
            const XGrad xg = coulomb_grad(k, S, ST_UE(sub), ST_UI(sub), rho, inv_e, inv_i, kr, lcc_off);
            const float gX = ge1 - gi;
            ge = ge1 + gX * xg.due;
            gi = gi + gX * xg.dui;
            grho += gX * xg.drho;
            if (g_lc && !xg.clamped) {
                const float cl = gX * xg.X * kLn2;
                atomicAdd(&glc_s[xg.ji * nC + xg.je], cl * (1.f - xg.wi) * (1.f - xg.we));
                atomicAdd(&glc_s[xg.ji * nC + xg.je + 1], cl * (1.f - xg.wi) * xg.we);
                atomicAdd(&glc_s[(xg.ji + 1) * nC + xg.je], cl * xg.wi * (1.f - xg.we));
                atomicAdd(&glc_s[(xg.ji + 1) * nC + xg.je + 1], cl * xg.wi * xg.we);
            }
        }
        g_rho[i] = grho;
        g_B[i] = gB;
        g_H[i] = gH;
        g_ue[i] = ge;
        g_ui[i] = gi;
    }
#undef ST_UE
#undef ST_UI
#undef ST_U1
#undef ST_US
#undef ST_BR
    __syncthreads();
    if (g_lb)
        for (int i = threadIdx.x; i < nT; i += blockDim.x)
            if (glb_s[i] != 0.f) atomicAdd(&g_lb[i], glb_s[i]);
    if (g_lc)
        for (int i = threadIdx.x; i < nC * nC; i += blockDim.x)
            if (glc_s[i] != 0.f) atomicAdd(&g_lc[i], glc_s[i]);
}

}  // namespace

cool_status launch_step_f32(const cool_table* t, const cool_params* p, long long n,
                            const float* rho, const float* B, const float* H,
                            const float* ue, const float* ui, float* ue_o, float* ui_o,
                            float* qc, float* qx, cool_counters* cnt, cudaStream_t st,
                            const cool_disk* disk, const float* r) {
    StepK k;
    fill_stepk(t, p, k);
    k.spin = disk ? (float)disk->spin : 0.f;
    k.h_floor = disk ? (float)disk->h_floor : 0.f;
    k.h_from_state = disk ? disk->h_from_state : 0;
    if (n == 0) return COOL_OK;
    bool vec = ((uintptr_t)rho | (uintptr_t)B | (uintptr_t)H | (uintptr_t)ue | (uintptr_t)ui |
                (uintptr_t)ue_o | (uintptr_t)ui_o | (uintptr_t)qc | (uintptr_t)qx | (uintptr_t)r) % 16 == 0;
    size_t smem = (size_t)(smem_table_floats(k) + kMaxW * kThreads) * sizeof(float);
    if (vec) smem += (size_t)kWarps * (disk ? 6 : 5) * kWarpCells * sizeof(float);
    using KFn = void (*)(StepK, long long, const float*, const float*, const float*, const float*, const float*,
                         float*, float*, float*, float*, cool_counters*, const float*);
    using KFnT = void (*)(StepK, long long, const float*, const float*, const float*, const float*, const float*,
                          float*, float*, float*, float*, cool_counters*);
#define COOL_KV(V, F) k_step_f32<V, F, 0>, k_step_f32<V, F, 1>, k_step_f32<V, F, 2>, k_step_f32<V, F, 3>
    static const KFn table_v[5][4] = {{COOL_KV(true, 0)}, {COOL_KV(true, 1)}, {COOL_KV(true, 2)},
                                      {COOL_KV(true, 3)}, {COOL_KV(true, 4)}};
    static const KFn table_s[5][4] = {{COOL_KV(false, 0)}, {COOL_KV(false, 1)}, {COOL_KV(false, 2)},
                                      {COOL_KV(false, 3)}, {COOL_KV(false, 4)}};
#undef COOL_KV
    // disk geometry: FP32 table only
    static const KFn disk_v[4] = {k_step_f32<true, 0, 4>, k_step_f32<true, 0, 5>, k_step_f32<true, 0, 6>,
                                  k_step_f32<true, 0, 7>};
    static const KFn disk_s[4] = {k_step_f32<false, 0, 4>, k_step_f32<false, 0, 5>, k_step_f32<false, 0, 6>,
                                  k_step_f32<false, 0, 7>};
    const int fmt = t->dev.fmt;
    if (fmt < 0 || fmt > 4) return COOL_EUNSUPPORTED;
    if (disk && (fmt != 0 || !r)) return COOL_EUNSUPPORTED;
    const int var = (p->mode == COOL_IMPLICIT_STIFF ? 1 : 0) | (p->fp64_critical ? 2 : 0);
    if (p->path == COOL_PATH_TMA_SMEM) {
        if (disk) return COOL_EUNSUPPORTED;
        if (!vec) return COOL_EALIGN;   // bulk copies need 16-byte aligned fields
#define COOL_KT(F) k_step_tma<F, 0>, k_step_tma<F, 1>, k_step_tma<F, 2>, k_step_tma<F, 3>
        static const KFnT table_t[5][4] = {{COOL_KT(0)}, {COOL_KT(1)}, {COOL_KT(2)}, {COOL_KT(3)}, {COOL_KT(4)}};
#undef COOL_KT
        static const int width[5] = {Fmt<0>::W, Fmt<1>::W, Fmt<2>::W, Fmt<3>::W, Fmt<4>::W};
        KFnT fn = table_t[fmt][var];
        const size_t sm_t = (size_t)(smem_table_floats(k) + width[fmt] * kThreads + kWarps * 2 * 5 * kWarpCells) *
                                sizeof(float) + kWarps * 2 * sizeof(uint64_t);
        cudaError_t et = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_t);
        if (et != cudaSuccess) return set_cuda_error(et);
        int per = 0;
        et = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, sm_t);
        if (et != cudaSuccess) return set_cuda_error(et);
        if (per < 1) per = 1;
        long long wk = (n + kWarps * kWarpCells - 1) / (kWarps * kWarpCells);
        long long cp = (long long)sm_count() * per;
        long long bl = wk < cp ? wk : cp;
        if (bl < 1) bl = 1;
        fn<<<(int)bl, kThreads, sm_t, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt);
        et = cudaGetLastError();
        return et == cudaSuccess ? COOL_OK : set_cuda_error(et);
    }
    KFn fn = disk ? (vec ? disk_v[var] : disk_s[var]) : (vec ? table_v[fmt][var] : table_s[fmt][var]);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (per_sm < 1) per_sm = 1;
    long long work = vec ? (n + kWarps * kWarpCells - 1) / (kWarps * kWarpCells) : (n + kThreads - 1) / kThreads;
    long long cap = (long long)sm_count() * per_sm;  // one resident wave, persistent blocks
    long long blocks = work < cap ? work : cap;
    if (blocks < 1) blocks = 1;
    fn<<<(int)blocks, kThreads, smem, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt, r);
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


cool_status launch_step_bwd_f32(const cool_table* t, const cool_params* p, long long n, const float* rho,
                                const float* B, const float* H, const float* ue, const float* ui,
                                const float* gue, const float* gui, float* g_rho, float* g_B, float* g_H,
                                float* g_ue, float* g_ui, float* g_lb, float* g_ls, float* g_lc, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    if (t->dev.fmt != 0 || p->fp64_critical || p->n_sub > kMaxSub) return COOL_EUNSUPPORTED;
    StepK k;
    fill_stepk(t, p, k);
    const bool sms = p->n_sub <= kSmemSub;
    size_t smem = (size_t)(smem_table_floats(k) + kMaxW * kThreads + t->dev.n[3] +
                           ((t->dev.n[4] * t->dev.n[4] + 3) & ~3)) * sizeof(float);
    if (sms) smem += (size_t)kSmemSub * kThreads * (4 * sizeof(float) + 1);
    auto fn = sms ? k_step_bwd_f32<true> : k_step_bwd_f32<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (per_sm < 1) per_sm = 1;
    long long work = (n + kThreads - 1) / kThreads;
    long long cap = (long long)sm_count() * per_sm;
    long long blocks = work < cap ? work : cap;
    fn<<<(int)blocks, kThreads, smem, st>>>(k, n, rho, B, H, ue, ui, gue, gui, g_rho, g_B, g_H, g_ue, g_ui, g_lb,
                                            g_ls, g_lc);
    e = cudaGetLastError();
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
