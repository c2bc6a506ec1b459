// cool_step_bwd.cu -- the adjoint of the FP32 step (cool_step_bwd).
#include "cool_step_cell.cuh"

namespace cool {
namespace {

// ---------------------------------------------------------------------------
// Adjoint (cool_step_bwd).  Per cell the forward sub-cycles are recomputed
// with the forward kernel's own functions (same trajectory, same branches)
// and differentiated with the hand-derived partial derivatives of the
// cooling energy q and of the Coulomb transfer X (below), the limiter's
// branch, and for an implicit sub-cycle the implicit-function theorem at
// the root (du*/du1 = 1/(1 + dq/du), du*/dtheta = -dq/dtheta / (1 + dq/du)).
// Input gradients alone: forward tangents (k_step_tan_f32), the 2x5
// Jacobian carried along the sub-cycles.  With table adjoints: each
// sub-cycle's state is kept and a reverse sweep (k_step_bwd_f32) sends the
// table adjoints to the natural layouts: synchrotron [nH nB nN nT] with
// global atomics, brems and Coulomb through shared-memory partial sums.
// ---------------------------------------------------------------------------
constexpr int kMaxSub = 64;
constexpr float kLn2 = 0.69314718056f;
constexpr float kInvLn2 = 1.44269504089f;

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
    const SelW s = select_sub<3, true>(k, axT + nT, nT, T.inv_dl[3], Te, dummy, dummy);
    const int j = s.j;
    const float wraw = s.r * T.inv_dl[3];
    const float wt = s.w;
    const float cT = (wraw > 0.f && wraw < 1.f) ? T.inv_dl[3] * kInvLn2 : 0.f;   // dwt / d ln Te
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
        const float rD = __fdividef(1.f, D);   // D >= 1
        kap = tau * (1.7320508f + 3.f * tau + 1.5f * c.tau_sca) * rD;
        ctau = (1.5f * kInvLn2) * tau * rD;
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

__device__ __forceinline__ XGrad coulomb_grad(const StepK& k, const Smem& S, float ue, float ui, float inv_rho,
                                              float inv_e, float inv_i, float kr, float lcc_off) {
    XGrad x;
    const DevTable& T = k.tab;
    const int nC = T.n[4];
    const float* axC = S.ax + T.axis_off[4];
    unsigned dummy = 0u;
    const SelW se = select_sub<4, true>(k, axC + nC, nC, T.inv_dl[4], ue * inv_e, dummy, dummy);
    const SelW si = select_sub<4, true>(k, axC + nC, nC, T.inv_dl[4], ui * inv_i, dummy, dummy);
    const float re = se.r * T.inv_dl[4], ri = si.r * T.inv_dl[4];
    const float we = se.w, wi = si.w;
    const float ce_w = (re > 0.f && re < 1.f) ? T.inv_dl[4] * kInvLn2 : 0.f;
    const float ci_w = (ri > 0.f && ri < 1.f) ? T.inv_dl[4] * kInvLn2 : 0.f;
    const int ls = k.lc_stride;
    const float* row = S.lc + si.j * ls + se.j;
    const float c00 = row[0], c01 = row[1], c10 = row[ls], c11 = row[ls + 1];
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
        x.due = __fdividef(X * kLn2 * dlC_we * ce_w * live, ue) - rate * kr * k.ce;
        x.dui = __fdividef(X * kLn2 * dlC_wi * ci_w * live, ui) + rate * kr * k.ci;
        // d ln X / d ln rho = ln2 dlC/d ln rho + 2 (n_e^2) - 1 (s_K/rho); a saturated
        // rate keeps only the -1
        x.drho = live > 0.f ? X * (1.f - kLn2 * (dlC_we * ce_w + dlC_wi * ci_w)) * inv_rho : -X * inv_rho;
    }
    x.X = X;
    x.ji = si.j;
    x.je = se.j;
    x.wi = wi;
    x.we = we;
    return x;
}

// The per-cell constants of both adjoint kernels, from (rho, B, H): the
// (H, B, n_e) selection (exact rule) with its weights, the weights'
// derivative constants, and the bridge's offsets.
__device__ __forceinline__ void bwd_cell(const StepK& k, const Smem& S, float rho, float B, float H,
                                         CellC& c, CellD& cd, unsigned& clamp) {
    const DevTable& T = k.tab;
    const float ne = rho * k.s_n, Bg = B * k.s_B, Hc = H * k.s_H;
    unsigned unused = 0u;
    const SelW sh = select_sub<0, true>(k, S.ax + T.axis_off[0] + T.n[0], T.n[0], T.inv_dl[0], Hc, clamp, unused);
    const SelW sb = select_sub<1, true>(k, S.ax + T.axis_off[1] + T.n[1], T.n[1], T.inv_dl[1], Bg, clamp, unused);
    const SelW sn = select_sub<2, true>(k, S.ax + T.axis_off[2] + T.n[2], T.n[2], T.inv_dl[2], ne, clamp, unused);
    const int rowf = 8 * T.nblk;
    c.oN = rowf;
    c.oB = rowf * T.n[2];
    c.oH = c.oB * T.n[1];
    c.row = T.lsb + (long long)((sh.j * T.n[1] + sb.j) * T.n[2] + sn.j) * rowf;
    const float rh = sh.r * T.inv_dl[0], rb = sb.r * T.inv_dl[1], rn = sn.r * T.inv_dl[2];
    c.wh = __saturatef(rh);
    c.wb = __saturatef(rb);
    c.wn = __saturatef(rn);
    cd.cH = (rh > 0.f && rh < 1.f) ? T.inv_dl[0] * kInvLn2 : 0.f;
    cd.cB = (rb > 0.f && rb < 1.f) ? T.inv_dl[1] * kInvLn2 : 0.f;
    cd.cN = (rn > 0.f && rn < 1.f) ? T.inv_dl[2] * kInvLn2 : 0.f;
    c.ls_off = k.l_hs_e;
    c.lb_off = fmaf(2.f, lg2a(ne), k.l_hs_e);
    c.lbb_off = k.l_bb - lg2a(Hc);
    c.tau_sca = k.two_sigT * ne * Hc;
}

// SMS: the per-sub-cycle state lives in shared memory (n_sub <= kSmemSub,
// column layout, conflict-free) instead of thread-local arrays.
constexpr int kSmemSub = 8;
constexpr int kStateFloats = 3;   // floats of per-sub-cycle state (ST_F) with the implicit root; 2 without

// With table adjoints requested (g_lb, g_ls or g_lc non-null); the input
// gradients alone come from k_step_tan_f32.  IMPL: the implicit mode's
// solve compiled in (and its root kept per sub-cycle).
// PASS 1 (implicit mode, without IMPL): a cell that turns stiff stops
// before any write and its index goes to the list dl ([0] the count, then
// the indices); PASS 2 (with IMPL) steps the listed cells, consecutive
// entries on consecutive lanes, instead of a solving lane holding its warp.
template <bool SMS, bool IMPL, int PASS = 0>
__global__ void __launch_bounds__(kThreads, IMPL ? 2 : 3) k_step_bwd_f32(
    StepK k, long long n, const float* __restrict__ rho_in, const float* __restrict__ B_in,
    const float* __restrict__ H_in, const float* __restrict__ ue_in, const float* __restrict__ ui_in,
    const float* __restrict__ gue_out, const float* __restrict__ gui_out, float* g_rho, float* g_B, float* g_H,
    float* g_ue, float* g_ui, float* g_lb, float* g_ls, float* g_lc, unsigned* dl) {
    extern __shared__ float sm[];
    load_smem(k, sm);
    const Smem S = smem_view(k, sm);
    float* win = sm + smem_table_floats(k) + threadIdx.x;           // 8-row window (FP32 table)
    float* glb_s = sm + smem_table_floats(k) + Fmt<0>::W * kThreads;  // partial brems adjoints
    float* glc_s = glb_s + k.tab.n[3];                             // partial Coulomb adjoints
    const DevTable& T = k.tab;
    const int nT = T.n[3], nC = T.n[4];
    for (int i = threadIdx.x; i < nT + nC * nC; i += blockDim.x) glb_s[i] = 0.f;
    __syncthreads();
    // per-sub-cycle state: u_e, u_i before the exchange, the implicit root
    // (IMPL) and the branch taken (0 free, 1 limited, 2 implicit); the
    // exchange (its X and partials, u_e after it) is evaluated again from
    // u_e, u_i in the reverse sweep, which needs its corners for the
    // Coulomb adjoint anyway
    constexpr int NSF = IMPL ? kStateFloats : kStateFloats - 1;
    float* sst = glc_s + ((nC * nC + 3) & ~3);
    unsigned char* sbr = reinterpret_cast<unsigned char*>(sst + NSF * kSmemSub * kThreads);
    float l_st[SMS ? 1 : NSF * kMaxSub];
    unsigned char l_br[SMS ? 1 : kMaxSub];
#define ST_F(sub, f) (*(SMS ? &sst[(NSF * (sub) + (f)) * kThreads + threadIdx.x] \
                            : &l_st[NSF * (sub) + (f)]))
#define ST_UE(sub) ST_F(sub, 0)
#define ST_UI(sub) ST_F(sub, 1)
#define ST_US(sub) ST_F(sub, 2)
#define ST_BR(sub) (*(SMS ? &sbr[(sub) * kThreads + threadIdx.x] : &l_br[(sub)]))
    // cells in chunks of 32 (one per lane): each warp's first chunk by its
    // index in the grid, the next ones from the tile counter (k.sched) as
    // it finishes, or round-robin without one
    const int lane = threadIdx.x & 31;
    const long long nitems = PASS == 2 ? (long long)dl[0] : n;
    const long long nchunks = (nitems + 31) / 32;
    const long long first = (long long)gridDim.x * kWarps;
    long long chunk = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    while (chunk < nchunks) {
        const long long t = chunk * 32 + lane;
        if (t < nitems) {
            const long long i = PASS == 2 ? (long long)dl[1 + t] : t;
            const float rho = rho_in[i], B = B_in[i], H = H_in[i];
            float ue = ue_in[i], ui = ui_in[i];
            const float ge_out = gue_out[i], gi_out = gui_out[i];
            if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
                !(rho > 0.f) || !(ue > 0.f) || !(ui > 0.f) || B < 0.f || H < 0.f) {
                g_rho[i] = 0.f; g_B[i] = 0.f; g_H[i] = 0.f; g_ue[i] = ge_out; g_ui[i] = gi_out;
                goto next_chunk;
            }
            unsigned clamp = 0u;
            const float inv_e = k.s_Te / rho, inv_i = k.s_Ti / rho, kr = k.s_K / rho;
            const float inv_rho = 1.f / rho;
            const float inv_B = B > 0.f ? 1.f / B : 0.f;   // used only where dq/dB != 0 (B above the first node)
            const float inv_H = H > 0.f ? 1.f / H : 0.f;
            CellC c;
            CellD cd;
            bwd_cell(k, S, rho, B, H, c, cd, clamp);
            const float lcc_off = c.lb_off;
            Cache cc;
            cc.base = -8;
            cc.win = win;
            cc.near = 0u;
            GCache gc;
            gc.j = -1;
            // ---- forward, recorded (the forward kernel's arithmetic) ----
            for (int sub = 0; sub < k.n_sub; ++sub) {
                ST_UE(sub) = ue;
                ST_UI(sub) = ui;
                const XGrad xg = coulomb_grad(k, S, ue, ui, inv_rho, inv_e, inv_i, kr, lcc_off);
                ue += xg.X;
                ui -= xg.X;
                const float q = cool_energy<0, true>(k, S, c, cc, ue * inv_e, clamp);
                if (PASS == 1 && q > k.limiter * ue) {
                    // stiff: listed for PASS 2, nothing written or added here
                    dl[1 + atomicAdd(dl, 1u)] = (unsigned)i;
                    goto next_chunk;
                }
                float du = fminf(q, k.limiter * ue);
                unsigned char br = q < k.limiter * ue ? 0 : 1;
                if (IMPL && q > k.limiter * ue) {
                    float u1;
                    if (implicit_fp32<0, true>(k, S, c, cc, inv_e, ue, q, u1)) {
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
            int ls_j = -1;                 // interval whose synchrotron adjoints are being summed
            float ls_a0 = 0.f, ls_a1 = 0.f;
            // add the summed adjoints of interval j to its 8 corner rows (natural layout)
            auto flush_ls = [&](int j, float a0, float a1) {
                if (j < 0) return;
                const long long r0 = (long long)(c.row - T.lsb) / (8 * T.nblk);
                const long long nN = T.n[2], nBN = (long long)T.n[1] * T.n[2];
                const long long rows[8] = {r0, r0 + 1, r0 + nN, r0 + nN + 1,
                                           r0 + nBN, r0 + nBN + 1, r0 + nBN + nN, r0 + nBN + nN + 1};
                const float wh[2] = {1.f - c.wh, c.wh}, wb[2] = {1.f - c.wb, c.wb}, wn[2] = {1.f - c.wn, c.wn};
#pragma unroll
                for (int cidx = 0; cidx < 8; ++cidx) {
                    const float wc = wh[cidx >> 2] * wb[(cidx >> 1) & 1] * wn[cidx & 1];
                    atomicAdd(&g_ls[rows[cidx] * nT + j], wc * a0);
                    atomicAdd(&g_ls[rows[cidx] * nT + j + 1], wc * a1);
                }
            };
            // the brems and Coulomb adjoints likewise summed in registers while
            // the sweep stays in one interval (brems: the synchrotron's T_e
            // interval) or one Coulomb cell, then added to the block's
            // shared partial sums
            int lb_j = -1;
            float lb_a0 = 0.f, lb_a1 = 0.f;
            int lc_k = -1;                 // i nC + j of the Coulomb cell being summed
            float lc00 = 0.f, lc01 = 0.f, lc10 = 0.f, lc11 = 0.f;
            auto flush_lb = [&]() {
                if (lb_j < 0) return;
                atomicAdd(&glb_s[lb_j], lb_a0);
                atomicAdd(&glb_s[lb_j + 1], lb_a1);
            };
            auto flush_lc = [&]() {
                if (lc_k < 0) return;
                atomicAdd(&glc_s[lc_k], lc00);
                atomicAdd(&glc_s[lc_k + 1], lc01);
                atomicAdd(&glc_s[lc_k + nC], lc10);
                atomicAdd(&glc_s[lc_k + nC + 1], lc11);
            };
            for (int sub = k.n_sub - 1; sub >= 0; --sub) {
                float ge1;
                // the exchange of this sub-cycle again (the forward's arithmetic:
                // the same X, so the same u_e after it)
                const XGrad xg = coulomb_grad(k, S, ST_UE(sub), ST_UI(sub), inv_rho, inv_e, inv_i, kr, lcc_off);
                const unsigned char br = ST_BR(sub);
                if (br == 1) {
                    ge1 = (1.f - k.limiter) * ge;
                } else {
                    const float u = (IMPL && br == 2) ? ST_US(sub) : ST_UE(sub) + xg.X;
                    const QGrad g = cool_grad(k, S, c, cd, gc, u, inv_e);
                    const float qu = __fdividef(g.q * g.du, u);
                    float sc;
                    if (br == 2) {
                        ge1 = __fdividef(ge, 1.f + qu);
                        sc = -ge1;
                    } else {
                        ge1 = ge * (1.f - qu);
                        sc = -ge;
                    }
                    grho += sc * g.q * g.drho * inv_rho;
                    if (g.dB != 0.f) gB += sc * g.q * g.dB * inv_B;
                    if (g.dH != 0.f) gH += sc * g.q * g.dH * inv_H;
                    if (g_ls) {
                        // the 16 corner entries of interval jt receive w_corner x
                        // (gs w_T): summed over the sub-cycles that stay in it
                        const float gs = sc * g.Gs;
                        if (g.jt != ls_j) {
                            flush_ls(ls_j, ls_a0, ls_a1);
                            ls_j = g.jt;
                            ls_a0 = 0.f;
                            ls_a1 = 0.f;
                        }
                        ls_a0 += gs * (1.f - g.wt);
                        ls_a1 += gs * g.wt;
                    }
                    if (g_lb) {
                        if (g.jt != lb_j) {
                            flush_lb();
                            lb_j = g.jt;
                            lb_a0 = 0.f;
                            lb_a1 = 0.f;
                        }
                        lb_a0 += sc * g.Gb * (1.f - g.wt);
                        lb_a1 += sc * g.Gb * g.wt;
                    }
                }
                const float gX = ge1 - gi;
                ge = ge1 + gX * xg.due;
                gi = gi + gX * xg.dui;
                grho += gX * xg.drho;
                if (g_lc) {
                    if (xg.clamped) continue;
                    const float cl = gX * xg.X * kLn2;
                    const int key = xg.ji * nC + xg.je;
                    if (key != lc_k) {
                        flush_lc();
                        lc_k = key;
                        lc00 = lc01 = lc10 = lc11 = 0.f;
                    }
                    lc00 += cl * (1.f - xg.wi) * (1.f - xg.we);
                    lc01 += cl * (1.f - xg.wi) * xg.we;
                    lc10 += cl * xg.wi * (1.f - xg.we);
                    lc11 += cl * xg.wi * xg.we;
                }
            }
            if (g_ls) flush_ls(ls_j, ls_a0, ls_a1);
            if (g_lb) flush_lb();
            if (g_lc) flush_lc();
            g_rho[i] = grho;
            g_B[i] = gB;
            g_H[i] = gH;
            g_ue[i] = ge;
            g_ui[i] = gi;
        }
    next_chunk:
        if (k.sched) {
            unsigned long long nt = 0;
            if (lane == 0) nt = atomicAdd(k.sched, 1ull);
            chunk = first + (long long)__shfl_sync(0xffffffffu, nt, 0);
        } else {
            chunk += first;
        }
    }
#undef ST_F
#undef ST_UE
#undef ST_UI
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

// One input gradient from the output adjoints and a column of the
// Jacobian; the same expression in tan_cell and k_jac_contract, so the
// gradients of cool_step_bwd_jac are cool_step_bwd's bit for bit.
__device__ __forceinline__ float jac_contract(float ge, float gi, float je, float ji) {
    return fmaf(ge, je, gi * ji);
}

// The input gradients without table adjoints, by forward tangents.  The
// step maps five inputs (rho, B, H, u_e, u_i) to two outputs, so the 2x5
// Jacobian d(u_e, u_i)/d(inputs) is carried through the sub-cycles in
// registers -- the chain rule applied in the forward order, with the same
// partials of X and q the reverse sweep uses -- and contracted with the
// output gradients at the end.  The product is the reverse sweep's
// (different FP32 rounding order), with no per-sub-cycle state.
// IMPL: the implicit mode's solve is compiled in; the explicit-only kernel
// fits 64 registers without spills, 4 blocks (32 warps) per SM.  DEFER
// (implicit mode, without IMPL): a cell that turns stiff stops, writes
// nothing and returns false; its index goes to a list that
// k_step_tan_list_f32 steps with the solve, the listed cells side by side
// on consecutive lanes instead of one solving lane holding its warp.
// JAC (cool_step_fwd_jac): instead of the contraction, the cell's outputs
// u_e, u_i (the forward step's, bit for bit: the same selections, exchange,
// bridge and solve) and its Jacobian go to jo, the Jacobian as ten SoA rows
// of jo.n floats: row x = d u_e / d in_x, row 5 + x = d u_i / d in_x for
// in = (rho, B, H, u_e, u_i).  The inputs are read before anything is
// written, so the outputs may overwrite them.
struct JacOut {
    float* ue;
    float* ui;
    float* jac;
    long long n;
};

template <bool IMPL, bool DEFER, bool JAC>
__device__ __forceinline__ bool tan_cell(const StepK& k, const Smem& S, float* win, long long i,
                                         const float* __restrict__ rho_in, const float* __restrict__ B_in,
                                         const float* __restrict__ H_in, const float* ue_in,
                                         const float* ui_in, const float* __restrict__ gue_out,
                                         const float* __restrict__ gui_out, float* g_rho, float* g_B, float* g_H,
                                         float* g_ue, float* g_ui, const JacOut& jo) {
    const float rho = rho_in[i], B = B_in[i], H = H_in[i];
    float ue = ue_in[i], ui = ui_in[i];
    const float ge_out = JAC ? 0.f : gue_out[i], gi_out = JAC ? 0.f : gui_out[i];
    if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
        !(rho > 0.f) || !(ue > 0.f) || !(ui > 0.f) || B < 0.f || H < 0.f) {
        if (JAC) {
            // passed through: the identity on (u_e, u_i)
            jo.ue[i] = ue;
            jo.ui[i] = ui;
#pragma unroll
            for (int x = 0; x < 5; ++x) {
                jo.jac[x * jo.n + i] = x == 3 ? 1.f : 0.f;
                jo.jac[(5 + x) * jo.n + i] = x == 4 ? 1.f : 0.f;
            }
        } else {
            g_rho[i] = 0.f; g_B[i] = 0.f; g_H[i] = 0.f; g_ue[i] = ge_out; g_ui[i] = gi_out;
        }
    } else {
        unsigned clamp = 0u;
        const float inv_e = k.s_Te / rho, inv_i = k.s_Ti / rho, kr = k.s_K / rho;
        const float inv_rho = 1.f / rho;
        const float inv_B = B > 0.f ? 1.f / B : 0.f;
        const float inv_H = H > 0.f ? 1.f / H : 0.f;
        CellC c;
        CellD cd;
        bwd_cell(k, S, rho, B, H, c, cd, clamp);
        const float lcc_off = c.lb_off;
        Cache cc;
        cc.base = -8;
        cc.win = win;
        cc.near = 0u;
        GCache gc;
        gc.j = -1;
        // tangents: je[x] = d u_e / d x, ji[x] = d u_i / d x for
        // x = rho, B, H, u_e(in), u_i(in)
        float je[5] = {0.f, 0.f, 0.f, 1.f, 0.f};
        float ji[5] = {0.f, 0.f, 0.f, 0.f, 1.f};
        for (int sub = 0; sub < k.n_sub; ++sub) {
            // exchange: u_e += X, u_i -= X
            const XGrad xg = coulomb_grad(k, S, ue, ui, inv_rho, inv_e, inv_i, kr, lcc_off);
            ue += xg.X;
            ui -= xg.X;
#pragma unroll
            for (int x = 0; x < 5; ++x) {
                float dX = fmaf(xg.due, je[x], xg.dui * ji[x]);
                if (x == 0) dX += xg.drho;
                je[x] += dX;
                ji[x] -= dX;
            }
            // cooling: free, limited or implicit, as the forward step
            QGrad g = cool_grad(k, S, c, cd, gc, ue, inv_e);
            const float q = g.q;
            if (DEFER && q > k.limiter * ue) return false;   // stiff: the list kernel steps it
            float du = fminf(q, k.limiter * ue);
            int br = q < k.limiter * ue ? 0 : 1;
            float u_at = ue;
            if (IMPL && q > k.limiter * ue) {
                float u1;
                if (implicit_fp32<0, true>(k, S, c, cc, inv_e, ue, q, u1)) {
                    du = ue - u1;
                    br = 2;
                    u_at = u1;
                    g = cool_grad(k, S, c, cd, gc, u1, inv_e);
                }
            }
            if (br == 1) {
                const float f = 1.f - k.limiter;
#pragma unroll
                for (int x = 0; x < 5; ++x) je[x] *= f;
            } else {
                // dq = qu du + q_rho drho + q_B dB + q_H dH
                const float qu = __fdividef(g.q * g.du, u_at);
                const float qx[3] = {g.q * g.drho * inv_rho, g.dB != 0.f ? g.q * g.dB * inv_B : 0.f,
                                     g.dH != 0.f ? g.q * g.dH * inv_H : 0.f};
                if (br == 2) {
                    // u* + q(u*) = u_e: du* = (du_e - q_x dx) / (1 + qu)
                    const float r = __fdividef(1.f, 1.f + qu);
#pragma unroll
                    for (int x = 0; x < 5; ++x) je[x] = (x < 3 ? je[x] - qx[x < 3 ? x : 0] : je[x]) * r;
                } else {
                    const float f = 1.f - qu;
#pragma unroll
                    for (int x = 0; x < 5; ++x) je[x] = x < 3 ? fmaf(je[x], f, -qx[x < 3 ? x : 0]) : je[x] * f;
                }
            }
            ue -= du;
        }
        if (JAC) {
            jo.ue[i] = ue;
            jo.ui[i] = ui;
#pragma unroll
            for (int x = 0; x < 5; ++x) {
                jo.jac[x * jo.n + i] = je[x];
                jo.jac[(5 + x) * jo.n + i] = ji[x];
            }
        } else {
            g_rho[i] = jac_contract(ge_out, gi_out, je[0], ji[0]);
            g_B[i] = jac_contract(ge_out, gi_out, je[1], ji[1]);
            g_H[i] = jac_contract(ge_out, gi_out, je[2], ji[2]);
            g_ue[i] = jac_contract(ge_out, gi_out, je[3], ji[3]);
            g_ui[i] = jac_contract(ge_out, gi_out, je[4], ji[4]);
        }
    }
    return true;
}

template <bool IMPL, bool DEFER, bool JAC>
__global__ void __launch_bounds__(kThreads, IMPL ? 2 : 4) k_step_tan_f32(
    StepK k, long long n, const float* __restrict__ rho_in, const float* __restrict__ B_in,
    const float* __restrict__ H_in, const float* ue_in, const float* ui_in,
    const float* __restrict__ gue_out, const float* __restrict__ gui_out, float* g_rho, float* g_B, float* g_H,
    float* g_ue, float* g_ui, unsigned* n_list, unsigned* list, JacOut jo) {
    extern __shared__ float sm[];
    load_smem(k, sm);
    const Smem S = smem_view(k, sm);
    float* win = sm + smem_table_floats(k) + threadIdx.x;           // 8-row window (FP32 table)
    const int lane = threadIdx.x & 31;
    const long long nchunks = (n + 31) / 32;
    const long long first = (long long)gridDim.x * kWarps;
    long long chunk = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    while (chunk < nchunks) {
        const long long i = chunk * 32 + lane;
        bool deferred = false;
        if (i < n)
            deferred = !tan_cell<IMPL, DEFER, JAC>(k, S, win, i, rho_in, B_in, H_in, ue_in, ui_in, gue_out, gui_out,
                                                   g_rho, g_B, g_H, g_ue, g_ui, jo);
        if (DEFER) {
            // the warp's deferred cells, appended with one atomic
            const unsigned bal = __ballot_sync(0xffffffffu, deferred);
            if (bal) {
                unsigned base = 0u;
                if (lane == 0) base = atomicAdd(n_list, (unsigned)__popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (deferred) list[base + __popc(bal & ((1u << lane) - 1u))] = (unsigned)i;
            }
        }
        if (k.sched) {
            unsigned long long nt = 0;
            if (lane == 0) nt = atomicAdd(k.sched, 1ull);
            chunk = first + (long long)__shfl_sync(0xffffffffu, nt, 0);
        } else {
            chunk += first;
        }
    }
}

// The cells k_step_tan_f32<false, true, JAC> deferred, by index, with the
// solve compiled in: consecutive list entries on consecutive lanes.
template <bool JAC>
__global__ void __launch_bounds__(kThreads, 2) k_step_tan_list_f32(
    StepK k, const unsigned* __restrict__ n_list, const unsigned* __restrict__ list,
    const float* __restrict__ rho_in, const float* __restrict__ B_in, const float* __restrict__ H_in,
    const float* ue_in, const float* ui_in, const float* __restrict__ gue_out,
    const float* __restrict__ gui_out, float* g_rho, float* g_B, float* g_H, float* g_ue, float* g_ui, JacOut jo) {
    extern __shared__ float sm[];
    load_smem(k, sm);
    const Smem S = smem_view(k, sm);
    float* win = sm + smem_table_floats(k) + threadIdx.x;
    const long long m = *n_list;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (long long)gridDim.x * blockDim.x)
        tan_cell<true, false, JAC>(k, S, win, (long long)list[t], rho_in, B_in, H_in, ue_in, ui_in, gue_out,
                                   gui_out, g_rho, g_B, g_H, g_ue, g_ui, jo);
}

// cool_step_bwd_jac: the input gradients from a stored Jacobian (the layout
// of JacOut) and the output adjoints.
__global__ void k_jac_contract(long long n, const float* __restrict__ jac, const float* __restrict__ gue,
                               const float* __restrict__ gui, float* g_rho, float* g_B, float* g_H, float* g_ue,
                               float* g_ui) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float ge = gue[i], gi = gui[i];
        g_rho[i] = jac_contract(ge, gi, jac[i], jac[5 * n + i]);
        g_B[i] = jac_contract(ge, gi, jac[n + i], jac[6 * n + i]);
        g_H[i] = jac_contract(ge, gi, jac[2 * n + i], jac[7 * n + i]);
        g_ue[i] = jac_contract(ge, gi, jac[3 * n + i], jac[8 * n + i]);
        g_ui[i] = jac_contract(ge, gi, jac[4 * n + i], jac[9 * n + i]);
    }
}

// The launches of one cool_step_bwd call: fn over the cells (persistent
// grid, dynamic chunk order), then, with a deferral list, the list kernel.
using TanFn = decltype(&k_step_tan_f32<false, false, false>);
using BwdFn = decltype(&k_step_bwd_f32<true, true, 0>);

cudaError_t launch_bwd(StepK& k, long long n, const void* fn, TanFn tf, BwdFn fb, bool tbl, size_t smem,
                       unsigned* scratch, const float* rho, const float* B, const float* H, const float* ue,
                       const float* ui, const float* gue, const float* gui, float* g_rho, float* g_B, float* g_H,
                       float* g_ue, float* g_ui, float* g_lb, float* g_ls, float* g_lc, const JacOut& jo,
                       cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long work = (n + kThreads - 1) / kThreads;
    long long cap = (long long)sm_count() * per_sm;
    long long blocks = work < cap ? work : cap;
    if ((n + 31) / 32 > blocks * kWarps) {
        // more chunks than warps: the dynamic order
        k.sched = sched_counter(st);
        if (k.sched) {
            e = cudaMemsetAsync(k.sched, 0, sizeof(unsigned long long), st);
            if (e != cudaSuccess) return e;
        }
    }
    if (tbl) {
        fb<<<(int)blocks, kThreads, smem, st>>>(k, n, rho, B, H, ue, ui, gue, gui, g_rho, g_B, g_H, g_ue, g_ui,
                                                g_lb, g_ls, g_lc, scratch);
        e = cudaGetLastError();
        if (e != cudaSuccess || !scratch) return e;
        // the listed stiff cells, with the solve (and its root in the state)
        const void* fl = (const void*)k_step_bwd_f32<true, true, 2>;
        const size_t sl = smem + (size_t)kSmemSub * kThreads * sizeof(float);
        e = cudaFuncSetAttribute(fl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fl, kThreads, sl);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        long long bl = (long long)sm_count() * per_sm;
        if (bl > work) bl = work;
        StepK kl = k;
        kl.sched = nullptr;   // the list in its fixed order
        k_step_bwd_f32<true, true, 2><<<(int)bl, kThreads, sl, st>>>(kl, n, rho, B, H, ue, ui, gue, gui, g_rho, g_B,
                                                                       g_H, g_ue, g_ui, g_lb, g_ls, g_lc, scratch);
        return cudaGetLastError();
    }
    unsigned* list = scratch ? scratch + 1 : nullptr;
    tf<<<(int)blocks, kThreads, smem, st>>>(k, n, rho, B, H, ue, ui, gue, gui, g_rho, g_B, g_H, g_ue, g_ui, scratch,
                                            list, jo);
    e = cudaGetLastError();
    if (e != cudaSuccess || !scratch) return e;
    const auto lf = jo.jac ? k_step_tan_list_f32<true> : k_step_tan_list_f32<false>;
    const void* fl = (const void*)lf;
    e = cudaFuncSetAttribute(fl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fl, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // the list's length is on the device: one resident wave strides over it
    long long bl = (long long)sm_count() * per_sm;
    if (bl > work) bl = work;
    lf<<<(int)bl, kThreads, smem, st>>>(k, scratch, list, rho, B, H, ue, ui, gue, gui, g_rho, g_B, g_H, g_ue, g_ui,
                                        jo);
    return cudaGetLastError();
}

}  // namespace

cool_status launch_step_bwd_f32(const cool_table* t, const cool_params* p, long long n, const float* rho,
                                const float* B, const float* H, const float* ue, const float* ui,
                                const float* gue, const float* gui, float* g_rho, float* g_B, float* g_H,
                                float* g_ue, float* g_ui, float* g_lb, float* g_ls, float* g_lc, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    const bool tbl = g_lb || g_ls || g_lc;
    if (t->dev.fmt != 0 || p->fp64_critical || p->n_sub > kMaxSub) return COOL_EUNSUPPORTED;
    StepK k;
    fill_stepk(t, p, k);
    const bool sms = p->n_sub <= kSmemSub;
    const bool impl = p->mode == COOL_IMPLICIT_STIFF;
    // implicit mode: stiff cells deferred to a list (n + 1 words: the
    // count, then the indices) stepped by a second pass with the solve --
    // for the input gradients, and for the table adjoints with the state in
    // shared memory (n_sub <= 8); without a list every lane solves its own
    unsigned* scratch = nullptr;
    bool owned = false;
    if (impl && (!tbl || sms) && n < 0xffffffffll) {
        cudaError_t em = cudaSuccess;
        scratch = list_for_call(st, n, &owned, &em);
        if (em != cudaSuccess) return set_cuda_error(em);
    }
    const bool defer = scratch != nullptr;
    // without table adjoints: forward tangents (the table parts and the
    // window in shared memory); with them: the recorded forward and the
    // reverse sweep (plus the partial sums and the sub-cycles' state: the
    // implicit root too where this pass solves)
    const bool solves = impl && !defer;
    size_t smem = (size_t)(smem_table_floats(k) + Fmt<0>::W * kThreads) * sizeof(float);
    if (tbl) {
        smem += (size_t)(t->dev.n[3] + ((t->dev.n[4] * t->dev.n[4] + 3) & ~3)) * sizeof(float);
        const int nsf = solves ? kStateFloats : kStateFloats - 1;
        if (sms) smem += (size_t)kSmemSub * kThreads * (nsf * sizeof(float) + 1);
    }
    const TanFn tf = !impl  ? k_step_tan_f32<false, false, false>
                     : defer ? k_step_tan_f32<false, true, false>
                             : k_step_tan_f32<true, false, false>;
    const BwdFn fb = sms ? (!impl ? k_step_bwd_f32<true, false, 0>
                            : defer ? k_step_bwd_f32<true, false, 1> : k_step_bwd_f32<true, true, 0>)
                         : (impl ? k_step_bwd_f32<false, true, 0> : k_step_bwd_f32<false, false, 0>);
    const void* fn = !tbl ? (const void*)tf : (const void*)fb;
    const JacOut none{nullptr, nullptr, nullptr, 0};
    cudaError_t e = launch_bwd(k, n, fn, tf, fb, tbl, smem, scratch, rho, B, H, ue, ui, gue, gui, g_rho, g_B, g_H,
                               g_ue, g_ui, g_lb, g_ls, g_lc, none, st);
    if (owned) {
        cudaError_t ef = cudaFreeAsync(scratch, st);
        if (e == cudaSuccess) e = ef;
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

cool_status launch_step_fwd_jac_f32(const cool_table* t, const cool_params* p, long long n, const float* rho,
                                    const float* B, const float* H, const float* ue, const float* ui, float* ue_out,
                                    float* ui_out, float* jac, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    if (t->dev.fmt != 0 || p->fp64_critical || p->n_sub > kMaxSub) return COOL_EUNSUPPORTED;
    StepK k;
    fill_stepk(t, p, k);
    const bool impl = p->mode == COOL_IMPLICIT_STIFF;
    // implicit mode: stiff cells deferred to the list kernel, as in cool_step_bwd
    unsigned* scratch = nullptr;
    bool owned = false;
    if (impl && n < 0xffffffffll) {
        cudaError_t em = cudaSuccess;
        scratch = list_for_call(st, n, &owned, &em);
        if (em != cudaSuccess) return set_cuda_error(em);
    }
    const bool defer = scratch != nullptr;
    const size_t smem = (size_t)(smem_table_floats(k) + Fmt<0>::W * kThreads) * sizeof(float);
    const TanFn tf = !impl  ? k_step_tan_f32<false, false, true>
                     : defer ? k_step_tan_f32<false, true, true>
                             : k_step_tan_f32<true, false, true>;
    const JacOut jo{ue_out, ui_out, jac, n};
    cudaError_t e = launch_bwd(k, n, (const void*)tf, tf, nullptr, false, smem, scratch, rho, B, H, ue, ui, nullptr,
                               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, jo, st);
    if (owned) {
        cudaError_t ef = cudaFreeAsync(scratch, st);
        if (e == cudaSuccess) e = ef;
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

cool_status launch_jac_contract_f32(long long n, const float* jac, const float* gue, const float* gui, float* g_rho,
                                    float* g_B, float* g_H, float* g_ue, float* g_ui, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    long long blocks = (n + kThreads - 1) / kThreads;
    const long long cap = (long long)sm_count() * 8;   // streaming: a few waves of 256 threads per SM
    if (blocks > cap) blocks = cap;
    k_jac_contract<<<(int)blocks, kThreads, 0, st>>>(n, jac, gue, gui, g_rho, g_B, g_H, g_ue, g_ui);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

}  // namespace cool
