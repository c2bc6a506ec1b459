// cool_sur_step.cu -- the cooling step with the learned surrogate of the
// synchrotron channel (cool_surrogate_infer; not in the paper).
#include <cuda_bf16.h>

#include "cool_mlp.cuh"
#include "cool_mma.cuh"
#include "cool_step_common.cuh"
#include "cool_bridge.cuh"

namespace cool {
namespace {

// ---------------------------------------------------------------------------
// The step with the learned surrogate (cool_surrogate_infer): the network
// replaces the synchrotron-table read.  A CTA steps a tile of 128 cells (one
// per thread); each sub-cycle the tile's four log2 coordinates (H, B, n_e,
// T_e, normalised) form a 128 x 16 bf16 operand and the two hidden layers
// run as tcgen05.mma (FP32 in TMEM), the 128 -> 1 output on the CUDA cores.
// Cells whose 4-D table cell carries the fallback bit read the table instead;
// a sub-cycle where every cell of the tile falls back skips the network.
// Explicit mode, FP32 fields, FP32 table.
// ---------------------------------------------------------------------------
struct SurK {
    const __nv_bfloat16* W1b;
    const __nv_bfloat16* W2b;
    const float* p;
    float mean, std;
    float l0[4], sc[4];        // x = (l - l0) sc - 1, sc = 2 / span
    float xs;                  // normalised log2 of the K2 switch temperature
    const uint32_t* mask;      // fallback bits (nullable: never fall back)
};

constexpr int kSurT = 128;

// Table fallback: the two T_e nodes j, j + 1 of the 8 (H, B, n_e) corners
// (both in block j / 7 of the FP32 layout, one 32-byte sector per corner),
// collapsed trilinearly into v[0], v[1]; kept while the cell stays in T_e
// interval j (the common case from one sub-cycle to the next).
__device__ __forceinline__ void table_pair(const CellC& c, int j, float (&v)[2]) {
    const float* p = reinterpret_cast<const float*>(c.row) + (j / 7) * 8 + (j % 7);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float* q = p + e;
        const float a = lerpf(lerpf(__ldg(q), __ldg(q + c.oN), c.wn),
                              lerpf(__ldg(q + c.oB), __ldg(q + c.oB + c.oN), c.wn), c.wb);
        const float* r = q + c.oH;
        const float b = lerpf(lerpf(__ldg(r), __ldg(r + c.oN), c.wn),
                              lerpf(__ldg(r + c.oB), __ldg(r + c.oB + c.oN), c.wn), c.wb);
        v[e] = lerpf(a, b, c.wh);
    }
}

// Shared memory of the surrogate step: axes and brems channel (the Coulomb
// table is read through L1), then the network operands.
__host__ __device__ __forceinline__ int sur_table_floats(const StepK& k) {
    return (k.axes_floats + k.tab.n[3] + 3) & ~3;
}

__global__ void __launch_bounds__(kSurT) k_step_surrogate(StepK k, SurK m, long long n, const float* __restrict__ rho_in,
                                                         const float* __restrict__ B_in, const float* __restrict__ H_in,
                                                         const float* ue_in, const float* ui_in, float* ue_out,
                                                         float* ui_out, float* qc_out, float* qx_out,
                                                         cool_counters* cnt, unsigned* err) {
    extern __shared__ __align__(1024) float sms[];
    for (int i = threadIdx.x; i < k.axes_floats; i += blockDim.x) sms[i] = k.tab.axes[i];
    for (int i = threadIdx.x; i < k.tab.n[3]; i += blockDim.x) sms[k.axes_floats + i] = k.tab.lb[i];
    Smem S;
    S.ax = sms;
    S.lb = sms + k.axes_floats;
    S.lc = k.tab.lc;
    S.tn = nullptr;   // the T_e interval records are not staged here (no cool_energy)
    unsigned char* W1s = reinterpret_cast<unsigned char*>(sms + sur_table_floats(k));
    unsigned char* W2s = W1s + 128 * 16 * 2;
    unsigned char* H1s = W2s + 128 * 128 * 2;
    // X is consumed by the first product before H1 is written, and written
    // again only after the second product has consumed H1: they share space
    unsigned char* Xs = H1s;
    float* Ps = reinterpret_cast<float*>(H1s + 128 * 128 * 2);        // b1, b2, w3, b3
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Ps + 3 * 128 + 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(Ps + 3 * 128 + 6);
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    mma::load_kmajor(W1s, m.W1b, 128, 16);
    mma::load_kmajor(W2s, m.W2b, 128, 128);
    Ps[t] = m.p[kP_b1 + t];
    Ps[128 + t] = m.p[kP_b2 + t];
    Ps[256 + t] = m.p[kP_w3 + t];
    if (t == 0) Ps[384] = m.p[kP_b3];
    if (t == 0) {
        mma::mbar_init(mma::smem_addr(mbar), 1);
        mma::fence_mbar_init();
    }
    if (warp == 0) mma::tmem_alloc(mma::smem_addr(tslot), 128);
    mma::operands_ready();
    const uint32_t tm = *tslot;
    const uint32_t mb = mma::smem_addr(mbar);
    uint32_t phase = 0;
    const DevTable& T = k.tab;
    const int nB1 = T.n[1] - 1, nN1 = T.n[2] - 1, nT1 = T.n[3] - 1;
    const long long ntiles = (n + kSurT - 1) / kSurT;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long i = tile * kSurT + t;
        const bool live = i < n;
        float rho = 1.f, B = 1e-3f, H = 1.f, ue = 1e-3f, ui = 1e-3f;
        if (live) {
            rho = rho_in[i]; B = B_in[i]; H = H_in[i]; ue = ue_in[i]; ui = ui_in[i];
        }
        const float ue0 = ue, ui0 = ui;
        const bool valid = live && isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui) &&
                           rho > 0.f && ue > 0.f && ui > 0.f && B >= 0.f && H >= 0.f;
        if (!valid) { rho = 1.f; B = 1e-3f; H = 1.f; ue = 1e-3f; ui = 1e-3f; }
        unsigned clamp = 0u, band = 0u, fallback = 0u;
        const float ne = rho * k.s_n, Bg = B * k.s_B, Hc = H * k.s_H;
        const float inv_e = k.s_Te / rho, inv_i = k.s_Ti / rho, kr = k.s_K / rho;
        CellC c;
        float xH, xB, xN;
        int jh, jb, jn;
        {
            Sel sh = select_axis(S.ax + T.axis_off[0], T.n[0], T.inv_dl[0], Hc, clamp);
            Sel sb = select_axis(S.ax + T.axis_off[1], T.n[1], T.inv_dl[1], Bg, clamp);
            Sel sn = select_axis(S.ax + T.axis_off[2], T.n[2], T.inv_dl[2], ne, clamp);
            jh = sh.j; jb = sb.j; jn = sn.j;
            const int rowf = 8 * T.nblk;
            c.oN = rowf;
            c.oB = rowf * T.n[2];
            c.oH = c.oB * T.n[1];
            c.row = T.lsb + (long long)((sh.j * T.n[1] + sb.j) * T.n[2] + sn.j) * rowf;
            c.wh = __saturatef(sh.r * T.inv_dl[0]);
            c.wb = __saturatef(sb.r * T.inv_dl[1]);
            c.wn = __saturatef(sn.r * T.inv_dl[2]);
            const float lH = lg2a(Hc), lB = lg2a(Bg), lN = lg2a(ne);
            xH = fminf(fmaxf(fmaf(lH - m.l0[0], m.sc[0], -1.f), -1.f), 1.f);
            xB = fminf(fmaxf(fmaf(lB - m.l0[1], m.sc[1], -1.f), -1.f), 1.f);
            xN = fminf(fmaxf(fmaf(lN - m.l0[2], m.sc[2], -1.f), -1.f), 1.f);
            c.ls_off = k.l_hs_e;
            c.lb_off = fmaf(2.f, lN, k.l_hs_e);
            c.lbb_off = k.l_bb - lH;
            c.tau_sca = k.two_sigT * ne * Hc;
        }
        const float lcc_off = c.lb_off;
        const int nC = T.n[4];
        const float* axC = S.ax + T.axis_off[4];
        const int nT = T.n[3];
        const float* axT = S.ax + T.axis_off[3];
        float sum_q = 0.f, sum_x = 0.f;
        int pj = -1;             // T_e interval of the held fallback pair
        float pv[2] = {0.f, 0.f};
        for (int sub = 0; sub < k.n_sub; ++sub) {
            // ---- (i) Coulomb exchange (the forward kernel's FP32 form) ----
            const float Te = ue * inv_e, Ti = ui * inv_i;
            const Sel se = select_axis(axC, nC, T.inv_dl[4], Te, clamp);
            const Sel si = select_axis(axC, nC, T.inv_dl[4], Ti, clamp);
            const float we = __saturatef(se.r * T.inv_dl[4]), wi = __saturatef(si.r * T.inv_dl[4]);
            const float* row = S.lc + si.j * nC + se.j;
            const float lC = lerpf(lerpf(__ldg(row), __ldg(row + 1), we),
                                   lerpf(__ldg(row + nC), __ldg(row + nC + 1), we), wi);
            const float rate = ex2a(fminf(lC + lcc_off, 126.f));
            band |= fabsf(Te - Ti) <= k.eq_band * Ti ? 1u : 0u;
            const float pe = k.ce * ue;
            const float ee = fmaf(k.ce, ue, -pe);
            const float D = fmaf(k.ci, ui, -pe) - ee;
            float X = rate * (kr * D);
            const float lim = k.clamp * fabsf(D * k.inv_cec);
            X = fabsf(X) > lim ? copysignf(lim, X) : X;
            ue += X;
            ui -= X;
            sum_x += X;
            // ---- (ii) cooling: network or table for the synchrotron channel ----
            const float Te1 = ue * inv_e;
            const Sel st = select_axis(axT, nT, T.inv_dl[3], Te1, clamp);
            const float wt = __saturatef(st.r * T.inv_dl[3]);
            const float lT = axT[2 * nT + st.j] + st.r;
            bool flagged = false;
            if (m.mask) {
                const long long cell = (((long long)jh * nB1 + jb) * nN1 + jn) * nT1 + st.j;
                flagged = (m.mask[cell >> 5] >> (cell & 31)) & 1u;
            }
            float Ls;
            if (__syncthreads_or(valid && !flagged)) {
                const float xT = fminf(fmaxf(fmaf(lT - m.l0[3], m.sc[3], -1.f), -1.f), 1.f);
                {
                    const float xv[4] = {xH, xB, xN, xT};
                    __align__(16) __nv_bfloat16 tmp[16];
                    input_row(xv, m.xs, tmp);
                    *reinterpret_cast<uint4*>(Xs + mma::kmajor_offset(t, 0, 16)) = *reinterpret_cast<const uint4*>(tmp);
                    *reinterpret_cast<uint4*>(Xs + mma::kmajor_offset(t, 8, 16)) =
                        *reinterpret_cast<const uint4*>(tmp + 8);
                }
                mma::operands_ready();
                if (t == 0) {
                    mma::issue(tm, Xs, W1s, 16, 128);
                    mma::commit(mb);
                }
                mma::mma_done(mb, phase, err);
                phase ^= 1u;
#pragma unroll 1
                for (int c0 = 0; c0 < 128; c0 += 32) {
                    float z[32];
                    mma::tmem_ld32(tm + lane_off + c0, z);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float zz = z[j] + Ps[c0 + j];
                        z[j] = zz * mma::sigm(zz);
                    }
                    mma::st_row32(H1s, t, c0, 128, z);
                }
                mma::operands_ready();
                // Z2 overwrites Z1's columns: every thread has read Z1
                if (t == 0) {
                    mma::issue(tm, H1s, W2s, 128, 128);
                    mma::commit(mb);
                }
                mma::mma_done(mb, phase, err);
                phase ^= 1u;
                float yh = Ps[384];
#pragma unroll 1
                for (int c0 = 0; c0 < 128; c0 += 32) {
                    float z[32];
                    mma::tmem_ld32(tm + lane_off + c0, z);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float zz = z[j] + Ps[128 + c0 + j];
                        yh = fmaf(zz * mma::sigm(zz), Ps[256 + c0 + j], yh);
                    }
                }
                Ls = fmaf(m.std, yh, m.mean);
            } else {
                Ls = 0.f;
            }
            if (flagged) {
                if (st.j != pj) {
                    table_pair(c, st.j, pv);
                    pj = st.j;
                }
                Ls = lerpf(pv[0], pv[1], wt);
                fallback = 1u;
            }
            const float Lb = lerpf(S.lb[st.j], S.lb[st.j + 1], wt) + c.lb_off;
            const float q = bridge_energy(c, Ls + c.ls_off, Lb, lT);
            const float du = fminf(q, k.limiter * ue);
            ue -= du;
            sum_q += du;
        }
        if (live) {
            if (valid) {
                ue_out[i] = ue;
                ui_out[i] = ui;
                if (qc_out) qc_out[i] = sum_q;
                if (qx_out) qx_out[i] = sum_x;
            } else {
                ue_out[i] = ue0;
                ui_out[i] = ui0;
                if (qc_out) qc_out[i] = 0.f;
                if (qx_out) qx_out[i] = 0.f;
            }
        }
        if (cnt) {
            const unsigned f = !live ? 0u : (!valid ? 2u : (clamp | (band << 3) | (fallback << 5)));
            const unsigned full = __activemask();
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                if (b == 2 || b == 4) continue;
                const unsigned msk = __ballot_sync(full, (f >> b) & 1u);
                if (msk && (threadIdx.x & 31) == (__ffs(full) - 1)) {
                    unsigned long long* dst = b == 0 ? &cnt->n_clamped : b == 1 ? &cnt->n_nonfinite
                                            : b == 3 ? &cnt->n_fp64_coulomb : &cnt->n_fallback;
                    atomicAdd(dst, (unsigned long long)__popc(msk));
                }
            }
        }
    }
    mma::fence_before_sync();
    __syncthreads();
    if (warp == 0) mma::tmem_dealloc(tm, 128);
}


}  // namespace

cool_status launch_step_surrogate(const cool_surrogate* sg, const cool_table* t, const cool_params* p, long long n,
                                  const float* rho, const float* B, const float* H, const float* ue,
                                  const float* ui, float* ue_o, float* ui_o, float* qc, float* qx,
                                  cool_counters* cnt, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    if (t->dev.fmt != 0 || p->mode != COOL_EXPLICIT_LIMITED || p->fp64_critical) return COOL_EUNSUPPORTED;
    StepK k;
    fill_stepk(t, p, k);
    SurK m;
    m.W1b = sg->d_W1b;
    m.W2b = sg->d_W2b;
    m.p = sg->d_p;
    m.mean = (float)sg->mean;
    m.std = (float)sg->std;
    for (int d = 0; d < 4; ++d) {
        m.l0[d] = (float)sg->l0[d];
        m.sc[d] = (float)(2.0 / sg->span[d]);
    }
    m.xs = (float)sg->x_switch;
    m.mask = sg->d_mask;
    const size_t smem = (size_t)sur_table_floats(k) * sizeof(float) + 128 * 16 * 2 + 128 * 128 * 2 +
                        128 * 128 * 2 + (3 * 128 + 8) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_step_surrogate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    long long tiles = (n + kSurT - 1) / kSurT;
    // resident blocks per SM from the kernel's shared memory and registers
    // (the TMEM allows 4 blocks of 128 columns)
    int dev = 0, smem_sm = 0, smem_rsv = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa;
    int regs = 128;
    if (cudaFuncGetAttributes(&fa, k_step_surrogate) == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
    int per_sm = smem_sm / (int)(smem + smem_rsv);
    const int by_regs = 65536 / (regs * kSurT);
    if (by_regs < per_sm) per_sm = by_regs;
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
    long long cap = (long long)sm_count() * per_sm;
    long long blocks = tiles < cap ? tiles : cap;
    k_step_surrogate<<<(int)blocks, kSurT, smem, st>>>(k, m, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt,
                                                        sg->d_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

}  // namespace cool
