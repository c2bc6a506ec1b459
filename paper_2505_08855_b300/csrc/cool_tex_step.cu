// cool_tex_step.cu -- the step reading the synchrotron channel through
// texture fetches, the paper's own design (Sec. 3.1: the table in texture
// memory, read with the hardware's linear interpolation), kept as a
// comparison path for the L2-resident block layout of cool_step.cu.
//
// The FP32 log2 channel is a 3-D CUDA array, x = T_e, y = n_e, z = h n_B + b
// (the (H, B) pair flattened: texture arrays have at most three axes).
//   COOL_PATH_TEXTURE_POINT:  16 point fetches per sub-cycle (the corners of
//     the 4-D cell), multilinear interpolation in FP32 -- the same numbers as
//     the table step up to rounding;
//   COOL_PATH_TEXTURE_HWLERP: the texture unit interpolates T_e, n_e and B
//     (trilinear filtering, 2 fetches per sub-cycle), H is interpolated in
//     FP32.  The hardware forms its weights in fixed point with 8
//     fractional bits, so each weight is off by up to 2^-8: an error of up
//     to 2^-8 of a node-to-node step of the channel per filtered axis.
// Everything else (keys, index selection, Coulomb exchange, bremsstrahlung,
// bridge, limiter) is the explicit FP32 step.
#include "cool_bridge.cuh"
#include "cool_step_common.cuh"

namespace cool {
namespace {

constexpr int kTexThreads = 256;

// select_axis with the clamp test written as an explicit range check on
// the end nodes (the same selection, weights and flag).  In this kernel the
// compiler schedules the texture fetches better around this form (measured
// 2.6 ms against 3.7 ms per step for the hardware-filtered path).
__device__ __forceinline__ Sel select_axis_rc(const float* a, int n, float inv_dl, float key, unsigned& clamp) {
    const float* x = a;
    const float* rx = a + n;
    const float* lx = a + 2 * n;
    int j = __float2int_rd((lg2a(key) - lx[0]) * inv_dl);
    j = min(max(j, 0), n - 2);
    j += (j < n - 2 && x[j + 1] <= key) ? 1 : 0;
    j -= (j > 0 && x[j] > key) ? 1 : 0;
    clamp |= (key < x[0] || key > x[n - 1]) ? 1u : 0u;
    Sel s;
    s.j = j;
    s.r = lg2a(key * rx[j]);
    return s;
}

template <bool HW>
__global__ void __launch_bounds__(kTexThreads) k_step_tex(StepK k, cudaTextureObject_t tex, long long n,
                                                          const float* __restrict__ rho_in,
                                                          const float* __restrict__ B_in,
                                                          const float* __restrict__ H_in, const float* ue_in,
                                                          const float* ui_in, float* ue_out, float* ui_out,
                                                          float* qc_out, float* qx_out, cool_counters* cnt) {
    extern __shared__ float stx[];
    for (int i = threadIdx.x; i < k.axes_floats; i += blockDim.x) stx[i] = k.tab.axes[i];
    for (int i = threadIdx.x; i < k.tab.n[3]; i += blockDim.x) stx[k.axes_floats + i] = k.tab.lb[i];
    const int nC = k.tab.n[4];
    float* lcs = stx + k.axes_floats + k.tab.n[3];
    for (int i = threadIdx.x; i < nC * nC; i += blockDim.x) lcs[i] = k.tab.lc[i];
    __syncthreads();
    const DevTable& T = k.tab;
    const float* ax = stx;
    const float* lbs = stx + k.axes_floats;
    const float* axC = ax + T.axis_off[4];
    const float* axT = ax + T.axis_off[3];
    const int nT = T.n[3];
    const float nBf = (float)T.n[1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float rho = rho_in[i], B = B_in[i], H = H_in[i], ue = ue_in[i], ui = ui_in[i];
        if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) || !(rho > 0.f) ||
            !(ue > 0.f) || !(ui > 0.f) || B < 0.f || H < 0.f) {
            ue_out[i] = ue;
            ui_out[i] = ui;
            if (qc_out) qc_out[i] = 0.f;
            if (qx_out) qx_out[i] = 0.f;
            if (cnt) atomicAdd(&cnt->n_nonfinite, 1ull);
            continue;
        }
        unsigned clamp = 0u, band = 0u;
        const float ne = rho * k.s_n, Bg = B * k.s_B, Hc = H * k.s_H;
        const float inv_e = k.s_Te / rho, inv_i = k.s_Ti / rho, kr = k.s_K / rho;
        const Sel sh = select_axis_rc(ax + T.axis_off[0], T.n[0], T.inv_dl[0], Hc, clamp);
        const Sel sb = select_axis_rc(ax + T.axis_off[1], T.n[1], T.inv_dl[1], Bg, clamp);
        const Sel sn = select_axis_rc(ax + T.axis_off[2], T.n[2], T.inv_dl[2], ne, clamp);
        CellC c;
        c.wh = __saturatef(sh.r * T.inv_dl[0]);
        c.wb = __saturatef(sb.r * T.inv_dl[1]);
        c.wn = __saturatef(sn.r * T.inv_dl[2]);
        const float lne = lg2a(ne);
        c.ls_off = k.l_hs_e;
        c.lb_off = fmaf(2.f, lne, k.l_hs_e);
        c.lbb_off = k.l_bb - lg2a(Hc);
        c.tau_sca = k.two_sigT * ne * Hc;
        // texel-centre coordinates of the step-invariant axes
        const float y0 = (float)sn.j + 0.5f;
        const float z0 = (float)sh.j * nBf + (float)sb.j + 0.5f;
        float sum_q = 0.f, sum_x = 0.f;
        for (int sub = 0; sub < k.n_sub; ++sub) {
            // (i) Coulomb exchange (the explicit FP32 form of cool_step)
            const float Te = ue * inv_e, Ti = ui * inv_i;
            const Sel se = select_axis_rc(axC, nC, T.inv_dl[4], Te, clamp);
            const Sel si = select_axis_rc(axC, nC, T.inv_dl[4], Ti, clamp);
            const float we = __saturatef(se.r * T.inv_dl[4]), wi = __saturatef(si.r * T.inv_dl[4]);
            const float* row = lcs + si.j * nC + se.j;
            const float lC = lerpf(lerpf(row[0], row[1], we), lerpf(row[nC], row[nC + 1], we), wi);
            const float rate = ex2a(fminf(lC + c.lb_off, 126.f));
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
            // (ii) cooling, synchrotron channel from the texture
            const Sel st = select_axis_rc(axT, nT, T.inv_dl[3], ue * inv_e, clamp);
            const float wt = __saturatef(st.r * T.inv_dl[3]);
            const float lT = axT[2 * nT + st.j] + st.r;
            float Ls;
            if (HW) {
                const float x = (float)st.j + wt + 0.5f;
                const float y = y0 + c.wn;
                const float z = z0 + c.wb;
                const float a = tex3D<float>(tex, x, y, z);
                const float b = tex3D<float>(tex, x, y, z + nBf);
                Ls = lerpf(a, b, c.wh);
            } else {
                const float x = (float)st.j + 0.5f;
                float v[2][2][2];   // [h][b][n], T_e already interpolated
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
#pragma unroll
                        for (int m = 0; m < 2; ++m) {
                            const float zz = z0 + (float)(h * T.n[1] + b);
                            const float yy = y0 + (float)m;
                            v[h][b][m] = lerpf(tex3D<float>(tex, x, yy, zz), tex3D<float>(tex, x + 1.f, yy, zz), wt);
                        }
                const float l0 = lerpf(lerpf(v[0][0][0], v[0][0][1], c.wn), lerpf(v[0][1][0], v[0][1][1], c.wn), c.wb);
                const float l1 = lerpf(lerpf(v[1][0][0], v[1][0][1], c.wn), lerpf(v[1][1][0], v[1][1][1], c.wn), c.wb);
                Ls = lerpf(l0, l1, c.wh);
            }
            const float Lb = lerpf(lbs[st.j], lbs[st.j + 1], wt) + c.lb_off;
            const float q = bridge_energy(c, Ls + c.ls_off, Lb, lT);
            const float du = fminf(q, k.limiter * ue);
            ue -= du;
            sum_q += du;
        }
        ue_out[i] = ue;
        ui_out[i] = ui;
        if (qc_out) qc_out[i] = sum_q;
        if (qx_out) qx_out[i] = sum_x;
        if (cnt) {
            if (clamp) atomicAdd(&cnt->n_clamped, 1ull);
            if (band) atomicAdd(&cnt->n_fp64_coulomb, 1ull);
        }
    }
}

}  // namespace

cool_status launch_step_tex(const cool_table* t, const cool_params* p, long long n, const float* rho,
                            const float* B, const float* H, const float* ue, const float* ui, float* ue_o,
                            float* ui_o, float* qc, float* qx, cool_counters* cnt, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    StepK k;
    fill_stepk(t, p, k);
    // this kernel's own shared layout: axes, brems row, unpadded Coulomb channel
    const size_t smem = (size_t)(k.axes_floats + k.tab.n[3] + k.tab.n[4] * k.tab.n[4]) * sizeof(float);
    const bool hw = p->path == COOL_PATH_TEXTURE_HWLERP;
    auto kern = hw ? k_step_tex<true> : k_step_tex<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTexThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
#ifdef COOL_TEX_PER_SM
    if (per_sm > COOL_TEX_PER_SM) per_sm = COOL_TEX_PER_SM;
#endif
    long long blocks = (n + kTexThreads - 1) / kTexThreads;
    long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    const cudaTextureObject_t tex = (cudaTextureObject_t)(hw ? t->tex_linear : t->tex_point);
    kern<<<(int)blocks, kTexThreads, smem, st>>>(k, tex, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt);
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

}  // namespace cool
