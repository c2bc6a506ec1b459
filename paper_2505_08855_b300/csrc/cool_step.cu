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
//        u' = u_e - q(u') (Sec. 3.2.1 (ii)): Illinois iterations in FP32, or
//        bisection in log2 u in FP64 with fp64_critical.
//
// FP32 path design (B300):
//   - fields are SoA; 16-byte aligned arrays are read and written with
//     128-bit accesses, staged per warp in tiles of 128 cells, which warps
//     take in a dynamic order from a per-stream counter;
//   - node arrays, the 1-D bremsstrahlung and the 2-D Coulomb channels live
//     in shared memory (loaded once per persistent block; Coulomb rows at a
//     stride of 5 mod 32 against bank conflicts, one 16-byte record per
//     cooling T_e interval);
//   - the 4-D synchrotron channel stays in global memory, L2-resident by its
//     reuse: the step-invariant H, B, n_e axes are collapsed once per visited
//     T_e block (8 corners x one 32-byte block of nodes, T_e fastest in
//     memory, two L2 round trips), so a sub-cycle that stays in its block
//     reads no table memory;
//   - index selection without node loads (a log2 guess confirmed by its
//     weight); the few cells with a key near a node are redone after their
//     tile with node compares, so every index equals the node-compare rule;
//   - the bridge is evaluated in log2 space so that no intermediate
//     over/underflows FP32 over the table's 60-decade range.
#include <string.h>

#include "cool_step_kernel.cuh"

namespace cool {
namespace {


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
            c.jt = -1;
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
                    double u1;
                    if (implicit_fp64(k, c, r, ue, u1, nan64(), nan64())) {
                        du = ue - u1;
                    } else {
                        fail = 1u;
                        du = k.limiter * ue;
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

// axis 0..4: select_axis (node compares, the oracle's rule); 5..9:
// select_sub on axes 0..4 (the same rule as the step computes it)
__global__ void k_debug_lookup(StepK k, int axis, long long n, const float* keys, int* idx, float* w) {
    const DevTable& T = k.tab;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned clamp = 0u;
        if (axis < 5) {
            Sel s = select_axis(T.axes + T.axis_off[axis], T.n[axis], T.inv_dl[axis], keys[i], clamp);
            idx[i] = s.j;
            w[i] = __saturatef(s.r * T.inv_dl[axis]);
        } else {
            const int a = axis - 5;
            const float* rx = T.axes + T.axis_off[a] + T.n[a];
            SelW s;
            unsigned near = 0u;
            switch (a) {
            case 0: s = select_sub<0, false>(k, rx, T.n[a], T.inv_dl[a], keys[i], clamp, near); break;
            case 1: s = select_sub<1, false>(k, rx, T.n[a], T.inv_dl[a], keys[i], clamp, near); break;
            case 2: s = select_sub<2, false>(k, rx, T.n[a], T.inv_dl[a], keys[i], clamp, near); break;
            case 3: s = select_sub<3, false>(k, rx, T.n[a], T.inv_dl[a], keys[i], clamp, near); break;
            default: s = select_sub<4, false>(k, rx, T.n[a], T.inv_dl[a], keys[i], clamp, near); break;
            }
            // near a node: node compares, as the step redoes such a cell
            if (near) {
                const Sel e = select_axis(rx - T.n[a], T.n[a], T.inv_dl[a], keys[i], clamp);
                s.j = e.j;
                s.w = __saturatef(e.r * T.inv_dl[a]);
            }
            idx[i] = s.j;
            w[i] = s.w;
        }
    }
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
    const int fmt = t->dev.fmt;
    if (fmt < 0 || fmt > 4) return COOL_EUNSUPPORTED;
    // shared memory: the table parts, the window (one row per node of a
    // block of this format) and the warps' field tiles
    size_t smem = (size_t)(smem_table_floats(k) + fmt_nodes(fmt) * kThreads) * sizeof(float);
    if (vec) smem += (size_t)kWarps * (disk ? 6 : 5) * kWarpCells * sizeof(float);
    if (vec && (p->fp64_critical || p->mode == COOL_IMPLICIT_STIFF))
        smem += (size_t)kWarps * kWarpCells;   // the deferred cells' lists
    // the kernels are indexed by implicit | fp64_critical << 1 | counters << 2
    // (template bits 0, 1 and 3); 16-bit formats come from cool_step_f16.cu
    // and cool_step_f16s.cu
#define COOL_KV(V, F) k_step_f32<V, F, 0>, k_step_f32<V, F, 1>, k_step_f32<V, F, 2>, k_step_f32<V, F, 3>, \
                      k_step_f32<V, F, 8>, k_step_f32<V, F, 9>, k_step_f32<V, F, 10>, k_step_f32<V, F, 11>
    static const StepKernelFn table_v[8] = {COOL_KV(true, 0)};
    // implicit / fp64_critical with the flagged cells listed (template bit 6)
    // and the list kernels that step them
    static const StepKernelFn table_lv[8] = {nullptr, k_step_f32<true, 0, 65>, k_step_f32<true, 0, 66>,
                                             k_step_f32<true, 0, 67>, nullptr, k_step_f32<true, 0, 73>,
                                             k_step_f32<true, 0, 74>, k_step_f32<true, 0, 75>};
    static const StepKernelFn list_v[8] = {nullptr, k_step_list_f32<0, 1>, k_step_list_f32<0, 2>,
                                           k_step_list_f32<0, 3>, nullptr, k_step_list_f32<0, 9>,
                                           k_step_list_f32<0, 10>, k_step_list_f32<0, 11>};
    static const StepKernelFn table_s[8] = {COOL_KV(false, 0)};
#undef COOL_KV
    // disk geometry (template bit 2): FP32 table only
#define COOL_KD(V) k_step_f32<V, 0, 4>, k_step_f32<V, 0, 5>, k_step_f32<V, 0, 6>, k_step_f32<V, 0, 7>, \
                   k_step_f32<V, 0, 12>, k_step_f32<V, 0, 13>, k_step_f32<V, 0, 14>, k_step_f32<V, 0, 15>
    static const StepKernelFn disk_v[8] = {COOL_KD(true)};
    static const StepKernelFn disk_s[8] = {COOL_KD(false)};
    static const StepKernelFn disk_lv[8] = {nullptr, k_step_f32<true, 0, 69>, k_step_f32<true, 0, 70>,
                                            k_step_f32<true, 0, 71>, nullptr, k_step_f32<true, 0, 77>,
                                            k_step_f32<true, 0, 78>, k_step_f32<true, 0, 79>};
    static const StepKernelFn disk_list_v[8] = {nullptr, k_step_list_f32<0, 5>, k_step_list_f32<0, 6>,
                                                k_step_list_f32<0, 7>, nullptr, k_step_list_f32<0, 13>,
                                                k_step_list_f32<0, 14>, k_step_list_f32<0, 15>};
#undef COOL_KD
    // the paper's table layout (template bit 4): explicit, FP32 table, no geometry
    static const StepKernelFn tot_v[2] = {k_step_f32<true, 0, 16>, k_step_f32<true, 0, 24>};
    static const StepKernelFn tot_s[2] = {k_step_f32<false, 0, 16>, k_step_f32<false, 0, 24>};
    if (disk && (fmt != 0 || !r)) return COOL_EUNSUPPORTED;
    const bool tot = p->path == COOL_PATH_QTOTAL;
    if (tot && (disk || fmt != 0 || p->mode != COOL_EXPLICIT_LIMITED || p->fp64_critical || !t->dev.lst))
        return COOL_EUNSUPPORTED;
    const int var = (p->mode == COOL_IMPLICIT_STIFF ? 1 : 0) | (p->fp64_critical ? 2 : 0) | (cnt ? 4 : 0);
    const void* fn = tot    ? (const void*)(vec ? tot_v[cnt ? 1 : 0] : tot_s[cnt ? 1 : 0])
                     : disk ? (const void*)(vec ? disk_v[var] : disk_s[var])
                     : fmt == 0 ? (const void*)(vec ? table_v[var] : table_s[var])
                     : (fmt <= 2 ? step_kernel_f16(fmt, vec, var) : step_kernel_f16s(fmt, vec, var));
    if (!fn) return COOL_EUNSUPPORTED;
    // implicit mode and fp64_critical on the FP32 table with aligned fields
    // (with or without the disk geometry): the flagged cells go to a list
    // (n + 1 words: the count, then the indices), stepped by k_step_list_f32
    // after the tile pass; without a list each warp steps its own
    unsigned* scratch = nullptr;
    bool owned = false;
    if (vec && !tot && fmt == 0 && (var & 3) && n < 0xffffffffll) {
        cudaError_t em = cudaSuccess;
        scratch = list_for_call(st, n, &owned, &em);
        if (em != cudaSuccess) return set_cuda_error(em);
        if (scratch) {
            fn = (const void*)(disk ? disk_lv[var] : table_lv[var]);
            k.dlist = scratch;
        }
    }
    auto tile_pass = [&]() -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        long long work = vec ? (n + kWarps * kWarpCells - 1) / (kWarps * kWarpCells) : (n + kThreads - 1) / kThreads;
        long long cap = (long long)sm_count() * per_sm;  // one resident wave, persistent blocks
        long long blocks = work < cap ? work : cap;
        if (blocks < 1) blocks = 1;
        if (vec && n / kWarpCells > blocks * kWarps) {
            // more tiles than warps: the dynamic tile order (a no-op otherwise)
            k.sched = sched_counter(st);
            if (k.sched) {
                e = cudaMemsetAsync(k.sched, 0, sizeof(unsigned long long), st);
                if (e != cudaSuccess) return e;
            }
        }
        // with cool_table_l2_persist on: the packed 4-D channel as a persisting
        // L2 access-policy window of this launch (the stream's own attributes are
        // left alone)
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        int max_win = 0;
        size_t limit = 0;
        if (t->l2_persist && t->ls_bytes > 0 &&
            cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, t->device) == cudaSuccess &&
            max_win > 0 && cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize) == cudaSuccess && limit > 0) {
            const size_t win = t->ls_bytes < (size_t)max_win ? t->ls_bytes : (size_t)max_win;
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
            attr[0].val.accessPolicyWindow.base_ptr = (void*)t->dev.lsb;
            attr[0].val.accessPolicyWindow.num_bytes = win;
            attr[0].val.accessPolicyWindow.hitRatio = limit >= win ? 1.f : (float)limit / (float)win;
            attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
            attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
        }
        void* args[] = {&k, &n, &rho, &B, &H, &ue, &ui, &ue_o, &ui_o, &qc, &qx, &cnt, &r};
        e = cudaLaunchKernelExC(&cfg, fn, args);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    };
    cudaError_t e = tile_pass();
    if (scratch) {
        if (e == cudaSuccess) {
            // the listed cells: one resident wave strides over the list,
            // whose length is on the device
            const StepKernelFn fl = disk ? disk_list_v[var] : list_v[var];
            const size_t sl = (size_t)(smem_table_floats(k) + fmt_nodes(fmt) * kThreads) * sizeof(float);
            e = cudaFuncSetAttribute((const void*)fl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
            int pl = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl, (const void*)fl, kThreads, sl);
            if (e == cudaSuccess) {
                if (pl < 1) pl = 1;
                long long bl = (long long)sm_count() * pl;
                const long long need = (n + kThreads - 1) / kThreads;
                if (bl > need) bl = need;
                fl<<<(int)bl, kThreads, sl, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt, r);
                e = cudaGetLastError();
            }
        }
        if (owned) {
            const cudaError_t ef = cudaFreeAsync(scratch, st);
            if (e == cudaSuccess) e = ef;
        }
    }
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
    cool_params p;
    cool_params_default(&p);
    StepK k;
    fill_stepk(t, &p, k);
    k_debug_lookup<<<(int)blocks, 256, 0, st>>>(k, axis, n, keys, idx, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}
}  // namespace cool
