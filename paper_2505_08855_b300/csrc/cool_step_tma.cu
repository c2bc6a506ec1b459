// cool_step_tma.cu -- the step with its field staging done by the TMA engine
// (COOL_PATH_TMA_SMEM).
#include "cool_step_cell.cuh"
#include "cool_tma.cuh"

namespace cool {
namespace {

// COOL_PATH_TMA_SMEM: the vector kernel with its field staging done by the
// TMA engine.  Each warp owns two staging buffers (5 fields x 128 cells) and
// two mbarriers; while the warp steps one tile from one buffer, lane 0 has
// the bulk copies of its next tile (five 512-byte copies; the tile taken
// from the tile counter when there is one, as in k_step_f32) landing in
// the other, so
// the fields of the next tile need no load instructions and no wait at the
// start of the tile.  Outputs overwrite the inputs of their cell in the
// buffer and leave by 128-bit streaming stores, as in k_step_f32.  The
// window holds only the W nodes of the table format's block.  Waits are
// bounded: a copy that does not complete sets g_tma_err bit 0 (read by the
// host after the launch); the warp then issues no further copy, waits
// (bounded) for those in flight and stops stepping tiles, so none of its
// later tiles is computed from a partly filled buffer.
__device__ unsigned g_tma_err;

template <int FMT, int VAR>
__global__ void __launch_bounds__(kThreads, COOL_MINB) k_step_tma(const __grid_constant__ StepK k, long long n,
                                                                  const float* __restrict__ rho,
                                                         const float* __restrict__ Bf, const float* __restrict__ Hf,
                                                         const float* ue_in, const float* ui_in, float* ue_out,
                                                         float* ui_out, float* qc_out, float* qx_out,
                                                         cool_counters* cnt) {
    constexpr int W = Fmt<FMT>::W;
    constexpr int TILE = 5 * kWarpCells;     // floats per buffer
    extern __shared__ __align__(16) float smt[];
    load_smem(k, smt);
    const Smem S = smem_view(k, smt);
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
    while (tw < ntiles) {
        // the next tile: from the tile counter (dynamic order, taken one
        // tile ahead so that its copies overlap this tile) or round-robin
        long long nx = tw + step;
        if (k.sched) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(k.sched, 1ull);
            nx = step + (long long)__shfl_sync(0xffffffffu, t, 0);
        }
        if (lane == 0 && nx < ntiles) {
            mma::fence_async_smem();   // the other buffer's generic reads and writes are done (warp-synchronised)
            issue(nx, b ^ 1);
        }
        // warp-uniform: every lane polls, and the tile is used only if all saw it land
        const bool ok = __all_sync(0xffffffffu, mma::mbar_wait(mbar[b], phase[b], 1 << 22));
        if (!ok) {
            // a copy did not complete: report it, issue nothing more, wait
            // (bounded) for the copies still in flight into either buffer and
            // leave the tile loop; no tile output is written after this
            if (lane == 0) atomicOr(&g_tma_err, 1u);
            mma::mbar_wait(mbar[b], phase[b], 1 << 22);
            if (nx < ntiles) mma::mbar_wait(mbar[b ^ 1], phase[b ^ 1], 1 << 22);
            __syncwarp();
            break;
        }
        phase[b] ^= 1u;
        float* tile = bufs + b * TILE;
        float4* t4 = reinterpret_cast<float4*>(tile);
        const long long q = tw * 32 + lane;
        {
            unsigned redo = 0u;   // cells with a key near a node, redone below (as k_step_f32)
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int j = c * 32 + lane;
                const Out o = step_cell<FMT, (VAR & ~8), false>(k, S, win, tile[j], tile[kWarpCells + j],
                                                             tile[2 * kWarpCells + j], tile[3 * kWarpCells + j],
                                                             tile[4 * kWarpCells + j], 0.f);
                if (o.near) {
                    redo |= 1u << c;
                } else {
                    tile[3 * kWarpCells + j] = o.ue;
                    tile[4 * kWarpCells + j] = o.ui;
                    tile[0 * kWarpCells + j] = o.qc;
                    tile[1 * kWarpCells + j] = o.qx;
                    if (VAR & 8) count_flags(o.flags, cnt);
                }
            }
            if (__any_sync(0xffffffffu, redo != 0u)) {
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    if (!((redo >> c) & 1u)) continue;
                    const int j = c * 32 + lane;
                    const Out o = step_cell<FMT, (VAR & ~8), true>(k, S, win, tile[j], tile[kWarpCells + j],
                                                                tile[2 * kWarpCells + j], tile[3 * kWarpCells + j],
                                                                tile[4 * kWarpCells + j], 0.f);
                    tile[3 * kWarpCells + j] = o.ue;
                    tile[4 * kWarpCells + j] = o.ui;
                    tile[0 * kWarpCells + j] = o.qc;
                    tile[1 * kWarpCells + j] = o.qx;
                    if (VAR & 8) count_flags(o.flags | kFlagRedo, cnt);
                }
            }
            __syncwarp();
            __stcs(reinterpret_cast<float4*>(ue_out) + q, t4[3 * 32 + lane]);
            __stcs(reinterpret_cast<float4*>(ui_out) + q, t4[4 * 32 + lane]);
            if (qc_out) __stcs(reinterpret_cast<float4*>(qc_out) + q, t4[0 * 32 + lane]);
            if (qx_out) __stcs(reinterpret_cast<float4*>(qx_out) + q, t4[1 * 32 + lane]);
        }
        __syncwarp();
        b ^= 1;
        tw = nx;
    }
    const long long scalar_start = ntiles * kWarpCells;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = scalar_start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Out o = step_cell<FMT, (VAR & ~8), false>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], 0.f);
        unsigned rf = 0u;
        if (o.near) {
            o = step_cell<FMT, (VAR & ~8), true>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], 0.f);
            rf = kFlagRedo;
        }
        ue_out[i] = o.ue;
        ui_out[i] = o.ui;
        if (qc_out) qc_out[i] = o.qc;
        if (qx_out) qx_out[i] = o.qx;
        if (VAR & 8) count_flags(o.flags | rf, cnt);
    }
}

}  // namespace

cool_status launch_step_tma(const cool_table* t, const cool_params* p, long long n, const float* rho,
                            const float* B, const float* H, const float* ue, const float* ui, float* ue_o,
                            float* ui_o, float* qc, float* qx, cool_counters* cnt, cudaStream_t st) {
    StepK k;
    fill_stepk(t, p, k);
    if (n == 0) return COOL_OK;
    const bool vec = ((uintptr_t)rho | (uintptr_t)B | (uintptr_t)H | (uintptr_t)ue | (uintptr_t)ui |
                      (uintptr_t)ue_o | (uintptr_t)ui_o | (uintptr_t)qc | (uintptr_t)qx) % 16 == 0;
    if (!vec) return COOL_EALIGN;   // bulk copies need 16-byte aligned fields
    const int fmt = t->dev.fmt;
    if (fmt < 0 || fmt > 4) return COOL_EUNSUPPORTED;
    // indexed by implicit | fp64_critical << 1 | counters << 2 (template bits 0, 1, 3)
    const int var = (p->mode == COOL_IMPLICIT_STIFF ? 1 : 0) | (p->fp64_critical ? 2 : 0) | (cnt ? 4 : 0);
    using KFnT = void (*)(StepK, long long, const float*, const float*, const float*, const float*, const float*,
                          float*, float*, float*, float*, cool_counters*);
#define COOL_KT(F) k_step_tma<F, 0>, k_step_tma<F, 1>, k_step_tma<F, 2>, k_step_tma<F, 3>, \
                   k_step_tma<F, 8>, k_step_tma<F, 9>, k_step_tma<F, 10>, k_step_tma<F, 11>
    static const KFnT table_t[5][8] = {{COOL_KT(0)}, {COOL_KT(1)}, {COOL_KT(2)}, {COOL_KT(3)}, {COOL_KT(4)}};
#undef COOL_KT
    static const int width[5] = {Fmt<0>::W, Fmt<1>::W, Fmt<2>::W, Fmt<3>::W, Fmt<4>::W};
    KFnT fn = table_t[fmt][var];
    const size_t sm_t = (size_t)(smem_table_floats(k) + width[fmt] * kThreads + kWarps * 2 * 5 * kWarpCells) *
                            sizeof(float) + kWarps * 2 * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_t);
    if (e != cudaSuccess) return set_cuda_error(e);
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, sm_t);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (per < 1) per = 1;
    long long wk = (n + kWarps * kWarpCells - 1) / (kWarps * kWarpCells);
    long long cp = (long long)sm_count() * per;
    long long bl = wk < cp ? wk : cp;
    if (bl < 1) bl = 1;
    if (n / kWarpCells > bl * kWarps) {
        // more tiles than warps: the dynamic order of the default step
        k.sched = sched_counter(st);
        if (k.sched) {
            e = cudaMemsetAsync(k.sched, 0, sizeof(unsigned long long), st);
            if (e != cudaSuccess) return set_cuda_error(e);
        }
    }
    fn<<<(int)bl, kThreads, sm_t, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt);
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

}  // namespace cool

// Error word of the TMA-staged step on the current device: bit 0 = a bulk
// copy that never completed (see k_step_tma).  Synchronous.
extern "C" cool_status cool_tma_error(unsigned* err_out, int clear) {
    using namespace cool;
    if (!err_out) return COOL_ENULL;
    if (clear != 0 && clear != 1) return COOL_EINVAL;
    cudaError_t e = cudaMemcpyFromSymbol(err_out, g_tma_err, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_tma_err, &zero, sizeof(unsigned));
    }
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}
