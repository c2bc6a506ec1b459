// cool_step_kernel.cuh -- the FP32 step kernel template k_step_f32
// (vector and scalar paths), instantiated per table format in cool_step.cu
// (FP32 table, disk geometry, the paper's layout), cool_step_f16.cu (plain
// BF16/FP16) and cool_step_f16s.cu (block-scaled BF16/FP16), so that the
// instantiations compile in parallel.
#pragma once

#include "cool_step_cell.cuh"

namespace cool {
namespace {

// VAR: the step_cell variant bits (0 implicit, 1 fp64_critical, 2 disk
// geometry) and bit 3, counters requested: without it no counter flag is
// formed (the flag arithmetic of step_cell is dead code) and nothing is
// counted.  Shared memory after the warps' staging tiles: one list of up to
// 128 tile indices per warp (the deferred cells: stiff ones in implicit
// mode, and with fp64_critical those entering the equilibrium band).
// VEC: all arrays 16-byte aligned.  Each warp walks tiles of 128 cells: its
// first tile by its index in the grid, the next ones from a device counter
// (k.sched) as it finishes, so the warps that draw cheap tiles take more of
// them (static round-robin order when k.sched is null).  Per tile the five
// input fields arrive by 128-bit streaming loads into the
// warp's staging area, each lane steps cells lane, lane+32, lane+64, lane+96
// (one cell's state in registers at a time), the outputs overwrite the
// staging area and leave by 128-bit streaming stores.  Warps synchronise
// only with themselves (__syncwarp), so a slow cell delays one warp, not the
// block.  The remainder (and unaligned arrays) take a scalar loop.
// A tile-pass result that defers the cell: it entered the equilibrium band
// (fp64_critical) or turned stiff (implicit mode).
template <int VAR>
__device__ __forceinline__ bool deferred_flags(unsigned f) {
    return ((VAR & 2) && (f & 8u)) || ((VAR & 1) && (f & 4u));
}

template <bool VEC, int FMT, int VAR>
__global__ void __launch_bounds__(kThreads, COOL_MINB) k_step_f32(const __grid_constant__ StepK k, long long n,
                                                                  const float* __restrict__ rho,
                                                         const float* __restrict__ Bf, const float* __restrict__ Hf,
                                                         const float* ue_in, const float* ui_in, float* ue_out,
                                                         float* ui_out, float* qc_out, float* qx_out,
                                                         cool_counters* cnt, const float* __restrict__ rr) {
    constexpr int NF = (VAR & 4) ? 6 : 5;   // staged input fields
    // the tile pass's variant: in implicit mode (bit 0) a stiff cell takes
    // the limited step instead of a solve (bit 5) and is only flagged; with
    // fp64_critical (bit 1) every cell is first stepped in FP32 (bit 1
    // cleared) and also flagged when it enters the equilibrium band.  Up to
    // that sub-cycle the tile pass and the full variant are the same
    // arithmetic, so an unflagged cell's result is the full variant's; a
    // flagged cell is stepped again below with the full variant, the
    // deferred cells of the tile gathered onto consecutive lanes, so that
    // the solves run side by side instead of one lane at a time in most
    // passes of the tile.
    // bit 6 (LIST): the flagged cells go to the list k.dlist, stepped by
    // k_step_list_f32 after this kernel, instead of the warp's own pass
    constexpr bool LIST = (VAR & 64) != 0;
    constexpr int V = VAR & ~64;
    constexpr int VF = (V & 2) ? ((V & ~(2 | 8)) | 32) : (V & 1) ? ((V & ~8) | 32) : (V & ~8);
    extern __shared__ float sm[];
    load_smem(k, sm);
    const Smem S = smem_view(k, sm);
    constexpr int WR = Fmt<FMT>::W;                          // window rows of this format
    float* win = sm + smem_table_floats(k) + threadIdx.x;   // WR x kThreads window
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    long long scalar_start = 0;
    if (VEC) {
        float* tile = sm + smem_table_floats(k) + WR * kThreads + warp * NF * kWarpCells;
        float4* t4 = reinterpret_cast<float4*>(tile);
        const long long ntiles = n / kWarpCells;
        const long long first = (long long)gridDim.x * kWarps;   // tiles taken statically
        long long tw = (long long)blockIdx.x * kWarps + warp;
        while (tw < ntiles) {
            const long long q = tw * 32 + lane;  // float4 index of this lane
            t4[0 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(rho) + q);
            t4[1 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(Bf) + q);
            t4[2 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(Hf) + q);
            t4[3 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(ue_in) + q);
            t4[4 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(ui_in) + q);
            if (VAR & 4) t4[5 * 32 + lane] = __ldcs(reinterpret_cast<const float4*>(rr) + q);
            __syncwarp();
            unsigned redo = 0u;    // cells with a key near a node, redone below
            unsigned defer = 0u;   // cells redone below with the full variant
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int j = c * 32 + lane;
                const Out o = step_cell<FMT, VF, false>(k, S, win, tile[j], tile[kWarpCells + j],
                                                        tile[2 * kWarpCells + j], tile[3 * kWarpCells + j],
                                                        tile[4 * kWarpCells + j],
                                                        (VAR & 4) ? tile[5 * kWarpCells + j] : 0.f);
                if (deferred_flags<VAR>(o.flags)) {
                    defer |= 1u << c;  // its inputs stay in the tile
                } else if (o.near) {
                    redo |= 1u << c;   // its inputs stay in the tile
                } else {
                    // inputs of cell j are consumed: outputs reuse its slots
                    tile[3 * kWarpCells + j] = o.ue;
                    tile[4 * kWarpCells + j] = o.ui;
                    tile[0 * kWarpCells + j] = o.qc;
                    tile[1 * kWarpCells + j] = o.qx;
                    if (VAR & 8) count_flags(o.flags, cnt);
                }
            }
            if (__any_sync(0xffffffffu, redo != 0u)) {
                // a few cells in a million: every index by the exact rule
                // (node compares where the lg2 guess is in doubt), kept out of
                // the loop above so that it leaves its code alone
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    if (!((redo >> c) & 1u)) continue;
                    const int j = c * 32 + lane;
                    // with LIST the flag-only variant: a cell that turns stiff
                    // (or enters the band) on the exact trajectory is listed
                    constexpr int VR = LIST ? VF : (V & ~8);
                    const Out o = step_cell<FMT, VR, true>(k, S, win, tile[j], tile[kWarpCells + j],
                                                           tile[2 * kWarpCells + j], tile[3 * kWarpCells + j],
                                                           tile[4 * kWarpCells + j],
                                                           (VAR & 4) ? tile[5 * kWarpCells + j] : 0.f);
                    if (LIST && deferred_flags<VAR>(o.flags)) {
                        k.dlist[1 + atomicAdd(k.dlist, 1u)] = (unsigned)(tw * kWarpCells + j);
                        continue;   // its slots keep the inputs
                    }
                    tile[3 * kWarpCells + j] = o.ue;
                    tile[4 * kWarpCells + j] = o.ui;
                    tile[0 * kWarpCells + j] = o.qc;
                    tile[1 * kWarpCells + j] = o.qx;
                    if (VAR & 8) count_flags(o.flags | kFlagRedo, cnt);
                }
            }
            if (LIST) {
                // the tile's flagged cells, appended with one atomic; their
                // slots keep the inputs, which the stores below write out and
                // k_step_list_f32 overwrites
                unsigned bal[4], tot = 0u;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    bal[c] = __ballot_sync(0xffffffffu, (defer >> c) & 1u);
                    tot += __popc(bal[c]);
                }
                if (tot) {
                    unsigned base = 0u;
                    if (lane == 0) base = atomicAdd(k.dlist, tot);
                    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if ((defer >> c) & 1u)
                            k.dlist[1 + base + __popc(bal[c] & ((1u << lane) - 1u))] =
                                (unsigned)(tw * kWarpCells + c * 32 + lane);
                        base += __popc(bal[c]);
                    }
                }
            } else if ((VAR & 3) && __any_sync(0xffffffffu, defer != 0u)) {
                // the deferred cells, gathered onto consecutive lanes (their
                // tile indices in the warp's list), stepped again from their
                // inputs with the full variant: one pass per 32 of them
                // instead of a solve (or FP64 code) in most passes
                unsigned char* list = reinterpret_cast<unsigned char*>(
                                          sm + smem_table_floats(k) + WR * kThreads + kWarps * NF * kWarpCells) +
                                      warp * kWarpCells;
                int m = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool d = (defer >> c) & 1u;
                    const unsigned bal = __ballot_sync(0xffffffffu, d);
                    if (d) list[m + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)(c * 32 + lane);
                    m += __popc(bal);
                }
                __syncwarp();
#pragma unroll 1
                for (int b = 0; b < m; b += 32) {
                    if (b + lane < m) {
                        const int j = list[b + lane];
                        Out o = step_cell<FMT, (V & ~8), false>(k, S, win, tile[j], tile[kWarpCells + j],
                                                                  tile[2 * kWarpCells + j], tile[3 * kWarpCells + j],
                                                                  tile[4 * kWarpCells + j],
                                                                  (VAR & 4) ? tile[5 * kWarpCells + j] : 0.f);
                        unsigned rf = 0u;
                        if (o.near) {
                            o = step_cell<FMT, (V & ~8), true>(k, S, win, tile[j], tile[kWarpCells + j],
                                                                 tile[2 * kWarpCells + j], tile[3 * kWarpCells + j],
                                                                 tile[4 * kWarpCells + j],
                                                                 (VAR & 4) ? tile[5 * kWarpCells + j] : 0.f);
                            rf = kFlagRedo;
                        }
                        tile[3 * kWarpCells + j] = o.ue;
                        tile[4 * kWarpCells + j] = o.ui;
                        tile[0 * kWarpCells + j] = o.qc;
                        tile[1 * kWarpCells + j] = o.qx;
                        if (VAR & 8) count_flags(o.flags | rf, cnt);
                    }
                }
            }
            __syncwarp();
            __stcs(reinterpret_cast<float4*>(ue_out) + q, t4[3 * 32 + lane]);
            __stcs(reinterpret_cast<float4*>(ui_out) + q, t4[4 * 32 + lane]);
            if (qc_out) __stcs(reinterpret_cast<float4*>(qc_out) + q, t4[0 * 32 + lane]);
            if (qx_out) __stcs(reinterpret_cast<float4*>(qx_out) + q, t4[1 * 32 + lane]);
            __syncwarp();
            if (k.sched) {
                unsigned long long nt = 0;
                if (lane == 0) nt = atomicAdd(k.sched, 1ull);
                tw = first + (long long)__shfl_sync(0xffffffffu, nt, 0);
            } else {
                tw += first;
            }
        }
        scalar_start = ntiles * kWarpCells;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = scalar_start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float ri = (VAR & 4) ? rr[i] : 0.f;
        // with LIST the flag-only variant, a flagged cell listed
        constexpr int VS = LIST ? VF : (V & ~8);
        Out o = step_cell<FMT, VS, false>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], ri);
        unsigned rf = 0u;
        if (o.near && !(LIST && deferred_flags<VAR>(o.flags))) {
            o = step_cell<FMT, VS, true>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], ri);
            rf = kFlagRedo;
        }
        if (LIST && deferred_flags<VAR>(o.flags)) {
            k.dlist[1 + atomicAdd(k.dlist, 1u)] = (unsigned)i;
            continue;
        }
        ue_out[i] = o.ue;
        ui_out[i] = o.ui;
        if (qc_out) qc_out[i] = o.qc;
        if (qx_out) qx_out[i] = o.qx;
        if (VAR & 8) count_flags(o.flags | rf, cnt);
    }
}

// The cells a LIST tile pass listed in k.dlist, stepped from their inputs
// with the full variant VAR (the solve, the FP64 options): consecutive list
// entries on consecutive lanes, so that the solves run side by side.
template <int FMT, int VAR>
__global__ void __launch_bounds__(kThreads, 2) k_step_list_f32(const __grid_constant__ StepK k, long long n,
                                                               const float* __restrict__ rho,
                                                               const float* __restrict__ Bf,
                                                               const float* __restrict__ Hf, const float* ue_in,
                                                               const float* ui_in, float* ue_out, float* ui_out,
                                                               float* qc_out, float* qx_out, cool_counters* cnt,
                                                               const float* __restrict__ rr) {
    extern __shared__ float sm[];
    load_smem(k, sm);
    const Smem S = smem_view(k, sm);
    float* win = sm + smem_table_floats(k) + threadIdx.x;   // window rows of this format x kThreads
    const long long m = k.dlist[0];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = k.dlist[1 + t];
        const float ri = (VAR & 4) ? rr[i] : 0.f;
        Out o = step_cell<FMT, (VAR & ~8), false>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], ri);
        unsigned rf = 0u;
        if (o.near) {
            o = step_cell<FMT, (VAR & ~8), true>(k, S, win, rho[i], Bf[i], Hf[i], ue_in[i], ui_in[i], ri);
            rf = kFlagRedo;
        }
        ue_out[i] = o.ue;
        ui_out[i] = o.ui;
        if (qc_out) qc_out[i] = o.qc;
        if (qx_out) qx_out[i] = o.qx;
        if (VAR & 8) count_flags(o.flags | rf, cnt);
    }
}

using StepKernelFn = void (*)(StepK, long long, const float*, const float*, const float*, const float*, const float*,
                              float*, float*, float*, float*, cool_counters*, const float*);

}  // namespace
}  // namespace cool
