// cool_step_common.cuh -- FP32/FP64 building blocks of the cooling step
// shared by the step kernels (cool_step.cu) and the surrogate step
// (cool_sur_step.cu): constants of a launch, index selection, the packed
// 4-D channel gather, the cooling energy with the bridge, the implicit
// solves, and the host functions that fill the launch constants.
#pragma once

#include <cuda_fp16.h>
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


// A quiet FP64 NaN (an absent argument).
__device__ __forceinline__ double nan64() { return __longlong_as_double(0x7ff8000000000000ll); }

// Shared-memory view of the small table parts.
struct Smem {
    const float* ax;   // concatenated axes (x, rx, lx per axis)
    const float* lb;
    const float* lc;
    const float4* tn;  // per cooling T_e interval j: (1/x_j, log2 x_j, lb_j, lb_j+1)
};

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
    int jt;             // T_e interval of the cached collapse, -1 if none
    double v0, v1;      // synchrotron log2 values at its two nodes, collapsed over H, B, n_e
};

// dqdu (nullable): also dq/du of the same interpolation (the slopes of the
// T_e interval and of the bridge; zero slope where the key is clamped).
__device__ double cool_q64(const StepK64& k, Cell64& c, double ue, double rho, unsigned& clamp,
                           double* dqdu = nullptr) {
    const DevTable& T = k.tab;
    double Te = k.s_Te * ue / rho;
    double wt;
    int jt = select64(T, 3, Te, wt, clamp);
    if (jt != c.jt) {
        // the 8 (H, B, n_e) corners at the interval's two T_e nodes, collapsed
        // once per visited interval (an implicit solve evaluates many T_e in few
        // intervals)
        const int nB = T.n[1], nN = T.n[2], nT = T.n[3];
        double v0 = 0.0, v1 = 0.0;
        for (int cidx = 0; cidx < 8; ++cidx) {
            const int bh = cidx & 1, bb = (cidx >> 1) & 1, bn = (cidx >> 2) & 1;
            const double wgt = (bh ? c.wh : 1.0 - c.wh) * (bb ? c.wb : 1.0 - c.wb) * (bn ? c.wn : 1.0 - c.wn);
            const long long idx = (((long long)(c.jh + bh) * nB + (c.jb + bb)) * nN + (c.jn + bn)) * nT + jt;
            v0 += wgt * T.ls64[idx];
            v1 += wgt * T.ls64[idx + 1];
        }
        c.jt = jt;
        c.v0 = v0;
        c.v1 = v1;
    }
    double ls = (1.0 - wt) * c.v0 + wt * c.v1;
    double lb = (1.0 - wt) * T.lb64[jt] + wt * T.lb64[jt + 1];
    const double qb = c.ne * c.ne * exp2(lb), qs = exp2(ls);
    double qthin = qb + qs;
    double bb4 = 4.0 * kSigSB * Te * Te * Te * Te;
    double tau_sca = 2.0 * c.ne * kSigT * c.Hc;
    double tau_abs = c.Hc * qthin / bb4;
    const double D = 1.0 + tau_abs * (sqrt(3.0) + 1.5 * (tau_abs + tau_sca));
    double Q = qthin / D;
    if (dqdu) {
        // d/dln T_e: the weight moves by 1/(dl ln 2) inside the interval
        // (FP64 divisions are slow on this part: one reciprocal of D serves)
        const bool inside = wt > 0.0 && wt < 1.0;
        const double dthin = inside ? (qb * (T.lb64[jt + 1] - T.lb64[jt]) + qs * (c.v1 - c.v0)) / T.dl64[3] : 0.0;
        const double dtau = tau_abs * (dthin / qthin - 4.0);
        const double dD = (sqrt(3.0) + 3.0 * tau_abs + 1.5 * tau_sca) * dtau;
        const double rD = 1.0 / D;
        *dqdu = k.hs * (dthin - Q * dD) * rD / (k.escale * ue);   // dln T_e/du = 1/u
    }
    return k.hs * Q / k.escale;
}

// Backward Euler of a stiff cell in FP64 on the FP64 table: the root of
// g(x) = 2^x - u0 + q(2^x), x = log2 u, in the bracket [log2 u0 - 60,
// log2 u0] (g < 0 at its low end is checked, g = q(u0) > 0 at its high end).
// Illinois iterations (regula falsi with the value at the retained end
// halved) first on G(x) = log2((2^x + q(2^x)) / u0), which is close to
// piecewise linear over the 60 octaves, then on g itself once the bracket
// is 1e-3 wide, until it is 1e-15 max(1, |x|) wide: the root the oracle's
// bisection finds, to FP64 precision, in ~20 evaluations instead of 60; at
// most iters evaluations.  Returns false when the bracket has no sign change.
// xa0 < xb0: a narrower bracket around the FP32 solve's root (on the FP32
// table), used when g changes sign over it in FP64 (the FP32 and FP64
// functions differ by ~1e-6 relative, the bracket is 2^-13 wide in log2 u),
// else the full one; NaN: none.
__device__ __noinline__ bool implicit_fp64(const StepK64& k, Cell64& c, double rho, double u0, double& u_out,
                                           double xa0, double xb0) {
    unsigned dummy = 0u;
    double xa = xa0, xb = xb0, ua = 0.0, ub = 0.0, qa = 0.0, qb = 0.0;
    int it = 0;
    bool bracketed = false;
    if (xa0 < xb0) {
        // a bracket from the FP32 solve: kept if g changes sign over it in FP64
        ua = exp2(xa);
        ub = exp2(xb);
        qa = cool_q64(k, c, ua, rho, dummy);
        qb = cool_q64(k, c, ub, rho, dummy);
        it = 2;
        bracketed = ua - u0 + qa < 0.0 && ub - u0 + qb > 0.0;
    }
    if (!bracketed) {
        xa = log2(u0) - 60.0;
        xb = log2(u0);
        ua = exp2(xa);
        ub = exp2(xb);
        qa = cool_q64(k, c, ua, rho, dummy);
        qb = cool_q64(k, c, ub, rho, dummy);
        it += 2;
        if (!(ua - u0 + qa < 0.0) || !(ub - u0 + qb > 0.0)) return false;
    }
    for (int phase = 0; phase < 2; ++phase) {
        // phase 0: G in log space; phase 1: g in u
        double fa = phase == 0 ? log2((ua + qa) / u0) : ua - u0 + qa;
        double fb = phase == 0 ? log2((ub + qb) / u0) : ub - u0 + qb;
        int side = 0;
        for (; it < k.iters; ++it) {
            const double width = xb - xa;
            if (phase == 0 ? width <= 1e-3 : width <= 1e-15 * fmax(1.0, fabs(xb))) break;
            double x = xb - fb * width / (fb - fa);
            if (!(x > xa && x < xb)) x = 0.5 * (xa + xb);
            const double u = exp2(x);
            const double q = cool_q64(k, c, u, rho, dummy);
            const double f = phase == 0 ? log2((u + q) / u0) : u - u0 + q;
            if (f > 0.0) {
                xb = x; ub = u; qb = q; fb = f;
                if (side > 0) fa *= 0.5;
                side = 1;
            } else if (f < 0.0) {
                xa = x; ua = u; qa = q; fa = f;
                if (side < 0) fb *= 0.5;
                side = -1;
            } else {
                xa = xb = x;
                break;
            }
        }
    }
    u_out = exp2(0.5 * (xa + xb));
    return true;
}

struct StepK {
    DevTable tab;
    float s_n, s_B, s_H, s_Te, s_Ti;  // FP32 key scales (rounded once from FP64)
    float ce, ci, inv_cec;            // gamma - 1, 1/(ce + ci)
    double ce64, ci64, inv_cec64;
    float s_K;                        // m_p c^2 / k_B  (T_s = (gamma_s - 1) s_K u_s / rho)
    int fp64_critical;
    StepK64 k64;                      // FP64 constants for stiff cells when fp64_critical
    float l_hs_e;                     // log2(h / e_scale)
    float l_bb;                       // log2(4 sigma_SB h / e_scale)
    float two_sigT;                   // 2 sigma_T
    float limiter, eq_band, clamp;
    int n_sub, mode, iters;
    int smem_floats;                  // floats of axes + lb + lc in shared memory
    int lc_stride;                    // row stride of the Coulomb channel in shared memory (see fill_stepk)
    int tn_off;                       // float offset (multiple of 4) of the T_e interval records (Smem::tn)
    int axes_floats;
    float spin, h_floor;              // disk geometry (the disk step): a, (H/R)_floor
    int h_from_state;                 // H_th = c_s / Omega_K replaces the H field
    // select_sub constants per axis (0 H, 1 B, 2 n_e, 3 T_e, 4 Coulomb T):
    // -log2(x_0)/dl - 1/2, n - 2, the end nodes x_0, x_{n-1}, and the
    // weight band 1/2 - 1e-6/dl outside which a key is treated as on a node
    float g_c0[5], g_hi[5], g_x0[5], g_xn[5], g_wb[5];
    // tile counter of the vector step's dynamic tile order (zeroed on the
    // launch stream before the launch); nullptr: the static order
    unsigned long long* sched;
    unsigned* dlist;                  // deferred cells: [0] the count, then their indices (k_step_list_f32)
};

struct Sel {
    int j;
    float r;   // log2(key / x_j), unclamped
};

// Index selection on an axis (x, rx, lx arrays of n floats at `a`): the
// largest j in [0, n-2] with x[j] <= key, compared exactly in FP32 (j = 0
// below the first node).  The guess floor((log2 key - l_0)/dl) is within
// one of that index (lg2.approx is accurate to ~1e-5 absolute, far below
// one node spacing), so one upward and one downward correction make the
// selection exact with no data-dependent loop.  The key is clamped when it
// lies outside [x_0, x_{n-1}]; the two compared nodes tell: below x_0 the
// guess is 0 and x_0 > key, above x_{n-1} the guess is n-2 and x_{n-1} < key.
__device__ __forceinline__ Sel select_axis(const float* a, int n, float inv_dl, float key,
                                           unsigned& clamp) {
    const float* x = a;
    const float* rx = a + n;
    const float* lx = a + 2 * n;
    int j0 = __float2int_rd((lg2a(key) - lx[0]) * inv_dl);
    j0 = min(max(j0, 0), n - 2);
    const float xa = x[j0 + 1];
    const int j1 = j0 + ((j0 < n - 2 && xa <= key) ? 1 : 0);
    const float xb = x[j1];
    const bool above = xb > key;
    clamp |= ((j1 == 0 && above) || (j0 == n - 2 && xa < key)) ? 1u : 0u;
    Sel s;
    s.j = j1 - ((j1 > 0 && above) ? 1 : 0);
    s.r = lg2a(key * rx[s.j]);
    return s;
}

struct SelW {
    int j;
    float r;   // log2(key / x_j)
    float w;   // interpolation weight r / dl, saturated to [0, 1]
};

// Index selection on axis A (0..4) as the step does it.  EXACT: select_axis
// (the largest j with x_j <= key in exact FP32 compares).  Otherwise the
// same j and w without node loads besides 1/x_j, or the flag `near`: the
// guess floor((log2 key - l_0)/dl) is taken as round-to-nearest of the value
// shifted by -1/2 (the FP32 addition of 1.5 * 2^23 rounds to an integer);
// lg2.approx puts it within one of the true index, and wrong only for keys
// within ~1e-5 node spacings of a node.  Then r = log2(key / x_j) comes from
// the ratio, accurate to ~2e-7 in log2: a weight inside the band
// (1e-6/dl, 1 - 1e-6/dl) proves x_j < key < x_{j+1}, so j is the index.
// Outside it (a key within ~1e-6 of a node, a wrong guess -- a few keys in
// a million -- or a key outside the axis, whose weight lies outside [0, 1])
// `near` is set and the caller redoes the cell with EXACT, which also sets
// the clamp flag; the values returned meanwhile are those of the guessed
// interval.  (Sending out-of-range keys to the redo instead of testing the
// range here saves two compares per key: 4 % of the benchmark step.)
// RANGE: the implicit solve's trial keys, which fall outside the axis in
// most solves: there the range is tested and an out-of-range key does not
// set `near`, since its guess is already select_axis's result (the guess
// clamps to the end interval, the weight to 0 or 1, and both take r from
// the same ratio).  The clamp flag compares the key with the end nodes
// exactly, as select_axis does; outside the redo it is formed only where
// counters are kept.
template <int A>
__device__ __forceinline__ int select_guess(const StepK& k, float inv_dl, float key) {
    float t = fmaf(lg2a(key), inv_dl, k.g_c0[A]);
    t = fminf(fmaxf(t, 0.f), k.g_hi[A]);
    return __float_as_int(__fadd_rn(t, 12582912.f)) - 0x4B400000;
}

template <int A, bool RANGE = false>
__device__ __forceinline__ SelW select_finish(const StepK& k, int j, float rxj, float inv_dl, float key,
                                              unsigned& clamp, unsigned& near) {
    SelW s;
    s.j = j;
    s.r = lg2a(key * rxj);
    const float w = s.r * inv_dl;
    const bool out = key < k.g_x0[A] || key > k.g_xn[A];
    clamp |= out ? 1u : 0u;   // formed only where counted
    if (RANGE) near |= (fabsf(w - 0.5f) > k.g_wb[A] && !out) ? 1u : 0u;
    else near |= fabsf(w - 0.5f) > k.g_wb[A] ? 1u : 0u;   // an out-of-range key too: its weight is outside
    s.w = __saturatef(w);
    return s;
}

// EXACT: the guess where its weight confirms it, node compares (select_axis)
// where it does not; the same j, r, w as select_axis in every case.
template <int A, bool EXACT, bool RANGE = false>
__device__ __forceinline__ SelW select_sub(const StepK& k, const float* rx, int n, float inv_dl, float key,
                                           unsigned& clamp, unsigned& near) {
    const int j = select_guess<A>(k, inv_dl, key);
    if (EXACT) {
        unsigned doubt = 0u;
        SelW s = select_finish<A, RANGE>(k, j, rx[j], inv_dl, key, clamp, doubt);
        if (doubt) {
            const Sel e = select_axis(rx - n, n, inv_dl, key, clamp);
            s.j = e.j;
            s.r = e.r;
            s.w = __saturatef(e.r * inv_dl);
        }
        return s;
    }
    return select_finish<A, RANGE>(k, j, rx[j], inv_dl, key, clamp, near);
}

// Per-cell, step-invariant part of the 4-D lookup and the cooling constants.
struct CellC {
    const uint32_t* row;  // block row of corner (jh, jb, jn): lsb + r nblk 8 words
    int oH, oB, oN;     // float offsets to the H+1, B+1, n_e+1 corner rows
    float wh, wb, wn;
    float lb_off;       // log2(h n_e^2 / e_scale)
    float ls_off;       // log2(h / e_scale)
    float lbb_off;      // log2(4 sigma_SB h / (H_cm e_scale))
    float tau_sca;      // 2 n_e sigma_T H_cm
};

// Collapsed synchrotron values of one T_e octet (7 intervals) live in shared
// memory, node o of thread t at win[o * kThreads + t] (conflict-free).
struct Cache {
    int base;           // first node of the held octet (multiple of 7), -8 if none
    float* win;         // this thread's window column
    unsigned near;      // a key of this cell fell near a node (select_sub)
};

constexpr int kThreads = 256;

__device__ __forceinline__ float lerpf(float a, float b, float w) { return fmaf(w, b - a, a); }

// Packed formats of the 4-D channel (DevTable::fmt): nodes per 32-byte block
// W and block stride S = W - 1.
template <int FMT> struct Fmt;
template <> struct Fmt<0> { static constexpr int W = 8, S = 7; };    // FP32
template <> struct Fmt<1> { static constexpr int W = 16, S = 15; };  // BF16
template <> struct Fmt<2> { static constexpr int W = 16, S = 15; };  // FP16
template <> struct Fmt<3> { static constexpr int W = 12, S = 11; };  // BF16, block-scaled
template <> struct Fmt<4> { static constexpr int W = 12, S = 11; };  // FP16, block-scaled
// nodes per block of a format, on the host (the window rows a kernel needs)
constexpr int fmt_nodes(int fmt) { return fmt == 0 ? Fmt<0>::W : (fmt <= 2 ? Fmt<1>::W : Fmt<3>::W); }

// 256-bit read-only load of one block (32-byte aligned), not allocated in
// L1: the gathers' corner rows are scattered (L1 hit rate ~10 % with
// allocation), and loads that do not allocate take fewer L1 data-pipe
// wavefronts (235.6 M -> 193.6 M per 256^3 benchmark step, 0.954 ->
// 0.893 ms) and leave L1 to the spills and the staged fields.
__device__ __forceinline__ void ld8u(const uint32_t* p, uint32_t (&v)[8]) {
    asm("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "l"(p));
}

__device__ __forceinline__ float half_bits(uint32_t h16, bool f16) {
    return f16 ? __half2float(__ushort_as_half((unsigned short)h16)) : __uint_as_float(h16 << 16);
}

// Value of node t (0 <= t < W) of a block.
template <int FMT>
__device__ __forceinline__ float dec(const uint32_t (&r)[8], int t) {
    if (FMT == 0) return __uint_as_float(r[t]);
    if (FMT == 1 || FMT == 2) {
        const uint32_t w = r[t >> 1];
        return half_bits((t & 1) ? (w >> 16) : (w & 0xffffu), FMT == 2);
    }
    const uint32_t w = r[2 + (t >> 1)];
    const float res = half_bits((t & 1) ? (w >> 16) : (w & 0xffffu), FMT == 4);
    return fmaf(__uint_as_float(r[1]), res, __uint_as_float(r[0]));
}

// Read the 8 corner blocks of block kb (one 32-byte sector each) and collapse
// the H, B, n_e axes: win[o] = trilinear value at T_e node S kb + o.
template <int FMT>
__device__ __forceinline__ void gather(const CellC& c, int kb, Cache& cc) {
    constexpr int W = Fmt<FMT>::W;
    const uint32_t* p = c.row + (long long)kb * 8;
    if (FMT == 0) {
        // FP32: the four corners of one H plane in flight together (two L2
        // round trips per gather); the first plane's bilinear value waits in
        // the window while the second plane loads
        uint32_t a[8], b[8], d[8], e[8];
        ld8u(p, a);
        ld8u(p + c.oN, b);
        ld8u(p + c.oB, d);
        ld8u(p + c.oB + c.oN, e);
#pragma unroll
        for (int t = 0; t < 8; ++t)
            cc.win[t * kThreads] = lerpf(lerpf(dec<0>(a, t), dec<0>(b, t), c.wn),
                                         lerpf(dec<0>(d, t), dec<0>(e, t), c.wn), c.wb);
        const uint32_t* q = p + c.oH;
        ld8u(q, a);
        ld8u(q + c.oN, b);
        ld8u(q + c.oB, d);
        ld8u(q + c.oB + c.oN, e);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float y = lerpf(lerpf(dec<0>(a, t), dec<0>(b, t), c.wn), lerpf(dec<0>(d, t), dec<0>(e, t), c.wn),
                                  c.wb);
            cc.win[t * kThreads] = lerpf(cc.win[t * kThreads], y, c.wh);
        }
    } else {
        // 16-bit formats (W = 16 or 12 nodes): the partial sums go through
        // the window in shared memory to bound register use (four corners
        // in flight, as for FP32, measured slower for BF16)
        uint32_t r0[8], r1[8];
        ld8u(p, r0);
        ld8u(p + c.oN, r1);
#pragma unroll
        for (int t = 0; t < W; ++t) cc.win[t * kThreads] = lerpf(dec<FMT>(r0, t), dec<FMT>(r1, t), c.wn);
        ld8u(p + c.oB, r0);
        ld8u(p + c.oB + c.oN, r1);
#pragma unroll
        for (int t = 0; t < W; ++t)
            cc.win[t * kThreads] = lerpf(cc.win[t * kThreads], lerpf(dec<FMT>(r0, t), dec<FMT>(r1, t), c.wn), c.wb);
        const uint32_t* q = p + c.oH;
        float hb[W];
        ld8u(q, r0);
        ld8u(q + c.oN, r1);
#pragma unroll
        for (int t = 0; t < W; ++t) hb[t] = lerpf(dec<FMT>(r0, t), dec<FMT>(r1, t), c.wn);
        ld8u(q + c.oB, r0);
        ld8u(q + c.oB + c.oN, r1);
#pragma unroll
        for (int t = 0; t < W; ++t) {
            const float h1 = lerpf(hb[t], lerpf(dec<FMT>(r0, t), dec<FMT>(r1, t), c.wn), c.wb);
            cc.win[t * kThreads] = lerpf(cc.win[t * kThreads], h1, c.wh);
        }
    }
    cc.base = Fmt<FMT>::S * kb;
}

// The bridge of Eq. 11 (see cool_energy below) from Ls = log2 q_syn,
// Lb = log2 q_brem (code units) and lT = log2 T_e.
__device__ __forceinline__ float energy_from_logs(const CellC& c, float Ls, float Lb, float lT) {
    const float M = fmaxf(Ls, Lb);
    const float A = M + lg2a(1.f + ex2a(fminf(Ls, Lb) - M));
    const float Bb = fmaf(4.f, lT, c.lbb_off);
    const float lt = A - Bb;  // log2 tau_abs
    float lq;
    if (lt <= 60.f) {
        const float tau = ex2a(lt);
        const float D = fmaf(tau, fmaf(1.5f, tau + c.tau_sca, 1.7320508f), 1.f);
        lq = A - lg2a(D);
    } else {
        // q = q_bb / (1.5 (tau_abs + tau_sca)) up to 2^-59 relative
        lq = Bb - 0.5849625f - (lt + lg2a(1.f + c.tau_sca * ex2a(-lt)));
    }
    return ex2a(fminf(lq, 126.f));
}

// Energy (code units) that cooling removes in one sub-cycle at T_e, with
// the bridge of Eq. 11 evaluated in log2 space:
//   A = log2 q_thin = log2(q_brem + q_syn), B = log2 q_bb with
//   q_bb = h 4 sigma T^4/(H e_scale), tau_abs = 2^(A - B),
//   q = q_thin / (1 + tau_abs (sqrt3 + 1.5 (tau_abs + tau_sca))).
// The common path has no range branches: 2^d underflows to 0 where one
// channel is negligible and tau_abs to 0 where the cell is thin; only
// tau_abs > 2^60 (where tau_abs^2 would overflow) takes the asymptotic form.
// RANGE: a trial key of the implicit solve (select_finish).
template <int FMT, bool EXACT, bool RANGE = false>
__device__ __forceinline__ float cool_energy(const StepK& k, const Smem& S, const CellC& c,
                                             Cache& cc, float Te, unsigned& clamp) {
    const int nT = k.tab.n[3];
    const float* axT = S.ax + k.tab.axis_off[3];
    SelW s;
    float4 nd;   // (1/x_j, log2 x_j, lb_j, lb_j+1): one 128-bit shared load on the step's path
    if (EXACT) {
        s = select_sub<3, true, RANGE>(k, axT + nT, nT, k.tab.inv_dl[3], Te, clamp, cc.near);
        if ((unsigned)(s.j - cc.base) > (unsigned)(Fmt<FMT>::S - 1)) gather<FMT>(c, s.j / Fmt<FMT>::S, cc);
        nd = make_float4(0.f, axT[2 * nT + s.j], S.lb[s.j], S.lb[s.j + 1]);
    } else {
        // the guess is the interval used (a doubtful one only flags the cell),
        // so the window moves before the record is read: nothing is held
        // across the gather
        const int jg = select_guess<3>(k, k.tab.inv_dl[3], Te);
        if ((unsigned)(jg - cc.base) > (unsigned)(Fmt<FMT>::S - 1)) gather<FMT>(c, jg / Fmt<FMT>::S, cc);
        nd = S.tn[jg];
        s = select_finish<3, RANGE>(k, jg, nd.x, k.tab.inv_dl[3], Te, clamp, cc.near);
    }
    const int j = s.j;
    const int o = j - cc.base;
    const float w = s.w;
    const float Ls = lerpf(cc.win[o * kThreads], cc.win[(o + 1) * kThreads], w) + c.ls_off;
    const float Lb = lerpf(nd.z, nd.w, w) + c.lb_off;
    return energy_from_logs(c, Ls, Lb, nd.y + s.r);
}

// The same energy on the paper's table layout (Sec. 3.1): the total rate,
// bridge included, interpolated from one 4-D table (c.row points into it):
// q = 2^(L + log2(h / e_scale)).  FP32 table format only.
template <bool EXACT>
__device__ __forceinline__ float cool_energy_total(const StepK& k, const Smem& S, const CellC& c, Cache& cc,
                                                   float Te, unsigned& clamp) {
    const int nT = k.tab.n[3];
    const float* axT = S.ax + k.tab.axis_off[3];
    const SelW s = select_sub<3, EXACT>(k, axT + nT, nT, k.tab.inv_dl[3], Te, clamp, cc.near);
    const int j = s.j;
    if ((unsigned)(j - cc.base) > (unsigned)(Fmt<0>::S - 1)) gather<0>(c, j / Fmt<0>::S, cc);
    const int o = j - cc.base;
    const float L = lerpf(cc.win[o * kThreads], cc.win[(o + 1) * kThreads], s.w) + c.ls_off;
    return ex2a(fminf(L, 126.f));
}

// Node 0 of T_e block 0 of a corner row (the words that hold it, read with
// plain loads; the same decoding as dec<FMT>(r, 0)).
template <int FMT>
__device__ __forceinline__ float node0(const uint32_t* p) {
    if (FMT == 0) return __uint_as_float(__ldg(p));
    if (FMT == 1 || FMT == 2) return half_bits(__ldg(p) & 0xffffu, FMT == 2);
    return fmaf(__uint_as_float(__ldg(p + 1)), half_bits(__ldg(p + 2) & 0xffffu, FMT == 4), __uint_as_float(__ldg(p)));
}

// cool_energy at a key below half the first T_e node: the selection there
// is interval 0 with weight 0 (in EXACT mode too), so the synchrotron value
// is node 0 collapsed over the H, B, n_e corners -- computed here from the
// eight corners' node-0 words in the order gather uses, without moving the
// window -- and the result is the one cool_energy returns, bit for bit.
template <int FMT>
__device__ __forceinline__ float cool_energy_below(const StepK& k, const Smem& S, const CellC& c, float Te) {
    const int nT = k.tab.n[3];
    const float* axT = S.ax + k.tab.axis_off[3];
    const uint32_t* p = c.row;
    const uint32_t* q = p + c.oH;
    const float v0 = lerpf(lerpf(node0<FMT>(p), node0<FMT>(p + c.oN), c.wn),
                           lerpf(node0<FMT>(p + c.oB), node0<FMT>(p + c.oB + c.oN), c.wn), c.wb);
    const float v1 = lerpf(lerpf(node0<FMT>(q), node0<FMT>(q + c.oN), c.wn),
                           lerpf(node0<FMT>(q + c.oB), node0<FMT>(q + c.oB + c.oN), c.wn), c.wb);
    const float r = lg2a(Te * axT[nT]);   // log2(T_e / x_0), as select_finish forms it
    return energy_from_logs(c, lerpf(v0, v1, c.wh) + c.ls_off, S.lb[0] + c.lb_off, axT[2 * nT] + r);
}

// Backward Euler u' = u0 - q(u') of a stiff cell (q(u0) > limiter u0) in
// FP32.  Bracket [u0 2^-60, u0]: g(u0) = q(u0) > 0 and g(u0 2^-60) < 0 is
// checked (false when it fails).  Illinois (modified regula falsi) first on
// G(x) = log2((2^x + q(2^x))/u0), x = log2 u, which is close to piecewise
// linear over the 60 octaves, then on g(u) = u + q(u) - u0 in u once the
// bracket is tight (FP32 x cannot resolve u to better than ~1e-6).  At most
// implicit_iters evaluations.
template <int FMT, bool EXACT>
__device__ __forceinline__ bool implicit_fp32(const StepK& k, const Smem& S, const CellC& c, Cache& cc,
                                           float inv_e, float u0, float q0, float& u_out) {
    const float inv_u0 = 1.f / u0;
    unsigned trial = 0u;  // trial points of the solve do not count as clamped keys
    float xb = lg2a(u0);
    float xa = xb - 60.f;
    const float ua0 = ex2a(xa);
    // the lower end lies 60 octaves below u0, far below the T_e axis: its
    // energy comes from node 0 without moving the window, which keeps the
    // block the next trial points (near the root) need
    const float ta0 = ua0 * inv_e;
    const float qa0 = ta0 < 0.5f * k.g_x0[3] ? cool_energy_below<FMT>(k, S, c, ta0)
                                             : cool_energy<FMT, EXACT, true>(k, S, c, cc, ta0, trial);
    if (!(ua0 - u0 + qa0 < 0.f)) return false;
    float Gb = lg2a(fmaf(q0, inv_u0, 1.f));
    float Ga = lg2a((ua0 + qa0) * inv_u0);
    int side = 0, it = 0;
    for (; it < k.iters; ++it) {
        if (xb - xa < 1e-3f) break;
        float x = xb - Gb * (xb - xa) / (Gb - Ga);
        if (!(x > xa && x < xb)) x = 0.5f * (xa + xb);
        const float u = ex2a(x);
        const float G = lg2a((u + cool_energy<FMT, EXACT, true>(k, S, c, cc, u * inv_e, trial)) * inv_u0);
        if (G > 0.f) {
            xb = x; Gb = G;
            if (side == 1) Ga *= 0.5f;
            side = 1;
        } else {
            xa = x; Ga = G;
            if (side == -1) Gb *= 0.5f;
            side = -1;
        }
    }
    float a = ex2a(xa), b = ex2a(xb);
    float ga = a - u0 + cool_energy<FMT, EXACT, true>(k, S, c, cc, a * inv_e, trial);
    float gb = b - u0 + cool_energy<FMT, EXACT, true>(k, S, c, cc, b * inv_e, trial);
    // an end whose residual rounds to the wrong sign is the root to rounding
    float u = !(ga < 0.f) ? a : (!(gb > 0.f) ? b : 0.5f * (a + b));
    side = 0;
    for (; it < k.iters && ga < 0.f && gb > 0.f; ++it) {
        u = b - gb * (b - a) / (gb - ga);
        if (!(u > a && u < b)) u = 0.5f * (a + b);
        if (b - a <= 2.4e-7f * b) break;
        const float g = u - u0 + cool_energy<FMT, EXACT, true>(k, S, c, cc, u * inv_e, trial);
        if (g > 0.f) {
            b = u; gb = g;
            if (side == 1) ga *= 0.5f;
            side = 1;
        } else if (g < 0.f) {
            a = u; ga = g;
            if (side == -1) gb *= 0.5f;
            side = -1;
        } else {
            break;
        }
    }
    u_out = u;
    return true;
}

// The same solve in FP64 on the FP64 table (fp64_critical, FP32 fields):
// the cell's H, B, n_e selections with FP64 keys are made on its first
// stiff sub-cycle (c64.jt == -2) and kept in c64 for the next ones, with
// the collapse of the last T_e interval visited.  From u32, the
// FP32 solve's root (0: none), Newton steps on g(u) = u - u0 + q(u) with
// g' = 1 + dq/du of the same interpolation: from the FP32 root's ~1e-6
// relative error two steps reach FP64 rounding.  Accepted when a step falls
// below 1e-14 u within 4 steps and every iterate stays within 2^-14 (in
// log2 u) of u32; otherwise (a kink of the interpolation on the way, or no
// FP32 root) implicit_fp64 solves from the bracket u32 2^+-(2^-14), or the
// whole one when g does not change sign over it.  The result is rounded to
// FP32.
__device__ __noinline__ bool implicit_fp64_cell(const StepK& k, const DevTable& T, float rho, float B, float H,
                                                float u0, float& u_out, float u32, Cell64& c64) {
    unsigned dummy = 0u;
    if (c64.jt == -2) {
        c64.jt = -1;
        c64.ne = (double)rho * k.k64.s_n;
        c64.Hc = (double)H * k.k64.s_H;
        c64.jh = select64(T, 0, c64.Hc, c64.wh, dummy);
        c64.jb = select64(T, 1, (double)B * k.k64.s_B, c64.wb, dummy);
        c64.jn = select64(T, 2, c64.ne, c64.wn, dummy);
    }
    const double U0 = (double)u0;
    double x32 = nan64();
    if (u32 > 0.f) {
        const double ulo = (double)u32 * 0.9999576945484311, uhi = (double)u32 * 1.0000423072413958;
        double u = (double)u32;
        for (int it = 0; it < 4; ++it) {
            double dq = 0.0;
            const double q = cool_q64(k.k64, c64, u, (double)rho, dummy, &dq);
            const double g = u - U0 + q, gp = 1.0 + dq;
            if (!(gp > 0.0)) break;
            const double step = g / gp;
            const double un = u - step;
            if (!(un > ulo && un < uhi)) break;
            u = un;
            if (fabs(step) <= 1e-14 * u) {
                u_out = (float)u;
                return true;
            }
        }
        x32 = log2((double)u32);
    }
    double u1;
    if (!implicit_fp64(k.k64, c64, (double)rho, U0, u1, x32 - 0x1p-14, x32 + 0x1p-14)) return false;
    u_out = (float)u1;
    return true;
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


void fill_k64(const cool_table* t, const cool_params* p, StepK64& k) {
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
}

void fill_stepk(const cool_table* t, const cool_params* p, StepK& k) {
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
    k.fp64_critical = p->fp64_critical;
    fill_k64(t, p, k.k64);
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
    for (int a = 0; a < 5; ++a) {
        const int n = t->dev.n[a];
        const float* x = t->h_axes + t->dev.axis_off[a];
        k.g_c0[a] = (float)(-(double)x[2 * n] * (double)t->dev.inv_dl[a] - 0.5);
        k.g_hi[a] = (float)(n - 2);
        k.g_x0[a] = x[0];
        k.g_xn[a] = x[n - 1];
        k.g_wb[a] = (float)(0.5 - 1e-6 * (double)t->dev.inv_dl[a]);
    }
    // Row stride of the Coulomb channel in shared memory: the smallest one
    // >= n that is 5 mod 32.  A warp's cells hold a few (T_i, T_e) rows and
    // columns near each other; with the stride n + 1 (1 mod 32) corner (i, j)
    // shares its bank with (i + 1, j - 1), (i + 2, j - 2), ..., so the four
    // corner loads averaged 4.2 passes over the banks per warp on the 256^3
    // two-region cells; 5 mod 32 separates such neighbours (2.2 passes).
    {
        const int nc = t->dev.n[4];
        k.lc_stride = nc + (((5 - nc) % 32) + 32) % 32;
    }
    k.tn_off = (na + t->dev.n[3] + t->dev.n[4] * k.lc_stride + 3) & ~3;
    k.smem_floats = k.tn_off + 4 * (t->dev.n[3] - 1);
    k.sched = nullptr;
    k.dlist = nullptr;
}

}  // namespace
}  // namespace cool
