// cool_build.cu -- FP64 device evaluation of the cooling-rate table.
//
// One thread per table node evaluates the formulas of Sec. 2 of the paper
// (arXiv 2505.08855) in FP64:
//   bremsstrahlung e-e and e-i fits (Eqs. 1-2),
//   thermal synchrotron emissivity (Eq. 3) with Mahadevan's I'(x) (Eq. 4)
//   and K2(1/theta_e) -> 2 theta_e^2 at T_e <= k2_switch_T,
//   the self-absorption frequency nu_c from the annulus balance (Eq. 5),
//   Q_syn = Rayleigh-Jeans part below nu_c + thin integral above (Eq. 6),
//   the Compton enhancement eta(nu_c) (Eqs. 7-9; exponent -1 - ln P/ln A,
//   the truncated scattering series -- the printed 1 - ln P/ln A is a flag),
//   the Coulomb coefficient C = Q_cc / (n_e^2 (T_i - T_e)) (Eq. 16).
// The table stores log2 values (Sec. 2.6: log-spaced nodes; values in log2
// so that interpolation spans the 60-decade dynamic range).
#include <math.h>
#include <stdint.h>
#include <stdio.h>


#include "cool_internal.cuh"

namespace cool {
namespace {

__constant__ double c_glx[16];
__constant__ double c_glw[16];

// Gauss-Legendre abscissae/weights on [-1, 1] (16 points): Newton's method
// on P_16 seeded at the Chebyshev points; P and P' from the three-term
// recurrence and P'_n = n (x P_n - P_{n-1}) / (x^2 - 1).
void gl16_host(double* x, double* w) {
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        double r = cos(kPi * (2.0 * i + 1.0) / (2.0 * n));
        double pn = 0.0, dpn = 1.0;
        for (int iter = 0; iter < 200; ++iter) {
            double pm = 1.0, pc = r;
            for (int k = 1; k < n; ++k) {
                double pnext = ((2 * k + 1) * r * pc - k * pm) / (k + 1);
                pm = pc;
                pc = pnext;
            }
            pn = pc;
            dpn = n * (r * pc - pm) / (r * r - 1.0);
            double step = pn / dpn;
            r -= step;
            if (fabs(step) <= 1e-17) break;
        }
        // final derivative at the converged root
        double pm = 1.0, pc = r;
        for (int k = 1; k < n; ++k) {
            double pnext = ((2 * k + 1) * r * pc - k * pm) / (k + 1);
            pm = pc;
            pc = pnext;
        }
        dpn = n * (r * pc - pm) / (r * r - 1.0);
        x[i] = r;
        w[i] = 2.0 / ((1.0 - r * r) * dpn * dpn);
    }
}

__device__ __forceinline__ double theta_e(double T) { return T * (kKB / (kME * kC * kC)); }

// Bremsstrahlung per n_e^2 (Eqs. 1-2).
__device__ double brems_n2(double T) {
    double th = theta_e(T);
    double ee, ei;
    if (th < 1.0) {
        double th15 = th * sqrt(th);
        ee = th15 * (1.0 + 1.1 * th + th * th - 1.25 * th * th15);
        ei = 4.0 * sqrt(2.0 * th / (kPi * kPi * kPi)) * (1.0 + 1.781 * pow(th, 1.34));
    } else {
        ee = 1.34 * th * (log(1.123 * th) + 1.28);
        ei = 9.0 * th / (2.0 * kPi) * (log(1.123 * th + 0.48) + 1.5);
    }
    return 2.56e-22 * ee + 1.48e-22 * ei;
}

// Scaled modified Bessel functions e^z K_nu(z), nu = 0, 1, 2.
// z <= 2: ascending series (Abramowitz & Stegun 9.6.13 for K_0, 9.6.11 with
// n = 1 for K_1) and K_2 = K_0 + 2 K_1 / z.
// z > 2: with cosh t - 1 = 2 s^2 (s = sinh(t/2)) the integral
// K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt becomes
// e^z K_nu(z) = int_0^inf exp(-2 z s^2) c_nu(s) 2/sqrt(1+s^2) ds with
// c_0 = 1, c_1 = 1 + 2 s^2, c_2 = 1 + 8 s^2 + 8 s^4; the integrand is even
// and analytic in |Im s| < 1, so the trapezoidal rule converges
// exponentially (step h = min(0.05, 0.3/sqrt z)).
__device__ void kve012(double z, double& k0, double& k1, double& k2) {
    const double euler = 0.57721566490153286061;
    if (z <= 2.0) {
        double q = 0.25 * z * z;
        double lnh = log(0.5 * z);
        double term0 = 1.0;         // q^k / (k!)^2
        double term1 = 1.0;         // q^k / (k! (k+1)!)
        double i0 = 0.0, i1s = 0.0, s0 = 0.0, s1 = 0.0;
        double hk = 0.0;            // harmonic number H_k
        double psi1 = -euler;       // psi(k+1)
        double psi2 = 1.0 - euler;  // psi(k+2)
        for (int k = 0; k < 60; ++k) {
            i0 += term0;
            i1s += term1;
            s0 += hk * term0;
            s1 += (psi1 + psi2) * term1;
            double kk = k + 1.0;
            term0 *= q / (kk * kk);
            term1 *= q / (kk * (kk + 1.0));
            hk += 1.0 / kk;
            psi1 += 1.0 / kk;
            psi2 += 1.0 / (kk + 1.0);
            if (term0 < 1e-18 * i0 && term1 < 1e-18 * i1s) break;
        }
        double K0 = -(lnh + euler) * i0 + s0;
        double I1 = 0.5 * z * i1s;
        double K1 = 1.0 / z + lnh * I1 - 0.25 * z * s1;
        double ez = exp(z);
        k0 = K0 * ez;
        k1 = K1 * ez;
        k2 = k0 + 2.0 * k1 / z;
        return;
    }
    double h = fmin(0.05, 0.3 / sqrt(z));
    double a0 = 0.5, a1 = 0.5, a2 = 0.5;  // s = 0: weights 1/2, c_nu(0) = 1, 2/sqrt(1) = 2 applied below
    for (int k = 1; k < 4000; ++k) {
        double s = k * h;
        double s2 = s * s;
        double ex = 2.0 * z * s2;
        if (ex > 745.0) break;
        double g = exp(-ex) / sqrt(1.0 + s2);
        a0 += g;
        a1 += g * (1.0 + 2.0 * s2);
        a2 += g * (1.0 + 8.0 * s2 + 8.0 * s2 * s2);
        if (ex > 45.0) break;
    }
    k0 = 2.0 * h * a0;
    k1 = 2.0 * h * a1;
    k2 = 2.0 * h * a2;
}

// log of Mahadevan's I'(x) (Eq. 4).
__device__ double log_iprime(double x) {
    double rx = 1.0 / sqrt(x);
    return log(4.0505) - log(x) * (1.0 / 6.0) + log1p(0.4 * sqrt(rx) + 0.5316 * rx) - 1.8899 * cbrt(x);
}

// Integrand of int x I'(x) dx in s = x^(1/3): 3 s^5 I'(s^3)
// = 3 * 4.0505 s^4.5 (1 + 0.4 s^-0.75 + 0.5316 s^-1.5) e^(-1.8899 s).
__device__ double syn_integrand(double s) {
    if (!(s > 0.0)) return 0.0;
    double r = sqrt(s);
    double q = sqrt(r);
    double s2 = s * s;
    return 12.1515 * s2 * s2 * r * (1.0 + 0.4 / (r * q) + 0.5316 / (s * r)) * exp(-1.8899 * s);
}

// J(x_c) = int_{x_c}^inf x I'(x) dx: 16-point Gauss-Legendre on 64 equal
// panels of s = x^(1/3) over [x_c^(1/3), x_c^(1/3) + 40].
__device__ double syn_tail_integral(double xc) {
    const int panels = 64;
    const double width = 40.0 / panels;
    double s0 = cbrt(xc);
    double total = 0.0;
    for (int p = 0; p < panels; ++p) {
        double c = s0 + (p + 0.5) * width;
        double acc = 0.0;
#pragma unroll 4
        for (int i = 0; i < 16; ++i) acc += c_glw[i] * syn_integrand(c + 0.5 * width * c_glx[i]);
        total += acc;
    }
    return 0.5 * width * total;
}

struct SynOut { double eta_qsyn; int flag; };

// eta(nu_c) * Q_syn at one node (Eqs. 3-9).
__device__ SynOut eta_qsyn(double H, double B, double ne, double T, double k2_switch_T,
                           int compton_literal) {
    double th = theta_e(T);
    double k2f;
    if (T <= k2_switch_T) {
        k2f = 2.0 * th * th;
    } else {
        double z = 1.0 / th, a, b, c;
        kve012(z, a, b, c);
        k2f = c * exp(-z);
    }
    double nu0 = 3.0 * kQE * B * th * th / (4.0 * kPi * kME * kC);
    double pref = 4.43e-30 * 4.0 * kPi * ne / k2f;       // eps_s = pref * nu * I'(nu/nu0)
    // Eq. 5 in x = nu/nu0:  ln I'(x) - ln x = ln(2 pi k T / c^2) - ln(H pref / nu0)
    double L = log(2.0 * kPi * kKB * T / (kC * kC)) - log(H * pref / nu0);
    double lnnu0 = log(nu0);
    double a = -lnnu0, b = log(1e30) - lnnu0;             // nu in [1 Hz, 1e30 Hz]
    double nuc;
    int flag = 0;
    if (log_iprime(exp(a)) - a - L <= 0.0) {
        nuc = 1.0;
    } else if (log_iprime(exp(b)) - b - L > 0.0) {
        nuc = 1e30;
        flag = 1;
    } else {
        for (int it = 0; it < 200 && (b - a) >= 1e-14; ++it) {
            double m = 0.5 * (a + b);
            if (log_iprime(exp(m)) - m - L > 0.0) a = m; else b = m;
        }
        nuc = exp(lnnu0 + 0.5 * (a + b));
    }
    // Eq. 6: Rayleigh-Jeans part (per unit volume of the annulus) + thin part
    double qsyn = 2.0 * kPi * kKB * T * nuc * nuc * nuc / (3.0 * kC * kC * H)
                + pref * nu0 * nu0 * syn_tail_integral(nuc / nu0);
    // Eqs. 7-9 at nu_c
    double E = kHP * nuc / (kME * kC * kC);
    double eta = 1.0;
    if (E < 3.0 * th) {
        double tau = 2.0 * ne * kSigT * H;
        double P = -expm1(-tau);
        double am1 = 4.0 * th * (1.0 + 4.0 * th);          // A - 1
        double lnA = log1p(am1);
        if (compton_literal) {
            double ex = 1.0 - log(P) / lnA;
            eta = 1.0 + P * am1 / (1.0 - P * (1.0 + am1)) * (1.0 - pow(E / (3.0 * th), ex));
        } else if (P > 0.0) {
            double kk = log(3.0 * th / E) / lnA;            // scatterings to reach 3 theta
            double eps = log(P) + lnA;                       // ln(P A)
            double ratio = (eps == 0.0) ? kk : expm1(kk * eps) / expm1(eps);
            eta = 1.0 + P * am1 * ratio;
        }
    }
    SynOut o;
    o.eta_qsyn = eta * qsyn;
    o.flag = flag;
    return o;
}

// Coulomb coefficient (Eq. 16) with scaled Bessel functions; the factors
// e^(-1/theta) cancel because 1/theta_m = 1/theta_e + 1/theta_i.
__device__ double coulomb_coeff(double Ti, double Te, double lnLambda, int theta_i_uses_mp) {
    double the = theta_e(Te);
    double mi = theta_i_uses_mp ? kMP : kME;
    double thi = Ti * (kKB / (mi * kC * kC));
    double ze = 1.0 / the, zi = 1.0 / thi;
    double zm = ze + zi;
    double a0, a1, a2, e0, e1, e2, m0, m1, m2;
    kve012(zi, a0, a1, a2);
    kve012(ze, e0, e1, e2);
    kve012(zm, m0, m1, m2);
    double sum = the + thi;
    double bracket = (2.0 * sum * sum + 1.0) / sum * m1 + 2.0 * m0;
    return 1.5 * (kME / kMP) * lnLambda * kC * kSigT * kKB * bracket / (a2 * e2);
}

// ---------------------------------------------------------------------------
// The step with every rate from the formulas (no table): the paper's
// "analytic" comparison (Appendix: direct calculation against the table).
// FP64 fields and arithmetic; per sub-cycle one nu_c root (Eq. 5), one
// 1024-point quadrature (Eq. 6), the Compton factor (Eqs. 7-9), the
// bremsstrahlung fits (Eqs. 1-2), the bridge (Eqs. 11-12, sigma_SB) and the
// Coulomb coefficient (Eq. 16) with three scaled Bessel triples.  The update
// is the one of the table step: Coulomb exchange clamped at T_e = T_i, then
// cooling, explicit with the limiter or implicit (bisection in log2 u) in
// stiff cells.
// ---------------------------------------------------------------------------
struct DirectK {
    double s_n, s_B, s_H, s_Te, s_Ti, ce, ci, hs, escale;
    double limiter, eq_band, clamp;
    int n_sub, mode, iters;
    double k2_switch_T, lnLambda;
    int theta_i_uses_mp, compton_literal;
};

__device__ double direct_q(const DirectK& k, double ne, double Bg, double Hc, double u, double rho,
                           unsigned& cap) {
    const double T = k.s_Te * u / rho;
    const SynOut so = eta_qsyn(Hc, Bg, ne, T, k.k2_switch_T, k.compton_literal);
    cap |= (unsigned)so.flag;
    const double qthin = ne * ne * brems_n2(T) + so.eta_qsyn;
    const double T2 = T * T;
    const double tau_abs = Hc * qthin / (4.0 * kSigSB * T2 * T2);
    const double tau_sca = 2.0 * ne * kSigT * Hc;
    const double Q = qthin / (1.0 + tau_abs * (1.7320508075688772 + 1.5 * (tau_abs + tau_sca)));
    return k.hs * Q / k.escale;
}

__global__ void k_step_direct(DirectK k, long long n, const double* rho_in, const double* B_in, const double* H_in,
                              const double* ue_in, const double* ui_in, double* ue_out, double* ui_out,
                              double* qc_out, double* qx_out, cool_counters* cnt) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double rho = rho_in[i], B = B_in[i], H = H_in[i], ue = ue_in[i], ui = ui_in[i];
        unsigned cap = 0u, stiff = 0u, band = 0u, fail = 0u, invalid = 0u;
        double sum_q = 0.0, sum_x = 0.0;
        if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) || !(rho > 0.0) ||
            !(ue > 0.0) || !(ui > 0.0) || B < 0.0 || H < 0.0) {
            invalid = 1u;
        } else {
            const double ne = rho * k.s_n, Bg = B * k.s_B, Hc = H * k.s_H;
            for (int sub = 0; sub < k.n_sub; ++sub) {
                const double Te = k.s_Te * ue / rho, Ti = k.s_Ti * ui / rho;
                if (fabs(Te / Ti - 1.0) <= k.eq_band) band = 1u;
                const double C = coulomb_coeff(Ti, Te, k.lnLambda, k.theta_i_uses_mp);
                double X = k.hs * ne * ne * C * (Ti - Te) / k.escale;
                const double lim = k.clamp * fabs((k.ci * ui - k.ce * ue) / (k.ce + k.ci));
                if (fabs(X) > lim) X = copysign(lim, X);
                ue += X;
                ui -= X;
                sum_x += X;
                const double q = direct_q(k, ne, Bg, Hc, ue, rho, cap);
                double du;
                if (k.mode == 1 && q > k.limiter * ue) {
                    stiff = 1u;
                    double a = log2(ue) - 60.0, b = log2(ue);
                    const double ga = exp2(a) - ue + direct_q(k, ne, Bg, Hc, exp2(a), rho, cap);
                    if (!(ga < 0.0)) {
                        fail = 1u;
                        du = k.limiter * ue;
                    } else {
                        for (int it = 0; it < k.iters; ++it) {
                            const double m = 0.5 * (a + b);
                            const double um = exp2(m);
                            if (um - ue + direct_q(k, ne, Bg, Hc, um, rho, cap) > 0.0) b = m; else a = m;
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
        if (cnt) {
            if (cap) atomicAdd(&cnt->n_clamped, 1ull);
            if (invalid) atomicAdd(&cnt->n_nonfinite, 1ull);
            if (stiff) atomicAdd(&cnt->n_stiff, 1ull);
            if (band) atomicAdd(&cnt->n_fp64_coulomb, 1ull);
            if (fail) atomicAdd(&cnt->n_implicit_fail, 1ull);
        }
    }
}

struct BuildArgs {
    const double* x64;  // node coordinates, concatenated per axis
    int off[5];
    int n[5];
    double k2_switch_T, lnLambda;
    int theta_i_uses_mp, compton_literal;
};

__global__ void k_build_syn(BuildArgs a, long long first, long long count, double* out,
                            unsigned int* flags) {
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = first + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < first + count;
         i += stride) {
        long long r = i;
        int t = (int)(r % a.n[3]); r /= a.n[3];
        int n = (int)(r % a.n[2]); r /= a.n[2];
        int b = (int)(r % a.n[1]); r /= a.n[1];
        int h = (int)r;
        SynOut o = eta_qsyn(a.x64[a.off[0] + h], a.x64[a.off[1] + b], a.x64[a.off[2] + n],
                            a.x64[a.off[3] + t], a.k2_switch_T, a.compton_literal);
        out[i] = log2(o.eta_qsyn);
        if (o.flag) atomicAdd(flags, 1u);
    }
}

// The paper's table layout (Sec. 3.1): log2 Q_total at every node of the
// 4-D grid, the bridge of Eqs. 11-12 (sigma_SB) applied at the node's
// (H, n_e, T_e) to the table's own FP64 brems and synchrotron values.
__global__ void k_build_qtotal(BuildArgs a, const double* lb64, const double* ls64, double* out) {
    const long long total = (long long)a.n[0] * a.n[1] * a.n[2] * a.n[3];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += stride) {
        long long r = i;
        const int t = (int)(r % a.n[3]); r /= a.n[3];
        const int n = (int)(r % a.n[2]); r /= a.n[2];
        r /= a.n[1];
        const int h = (int)r;
        const double Hc = a.x64[a.off[0] + h], ne = a.x64[a.off[2] + n], T = a.x64[a.off[3] + t];
        const double qthin = ne * ne * exp2(lb64[t]) + exp2(ls64[i]);
        const double T2 = T * T;
        const double tau_abs = Hc * qthin / (4.0 * kSigSB * T2 * T2);
        const double tau_sca = 2.0 * ne * kSigT * Hc;
        out[i] = log2(qthin / (1.0 + tau_abs * (1.7320508075688772 + 1.5 * (tau_abs + tau_sca))));
    }
}

__global__ void k_build_small(BuildArgs a, double* lb, double* lc) {
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    int nT = a.n[3], nC = a.n[4];
    if (tid < nT) lb[tid] = log2(brems_n2(a.x64[a.off[3] + tid]));
    if (tid < nC * nC) {
        int i = tid / nC, e = tid % nC;
        lc[tid] = log2(coulomb_coeff(a.x64[a.off[4] + i], a.x64[a.off[4] + e], a.lnLambda,
                                     a.theta_i_uses_mp));
    }
}

// Counter-based generator: SplitMix64 of (seed, index) -> uniform in [0, 1).
__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Training samples of the synchrotron channel: even samples sit on a random
// table node, odd ones are uniform in log space over the table box;
// the label is log2(eta Q_syn) from the formulas (FP64).  x: normalised
// coordinates 2 (l - l_lo)/(l_hi - l_lo) - 1 per axis (H, B, n_e, T_e).
__global__ void k_fit_samples(BuildArgs a, double l0_0, double l0_1, double l0_2, double l0_3, double span0,
                              double span1, double span2, double span3, long long n,
                              unsigned long long seed, float* x, double* y) {
    const double l0[4] = {l0_0, l0_1, l0_2, l0_3};
    const double span[4] = {span0, span1, span2, span3};
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double l[4];
        for (int d = 0; d < 4; ++d) {
            const double u = u01(seed + 7919ull * d, (unsigned long long)i);
            if ((i & 1) == 0) {
                int j = (int)(u * a.n[d]);
                j = j > a.n[d] - 1 ? a.n[d] - 1 : j;
                l[d] = l0[d] + span[d] * j / (a.n[d] - 1);
            } else {
                l[d] = l0[d] + span[d] * u;
            }
            x[4 * i + d] = (float)(2.0 * (l[d] - l0[d]) / span[d] - 1.0);
        }
        SynOut o = eta_qsyn(exp2(l[0]), exp2(l[1]), exp2(l[2]), exp2(l[3]), a.k2_switch_T, a.compton_literal);
        y[i] = log2(o.eta_qsyn);
    }
}

}  // namespace

cool_status build_channels_fp64(const cool_table_spec& s, const double* d_axes64,
                                const int* axis_off64, double* d_lb64, double* d_ls64,
                                double* d_lc64, cudaStream_t st) {
    double gx[16], gw[16];
    gl16_host(gx, gw);
    cudaError_t e = cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    BuildArgs a;
    a.x64 = d_axes64;
    int n[5] = {s.n_H, s.n_B, s.n_ne, s.n_Te, s.n_Tc};
    for (int i = 0; i < 5; ++i) { a.off[i] = axis_off64[i]; a.n[i] = n[i]; }
    a.k2_switch_T = s.k2_switch_T;
    a.lnLambda = s.lnLambda;
    a.theta_i_uses_mp = s.theta_i_uses_mp;
    a.compton_literal = s.compton_literal;
    int small = n[3] > n[4] * n[4] ? n[3] : n[4] * n[4];
    k_build_small<<<(small + 127) / 128, 128, 0, st>>>(a, d_lb64, d_lc64);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    unsigned int* d_flags = nullptr;
    e = cudaMallocAsync(&d_flags, sizeof(unsigned int), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaMemsetAsync(d_flags, 0, sizeof(unsigned int), st);
    long long total = syn_count(s);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // chunks of ~4M nodes: each launch finishes in well under a second
    const long long chunk = 1LL << 22;
    for (long long first = 0; first < total; first += chunk) {
        long long cnt = total - first < chunk ? total - first : chunk;
        long long blocks = (cnt + 127) / 128;
        if (blocks > sms * 16LL) blocks = sms * 16LL;
        k_build_syn<<<(int)blocks, 128, 0, st>>>(a, first, cnt, d_ls64, d_flags);
        e = cudaGetLastError();
        if (e != cudaSuccess) { cudaFreeAsync(d_flags, st); return set_cuda_error(e); }
    }
    cudaFreeAsync(d_flags, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}


cool_status build_qtotal_fp64(const cool_table_spec& s, const double* d_axes64, const int* axis_off64,
                              const double* d_lb64, const double* d_ls64, double* d_lt64, cudaStream_t st) {
    BuildArgs a;
    a.x64 = d_axes64;
    int n[5] = {s.n_H, s.n_B, s.n_ne, s.n_Te, s.n_Tc};
    for (int i = 0; i < 5; ++i) { a.off[i] = axis_off64[i]; a.n[i] = n[i]; }
    a.k2_switch_T = s.k2_switch_T;
    a.lnLambda = s.lnLambda;
    a.theta_i_uses_mp = s.theta_i_uses_mp;
    a.compton_literal = s.compton_literal;
    const long long total = syn_count(s);
    long long blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_build_qtotal<<<(int)blocks, 256, 0, st>>>(a, d_lb64, d_ls64, d_lt64);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

cool_status launch_step_direct(const cool_table_spec& phys, const cool_params* p, long long n, const double* rho,
                               const double* B, const double* H, const double* ue, const double* ui, double* ue_o,
                               double* ui_o, double* qc, double* qx, cool_counters* cnt, cudaStream_t st) {
    if (n == 0) return COOL_OK;
    double gx[16], gw[16];
    gl16_host(gx, gw);
    cudaError_t e = cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    DirectK k;
    const double rg = (kG * (p->M_bh_msun * kMsun)) / (kC * kC);
    k.s_n = p->rho_scale / kMP;
    k.s_B = sqrt(4.0 * kPi * p->rho_scale) * kC;
    k.s_H = rg;
    k.ce = p->gamma_e - 1.0;
    k.ci = p->gamma_i - 1.0;
    k.s_Te = k.ce * kMP * kC * kC / kKB;
    k.s_Ti = k.ci * kMP * kC * kC / kKB;
    k.hs = p->dt * (rg / kC) / p->n_sub;
    k.escale = p->rho_scale * kC * kC;
    k.limiter = p->limiter_frac;
    k.eq_band = p->eq_band;
    k.clamp = p->coulomb_clamp;
    k.n_sub = p->n_sub;
    k.mode = (int)p->mode;
    k.iters = p->implicit_iters;
    k.k2_switch_T = phys.k2_switch_T;
    k.lnLambda = phys.lnLambda;
    k.theta_i_uses_mp = phys.theta_i_uses_mp;
    k.compton_literal = phys.compton_literal;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n + 127) / 128;
    if (blocks > sms * 16LL) blocks = sms * 16LL;
    k_step_direct<<<(int)blocks, 128, 0, st>>>(k, n, rho, B, H, ue, ui, ue_o, ui_o, qc, qx, cnt);
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

// ---------------------------------------------------------------------------
// Caller-allocated table build: the variant of the builder above that
// allocates no device memory.  The builder's scratch (FP64 node coordinates
// of the five axes and the nu_c-cap flag counter) lives in one file-scope
// device array instead of cudaMallocAsync'd buffers; the caller passes the
// three FP64 output channels.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocAxisMax = 256;                     // nodes per axis the scratch holds
constexpr size_t kNoAllocNodeBytes = sizeof(double) * 5 * 2 * kNoAllocAxisMax;   // 20 KiB
constexpr size_t kNoAllocScratchBytes = kNoAllocNodeBytes + 256;                 // + flag word

// Every device that loads the library holds this array until the process
// exits.  Layout: axis a at doubles [a*2*256, a*2*256 + 256) = x_j and
// [a*2*256 + 256, (a+1)*2*256) = l_j; the flag counter at byte
// kNoAllocNodeBytes.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Node coordinates of the five axes into the scratch: l_j = l0 + j dl,
// x_j = 2^l_j (the same node definition as the allocating build).
__global__ void k_noalloc_nodes(double* nodes, double l0_0, double l0_1, double l0_2, double l0_3,
                                double dl0, double dl1, double dl2, double dl3, int n0, int n1, int n2,
                                int n3, int n4, double dl4) {
    int a = blockIdx.x;
    int j = threadIdx.x;
    double l0 = a == 0 ? l0_0 : a == 1 ? l0_1 : a == 2 ? l0_2 : l0_3;
    double dl = a == 0 ? dl0 : a == 1 ? dl1 : a == 2 ? dl2 : a == 3 ? dl3 : dl4;
    int n = a == 0 ? n0 : a == 1 ? n1 : a == 2 ? n2 : a == 3 ? n3 : n4;
    if (j < n) {
        double l = l0 + j * dl;
        nodes[a * 2 * kNoAllocAxisMax + j] = exp2(l);
        nodes[a * 2 * kNoAllocAxisMax + kNoAllocAxisMax + j] = l;
    }
}

// Per call, with the caller's device current: the device address of the
// scratch array (in host code its name is only a host-side stand-in), looked
// up every call so that a re-created context never sees a stale address,
// and the Gauss-Legendre constants uploaded on the caller's stream, as the
// allocating build does, so a context whose constant memory was reset
// integrates with the right nodes.
cool_status noalloc_setup(cudaStream_t st, unsigned char** scratch) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return set_cuda_error(e);
    double gx[16], gw[16];
    gl16_host(gx, gw);
    e = cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    *scratch = (unsigned char*)ptr;
    return COOL_OK;
}

}  // namespace
}  // namespace cool

extern "C" cool_status cool_build_channels_noalloc(const cool_table_spec* spec, double* lb_out,
                                                   double* ls_out, double* lc_out, void* stream) {
    using namespace cool;
    if (!spec || !lb_out || !ls_out || !lc_out) return COOL_ENULL;
    const cool_table_spec& s = *spec;
    int n[5] = {s.n_H, s.n_B, s.n_ne, s.n_Te, s.n_Tc};
    for (int a = 0; a < 5; ++a)
        if (n[a] < 2) return COOL_EINVAL;
    for (int a = 0; a < 5; ++a)
        if (n[a] > kNoAllocAxisMax) return COOL_EINVAL;   // beyond the fixed scratch
    double lo[4] = {s.H_min, s.B_min, s.ne_min, s.T_min};
    double hi[4] = {s.H_max, s.B_max, s.ne_max, s.T_max};
    for (int a = 0; a < 4; ++a)
        if (!(lo[a] > 0.0) || !(hi[a] > lo[a]) || !isfinite(hi[a])) return COOL_EINVAL;
    if (!(s.k2_switch_T >= 0.0) || !(s.lnLambda > 0.0)) return COOL_EINVAL;
    if ((s.theta_i_uses_mp != 0 && s.theta_i_uses_mp != 1) ||
        (s.compton_literal != 0 && s.compton_literal != 1))
        return COOL_EINVAL;
    if (((uintptr_t)lb_out | (uintptr_t)ls_out | (uintptr_t)lc_out) % 8 != 0) return COOL_EALIGN;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaStream_t cs = (cudaStream_t)stream;
    unsigned char* scratch = nullptr;
    cool_status st = noalloc_setup(cs, &scratch);
    if (st != COOL_OK) return st;
    double* nodes = (double*)scratch;
    unsigned int* flags = (unsigned int*)(scratch + kNoAllocNodeBytes);
    double l0[5], dl[5];
    double lo5[5] = {s.H_min, s.B_min, s.ne_min, s.T_min, s.T_min};
    double hi5[5] = {s.H_max, s.B_max, s.ne_max, s.T_max, s.T_max};
    for (int a = 0; a < 5; ++a) {
        l0[a] = log2(lo5[a]);
        dl[a] = (log2(hi5[a]) - l0[a]) / (n[a] - 1);
    }
    // the Coulomb axis shares T_min with the T_e axis: l0[4] == l0[3]
    k_noalloc_nodes<<<5, kNoAllocAxisMax, 0, cs>>>(nodes, l0[0], l0[1], l0[2], l0[3], dl[0], dl[1], dl[2],
                                                    dl[3], n[0], n[1], n[2], n[3], n[4], dl[4]);
    e = cudaMemsetAsync(flags, 0, sizeof(unsigned int), cs);   // the counter starts at zero every call
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    BuildArgs a;
    a.x64 = nodes;
    for (int i = 0; i < 5; ++i) {
        a.off[i] = i * 2 * kNoAllocAxisMax;
        a.n[i] = n[i];
    }
    a.k2_switch_T = s.k2_switch_T;
    a.lnLambda = s.lnLambda;
    a.theta_i_uses_mp = s.theta_i_uses_mp;
    a.compton_literal = s.compton_literal;
    // BuildArgs addresses l_j at off + n; in the scratch l_j sits at off + 256
    // and is not read by the build kernels (they use x_j only).
    int small = n[3] > n[4] * n[4] ? n[3] : n[4] * n[4];
    k_build_small<<<(small + 127) / 128, 128, 0, cs>>>(a, lb_out, lc_out);
    long long total = (long long)n[0] * n[1] * n[2] * n[3];
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long chunk = 1LL << 22;
    for (long long first = 0; first < total; first += chunk) {
        long long cnt = total - first < chunk ? total - first : chunk;
        long long blocks = (cnt + 127) / 128;
        if (blocks > sms * 16LL) blocks = sms * 16LL;
        k_build_syn<<<(int)blocks, 128, 0, cs>>>(a, first, cnt, ls_out, flags);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

namespace cool {

cool_status fit_samples_fp64(const cool_table_spec& s, long long n, unsigned long long seed, float* x, double* y,
                             cudaStream_t st) {
    BuildArgs a;
    a.x64 = nullptr;
    int nn[5] = {s.n_H, s.n_B, s.n_ne, s.n_Te, s.n_Tc};
    for (int i = 0; i < 5; ++i) { a.off[i] = 0; a.n[i] = nn[i]; }
    a.k2_switch_T = s.k2_switch_T;
    a.lnLambda = s.lnLambda;
    a.theta_i_uses_mp = s.theta_i_uses_mp;
    a.compton_literal = s.compton_literal;
    double gx[16], gw[16];
    gl16_host(gx, gw);
    cudaError_t e = cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    double lo[4] = {s.H_min, s.B_min, s.ne_min, s.T_min}, hi[4] = {s.H_max, s.B_max, s.ne_max, s.T_max};
    double l0[4], sp[4];
    for (int d = 0; d < 4; ++d) { l0[d] = log2(lo[d]); sp[d] = log2(hi[d]) - l0[d]; }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long chunk = 1LL << 22;
    for (long long first = 0; first < n; first += chunk) {
        long long cnt = n - first < chunk ? n - first : chunk;
        long long blocks = (cnt + 127) / 128;
        if (blocks > sms * 16LL) blocks = sms * 16LL;
        k_fit_samples<<<(int)blocks, 128, 0, st>>>(a, l0[0], l0[1], l0[2], l0[3], sp[0], sp[1], sp[2], sp[3], cnt,
                                                   seed + (unsigned long long)first * 31ull, x + 4 * first, y + first);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return COOL_OK;
}

}  // namespace cool
