/*
 * cool_oracle.c -- plain, slow, FP64 CPU oracle of the two-temperature
 * cooling source step (Motta et al., arXiv 2505.08855).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link or call this file.  It is used by
 * tests/, by __graft_entry__.smoke() and by the cpu_baseline leg of bench.py.
 * It shares no code, header, constant table or helper with the CUDA path.
 *
 * Two levels (both FP64, cgs units):
 *   O1  the direct formulas of Sec. 2 (bremsstrahlung Eqs. 1-2, synchrotron
 *       Eqs. 3-6, Compton enhancement Eqs. 7-9, thin cooling Eq. 10, the
 *       optically-thick bridge Eqs. 11-12, Coulomb exchange Eq. 16);
 *   O2  the table of Sec. 2.6 / 2.8 built from O1 on log-spaced nodes, read by
 *       multilinear interpolation in log2 space, and the sub-cycled energy
 *       update of Sec. 3.2 (explicit with the 30 % limiter, or implicit).
 *
 * Readings of the paper where it is silent, garbled or inconsistent:
 *   - sigma in Eq. 11 and in tau_abs (Eq. 12) is Stefan-Boltzmann's constant
 *     (the printed sigma_T is dimensionally impossible there);
 *   - the Compton exponent is -1 - ln P / ln A (the truncated geometric series
 *     of scatterings); the printed 1 - ln P / ln A is available as a flag;
 *   - ln(Lambda) = 20 by default (spec field), theta_i = kT_i/(m_p c^2) by
 *     default (flag for the printed m_e);
 *   - nu_c is the root of Eq. 5, found by bisection in ln(nu);
 *   - K2(1/theta_e) -> 2 theta_e^2 for T_e <= k2_switch_T (1e8 K), literally;
 *   - the table stores log2 values; brems and Coulomb are factored by n_e^2
 *     (exact), the synchrotron channel is eta*Q_syn on the 4-D grid;
 *   - the optically-thick bridge is applied at run time per sub-cycle.
 *
 * Parity pins: every function below is pinned by tests/test_oracle_*.py to
 * closed forms, limits, library special functions or brute force; see the
 * per-function comments.  No function here is "parity unpinned" except the
 * absolute agreement with the authors' own (unpublished) table values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Physical constants, cgs, CODATA 2018.                                  */
/* ---------------------------------------------------------------------- */
#define O_C     2.99792458e10
#define O_KB    1.380649e-16
#define O_ME    9.1093837015e-28
#define O_MP    1.67262192369e-24
#define O_QE    4.80320471e-10
#define O_H     6.62607015e-27
#define O_SIGT  6.6524587321e-25
#define O_SIGSB 5.670374419e-5
#define O_G     6.6743e-8
#define O_MSUN  1.98847e33
#define O_PI    3.14159265358979323846

double orc_const(int i) {
    switch (i) {
    case 0: return O_C;   case 1: return O_KB;  case 2: return O_ME;
    case 3: return O_MP;  case 4: return O_QE;  case 5: return O_H;
    case 6: return O_SIGT; case 7: return O_SIGSB; case 8: return O_G;
    case 9: return O_MSUN;
    default: return NAN;
    }
}

/* ---------------------------------------------------------------------- */
/* Spec / params (the oracle's own definitions).                          */
/* ---------------------------------------------------------------------- */
typedef struct {
    int n[5];          /* axis sizes: 0 H, 1 B, 2 n_e, 3 T_e (cooling), 4 T (Coulomb, both axes) */
    double lo[5], hi[5];
    double k2_switch_T;
    double lnLambda;
    int theta_i_uses_mp;
    int compton_literal;
} orc_spec;

typedef struct {
    double rho_scale, M_bh_msun, gamma_e, gamma_i, dt;
    int n_sub, mode;               /* mode 0: explicit limited, 1: implicit in stiff cells */
    double limiter_frac, eq_band, coulomb_clamp;
    int implicit_iters;
} orc_params;

/* Disk geometry of a cell (Sec. 2.7 scale height, Sec. 3.2.3 temperature
 * floor): r in r_g per cell, the black-hole spin a.  h_from_state: the
 * thermal scale height H_th = c_s / Omega_K from the cell's own state
 * replaces the H field; h_floor > 0: no cooling in a sub-cycle whose gas
 * temperature P/rho is below T_floor = (pi/2) (h_floor Omega_K r)^2. */
typedef struct {
    double spin, h_floor;
    int h_from_state;
} orc_disk;

/* ---------------------------------------------------------------------- */
/* Exponentially scaled modified Bessel functions of the second kind,     */
/* Kt_nu(z) = e^z K_nu(z), nu = 0, 1, 2, z > 0.                           */
/* Method: the integral representation K_nu(z) = int_0^inf               */
/* exp(-z cosh t) cosh(nu t) dt (DLMF 10.32.9) evaluated by the           */
/* trapezoidal rule, which converges exponentially for this analytic,     */
/* double-exponentially decaying integrand (Trefethen & Weideman 2014,    */
/* SIAM Rev. 56, 385).  cosh t - 1 is formed as 2 sinh^2(t/2).            */
/* Pinned against scipy.special.kve and the recurrence K2 = K0 + 2K1/z.   */
/* ---------------------------------------------------------------------- */
double orc_kve(int nu, double z) {
    if (!(z > 0.0)) return INFINITY;
    double h = 0.125;
    if (z > 1.0) h = 0.125 / sqrt(z);
    double sum = 0.5; /* t = 0 term: exp(0) * cosh(0) = 1, half weight */
    for (int k = 1; k < 100000; ++k) {
        double t = k * h;
        double sh = sinh(0.5 * t);
        double ex = z * 2.0 * sh * sh;
        if (ex > 745.0) break;
        double term = exp(-ex) * cosh(nu * t);
        sum += term;
        if (term < 1e-18 * sum && ex > 40.0) break;
    }
    return h * sum;
}

/* ---------------------------------------------------------------------- */
/* Bremsstrahlung, Sec. 2.1 (Eqs. 1-2), per n_e^2, erg cm^3 s^-1.          */
/* Pinned: branch continuity at theta = 1, the non-relativistic sqrt(T)   */
/* free-free law, the n_e^2 scaling.                                      */
/* ---------------------------------------------------------------------- */
double orc_theta_e(double T) { return O_KB * T / (O_ME * O_C * O_C); }

double orc_brems_ee(double T) {
    double th = orc_theta_e(T);
    double f;
    if (th < 1.0) f = pow(th, 1.5) * (1.0 + 1.1 * th + th * th - 1.25 * pow(th, 2.5));
    else          f = 1.34 * th * (log(1.123 * th) + 1.28);
    return 2.56e-22 * f;
}

double orc_brems_ei(double T) {
    double th = orc_theta_e(T);
    double f;
    if (th < 1.0) f = 4.0 * sqrt(2.0 * th / (O_PI * O_PI * O_PI)) * (1.0 + 1.781 * pow(th, 1.34));
    else          f = 9.0 * th / (2.0 * O_PI) * (log(1.123 * th + 0.48) + 1.5);
    return 1.48e-22 * f;
}

double orc_brems(double T) { return orc_brems_ee(T) + orc_brems_ei(T); }

/* ---------------------------------------------------------------------- */
/* Synchrotron, Sec. 2.2.                                                  */
/* ---------------------------------------------------------------------- */

/* Mahadevan's fit I'(x), Eq. 4; log form to avoid underflow. */
double orc_log_Iprime(double x) {
    return log(4.0505) - log(x) / 6.0
         + log(1.0 + 0.4 * pow(x, -0.25) + 0.5316 * pow(x, -0.5))
         - 1.8899 * cbrt(x);
}
double orc_Iprime(double x) { return exp(orc_log_Iprime(x)); }

/* The K2(1/theta_e) factor of Eq. 3, with the low-temperature substitution
 * K2 -> 2 theta_e^2 for T_e <= k2_switch_T (Sec. 2.2, last paragraph). */
double orc_k2_factor(double T, double k2_switch_T) {
    double th = orc_theta_e(T);
    if (T <= k2_switch_T) return 2.0 * th * th;
    double z = 1.0 / th;
    return orc_kve(2, z) * exp(-z);
}

/* nu_0 such that x_M = nu / nu_0 (Eq. 3). */
double orc_nu0(double B, double T) {
    double th = orc_theta_e(T);
    return 3.0 * O_QE * B * th * th / (4.0 * O_PI * O_ME * O_C);
}

/* Emissivity eps_s(nu), Eq. 3, erg cm^-3 s^-1 Hz^-1. */
double orc_eps_syn(double nu, double ne, double B, double T, double k2_switch_T) {
    double x = nu / orc_nu0(B, T);
    return 4.43e-30 * 4.0 * O_PI * nu * ne / orc_k2_factor(T, k2_switch_T) * orc_Iprime(x);
}

/* ln of the ratio (annulus emission)/(Rayleigh-Jeans surface emission) in
 * Eq. 5, i.e. ln[ 2H eps_s(nu) / (2 * 2 pi nu^2 k T / c^2) ]. */
static double log_ratio_bb(double lnnu, double H, double ne, double T,
                           double k2f, double nu0) {
    double nu = exp(lnnu);
    double x = nu / nu0;
    double lhs = log(H) + log(4.43e-30 * 4.0 * O_PI * ne / k2f) + lnnu + orc_log_Iprime(x);
    double rhs = log(2.0 * O_PI * O_KB * T / (O_C * O_C)) + 2.0 * lnnu;
    return lhs - rhs;
}

/* Critical frequency nu_c: root of Eq. 5 by bisection in ln(nu) on
 * [ln 1 Hz, ln 1e30 Hz] to |d ln nu| < 1e-14, at most 200 halvings.
 * If the ratio is <= 1 already at 1 Hz, nu_c = 1 Hz.  If it is > 1 at
 * 1e30 Hz, nu_c = 1e30 Hz and *flag = 1.  Pinned by scipy's brentq on
 * the same equation and the residual test. */
double orc_nu_c(double H, double B, double ne, double T, double k2_switch_T, int* flag) {
    double k2f = orc_k2_factor(T, k2_switch_T);
    double nu0 = orc_nu0(B, T);
    double a = 0.0, b = log(1e30);
    if (flag) *flag = 0;
    if (log_ratio_bb(a, H, ne, T, k2f, nu0) <= 0.0) return 1.0;
    if (log_ratio_bb(b, H, ne, T, k2f, nu0) > 0.0) { if (flag) *flag = 1; return 1e30; }
    for (int it = 0; it < 200 && (b - a) >= 1e-14; ++it) {
        double m = 0.5 * (a + b);
        if (log_ratio_bb(m, H, ne, T, k2f, nu0) > 0.0) a = m; else b = m;
    }
    return exp(0.5 * (a + b));
}

/* Gauss-Legendre nodes/weights on [-1,1], n points: Newton iteration on
 * P_n from the asymptotic initial guess cos(pi (i - 1/4)/(n + 1/2)). */
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(O_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void orc_gl16(double* x, double* w) { gauss_legendre(16, x, w); }

static double gx[16], gw[16];
__attribute__((constructor)) static void gl16_init(void) { gauss_legendre(16, gx, gw); }

/* Integrand of J in s = x^(1/3): x I'(x) dx = 3 s^5 I'(s^3) ds. */
static double j_integrand(double s) {
    if (s <= 0.0) return 0.0;
    double rs = sqrt(s);
    double s45 = s * s * s * s * rs;          /* s^4.5 */
    double sm75 = 1.0 / (rs * sqrt(rs));     /* s^-0.75 */
    double sm15 = 1.0 / (s * rs);            /* s^-1.5 */
    return 3.0 * 4.0505 * s45 * (1.0 + 0.4 * sm75 + 0.5316 * sm15) * exp(-1.8899 * s);
}

/* J(x_c) = int_{x_c}^inf x I'(x) dx, by composite Gauss-Legendre (16 points)
 * over `panels` equal panels of s in [x_c^(1/3), x_c^(1/3) + 40].
 * Pinned against the closed form in upper incomplete gamma functions. */
double orc_J(double xc, int panels) {
    double s0 = cbrt(xc);
    double width = 40.0 / panels;
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        double a = s0 + p * width;
        double mid = a + 0.5 * width, half = 0.5 * width;
        double ps = 0.0;
        for (int i = 0; i < 16; ++i) ps += gw[i] * j_integrand(mid + half * gx[i]);
        sum += half * ps;
    }
    return sum;
}

/* Synchrotron cooling Q_syn, Eq. 6: Rayleigh-Jeans part below nu_c (per
 * unit volume, divided by H) plus the optically thin integral above nu_c. */
double orc_qsyn_nu(double H, double B, double ne, double T, double k2_switch_T,
                   double nuc, int panels) {
    double rj = 2.0 * O_PI * O_KB * T * nuc * nuc * nuc / (3.0 * O_C * O_C * H);
    double nu0 = orc_nu0(B, T);
    double pref = 4.43e-30 * 4.0 * O_PI * ne / orc_k2_factor(T, k2_switch_T);
    double thin = pref * nu0 * nu0 * orc_J(nuc / nu0, panels);
    return rj + thin;
}

/* Compton enhancement eta at nu_c, Eqs. 7-9 (Sec. 2.3).  Stable form of the
 * truncated geometric series: eta = 1 + P(A-1) [(PA)^k - 1]/(PA - 1),
 * k = ln(3 theta/E)/ln A, evaluated with expm1.  With literal != 0 the
 * exponent as printed, 1 - ln P/ln A, is used instead (for the test that
 * shows its sign failure). */
double orc_eta(double nuc, double T, double ne, double H, int literal) {
    double th = orc_theta_e(T);
    double E = O_H * nuc / (O_ME * O_C * O_C);
    if (E >= 3.0 * th) return 1.0;
    double tau = 2.0 * ne * O_SIGT * H;
    double P = -expm1(-tau);
    double am1 = 4.0 * th + 16.0 * th * th;
    double A = 1.0 + am1;
    double lnA = log1p(am1);
    if (literal) {
        double ex = 1.0 - log(P) / lnA;
        return 1.0 + P * am1 / (1.0 - P * A) * (1.0 - pow(E / (3.0 * th), ex));
    }
    if (!(P > 0.0)) return 1.0;
    double k = log(3.0 * th / E) / lnA;
    double eps = log(P) + lnA;
    double ratio = (eps == 0.0) ? k : expm1(k * eps) / expm1(eps);
    return 1.0 + P * am1 * ratio;
}

/* eta(nu_c) * Q_syn at one (H, B, n_e, T_e) point: the 4-D table channel. */
double orc_eta_qsyn(double H, double B, double ne, double T, const orc_spec* s, int* flag) {
    double nuc = orc_nu_c(H, B, ne, T, s->k2_switch_T, flag);
    double q = orc_qsyn_nu(H, B, ne, T, s->k2_switch_T, nuc, 64);
    return orc_eta(nuc, T, ne, H, s->compton_literal) * q;
}

/* Optically-thick bridge, Eqs. 11-12 (sigma read as Stefan-Boltzmann):
 * Q_total = (4 sigma T^4/H) / (3 tau/2 + sqrt 3 + 1/tau_abs),
 * tau_abs = H Q_thin/(4 sigma T^4), tau = tau_abs + tau_sca, written with
 * numerator and denominator multiplied by tau_abs,
 * Q_total = Q_thin / (1 + tau_abs (sqrt 3 + 1.5 (tau_abs + tau_sca))),
 * which is the same function and keeps its tau_abs -> 0 limit (Q_thin) at
 * H = 0 or Q_thin = 0.  Pinned by the thin and thick limits. */
double orc_bridge(double qthin, double T, double H, double ne) {
    double bb = 4.0 * O_SIGSB * T * T * T * T;
    double tau_sca = 2.0 * ne * O_SIGT * H;
    double tau_abs = H * qthin / bb;
    return qthin / (1.0 + tau_abs * (sqrt(3.0) + 1.5 * (tau_abs + tau_sca)));
}

/* Direct (O1) total cooling rate at one point, erg cm^-3 s^-1. */
double orc_qtotal_direct(double H, double B, double ne, double T, const orc_spec* s) {
    double qthin = ne * ne * orc_brems(T) + orc_eta_qsyn(H, B, ne, T, s, NULL);
    return orc_bridge(qthin, T, H, ne);
}

/* Coulomb exchange coefficient, Eq. 16: C = Q_cc / (n_e^2 (T_i - T_e)),
 * hydrogen (n_i = n_e = rho/m_p), with scaled Bessel functions so that the
 * exponentials cancel exactly (1/theta_m = 1/theta_e + 1/theta_i).
 * Pinned: non-relativistic (Spitzer) limit, symmetry, zero at T_e = T_i. */
double orc_coulomb_C(double Ti, double Te, const orc_spec* s) {
    double the = O_KB * Te / (O_ME * O_C * O_C);
    double mi = s->theta_i_uses_mp ? O_MP : O_ME;
    double thi = O_KB * Ti / (mi * O_C * O_C);
    double ze = 1.0 / the, zi = 1.0 / thi, zm = ze + zi;
    double ts = the + thi;
    double br = (2.0 * ts * ts + 1.0) / ts * orc_kve(1, zm) + 2.0 * orc_kve(0, zm);
    double pre = 1.5 * (O_ME / O_MP) * s->lnLambda * O_C * O_SIGT * O_KB;
    return pre * br / (orc_kve(2, zi) * orc_kve(2, ze));
}

/* ---------------------------------------------------------------------- */
/* Table nodes (Sec. 2.6): N log-spaced points, endpoints inclusive.       */
/* l_j = log2(lo) + j (log2(hi) - log2(lo))/(N-1), x_j = 2^l_j; stored also */
/* rounded to FP32 (the FP32 copy decides index selection).                */
/* ---------------------------------------------------------------------- */
#define ORC_MAXN 1024
typedef struct { int N; double l0, dl; float x32[ORC_MAXN]; } orc_axis;

static double axis_dl(const orc_spec* s, int a) {
    return (log2(s->hi[a]) - log2(s->lo[a])) / (s->n[a] - 1);
}
static double axis_l(const orc_spec* s, int a, int j) {
    return log2(s->lo[a]) + j * axis_dl(s, a);
}
static void axis_init(const orc_spec* s, int a, orc_axis* ax) {
    ax->N = s->n[a];
    ax->l0 = log2(s->lo[a]);
    ax->dl = axis_dl(s, a);
    for (int j = 0; j < ax->N && j < ORC_MAXN; ++j) ax->x32[j] = (float)exp2(axis_l(s, a, j));
}
void orc_nodes(const orc_spec* s, int a, double* x64, double* l64, float* x32) {
    for (int j = 0; j < s->n[a]; ++j) {
        double l = axis_l(s, a, j);
        double x = exp2(l);
        if (x64) x64[j] = x;
        if (l64) l64[j] = l;
        if (x32) x32[j] = (float)x;
    }
}

/* Table channels (log2 values):
 *   lb[t]              = log2(Q_brem/n_e^2)(T_t)
 *   ls[((h*nB+b)*nN+n)*nT+t] = log2(eta Q_syn)(H_h, B_b, n_n, T_t)
 *   lc[i*nC+e]         = log2 C(T_i = X_i, T_e = X_e)
 */
void orc_build_brems(const orc_spec* s, double* lb) {
    for (int t = 0; t < s->n[3]; ++t) lb[t] = log2(orc_brems(exp2(axis_l(s, 3, t))));
}

double orc_syn_node(const orc_spec* s, int h, int b, int n, int t) {
    double H = exp2(axis_l(s, 0, h)), B = exp2(axis_l(s, 1, b));
    double ne = exp2(axis_l(s, 2, n)), T = exp2(axis_l(s, 3, t));
    return log2(orc_eta_qsyn(H, B, ne, T, s, NULL));
}

void orc_build_syn(const orc_spec* s, double* ls, int nthreads) {
    long long total = (long long)s->n[0] * s->n[1] * s->n[2] * s->n[3];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (long long i = 0; i < total; ++i) {
        long long r = i;
        int t = (int)(r % s->n[3]); r /= s->n[3];
        int n = (int)(r % s->n[2]); r /= s->n[2];
        int b = (int)(r % s->n[1]); r /= s->n[1];
        int h = (int)r;
        ls[i] = orc_syn_node(s, h, b, n, t);
    }
}

/* The paper's table layout (Sec. 3.1): one 4-D table of the total rate,
 * ltot[((h*nB+b)*nN+n)*nT+t] = log2 Q_total(H_h, B_b, n_n, T_t) with
 * Q_total the bridge (Eqs. 11-12) of n_e^2 Q_brem/n_e^2 + eta Q_syn, from
 * the table's own brems and synchrotron channels at the node. */
void orc_build_qtotal(const orc_spec* s, const double* lb, const double* ls, double* ltot) {
    const long long total = (long long)s->n[0] * s->n[1] * s->n[2] * s->n[3];
    for (long long i = 0; i < total; ++i) {
        long long r = i;
        int t = (int)(r % s->n[3]); r /= s->n[3];
        int n = (int)(r % s->n[2]); r /= s->n[2];
        r /= s->n[1];
        int h = (int)r;
        double H = exp2(axis_l(s, 0, h)), ne = exp2(axis_l(s, 2, n)), T = exp2(axis_l(s, 3, t));
        double qthin = ne * ne * exp2(lb[t]) + exp2(ls[i]);
        ltot[i] = log2(orc_bridge(qthin, T, H, ne));
    }
}

/* Selected synchrotron nodes only: idx[k] are flat indices into the 4-D
 * table; out[k] receives the node value. */
void orc_build_syn_at(const orc_spec* s, long long m, const long long* idx, double* out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long long k = 0; k < m; ++k) {
        long long r = idx[k];
        int t = (int)(r % s->n[3]); r /= s->n[3];
        int n = (int)(r % s->n[2]); r /= s->n[2];
        int b = (int)(r % s->n[1]); r /= s->n[1];
        int h = (int)r;
        out[k] = orc_syn_node(s, h, b, n, t);
    }
}

void orc_build_coulomb(const orc_spec* s, double* lc) {
    int N = s->n[4];
    for (int i = 0; i < N; ++i)
        for (int e = 0; e < N; ++e)
            lc[i * N + e] = log2(orc_coulomb_C(exp2(axis_l(s, 4, i)), exp2(axis_l(s, 4, e)), s));
}

/* ---------------------------------------------------------------------- */
/* Interpolation (O2).                                                     */
/* Index: the largest j in [0, N-2] with node32[j] <= key (node32 = FP32    */
/* node, compared exactly); a key below node32[0] takes j = 0.  Weight:     */
/* w = (log2 key - l_j)/dl clamped to [0, 1] (constant extrapolation at    */
/* the table edges).  Returns 1 if the key lies outside [node32[0],        */
/* node32[N-1]] (a clamped key), else 0.                                   */
/* ---------------------------------------------------------------------- */
static int select_ax(const orc_axis* ax, double key, int* jout, double* wout) {
    int N = ax->N;
    int j = 0;
    int clamped = 0;
    if (!(key >= (double)ax->x32[0])) clamped = 1;
    else {
        /* plain linear scan over increasing nodes */
        for (int k = 1; k <= N - 2 && (double)ax->x32[k] <= key; ++k) j = k;
        if (key > (double)ax->x32[N - 1]) clamped = 1;
    }
    double w;
    if (!(key > 0.0)) w = 0.0;
    else w = (log2(key) - (ax->l0 + j * ax->dl)) / ax->dl;
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    *jout = j; *wout = w;
    return clamped;
}

int orc_select(const orc_spec* s, int a, double key, int* jout, double* wout) {
    orc_axis ax; axis_init(s, a, &ax);
    return select_ax(&ax, key, jout, wout);
}

/* Batch selection of FP32 keys on one axis (the twin of the GPU debug
 * lookup): idx[i], w[i] for keys[i]. */
void orc_select_f32(const orc_spec* s, int a, long long n, const float* keys, int* idx, double* w) {
    orc_axis ax; axis_init(s, a, &ax);
    for (long long i = 0; i < n; ++i) select_ax(&ax, (double)keys[i], &idx[i], &w[i]);
}

/* Lazy synchrotron table: entries equal to NaN are computed on first use
 * (single-threaded use only). */
static double syn_at(const orc_spec* s, double* ls, int lazy, int h, int b, int n, int t) {
    long long i = (((long long)h * s->n[1] + b) * s->n[2] + n) * s->n[3] + t;
    double v = ls[i];
    if (lazy && isnan(v)) { v = orc_syn_node(s, h, b, n, t); ls[i] = v; }
    return v;
}

/* Multilinear interpolation of the 4-D channel: sum over the 16 corners of
 * prod(weights) * value. */
static double interp4(const orc_spec* s, double* ls, int lazy, const int* j, const double* w) {
    double acc = 0.0;
    for (int c = 0; c < 16; ++c) {
        double wt = 1.0;
        int idx[4];
        for (int a = 0; a < 4; ++a) {
            int bit = (c >> a) & 1;
            idx[a] = j[a] + bit;
            wt *= bit ? w[a] : (1.0 - w[a]);
        }
        acc += wt * syn_at(s, ls, lazy, idx[0], idx[1], idx[2], idx[3]);
    }
    return acc;
}
static double interp1(const double* lb, int j, double w) {
    return (1.0 - w) * lb[j] + w * lb[j + 1];
}
static double interp2(const double* lc, int N, int ji, double wi, int je, double we) {
    return (1.0 - wi) * (1.0 - we) * lc[ji * N + je] + (1.0 - wi) * we * lc[ji * N + je + 1]
         + wi * (1.0 - we) * lc[(ji + 1) * N + je] + wi * we * lc[(ji + 1) * N + je + 1];
}

/* Public scalar interpolation helpers (tests). */
double orc_interp_syn(const orc_spec* s, double* ls, int lazy, double H, double B, double ne, double T) {
    int j[4]; double w[4];
    double k[4] = {H, B, ne, T};
    for (int a = 0; a < 4; ++a) orc_select(s, a, k[a], &j[a], &w[a]);
    return interp4(s, ls, lazy, j, w);
}
double orc_interp_brems(const orc_spec* s, const double* lb, double T) {
    int j; double w; orc_select(s, 3, T, &j, &w);
    return interp1(lb, j, w);
}
double orc_interp_coulomb(const orc_spec* s, const double* lc, double Ti, double Te) {
    int ji, je; double wi, we;
    orc_select(s, 4, Ti, &ji, &wi);
    orc_select(s, 4, Te, &je, &we);
    return interp2(lc, s->n[4], ji, wi, je, we);
}

/* ---------------------------------------------------------------------- */
/* The per-cell step (Sec. 3.2): unit conversion, N_sub sub-cycles of      */
/* (i) Coulomb exchange, (ii) radiative cooling with the bridge, applied   */
/* to the electron internal energy explicitly with the limiter, or         */
/* implicitly (backward Euler, bisection in log2 u) in stiff cells.        */
/* ---------------------------------------------------------------------- */
typedef struct {
    const orc_spec* s;
    const double* lb;
    double* ls;
    const double* lc;
    int lazy;
    int direct;       /* 1: O1 rates from the formulas instead of the table */
    const double* lsp;  /* optional: per-interval node pairs of the 4-D channel */
    const struct orc_net* net;  /* optional: the surrogate network replaces the 4-D channel */
    double* ltot;       /* optional: the paper's layout, log2 Q_total on the 4-D grid */
    orc_axis ax[5];
} orc_rates;

/* ---------------------------------------------------------------------- */
/* Surrogate network (not in the paper): an MLP 4 -> 128 -> 128 -> 1 with  */
/* SiLU standing in for the 4-D channel l(eta Q_syn).  Inputs: the four    */
/* log2 coordinates normalised to [-1, 1] over the table box, each as two  */
/* bf16 parts hi = bf16(x), lo = bf16(x - hi), and the side of the K2      */
/* switch (+1 above, -1 at or below).  Products in FP64 with the bf16      */
/* roundings of the tensor-core operands applied where they occur: input   */
/* parts, W1, W2 and the hidden activations H1.  A fallback bit per 4-D    */
/* table cell sends the lookup back to the table.                          */
/* ---------------------------------------------------------------------- */
typedef struct orc_net {
    double W1[128][9];    /* operand weights: hi parts, lo parts, switch side */
    double b1[128], W2[128][128], b2[128], w3[128], b3;
    double mean, std;     /* output log2 = mean + std * net */
    double l0[4], span[4], xs;
    const uint32_t* mask; /* fallback bits, cell ((h (nB-1) + b) (nN-1) + n) (nT-1) + t; nullable */
    int rounding;
} orc_net;

/* float64 -> float32 -> bfloat16, round to nearest even (finite values). */
static double bf16r(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double net_rnd(const orc_net* m, double v) { return m->rounding ? bf16r(v) : v; }

/* p: the library's flat FP32 parameter layout (W1 [128][16] with columns
 * 0..3 the coordinates and 4 the switch side, b1, W2 [out][in], b2, w3, b3). */
static void net_init(orc_net* m, const float* p, double mean, double stdv, const double* l0,
                     const double* span, double xs, const uint32_t* mask, int rounding) {
    m->rounding = rounding;
    for (int o = 0; o < 128; ++o) {
        for (int d = 0; d < 4; ++d) m->W1[o][d] = m->W1[o][4 + d] = net_rnd(m, p[o * 16 + d]);
        m->W1[o][8] = net_rnd(m, p[o * 16 + 4]);
        m->b1[o] = p[2048 + o];
        for (int i = 0; i < 128; ++i) m->W2[o][i] = net_rnd(m, p[2176 + o * 128 + i]);
        m->b2[o] = p[18560 + o];
        m->w3[o] = p[18688 + o];
    }
    m->b3 = p[18816];
    m->mean = mean; m->std = stdv;
    for (int d = 0; d < 4; ++d) { m->l0[d] = l0[d]; m->span[d] = span[d]; }
    m->xs = xs;
    m->mask = mask;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }

/* Network output in log2 units at normalised inputs x[4] (x in float32, as
 * the library receives it). */
static double net_eval(const orc_net* m, const double* x) {
    double X[9];
    for (int d = 0; d < 4; ++d) {
        double xd = m->rounding ? (double)(float)x[d] : x[d];
        X[d] = net_rnd(m, xd);
        X[4 + d] = net_rnd(m, xd - X[d]);
    }
    X[8] = ((m->rounding ? (double)(float)x[3] : x[3]) > (double)(float)m->xs) ? 1.0 : -1.0;
    double h1[128];
    for (int o = 0; o < 128; ++o) {
        double z = m->b1[o];
        for (int k = 0; k < 9; ++k) z += X[k] * m->W1[o][k];
        h1[o] = net_rnd(m, silu(z));
    }
    double y = m->b3;
    for (int o = 0; o < 128; ++o) {
        double z = m->b2[o];
        for (int i = 0; i < 128; ++i) z += h1[i] * m->W2[o][i];
        y += silu(z) * m->w3[o];
    }
    return m->mean + m->std * y;
}

/* Normalised coordinate of log2 value l on axis d, clamped to [-1, 1]. */
static double net_coord(const orc_net* m, int d, double l) {
    double x = 2.0 * (l - m->l0[d]) / m->span[d] - 1.0;
    return x < -1.0 ? -1.0 : (x > 1.0 ? 1.0 : x);
}

typedef struct {
    double ne, Bg, Hcm, hs, escale, sTe, sTi, ce, ci;
    int j[3]; double w[3]; /* H, B, n_e selections (step-invariant) */
    int* fallback;         /* set when the surrogate step read the table (nullable) */
} cell_ctx;

/* Multilinear interpolation of the 4-D channel when the table is given as
 * per-interval node pairs lsp[((row (nT-1)) + jt) 2 + bt] (a storage format
 * whose node values may depend on the interval, as a block-quantised table). */
static double interp4_pairs(const orc_spec* s, const double* lsp, const int* j, const double* w) {
    double acc = 0.0;
    for (int c = 0; c < 16; ++c) {
        double wt = 1.0;
        int idx[4];
        for (int a = 0; a < 4; ++a) {
            int bit = (c >> a) & 1;
            idx[a] = j[a] + bit;
            wt *= bit ? w[a] : (1.0 - w[a]);
        }
        long long row = ((long long)idx[0] * s->n[1] + idx[1]) * s->n[2] + idx[2];
        acc += wt * lsp[(row * (s->n[3] - 1) + j[3]) * 2 + ((c >> 3) & 1)];
    }
    return acc;
}

/* Cooling energy removed in one sub-cycle (code units) for electron energy
 * density ue, through T_e = s_Te ue/rho.  *clamp is or-ed with key clamping. */
static double cool_q(const orc_rates* R, const cell_ctx* c, double ue, double rho, int* clamp) {
    double Te = c->sTe * ue / rho;
    if (R->ltot) {
        /* the paper's layout: the total rate (bridge included) interpolated */
        int jt; double wt;
        int cl = select_ax(&R->ax[3], Te, &jt, &wt);
        if (clamp) *clamp |= cl;
        int j[4] = {c->j[0], c->j[1], c->j[2], jt};
        double w[4] = {c->w[0], c->w[1], c->w[2], wt};
        return c->hs * exp2(interp4(R->s, R->ltot, 0, j, w)) / c->escale;
    }
    double qthin;
    if (R->direct) {
        qthin = c->ne * c->ne * orc_brems(Te) + orc_eta_qsyn(c->Hcm, c->Bg, c->ne, Te, R->s, NULL);
    } else {
        int jt; double wt;
        int cl = select_ax(&R->ax[3], Te, &jt, &wt);
        if (clamp) *clamp |= cl;
        int j[4] = {c->j[0], c->j[1], c->j[2], jt};
        double w[4] = {c->w[0], c->w[1], c->w[2], wt};
        double lqs;
        const orc_net* m = R->net;
        int table = 1;
        if (m) {
            const int* n = R->s->n;
            long long cell = (((long long)j[0] * (n[1] - 1) + j[1]) * (n[2] - 1) + j[2]) * (n[3] - 1) + jt;
            table = m->mask && ((m->mask[cell >> 5] >> (cell & 31)) & 1u);
            if (table && c->fallback) *c->fallback = 1;
        }
        if (!table) {
            double x[4] = {net_coord(m, 0, log2(c->Hcm)), net_coord(m, 1, log2(c->Bg)),
                           net_coord(m, 2, log2(c->ne)), net_coord(m, 3, log2(Te))};
            lqs = net_eval(m, x);
        } else {
            lqs = R->lsp ? interp4_pairs(R->s, R->lsp, j, w) : interp4(R->s, R->ls, R->lazy, j, w);
        }
        double lqb = interp1(R->lb, jt, wt);
        qthin = c->ne * c->ne * exp2(lqb) + exp2(lqs);
    }
    double Q = orc_bridge(qthin, Te, c->Hcm, c->ne);
    return c->hs * Q / c->escale;
}

static double coulomb_rate(const orc_rates* R, double Ti, double Te, int* clamp) {
    if (R->direct) return orc_coulomb_C(Ti, Te, R->s);
    int ji, je; double wi, we;
    int cl = select_ax(&R->ax[4], Ti, &ji, &wi);
    cl |= select_ax(&R->ax[4], Te, &je, &we);
    if (clamp) *clamp |= cl;
    return exp2(interp2(R->lc, R->s->n[4], ji, wi, je, we));
}

/* Unit conversion of one cell (code units G = c = M = 1, 4 pi absorbed in
 * b; hydrogen, n_e = n_i = rho rho_scale/m_p; T_s = (gamma_s - 1) m_p c^2
 * (u_s/rho)/k_B) and the step-invariant H, B, n_e selections. */
static int cell_setup(const orc_rates* R, const orc_params* p, double rho, double B, double H,
                      cell_ctx* c) {
    double rg = (O_G * (p->M_bh_msun * O_MSUN)) / (O_C * O_C);
    double tg = rg / O_C;
    c->ne = rho * (p->rho_scale / O_MP);
    c->Bg = B * (sqrt(4.0 * O_PI * p->rho_scale) * O_C);
    c->Hcm = H * rg;
    c->hs = p->dt * tg / p->n_sub;
    c->escale = p->rho_scale * O_C * O_C;
    c->ce = p->gamma_e - 1.0; c->ci = p->gamma_i - 1.0;
    c->sTe = c->ce * O_MP * O_C * O_C / O_KB;
    c->sTi = c->ci * O_MP * O_C * O_C / O_KB;
    c->fallback = NULL;
    int clamp = 0;
    if (!R->direct) {
        double k[3] = {c->Hcm, c->Bg, c->ne};
        for (int a = 0; a < 3; ++a) clamp |= select_ax(&R->ax[a], k[a], &c->j[a], &c->w[a]);
    }
    return clamp;
}

/* Per-cell flags: bit 0 clamped key, 1 invalid input (non-finite or
 * non-positive; passed through unchanged), 2 stiff (implicit solve entered),
 * 3 Coulomb inside the equilibrium band |T_e/T_i - 1| <= eq_band,
 * 4 implicit solve without a sign change (limited explicit step taken). */
/* Omega_K = 1/(r^(3/2) + a) (code units, Sec. 2.7). */
static double omega_k(double r, double a) { return 1.0 / (r * sqrt(r) + a); }

/* H_th = c_s / Omega_K with c_s^2 = gamma P / (rho h), rho h = rho + u + P
 * (c = 1), P = (gamma_e - 1) u_e + (gamma_i - 1) u_i, u = u_e + u_i, and the
 * mixture's adiabatic index gamma = 1 + P/u (Sec. 2.7). */
double orc_h_thermal(const orc_params* p, double rho, double ue, double ui, double r, double a) {
    double P = (p->gamma_e - 1.0) * ue + (p->gamma_i - 1.0) * ui;
    double u = ue + ui;
    double gam = 1.0 + P / u;
    double cs = sqrt(gam * P / (rho + u + P));
    return cs / omega_k(r, a);
}

static void step_cell(const orc_rates* R, const orc_params* p, const orc_disk* dk, double r, double rho,
                      double B, double H, double ue, double ui, double* ue_out, double* ui_out,
                      double* qcool, double* qcc, unsigned* flags) {
    *flags = 0;
    if (dk && dk->h_from_state && isfinite(r) && r > 0.0 && isfinite(rho) && rho > 0.0 && isfinite(ue) &&
        ue > 0.0 && isfinite(ui) && ui > 0.0)
        H = orc_h_thermal(p, rho, ue, ui, r, dk->spin);
    if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue) && isfinite(ui)) ||
        !(rho > 0.0) || !(ue > 0.0) || !(ui > 0.0) || B < 0.0 || H < 0.0 ||
        (dk && !(isfinite(r) && r > 0.0))) {
        *ue_out = ue; *ui_out = ui;
        if (qcool) *qcool = 0.0;
        if (qcc) *qcc = 0.0;
        *flags = 1u << 1;
        return;
    }
    cell_ctx c;
    int clamp = cell_setup(R, p, rho, B, H, &c);
    double sum_cool = 0.0, sum_cc = 0.0;
    int stiff = 0, eqb = 0, fail = 0, fallback = 0, floored = 0;
    c.fallback = &fallback;
    double t_floor = -1.0;
    if (dk && dk->h_floor > 0.0) {
        double v = dk->h_floor * omega_k(r, dk->spin) * r;
        t_floor = 0.5 * O_PI * v * v;
    }
    for (int k = 0; k < p->n_sub; ++k) {
        /* (i) Coulomb exchange (Eq. 16), clamped so that the step does not
         * cross T_e = T_i. */
        double Te = c.sTe * ue / rho, Ti = c.sTi * ui / rho;
        if (fabs(Te / Ti - 1.0) <= p->eq_band) eqb = 1;
        double C = coulomb_rate(R, Ti, Te, &clamp);
        double X = c.hs * c.ne * c.ne * C * (Ti - Te) / c.escale;
        double Xeq = (c.ci * ui - c.ce * ue) / (c.ce + c.ci);
        double lim = p->coulomb_clamp * fabs(Xeq);
        if (fabs(X) > lim) X = (X >= 0.0 ? lim : -lim);
        ue += X; ui -= X; sum_cc += X;
        /* temperature floor: no cooling below T_floor (gas temperature P/rho) */
        if (((p->gamma_e - 1.0) * ue + (p->gamma_i - 1.0) * ui) / rho < t_floor) {
            floored = 1;
            continue;
        }
        /* (ii) cooling with the bridge (Eqs. 10-12) */
        double q = cool_q(R, &c, ue, rho, &clamp);
        double du;
        if (p->mode == 1 && q > p->limiter_frac * ue) {
            /* implicit backward Euler: g(u) = u - ue + q(u) = 0 on
             * [ue 2^-60, ue], bisection in log2 u */
            stiff = 1;
            double a = log2(ue) - 60.0, b = log2(ue);
            double ga = exp2(a) - ue + cool_q(R, &c, exp2(a), rho, NULL);
            if (!(ga < 0.0)) {
                fail = 1;
                du = p->limiter_frac * ue;
            } else {
                for (int it = 0; it < p->implicit_iters; ++it) {
                    double m = 0.5 * (a + b);
                    double um = exp2(m);
                    if (um - ue + cool_q(R, &c, um, rho, NULL) > 0.0) b = m; else a = m;
                }
                du = ue - exp2(0.5 * (a + b));
            }
        } else {
            du = q < p->limiter_frac * ue ? q : p->limiter_frac * ue;
        }
        ue -= du; sum_cool += du;
    }
    *ue_out = ue; *ui_out = ui;
    if (qcool) *qcool = sum_cool;
    if (qcc) *qcc = sum_cc;
    *flags = (clamp ? 1u : 0u) | (stiff ? 1u << 2 : 0u) | (eqb ? 1u << 3 : 0u) | (fail ? 1u << 4 : 0u) |
             (fallback ? 1u << 5 : 0u) | (floored ? 1u << 6 : 0u);
}

/* Step n cells.  counters[0..5] = cells with flag bit k set (bit 5: the
 * surrogate step read the table in some sub-cycle).  lazy: the 4-D channel
 * may hold NaN entries, computed on first use (forces one thread).
 * direct: O1 rates.  net: the surrogate network (nullable). */
static int step_impl(const orc_spec* s, const double* lb, double* ls, const double* lc, int lazy, int direct,
             const double* lsp, const orc_net* net, const orc_disk* dk, const double* rr, const orc_params* p,
             long long n, const double* rho, const double* B, const double* H, const double* ue, const double* ui,
             double* ue_out, double* ui_out, double* qcool, double* qcc,
             long long* counters, int nthreads) {
    orc_rates* R = (orc_rates*)malloc(sizeof(orc_rates));
    if (!R) return -1;
    R->s = s; R->lb = lb; R->ls = ls; R->lc = lc; R->lazy = lazy; R->direct = direct; R->lsp = lsp;
    R->net = net;
    R->ltot = NULL;
    for (int a = 0; a < 5; ++a) {
        if (s->n[a] < 2 || s->n[a] > ORC_MAXN) { free(R); return -2; }
        axis_init(s, a, &R->ax[a]);
    }
    long long cnt[7] = {0, 0, 0, 0, 0, 0, 0};
    if (lazy || direct) nthreads = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1024) reduction(+:cnt[:7]) if (nthreads != 1)
#endif
    for (long long i = 0; i < n; ++i) {
        unsigned f;
        double a, b;
        step_cell(R, p, dk, rr ? rr[i] : 0.0, rho[i], B[i], H ? H[i] : 0.0, ue[i], ui[i], &a, &b,
                  qcool ? &qcool[i] : NULL, qcc ? &qcc[i] : NULL, &f);
        ue_out[i] = a; ui_out[i] = b;
        for (int k = 0; k < 7; ++k) cnt[k] += (f >> k) & 1u;
    }
    if (counters) for (int k = 0; k < 7; ++k) counters[k] = cnt[k];
    free(R);
    return 0;
}

int orc_step(const orc_spec* s, const double* lb, double* ls, const double* lc, int lazy, int direct,
             const orc_params* p, long long n,
             const double* rho, const double* B, const double* H, const double* ue, const double* ui,
             double* ue_out, double* ui_out, double* qcool, double* qcc,
             long long* counters, int nthreads) {
    return step_impl(s, lb, ls, lc, lazy, direct, NULL, NULL, NULL, NULL, p, n, rho, B, H, ue, ui, ue_out,
                     ui_out, qcool, qcc, counters, nthreads);
}

/* The step on the paper's table layout: ltot (orc_build_qtotal) in place of
 * the brems and synchrotron channels and the run-time bridge. */
int orc_step_qtotal(const orc_spec* s, const double* lc, double* ltot, const orc_params* p, long long n,
                    const double* rho, const double* B, const double* H, const double* ue, const double* ui,
                    double* ue_out, double* ui_out, double* qcool, double* qcc,
                    long long* counters, int nthreads) {
    orc_rates* R = (orc_rates*)malloc(sizeof(orc_rates));
    if (!R) return -1;
    R->s = s; R->lb = NULL; R->ls = NULL; R->lc = lc; R->lazy = 0; R->direct = 0; R->lsp = NULL;
    R->net = NULL;
    R->ltot = ltot;
    for (int a = 0; a < 5; ++a) {
        if (s->n[a] < 2 || s->n[a] > ORC_MAXN) { free(R); return -2; }
        axis_init(s, a, &R->ax[a]);
    }
    long long cnt[7] = {0, 0, 0, 0, 0, 0, 0};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1024) reduction(+:cnt[:7]) if (nthreads != 1)
#endif
    for (long long i = 0; i < n; ++i) {
        unsigned f;
        double a, b;
        step_cell(R, p, NULL, 0.0, rho[i], B[i], H[i], ue[i], ui[i], &a, &b, qcool ? &qcool[i] : NULL,
                  qcc ? &qcc[i] : NULL, &f);
        ue_out[i] = a; ui_out[i] = b;
        for (int k = 0; k < 7; ++k) cnt[k] += (f >> k) & 1u;
    }
    if (counters) for (int k = 0; k < 7; ++k) counters[k] = cnt[k];
    free(R);
    return 0;
}

/* The step with the 4-D channel given as per-interval node pairs (the
 * values a packed storage format yields for each T_e interval). */
int orc_step_pairs(const orc_spec* s, const double* lb, const double* lsp, const double* lc,
                   const orc_params* p, long long n,
                   const double* rho, const double* B, const double* H, const double* ue, const double* ui,
                   double* ue_out, double* ui_out, double* qcool, double* qcc,
                   long long* counters, int nthreads) {
    return step_impl(s, lb, NULL, lc, 0, 0, lsp, NULL, NULL, NULL, p, n, rho, B, H, ue, ui, ue_out, ui_out,
                     qcool, qcc, counters, nthreads);
}

/* The step with the surrogate network in place of the 4-D channel, except
 * in table cells whose fallback bit is set (mask nullable: never).  l0,
 * span: log2 of the table box per axis (H, B, n_e, T_e); xs: normalised
 * log2 of the K2 switch; rounding: apply the bf16 operand roundings. */
int orc_step_surrogate(const orc_spec* s, const double* lb, const double* ls, const double* lc,
                       const float* params, double mean, double stdv, const double* l0, const double* span,
                       double xs, const uint32_t* mask, int rounding, const orc_params* p, long long n,
                       const double* rho, const double* B, const double* H, const double* ue, const double* ui,
                       double* ue_out, double* ui_out, double* qcool, double* qcc,
                       long long* counters, int nthreads) {
    orc_net* m = (orc_net*)malloc(sizeof(orc_net));
    if (!m) return -1;
    net_init(m, params, mean, stdv, l0, span, xs, mask, rounding);
    int rc = step_impl(s, lb, (double*)ls, lc, 0, 0, NULL, m, NULL, NULL, p, n, rho, B, H, ue, ui, ue_out,
                       ui_out, qcool, qcc, counters, nthreads);
    free(m);
    return rc;
}

/* The step with the disk geometry of each cell (r per cell, spin, optional
 * H_th from the state and the temperature floor); H may be NULL when
 * h_from_state.  counters[6] = cells floored in some sub-cycle. */
int orc_step_disk(const orc_spec* s, const double* lb, double* ls, const double* lc, int direct,
                  const orc_params* p, const orc_disk* dk, long long n, const double* rho, const double* B,
                  const double* H, const double* ue, const double* ui, const double* r, double* ue_out,
                  double* ui_out, double* qcool, double* qcc, long long* counters, int nthreads) {
    if (!H && !dk->h_from_state) return -4;
    return step_impl(s, lb, ls, lc, 0, direct, NULL, NULL, dk, r, p, n, rho, B, H, ue, ui, ue_out, ui_out,
                     qcool, qcc, counters, nthreads);
}

/* Network output (log2 units) at n normalised points x[n][4]. */
int orc_net_eval(const float* params, double mean, double stdv, double xs, int rounding, long long n,
                 const double* x, double* out) {
    orc_net* m = (orc_net*)malloc(sizeof(orc_net));
    if (!m) return -1;
    double l0[4] = {0, 0, 0, 0}, span[4] = {1, 1, 1, 1};
    net_init(m, params, mean, stdv, l0, span, xs, NULL, rounding);
    for (long long i = 0; i < n; ++i) out[i] = net_eval(m, x + 4 * i);
    free(m);
    return 0;
}

/* Cooling energy removed in one sub-cycle (code units) at electron energy
 * density ue for one cell (tests: implicit residual, limiter). */
double orc_cool_q_cell(const orc_spec* s, const double* lb, double* ls, const double* lc, int direct,
                       const orc_params* p, double rho, double B, double H, double ue) {
    orc_rates* R = (orc_rates*)malloc(sizeof(orc_rates));
    if (!R) return NAN;
    R->s = s; R->lb = lb; R->ls = ls; R->lc = lc; R->lazy = 0; R->direct = direct; R->lsp = NULL;
    R->net = NULL;
    R->ltot = NULL;
    for (int a = 0; a < 5; ++a) axis_init(s, a, &R->ax[a]);
    cell_ctx c;
    cell_setup(R, p, rho, B, H, &c);
    double q = cool_q(R, &c, ue, rho, NULL);
    free(R);
    return q;
}

/* Keys of the first sub-cycle formed in FP32 by the fixed operation sequence
 * that the GPU path also uses:  n_e = rho*s_n, B_G = B*s_B, H_cm = H*s_H,
 * inv = s_T / rho (IEEE division), T = u*inv, with the scale factors rounded
 * from FP64 once.  keys[5*i + {0..4}] = H_cm, B_G, n_e, T_e, T_i. */
void orc_keys_f32(const orc_params* p, long long n, const float* rho, const float* B, const float* H,
                  const float* ue, const float* ui, float* keys) {
    double rg = (O_G * (p->M_bh_msun * O_MSUN)) / (O_C * O_C);
    float s_n = (float)(p->rho_scale / O_MP);
    float s_B = (float)(sqrt(4.0 * O_PI * p->rho_scale) * O_C);
    float s_H = (float)rg;
    float s_Te = (float)((p->gamma_e - 1.0) * O_MP * O_C * O_C / O_KB);
    float s_Ti = (float)((p->gamma_i - 1.0) * O_MP * O_C * O_C / O_KB);
    for (long long i = 0; i < n; ++i) {
        volatile float inv_e = s_Te / rho[i];
        volatile float inv_i = s_Ti / rho[i];
        keys[5 * i + 0] = H[i] * s_H;
        keys[5 * i + 1] = B[i] * s_B;
        keys[5 * i + 2] = rho[i] * s_n;
        keys[5 * i + 3] = ue[i] * inv_e;
        keys[5 * i + 4] = ui[i] * inv_i;
    }
}

/* ===================================================================== */
/* Adjoint of the O2 step.                                                */
/* Reverse sweep over the sub-cycles (states recomputed by a forward pass */
/* and kept per sub-cycle); inside one sub-cycle the partial derivatives  */
/* of the Coulomb transfer X and of the cooling energy q come from        */
/* forward-mode dual numbers carrying d/d(u_e, u_i, rho, B, H) and one    */
/* seed used for d/d(Q_thin).  The implicit update is differentiated by   */
/* the implicit-function theorem at the root, not through the bisection.  */
/* Pinned by kink-aware central finite differences (tests).               */
/* ===================================================================== */
#define ND 6
typedef struct { double v, d[ND]; } dn;

static dn dc(double v) { dn r; r.v = v; for (int k = 0; k < ND; ++k) r.d[k] = 0.0; return r; }
static dn dvar(double v, int k) { dn r = dc(v); r.d[k] = 1.0; return r; }
static dn dadd(dn a, dn b) { dn r; r.v = a.v + b.v; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
static dn dsub(dn a, dn b) { dn r; r.v = a.v - b.v; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
static dn dmul(dn a, dn b) { dn r; r.v = a.v * b.v; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
static dn ddiv(dn a, dn b) {
    dn r; r.v = a.v / b.v;
    for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
static dn dscale(dn a, double s) { dn r; r.v = a.v * s; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * s; return r; }
static dn dshift(dn a, double s) { a.v += s; return a; }
static dn dlog2(dn a) { dn r; r.v = log2(a.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] / (a.v * log(2.0)); return r; }
static dn dexp2(dn a) { dn r; r.v = exp2(a.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * r.v * log(2.0); return r; }

/* Selection with a differentiable weight: w = (log2 key - l_j)/dl inside
 * the cell, constant where the weight is clamped (outside the table). */
static int sel_dn(const orc_axis* ax, dn key, int* j, dn* w, unsigned long long* sig) {
    double wv;
    int cl = select_ax(ax, key.v, j, &wv);
    double raw = (log2(key.v) - (ax->l0 + *j * ax->dl)) / ax->dl;
    if (raw < 0.0 || raw > 1.0) *w = dc(wv);
    else *w = dscale(dshift(dlog2(key), -(ax->l0 + *j * ax->dl)), 1.0 / ax->dl);
    if (sig) *sig = (*sig ^ (unsigned long long)(*j + 1000 * cl)) * 1099511628211ull;
    return cl;
}

typedef struct {
    double rg, hs, escale, sTe, sTi, ce, ci, s_n, s_B;
} bwd_const;

static void bwd_consts(const orc_params* p, bwd_const* k) {
    k->rg = (O_G * (p->M_bh_msun * O_MSUN)) / (O_C * O_C);
    k->hs = p->dt * (k->rg / O_C) / p->n_sub;
    k->escale = p->rho_scale * O_C * O_C;
    k->ce = p->gamma_e - 1.0; k->ci = p->gamma_i - 1.0;
    k->sTe = k->ce * O_MP * O_C * O_C / O_KB;
    k->sTi = k->ci * O_MP * O_C * O_C / O_KB;
    k->s_n = p->rho_scale / O_MP;
    k->s_B = sqrt(4.0 * O_PI * p->rho_scale) * O_C;
}

/* Cooling energy of one sub-cycle as a dual number (components 0 u_e,
 * 2 rho, 3 B, 4 H, 5 = d/dQ_thin), with what the table scatter needs. */
typedef struct {
    dn q;
    int jt; double wt;
    int j[3]; double w[3];
    double lqs, lqb, ne;
} qinfo;

static void q_dn(const orc_rates* R, const bwd_const* K, dn rho, dn B, dn H, dn ue, qinfo* o,
                 unsigned long long* sig) {
    dn ne = dscale(rho, K->s_n);
    dn Bg = dscale(B, K->s_B);
    dn Hc = dscale(H, K->rg);
    dn Te = ddiv(dscale(ue, K->sTe), rho);
    dn w[4];
    int j[4];
    sel_dn(&R->ax[0], Hc, &j[0], &w[0], sig);
    sel_dn(&R->ax[1], Bg, &j[1], &w[1], sig);
    sel_dn(&R->ax[2], ne, &j[2], &w[2], sig);
    sel_dn(&R->ax[3], Te, &j[3], &w[3], sig);
    dn lqs = dc(0.0);
    for (int c = 0; c < 16; ++c) {
        dn wt = dc(1.0);
        int idx[4];
        for (int a = 0; a < 4; ++a) {
            int bit = (c >> a) & 1;
            idx[a] = j[a] + bit;
            wt = dmul(wt, bit ? w[a] : dsub(dc(1.0), w[a]));
        }
        lqs = dadd(lqs, dscale(wt, syn_at(R->s, R->ls, R->lazy, idx[0], idx[1], idx[2], idx[3])));
    }
    dn lqb = dadd(dscale(dsub(dc(1.0), w[3]), R->lb[j[3]]), dscale(w[3], R->lb[j[3] + 1]));
    dn qthin = dadd(dmul(dmul(ne, ne), dexp2(lqb)), dexp2(lqs));
    qthin.d[5] = 1.0;
    dn T2 = dmul(Te, Te);
    dn bb = dscale(dmul(T2, T2), 4.0 * O_SIGSB);
    dn tau_sca = dscale(dmul(ne, Hc), 2.0 * O_SIGT);
    dn tau_abs = ddiv(dmul(Hc, qthin), bb);
    dn den = dadd(dc(1.0), dmul(tau_abs, dadd(dc(sqrt(3.0)), dscale(dadd(tau_abs, tau_sca), 1.5))));
    o->q = dscale(ddiv(qthin, den), K->hs / K->escale);
    o->jt = j[3]; o->wt = w[3].v;
    for (int a = 0; a < 3; ++a) { o->j[a] = j[a]; o->w[a] = w[a].v; }
    o->lqs = lqs.v; o->lqb = lqb.v; o->ne = ne.v;
}

/* Coulomb transfer X of one sub-cycle as a dual number (components 0 u_e,
 * 1 u_i, 2 rho). */
typedef struct {
    dn X;
    int clamped;
    int ji, je; double wi, we;
} xinfo;

static void x_dn(const orc_rates* R, const orc_params* p, const bwd_const* K, dn rho, dn ue, dn ui, xinfo* o,
                 unsigned long long* sig) {
    dn Te = ddiv(dscale(ue, K->sTe), rho);
    dn Ti = ddiv(dscale(ui, K->sTi), rho);
    dn wi, we;
    sel_dn(&R->ax[4], Ti, &o->ji, &wi, sig);
    sel_dn(&R->ax[4], Te, &o->je, &we, sig);
    int N = R->s->n[4];
    const double* lc = R->lc;
    dn lC = dadd(dadd(dscale(dmul(dsub(dc(1.0), wi), dsub(dc(1.0), we)), lc[o->ji * N + o->je]),
                      dscale(dmul(dsub(dc(1.0), wi), we), lc[o->ji * N + o->je + 1])),
                 dadd(dscale(dmul(wi, dsub(dc(1.0), we)), lc[(o->ji + 1) * N + o->je]),
                      dscale(dmul(wi, we), lc[(o->ji + 1) * N + o->je + 1])));
    dn ne = dscale(rho, K->s_n);
    dn X = dscale(dmul(dmul(dmul(ne, ne), dexp2(lC)), dsub(Ti, Te)), K->hs / K->escale);
    dn Xeq = dscale(dsub(dscale(ui, K->ci), dscale(ue, K->ce)), 1.0 / (K->ce + K->ci));
    double lim = p->coulomb_clamp * fabs(Xeq.v);
    o->clamped = 0;
    if (fabs(X.v) > lim) {
        double sgn = (X.v >= 0.0 ? 1.0 : -1.0) * (Xeq.v >= 0.0 ? 1.0 : -1.0);
        X = dscale(Xeq, p->coulomb_clamp * sgn);
        o->clamped = 1;
    }
    if (sig) *sig = (*sig ^ (unsigned long long)(o->clamped + 7)) * 1099511628211ull;
    o->X = X;
    o->wi = wi.v; o->we = we.v;
}

#define ORC_MAXSUB 64
typedef struct { double ue, ui, ue1, ustar; int branch; } sub_state;  /* branch: 0 free, 1 limited, 2 implicit */

/* Adjoint of one cell.  g_out_e, g_out_i: adjoints of u_e_out, u_i_out.
 * Returns the input adjoints; table adjoints are added (atomically) into
 * g_lb / g_ls / g_lc when given.  *sig hashes every discrete decision. */
static void cell_bwd(const orc_rates* R, const orc_params* p, double rho, double B, double H, double ue0,
                     double ui0, double g_out_e, double g_out_i, double* g, double* g_lb, double* g_ls,
                     double* g_lc, unsigned long long* sig, double* ue_out, double* ui_out) {
    bwd_const K;
    bwd_consts(p, &K);
    sub_state st[ORC_MAXSUB];
    for (int k = 0; k < 5; ++k) g[k] = 0.0;
    *sig = 1469598103934665603ull;
    if (!(isfinite(rho) && isfinite(B) && isfinite(H) && isfinite(ue0) && isfinite(ui0)) ||
        !(rho > 0.0) || !(ue0 > 0.0) || !(ui0 > 0.0) || B < 0.0 || H < 0.0 || p->n_sub > ORC_MAXSUB) {
        g[3] = g_out_e; g[4] = g_out_i;   /* pass-through cell */
        *ue_out = ue0; *ui_out = ui0;
        return;
    }
    dn drho = dc(rho), dB = dc(B), dH = dc(H);
    double ue = ue0, ui = ui0;
    /* forward, keeping the per-sub-cycle states and branches */
    for (int k = 0; k < p->n_sub; ++k) {
        xinfo xi;
        x_dn(R, p, &K, drho, dc(ue), dc(ui), &xi, sig);
        st[k].ue = ue; st[k].ui = ui;
        ue += xi.X.v; ui -= xi.X.v;
        st[k].ue1 = ue;
        qinfo qi;
        q_dn(R, &K, drho, dB, dH, dc(ue), &qi, sig);
        double q = qi.q.v, du;
        if (p->mode == 1 && q > p->limiter_frac * ue) {
            double a = log2(ue) - 60.0, b = log2(ue);
            qinfo qa;
            q_dn(R, &K, drho, dB, dH, dc(exp2(a)), &qa, NULL);
            if (!(exp2(a) - ue + qa.q.v < 0.0)) {
                st[k].branch = 1; du = p->limiter_frac * ue;
            } else {
                for (int it = 0; it < p->implicit_iters; ++it) {
                    double m = 0.5 * (a + b);
                    qinfo qm;
                    q_dn(R, &K, drho, dB, dH, dc(exp2(m)), &qm, NULL);
                    if (exp2(m) - ue + qm.q.v > 0.0) b = m; else a = m;
                }
                st[k].ustar = exp2(0.5 * (a + b));
                st[k].branch = 2; du = ue - st[k].ustar;
            }
        } else if (q < p->limiter_frac * ue) {
            st[k].branch = 0; du = q;
        } else {
            st[k].branch = 1; du = p->limiter_frac * ue;
        }
        *sig = (*sig ^ (unsigned long long)(st[k].branch + 17)) * 1099511628211ull;
        ue -= du;
    }
    *ue_out = ue; *ui_out = ui;
    /* reverse sweep */
    double ge = g_out_e, gi = g_out_i;     /* adjoints of (u_e, u_i) after sub-cycle k */
    double grho = 0.0, gB = 0.0, gH = 0.0;
    for (int k = p->n_sub - 1; k >= 0; --k) {
        /* (ii) cooling: u_e' = F(u_e1) */
        double ge1;
        if (st[k].branch == 1) {
            ge1 = (1.0 - p->limiter_frac) * ge;
        } else {
            double u = st[k].branch == 2 ? st[k].ustar : st[k].ue1;
            qinfo qi;
            q_dn(R, &K, dvar(rho, 2), dvar(B, 3), dvar(H, 4), dvar(u, 0), &qi, NULL);
            double scale;   /* d u_e' / d q_theta */
            if (st[k].branch == 2) {
                double den = 1.0 + qi.q.d[0];
                ge1 = ge / den;
                scale = -ge / den;
            } else {
                ge1 = ge * (1.0 - qi.q.d[0]);
                scale = -ge;
            }
            grho += scale * qi.q.d[2];
            gB += scale * qi.q.d[3];
            gH += scale * qi.q.d[4];
            /* table entries: dq/dls_c = dq/dQthin ln2 2^lqs W_c, dq/dlb = dq/dQthin ln2 ne^2 2^lqb (1-wt, wt) */
            double cs = scale * qi.q.d[5] * log(2.0) * exp2(qi.lqs);
            double cb = scale * qi.q.d[5] * log(2.0) * qi.ne * qi.ne * exp2(qi.lqb);
            if (g_ls) {
                for (int c = 0; c < 16; ++c) {
                    double wt = 1.0;
                    int idx[4];
                    for (int a = 0; a < 4; ++a) {
                        int bit = (c >> a) & 1;
                        double wa = a < 3 ? qi.w[a] : qi.wt;
                        int ja = a < 3 ? qi.j[a] : qi.jt;
                        idx[a] = ja + bit;
                        wt *= bit ? wa : (1.0 - wa);
                    }
                    long long ii = (((long long)idx[0] * R->s->n[1] + idx[1]) * R->s->n[2] + idx[2]) * R->s->n[3] + idx[3];
#ifdef _OPENMP
#pragma omp atomic
#endif
                    g_ls[ii] += cs * wt;
                }
            }
            if (g_lb) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                g_lb[qi.jt] += cb * (1.0 - qi.wt);
#ifdef _OPENMP
#pragma omp atomic
#endif
                g_lb[qi.jt + 1] += cb * qi.wt;
            }
        }
        /* (i) Coulomb: u_e1 = u_e + X, u_i1 = u_i - X */
        xinfo xi;
        x_dn(R, p, &K, dvar(rho, 2), dvar(st[k].ue, 0), dvar(st[k].ui, 1), &xi, NULL);
        double gX = ge1 - gi;
        double ge0 = ge1 + gX * xi.X.d[0];
        double gi0 = gi + gX * xi.X.d[1];
        grho += gX * xi.X.d[2];
        if (g_lc && !xi.clamped) {
            int N = R->s->n[4];
            double cl = gX * xi.X.v * log(2.0);
            double ws[4] = {(1.0 - xi.wi) * (1.0 - xi.we), (1.0 - xi.wi) * xi.we, xi.wi * (1.0 - xi.we), xi.wi * xi.we};
            int ids[4] = {xi.ji * N + xi.je, xi.ji * N + xi.je + 1, (xi.ji + 1) * N + xi.je, (xi.ji + 1) * N + xi.je + 1};
            for (int c = 0; c < 4; ++c) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                g_lc[ids[c]] += cl * ws[c];
            }
        }
        ge = ge0; gi = gi0;
    }
    g[0] = grho; g[1] = gB; g[2] = gH; g[3] = ge; g[4] = gi;
}

/* Adjoint of orc_step for n cells: grads[5 i + {0..4}] = dL/d(rho, B, H,
 * u_e_in, u_i_in) for L = sum(g_ue_out u_e_out + g_ui_out u_i_out);
 * g_lb / g_ls / g_lc (nullable, natural table layouts) accumulate dL/d(table
 * log2 values); sig (nullable) receives a hash of each cell's discrete
 * decisions; ue_out / ui_out (nullable) the forward outputs.  lazy: the 4-D
 * channel's NaN entries are computed on first use (one thread). */
int orc_step_bwd(const orc_spec* s, const double* lb, double* ls, const double* lc, const orc_params* p,
                 long long n, const double* rho, const double* B, const double* H, const double* ue,
                 const double* ui, const double* g_ue_out, const double* g_ui_out, double* grads,
                 double* g_lb, double* g_ls, double* g_lc, unsigned long long* sig, double* ue_out,
                 double* ui_out, int nthreads, int lazy) {
    orc_rates* R = (orc_rates*)malloc(sizeof(orc_rates));
    if (!R) return -1;
    R->s = s; R->lb = lb; R->ls = ls; R->lc = lc; R->lazy = lazy; R->direct = 0; R->lsp = NULL; R->net = NULL;
    if (lazy) nthreads = 1;
    R->ltot = NULL;
    for (int a = 0; a < 5; ++a) {
        if (s->n[a] < 2 || s->n[a] > ORC_MAXN) { free(R); return -2; }
        axis_init(s, a, &R->ax[a]);
    }
    if (p->n_sub > ORC_MAXSUB) { free(R); return -3; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long i = 0; i < n; ++i) {
        unsigned long long sg;
        double a, b;
        cell_bwd(R, p, rho[i], B[i], H[i], ue[i], ui[i], g_ue_out[i], g_ui_out[i], &grads[5 * i], g_lb, g_ls,
                 g_lc, &sg, &a, &b);
        if (sig) sig[i] = sg;
        if (ue_out) ue_out[i] = a;
        if (ui_out) ui_out[i] = b;
    }
    free(R);
    return 0;
}

/* ===================================================================== */
/* Radiation-pressure correction of T_e (Sec. 5.2, total-pressure Eq.): in */
/* optically thick cells the simulation's thermal pressure is read as gas  */
/* plus radiation, P = a T_e^4 + n k (T_e + T_i), and T_e is recomputed.   */
/* With P = n k (T_e,sim + T_i) (hydrogen, n = n_e = n_i) the ion terms    */
/* cancel: a T^4 + n k T = n k T_e,sim.                                    */
/* ===================================================================== */

/* The positive root of a x^4 + b x - c = 0 (a, b, c > 0; unique, since the
 * left side increases on x > 0), in closed form (Ferrari): with P = b/a and
 * q = c/a, x^4 + P x - q = 0; adding 2 m x^2 + m^2 to both sides makes
 * (x^2 + m)^2 = 2m x^2 - P x + m^2 + q a perfect square when m solves the
 * resolvent cubic 8 m^3 + 8 q m - P^2 = 0 (one positive root: the
 * trigonometric/hyperbolic Cardano form for a cubic with one real root).
 * Then x^2 + sqrt(2m) x + m - P/(2 sqrt(2m)) = 0 gives
 *   x = (A - B)/2,  A = sqrt(2P/sqrt(2m) - 2m),  B = sqrt(2m),
 * evaluated as 8 q m / (sqrt(2m) (P + sqrt(8 m^3)) (A + B)), which follows
 * from P^2 - 8 m^3 = 8 q m and has no cancellation. */
double orc_quartic_root(double a, double b, double c) {
    if (!(a > 0.0) || !(b > 0.0) || !(c > 0.0)) return NAN;
    double P = b / a, q = c / a;
    /* resolvent m^3 + q m - P^2/8 = 0: t^3 + pp t + qq = 0, pp > 0 */
    double pp = q, qq = -P * P / 8.0;
    double m = -2.0 * sqrt(pp / 3.0) * sinh(asinh(1.5 * qq / pp * sqrt(3.0 / pp)) / 3.0);
    double s2m = sqrt(2.0 * m);
    double A = sqrt((2.0 * P - sqrt(8.0 * m * m * m)) / s2m);
    return 8.0 * q * m / (s2m * (P + sqrt(8.0 * m * m * m)) * (A + s2m));
}

/* Per cell: tau_sca = n_e sigma_T H_cm (the local optical depth of Sec.
 * 5.2); where tau_sca > tau_crit the corrected T_e, else T_e,sim.  thick
 * (nullable) marks the corrected cells.  Invalid cells (non-finite or
 * non-positive rho, u_e; negative H) give NaN. */
void orc_radiation_te(const orc_params* p, double tau_crit, double a_rad, long long n, const double* rho,
                      const double* H, const double* ue, double* te_out, int* thick) {
    double rg = (O_G * (p->M_bh_msun * O_MSUN)) / (O_C * O_C);
    for (long long i = 0; i < n; ++i) {
        int th = 0;
        double t = NAN;
        if (isfinite(rho[i]) && isfinite(H[i]) && isfinite(ue[i]) && rho[i] > 0.0 && ue[i] > 0.0 && H[i] >= 0.0) {
            double ne = rho[i] * p->rho_scale / O_MP;
            double Te = (p->gamma_e - 1.0) * O_MP * O_C * O_C / O_KB * ue[i] / rho[i];
            double tau = ne * O_SIGT * H[i] * rg;
            t = Te;
            if (tau > tau_crit) {
                th = 1;
                t = orc_quartic_root(a_rad, ne * O_KB, ne * O_KB * Te);
            }
        }
        te_out[i] = t;
        if (thick) thick[i] = th;
    }
}
