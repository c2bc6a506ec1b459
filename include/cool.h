/*
 * cool.h -- C ABI of libcool, a B300-native (sm_103a) implementation of the
 * per-cell two-temperature radiative cooling source step of Motta et al.,
 * "Black hole spectral states revealed in GRMHD simulations with texture
 * memory accelerated cooling" (arXiv 2505.08855).
 *
 * What the library computes (paper sections / equations):
 *   - a log-space rate table (Sec. 2.6; Coulomb table Sec. 2.8) built on the
 *     GPU in FP64 from the cooling formulas of Sec. 2: bremsstrahlung
 *     (Eqs. 1-2), self-absorbed thermal synchrotron (Eqs. 3-6) with the
 *     low-temperature K2 substitution, the local Compton enhancement
 *     (Eqs. 7-9), thin cooling (Eq. 10), and the Coulomb exchange (Eq. 16);
 *   - the per-cell step: multilinear interpolation of the table, the
 *     optically-thick bridge (Eqs. 11-12, applied per sub-cycle), the
 *     Coulomb exchange, and the sub-cycled update of the electron and ion
 *     internal energies, explicit with the 30 % limiter or implicit in stiff
 *     cells (Sec. 3.2.1).
 *
 * Conventions for every entry point:
 *   - Pointers named "device" are CUDA device (or managed) pointers; pointers
 *     named "host" are host memory.  The caller owns every field array; the
 *     library owns cool_table objects (freed by cool_table_free).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Entry points that launch work are asynchronous on `stream`
 *     unless stated otherwise; they return after enqueueing.
 *   - Errors are returned as cool_status, never as exceptions, traps or
 *     device asserts.  Invalid arguments are detected on the host before any
 *     launch; nothing is written to outputs in that case.  A CUDA error is
 *     reported as COOL_ECUDA; cool_last_cuda_error() gives its code.
 *   - Field units are the paper's code units (G = c = M = 1, the 4 pi factor
 *     absorbed in b, Sec. 3.2): rho (rest-mass density; rho = 1 maps to
 *     rho_scale g/cm^3), B = |b|, H (thermal scale height in r_g), u_e, u_i
 *     (internal energy densities).  Hydrogen composition (n_e = n_i).
 */
#ifndef COOL_H
#define COOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    COOL_OK = 0,
    COOL_EINVAL = 1,        /* an argument is out of its documented range */
    COOL_ENULL = 2,         /* a required pointer is NULL */
    COOL_EALIGN = 3,        /* a field pointer is not 16-byte aligned (vector path) */
    COOL_ECUDA = 4,         /* a CUDA runtime call failed (see cool_last_cuda_error) */
    COOL_ENOMEM = 5,        /* device or host allocation failed */
    COOL_ESTATE = 6,        /* the object is in the wrong state (e.g. freed table) */
    COOL_EUNSUPPORTED = 7,  /* the combination of options is not implemented */
    COOL_EIO = 8            /* file could not be read/written or is malformed */
} cool_status;

typedef enum { COOL_F32 = 0, COOL_BF16 = 1, COOL_F16 = 2, COOL_F64 = 3 } cool_dtype;

/* Energy update of Sec. 3.2.1: (i) explicit with the limiter, (ii) implicit. */
typedef enum { COOL_EXPLICIT_LIMITED = 0, COOL_IMPLICIT_STIFF = 1 } cool_mode;

/* How the 4-D synchrotron channel is read.  L2WINDOW: the packed blocks in
 * global memory, L2-resident through their reuse; with
 * cool_table_l2_persist on, each step launch also carries an access-policy
 * window marking them persisting (all modes, formats and field types).
 * TEXTURE_POINT / TEXTURE_HWLERP (the paper's design, Sec. 3.1; comparison
 * paths, explicit mode with FP32 fields and an FP32 table only): the FP32
 * channel as a 3-D texture (x = T_e, y = n_e, z = h n_B + b, made on first
 * use, synchronously), read with 16 point fetches and FP32 interpolation, or
 * with the hardware's trilinear filtering (weights in fixed point with 8
 * fractional bits: an error of up to 2^-8 of a node step per filtered axis)
 * and FP32 interpolation in H.  TMA_SMEM: the L2WINDOW step with its field
 * staging done by bulk asynchronous copies into shared memory,
 * double-buffered per warp (FP32 fields, all arrays 16-byte aligned, else
 * COOL_EALIGN; same results as L2WINDOW).  QTOTAL (the paper's table layout,
 * Sec. 3.1; comparison path, explicit mode with FP32 fields and an FP32
 * table only): one 4-D table of log2 Q_total, the bridge of Eqs. 11-12
 * applied at each node to the table's brems and synchrotron values (made on
 * first use, synchronously; cool_table_export channel 3), interpolated in
 * place of the brems and synchrotron channels and the run-time bridge.
 * SURROGATE: COOL_EUNSUPPORTED in cool_step (the surrogate step is
 * cool_surrogate_infer). */
typedef enum {
    COOL_PATH_L2WINDOW = 0,
    COOL_PATH_TMA_SMEM = 1,
    COOL_PATH_TEXTURE_POINT = 2,
    COOL_PATH_TEXTURE_HWLERP = 3,
    COOL_PATH_SURROGATE = 4,
    COOL_PATH_QTOTAL = 5
} cool_path;

/* Table specification.  Axis nodes are log-spaced with inclusive endpoints
 * (Sec. 2.6): l_j = log2(min) + j (log2(max) - log2(min))/(n - 1), x_j = 2^l_j.
 * Channels: log2(Q_brem/n_e^2)(T_e) [n_Te], log2(eta Q_syn)(H, B, n_e, T_e)
 * [n_H x n_B x n_ne x n_Te, T_e fastest], log2 C(T_i, T_e) with
 * Q_cc = n_e^2 (T_i - T_e) C [n_Tc x n_Tc, T_e fastest].  Ranges in cgs.
 * Limits: 2 <= n <= 512 per axis, n_Tc <= 128; 0 < min < max. */
typedef struct {
    int n_H, n_B, n_ne, n_Te, n_Tc;
    double H_min, H_max;      /* cm   (paper: 1e3 .. 1e12) */
    double B_min, B_max;      /* G    (paper: 1 .. 1e10)   */
    double ne_min, ne_max;    /* cm^-3 (paper: 1e2 .. 1e25) */
    double T_min, T_max;      /* K    (paper: 1e2 .. 1e15), T_e and Coulomb axes */
    cool_dtype dtype;         /* storage of the 4-D channel: COOL_F32, COOL_BF16 or COOL_F16 */
    int row_scaled;           /* 16-bit storage only: 1 = each 32-byte block along T_e holds an FP32
                                 offset and scale and 12 16-bit residuals in [-1, 1]
                                 (value = offset + scale r); 0 = plain 16-bit log2 values */
    double k2_switch_T;       /* K2(1/theta) -> 2 theta^2 at T_e <= this (paper: 1e8 K) */
    double lnLambda;          /* Coulomb logarithm (default 20) */
    int theta_i_uses_mp;      /* 1: theta_i = kT_i/(m_p c^2) (default); 0: m_e as printed */
    int compton_literal;      /* 1: Compton exponent 1 - lnP/lnA as printed; 0: -1 - lnP/lnA */
} cool_table_spec;

/* Step parameters. */
typedef struct {
    double rho_scale;         /* g/cm^3 of rho = 1 (paper: 3e-7 .. 1e-9) */
    double M_bh_msun;         /* black-hole mass in solar masses (paper: 10) */
    double gamma_e, gamma_i;  /* adiabatic indices (paper: 5/3) */
    double dt;                /* step in code time units (r_g/c) */
    int n_sub;                /* sub-cycles per step, 1 .. 64 */
    cool_mode mode;
    double limiter_frac;      /* explicit cap on the electron energy removed per sub-cycle (0.3) */
    double eq_band;           /* equilibrium band |T_e - T_i| <= eq_band T_i (0.1), where T_i - T_e cancels */
    double coulomb_clamp;     /* the exchange may move at most this fraction of the way to T_e = T_i (1) */
    int implicit_iters;       /* evaluations of q(u) allowed to the implicit solve of a stiff cell,
                                 1 .. 200 (60).  The GPU solves backward Euler by Illinois (modified
                                 regula falsi) iterations, first on log2((u + q(u))/u_e) in log2 u,
                                 then on u + q(u) - u_e once the bracket is narrow, stopping at the
                                 FP32 (or, with fp64_critical, FP64) resolution of the root or after
                                 this many evaluations; the FP64 oracle bisects in log2 u instead. */
    cool_path path;           /* COOL_PATH_L2WINDOW (default), TMA_SMEM, TEXTURE_POINT, TEXTURE_HWLERP, QTOTAL */
    int fp64_critical;        /* FP32 fields only.  0 (default): the Coulomb difference
                                 (gamma_i-1) u_i - (gamma_e-1) u_e is formed with an error-free FP32
                                 product transformation in every cell, and stiff cells are solved in
                                 FP32.  1: FP64 inside the equilibrium band for the exchange, and the
                                 implicit solve of stiff cells in FP64 on the FP64 table. */
} cool_params;

/* Per-call diagnostics, accumulated (atomically) into a caller-owned device
 * struct when a pointer is given; counts are cells (not sub-cycles). */
typedef struct {
    unsigned long long n_clamped;        /* a table key outside the table range (edge value used) */
    unsigned long long n_nonfinite;      /* invalid cell (non-finite or non-positive rho/u, negative B/H): passed through */
    unsigned long long n_stiff;          /* implicit solve entered (mode IMPLICIT) */
    unsigned long long n_fp64_coulomb;   /* Coulomb exchange inside the equilibrium band in some sub-cycle
                                            (FP64 there when fp64_critical = 1; FP64 fields: always FP64) */
    unsigned long long n_implicit_fail;  /* implicit bracket without sign change: limited explicit step taken */
    unsigned long long n_fallback;       /* cool_surrogate_infer: the table read instead of the network in
                                            some sub-cycle */
    unsigned long long n_floor;          /* cool_step_disk: cooling skipped under the temperature floor in
                                            some sub-cycle */
    unsigned long long n_exact_redo;     /* FP32 step: cells stepped a second time with the exact index
                                            rule (node compares) because a key fell within ~1e-6 of a
                                            node or its guessed interval was in doubt; the outputs are
                                            the same, this counts the fast selection's extra work */
} cool_counters;

/* Disk geometry for cool_step_disk (Sec. 2.7 scale height, Sec. 3.2.3
 * temperature floor).  Omega_K = 1/(r^1.5 + spin) (code units, r in r_g).
 * h_from_state = 1: H_th = c_s / Omega_K with c_s^2 = gamma P/(rho + u + P),
 * P = (gamma_e - 1) u_e + (gamma_i - 1) u_i, u = u_e + u_i, gamma = 1 + P/u,
 * from the step's input state, replaces the H field.  h_floor > 0: a
 * sub-cycle whose gas temperature P/rho lies below T_floor = (pi/2)
 * (h_floor Omega_K r)^2 does not cool (the exchange still acts). */
typedef struct {
    double spin;               /* black-hole spin a (paper: 0.9375) */
    double h_floor;            /* (H/R)_floor (paper: 0.1); 0 = no floor */
    int h_from_state;          /* 0: H from the field; 1: H_th from the state */
} cool_disk;

typedef struct cool_table cool_table;    /* opaque; owns device memory */

/* Human-readable name of a status. */
const char* cool_strerror(cool_status s);

/* The cudaError_t of the last COOL_ECUDA returned on this thread (0 if none). */
int cool_last_cuda_error(void);

/* Fill *spec with the paper's ranges (Sec. 2.6, 2.8), 64 points per axis,
 * FP32 storage, k2_switch_T = 1e8 K, lnLambda = 20, theta_i with m_p. */
cool_status cool_table_spec_default(cool_table_spec* spec);

/* Fill *p with rho_scale 3e-7, M = 10 Msun, gamma 5/3, dt 1e-2, n_sub 8,
 * explicit mode, limiter 0.3, eq_band 0.1, clamp 1, 60 iterations, L2 path. */
cool_status cool_params_default(cool_params* p);

/* Build the table on the device in FP64 (Sec. 2.6: every node evaluates the
 * formulas of Sec. 2, including the nu_c root of Eq. 5 and the integral of
 * Eq. 6), then pack it for the step.  Synchronous: returns when the table is
 * ready (the build takes seconds for 64^4 nodes).  `stream` orders the work.
 * On success *out owns device memory until cool_table_free. */
cool_status cool_build_table(const cool_table_spec* spec, void* stream, cool_table** out);

/* Release a table (NULL is a no-op). */
cool_status cool_table_free(cool_table* t);

/* Reserve persisting L2 for the table's packed 4-D channel (on = 1) or give
 * it back (on = 0, the state of a new table).  On: the context's
 * persisting-L2 limit (cudaLimitPersistingL2CacheSize, one value per CUDA
 * context) is raised to min(packed bytes, the device maximum) if it is
 * lower, and every L2WINDOW step launch with this table attaches an
 * access-policy window over the packed channel (hit property persisting,
 * miss property streaming, hit ratio = limit / window, capped at 1).  Off:
 * persisting lines are reset to normal and the limit this call raised is
 * put back.  The carve-out is context-wide: L2 set aside for persisting
 * lines is not available to other kernels' ordinary accesses.  Measured on
 * B300 (8 sub-cycles, 16.8 M cells): the step does not gain, with a table
 * that fits L2 beside the streamed fields (75.5 MB: 1.170 ms off, 1.186 ms
 * on) or not (302 MB: 1.180 / 1.178 ms) -- the table's own reuse keeps it
 * in L2 -- while a streaming kernel run after it in the same context slows
 * down 1.7x (62 -> 105 us); hence off by default.  Freeing the table turns
 * it off.  Errors:
 * COOL_ENULL, COOL_ESTATE (not a live table), COOL_EINVAL (on not 0 or 1),
 * COOL_ECUDA. */
cool_status cool_table_l2_persist(cool_table* t, int on);

/* The spec a table was built with. */
cool_status cool_table_get_spec(const cool_table* t, cool_table_spec* spec);

/* Copy the FP64 log2 values of one channel to host memory.
 * channel 0: brems [n_Te]; 1: synchrotron [n_H*n_B*n_ne*n_Te]; 2: Coulomb
 * [n_Tc*n_Tc]; 3: the paper's layout, log2 Q_total [n_H*n_B*n_ne*n_Te]
 * (FP32 tables; made on first use).  host_out must hold that many
 * doubles.  Synchronous. */
cool_status cool_table_export(const cool_table* t, int channel, double* host_out, long long count);

/* FP32 node coordinates of one axis (0 H, 1 B, 2 n_e, 3 T_e, 4 Coulomb T)
 * to host memory (host_out holds n floats).  Synchronous. */
cool_status cool_table_nodes(const cool_table* t, int axis, float* host_out, int n);

/* The 4-D channel as packed for the step: 32-byte blocks along T_e, row
 * r = (h n_B + b) n_ne + n holding ceil((n_Te - 1)/S) blocks.  F32: 8 floats
 * (nodes S k .. S k + 7, S = 7).  BF16/F16 plain: 16 codes (S = 15), node
 * 2i in the low half of word i.  Row-scaled: words 0, 1 = FP32 offset and
 * scale, words 2..7 = 12 codes of (v - offset)/scale (S = 11).  Codes are
 * FP64 -> FP32 -> 16-bit, round to nearest even; nodes past n_Te - 1 repeat
 * the last node.  packed_bytes gives the size; export copies it to host
 * memory (synchronous). */
cool_status cool_table_packed_bytes(const cool_table* t, long long* bytes);
cool_status cool_table_export_packed(const cool_table* t, void* host_out, long long bytes);

/* Save / load a table (spec + FP64 channel values, binary, with a spec hash).
 * load rebuilds the packed device table from the stored values without
 * re-evaluating the formulas.  Synchronous. */
cool_status cool_table_save(const cool_table* t, const char* path);
cool_status cool_table_load(const char* path, void* stream, cool_table** out);

/* One cooling step over n_cells cells (Sec. 3.2): per cell, N_sub sub-cycles
 * of (i) Coulomb exchange (Eq. 16; the cancelling difference of T_i and T_e
 * formed exactly in FP32, or FP64 inside the equilibrium band with
 * fp64_critical) and (ii) radiative cooling from the table with the bridge
 * of Eq. 11, applied to u_e explicitly (min(h Q, limiter_frac u_e)) or, in
 * mode IMPLICIT for stiff cells (h Q > limiter_frac u_e), by backward Euler.
 * FP32 fields: every table index equals the node-compare rule of
 * cool_debug_lookup (axes 0..4).  Warps take tiles of cells from an 8-byte
 * tile counter that the step zeroes on `stream` before its kernel: one
 * counter per device and stream, keyed by the stream's unique id
 * (cudaStreamGetId, so cudaStreamPerThread on two host threads gets two),
 * allocated on first use.  Launches inside a stream capture never use the
 * counter (they take a fixed tile order, with the same results), so a graph
 * replayed on any stream cannot share it with a step running meanwhile.
 * Launches on one stream run in order, so no two launches that overlap in
 * time share a counter.  In mode IMPLICIT or with fp64_critical (FP32
 * fields, FP32 table, 16-byte aligned arrays, n_cells < 2^32 - 1) the
 * cells that turn stiff or enter the equilibrium band are listed in scratch
 * (4 (n_cells + 1) bytes) and stepped by a second kernel: device memory
 * kept per device and stream between calls and grown as needed (see
 * cool_release_scratch), or inside a stream capture stream-ordered memory
 * (cudaMallocAsync/cudaFreeAsync on `stream`) that the graph owns; where
 * it cannot be had each warp steps its own (bitwise the same results).
 *   field_dtype: COOL_F32 or COOL_F64 (all seven field arrays of that type).
 *   rho, B, H, u_e_in, u_i_in: device inputs, n_cells each.
 *   u_e_out, u_i_out: device outputs (may alias u_e_in / u_i_in).
 *   q_cool_out (nullable): electron energy removed by cooling during the step.
 *   q_cc_out (nullable): energy moved from ions to electrons by Coulomb.
 *     (u_e_out = u_e_in + q_cc - q_cool, u_i_out = u_i_in - q_cc.)
 *   counters (nullable, device): accumulated with atomics.
 * Invalid cells are copied through unchanged.  Out-of-range keys use the
 * table edge.  n_cells = 0 is a no-op.  Non-NULL pointers are required for
 * every non-nullable array when n_cells > 0.  For COOL_F32, arrays that are
 * 16-byte aligned use 128-bit loads; unaligned arrays take a scalar path. */
cool_status cool_step(const cool_table* t, const cool_params* p, long long n_cells,
                      cool_dtype field_dtype,
                      const void* rho, const void* B, const void* H,
                      const void* u_e_in, const void* u_i_in,
                      void* u_e_out, void* u_i_out,
                      void* q_cool_out, void* q_cc_out,
                      cool_counters* counters, void* stream);

/* Build the three FP64 channels of a table into caller-allocated device
 * arrays, allocating no device memory.  The paper has no counterpart: this
 * entry point serves callers that cannot let a library call cudaMalloc or
 * cudaFree -- for example a simulation code that reserves its whole device
 * memory as one arena at start-up and hands out slices of it, or a framework
 * whose caching allocator must own every device allocation.
 *   spec: as for cool_build_table, but every axis must have at most 256
 *     nodes (n_H, n_B, n_ne, n_Te, n_Tc <= 256); larger axes return
 *     COOL_EINVAL because the builder's scratch is a fixed-size array.
 *   lb_out [n_Te], ls_out [n_H n_B n_ne n_Te], lc_out [n_Tc n_Tc]: device
 *     arrays (8-byte aligned) that receive the same FP64 log2 values, in the
 *     same layouts, as cool_table_export returns for a table built from spec.
 *   stream: the work is enqueued on it; the call returns after enqueueing.
 * The builder's scratch (node coordinates and a counter) is one 20.25 KiB
 * file-scope device array that every GPU loading the library holds until the
 * process exits.  All calls share it and it keeps the last call's contents
 * (the counter is cleared at the start of each call), so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race:
 * order them on one stream.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, with the caller's device current) and enqueues the
 * quadrature constants on `stream` before its kernels; the first call on a
 * device may also load the library's device code, so make that first call
 * before any stream capture. */
cool_status cool_build_channels_noalloc(const cool_table_spec* spec, double* lb_out, double* ls_out,
                                        double* lc_out, void* stream);

/* Adjoint of cool_step (FP32 fields, FP32 table, fp64_critical = 0): for
 * L = sum(g_u_e_out u_e_out + g_u_i_out u_i_out) over the cells of one
 * cool_step with the same table, params and inputs, writes dL/d(rho, B, H,
 * u_e_in, u_i_in) per cell and, when the pointers are given, ADDS dL/d(log2
 * table values) into g_lb [n_Te], g_ls [n_H n_B n_ne n_Te] (natural layout,
 * T_e fastest) and g_lc [n_Tc n_Tc] (atomic accumulation: order of the FP32
 * additions is not deterministic).  The forward sub-cycles are recomputed,
 * not stored; explicit and limited sub-cycles are differentiated on the
 * branch taken, implicit ones by the implicit-function theorem at the root.
 * Without table gradients (all three NULL) the chain rule runs in the
 * forward order (the 2x5 Jacobian of the cell carried along the
 * sub-cycles); with any of them, in the reverse order over the kept
 * sub-cycle states.  The two give the same input gradients up to FP32
 * rounding order (not bitwise).  In implicit mode (with table gradients:
 * when n_sub <= 8) the stiff cells are deferred to a second kernel through
 * a list in the scratch cool_step uses for its own (4 (n_cells + 1) bytes,
 * kept per device and stream; stream-ordered inside a capture); where it
 * cannot be had every cell is solved in place (the same gradients to FP32
 * rounding).  Invalid cells pass the output adjoints
 * through.  The inputs must not alias
 * the gradient outputs.  Device pointers, asynchronous on stream; n_sub <= 64. */
cool_status cool_step_bwd(const cool_table* t, const cool_params* p, long long n_cells, const float* rho,
                          const float* B, const float* H, const float* u_e_in, const float* u_i_in,
                          const float* g_u_e_out, const float* g_u_i_out, float* g_rho, float* g_B, float* g_H,
                          float* g_u_e_in, float* g_u_i_in, float* g_lb, float* g_ls, float* g_lc, void* stream);

/* Forward step and its Jacobian in one pass (the adjoint of cool_step_bwd
 * split at the cell's Jacobian; Sec. 3.2's step, differentiated by the chain
 * rule in the forward order).  Writes u_e_out, u_i_out -- cool_step's
 * outputs for the same table, params and inputs, bit for bit -- and the
 * Jacobian of each cell's outputs with respect to its inputs, so that
 * cool_step_bwd_jac can later form the input gradients for any output
 * adjoints without stepping again.  jac: 10 n_cells floats (device,
 * caller-owned), ten rows of n_cells: row x = d u_e_out / d in_x and row
 * 5 + x = d u_i_out / d in_x, for in = (rho, B, H, u_e_in, u_i_in), x = 0..4.
 * Invalid cells pass through with the identity on (u_e, u_i).  The outputs
 * may overwrite u_e_in, u_i_in (each cell reads its inputs first); jac must
 * not alias the fields.  FP32 fields, an FP32 table, the L2WINDOW path,
 * explicit or implicit mode (stiff cells through the list scratch of
 * cool_step_bwd); fp64_critical: COOL_EUNSUPPORTED.  Device pointers,
 * asynchronous on stream; n_sub <= 64. */
cool_status cool_step_fwd_jac(const cool_table* t, const cool_params* p, long long n_cells, const float* rho,
                              const float* B, const float* H, const float* u_e_in, const float* u_i_in,
                              float* u_e_out, float* u_i_out, float* jac, void* stream);

/* Input gradients from a Jacobian of cool_step_fwd_jac (same layout, same
 * n_cells) and the output adjoints g_u_e_out, g_u_i_out:
 * g_x = g_u_e_out d u_e_out/d x + g_u_i_out d u_i_out/d x for x = rho, B,
 * H, u_e_in, u_i_in.  These are cool_step_bwd's input gradients (without
 * table gradients) bit for bit: the same Jacobian, contracted by the same
 * expression.  Device pointers, asynchronous on stream; the gradients must
 * not alias jac or the adjoints. */
cool_status cool_step_bwd_jac(long long n_cells, const float* jac, const float* g_u_e_out, const float* g_u_i_out,
                              float* g_rho, float* g_B, float* g_H, float* g_u_e_in, float* g_u_i_in, void* stream);

/* cool_step with the disk geometry of each cell: r (radius in r_g per
 * cell, FP32 device array, > 0) and `disk` (spin, optional H_th from the
 * state, optional temperature floor).  H may be NULL when
 * disk->h_from_state.  FP32 fields and an FP32 table (L2WINDOW path);
 * explicit or implicit, fp64_critical allowed; otherwise as cool_step.
 * counters->n_floor counts cells whose cooling the floor skipped in some
 * sub-cycle.  A cell with a non-finite or non-positive r is invalid
 * (passed through, counted). */
cool_status cool_step_disk(const cool_table* t, const cool_params* p, const cool_disk* disk, long long n_cells,
                           const float* rho, const float* B, const float* H, const float* u_e_in,
                           const float* u_i_in, const float* r, float* u_e_out, float* u_i_out,
                           float* q_cool_out, float* q_cc_out, cool_counters* counters, void* stream);

/* cool_step on HOST arrays (FP32; the L2WINDOW path): the cells are
 * streamed through the device in chunks of chunk_cells (0: n/12, at least
 * 65536; rounded to a multiple of 128), each chunk's five input copies,
 * its step and its two output copies on one of two internal streams, so that
 * host-to-device copies, steps and device-to-host copies of consecutive
 * chunks overlap.  The host arrays should be page-locked (cudaHostAlloc or
 * cudaHostRegister) for the copies to run asynchronously; they must stay
 * valid until `stream` reaches the end of the call's work.  Device staging
 * (14 chunk_cells floats) is allocated and freed stream-ordered on `stream`.
 * Outputs q_cool/q_cc are not produced.  counters: device pointer or NULL. */
cool_status cool_step_host(const cool_table* t, const cool_params* p, long long n_cells, const float* rho,
                           const float* B, const float* H, const float* u_e_in, const float* u_i_in,
                           float* u_e_out, float* u_i_out, long long chunk_cells, cool_counters* counters,
                           void* stream);

/* The step with every rate evaluated from the formulas instead of the
 * table: the paper's "analytic" comparison (Appendix, direct calculation
 * against the table).  Per cell and sub-cycle: the bremsstrahlung fits
 * (Eqs. 1-2), the nu_c root of Eq. 5 and the synchrotron integral of Eq. 6
 * (1024-point quadrature), the Compton factor (Eqs. 7-9), the bridge
 * (Eqs. 11-12) and the Coulomb coefficient (Eq. 16); the update is the one
 * of cool_step (explicit or implicit; fp64_critical and the texture paths
 * do not apply).  FP64 device arrays only (8-byte aligned).  `physics` gives
 * k2_switch_T, lnLambda, theta_i_uses_mp and compton_literal; its node
 * counts and ranges are ignored (no table, no clamping).  counters:
 * n_clamped counts cells whose nu_c hit the 1e30 Hz cap.  Asynchronous on
 * stream; FP64-bound on B300 (slow by design: the comparison point). */
cool_status cool_step_direct(const cool_table_spec* physics, const cool_params* p, long long n_cells,
                             const double* rho, const double* B, const double* H, const double* u_e_in,
                             const double* u_i_in, double* u_e_out, double* u_i_out, double* q_cool_out,
                             double* q_cc_out, cool_counters* counters, void* stream);

/* Radiation-pressure correction of the electron temperature (Sec. 5.2, the
 * total-pressure equation): where the local scattering depth tau_sca =
 * n_e sigma_T H exceeds tau_crit (4.6: fewer than 1 % of photons escape
 * unscattered), the thermal pressure is read as gas plus radiation,
 * P = a_rad T_e^4 + n k (T_e + T_i), and T_e recomputed; with P = n k (T_e +
 * T_i) from the fields this is a_rad T^4 + n k T = n k T_e,sim (u_i drops
 * out).  te_out[i] = the corrected T_e [K] in thick cells, T_e,sim
 * elsewhere, NaN for invalid cells (non-finite or non-positive rho, u_e,
 * negative H).  thick_out (nullable) = 1 where corrected.  FP32 device
 * arrays (4-byte aligned; 16-byte aligned with thick_out 4-byte aligned
 * takes the vector path).  a_rad: the paper prints 7.5646e-15 erg cm^-3
 * K^-4.  Uses rho_scale, M_bh_msun and gamma_e of p.  Asynchronous. */
cool_status cool_radiation_te(const cool_params* p, double tau_crit, double a_rad, long long n_cells,
                              const float* rho, const float* H, const float* u_e, float* te_out,
                              unsigned char* thick_out, void* stream);

/* ---- learned surrogate of the synchrotron channel (not in the paper) ------
 * An MLP 4 -> 128 -> 128 -> 1 with SiLU (inputs: the four log2 coordinates
 * normalised to [-1, 1] over the table box, each as two bf16 parts (value
 * and rounding residual), plus the side of the K2 switch temperature as
 * +-1, where the channel jumps; output: the standardised
 * log2(eta Q_syn)), BF16 weights and activations on the tensor cores
 * (tcgen05, FP32 accumulation), trained on the GPU by Adam on MSE in log2
 * space with samples labelled by the FP64 formulas (half on table nodes,
 * half uniform in log space).  A bit per 4-D table cell marks where the
 * network misses the table by more than fallback_tol (relative, checked at
 * the cell's corners and centre): there the table is used instead. */
typedef struct cool_surrogate cool_surrogate;   /* opaque; owns device memory */

typedef struct {
    int channel;               /* 1 = synchrotron (the only one supported) */
    long long n_samples;       /* training samples (default 2^24), multiple of batch */
    int batch;                 /* samples per Adam step, multiple of 128 (16384) */
    int epochs;                /* passes over the samples (16); 0 = initial weights only */
    double lr, lr_final;       /* Adam learning rate, cosine decay from lr to lr_final */
    unsigned long long seed;   /* samples and initial weights */
    double fallback_tol;       /* 1e-3 */
} cool_fit_spec;

typedef struct {
    double final_loss;         /* MSE (standardised units) of the last batch */
    long long steps;           /* Adam steps taken */
    long long mask_cells;      /* 4-D table cells */
    long long fallback_cells;  /* cells where the table is used instead of the network */
    long long param_bytes_bf16;/* bytes of the network as stored for inference */
    double mean, std;          /* output standardisation (log2 units) */
    double x_switch;           /* normalised log2 T_e of the K2 switch (input column 8 is +1 above it) */
} cool_surrogate_stats;

cool_status cool_fit_spec_default(cool_fit_spec* f);

/* Train a surrogate of table t's synchrotron channel (synchronous; device
 * memory for the samples is allocated and freed inside). */
cool_status cool_surrogate_fit(const cool_table* t, const cool_fit_spec* f, void* stream, cool_surrogate** out);
cool_status cool_surrogate_free(cool_surrogate* s);
cool_status cool_surrogate_info(const cool_surrogate* s, cool_surrogate_stats* out);

/* The 18817 FP32 parameters (W1 [128][16]: columns 0..3 the coordinates,
 * column 4 the switch side, columns 5..15 zero; b1 [128], W2 [128 out][128
 * in], b2 [128], w3 [128], b3), host memory. */
cool_status cool_surrogate_get_params(const cool_surrogate* s, float* host, int n);
cool_status cool_surrogate_set_params(cool_surrogate* s, const float* host, int n);

/* Gradients of the batch-mean squared error over n samples (device x4
 * [n][4] normalised inputs, y_std [n] standardised targets, n % 128 == 0)
 * into host grads [18817]; *loss_host (nullable) the loss.  Check entry of
 * the training kernel (synchronous). */
cool_status cool_surrogate_grads(cool_surrogate* s, long long n, const float* x4, const float* y_std,
                                 float* grads_host, float* loss_host, void* stream);

/* Network output in log2 units at n normalised points (device arrays). */
cool_status cool_surrogate_eval(const cool_surrogate* s, long long n, const float* x4, float* y, void* stream);

/* The fallback bits (one per 4-D table cell, cell index ((h (nB-1) + b)
 * (nne-1) + n) (nTe-1) + t), host memory of (cells + 31)/32 words. */
cool_status cool_surrogate_mask(const cool_surrogate* s, uint32_t* host_bits, long long words);

/* Replace the fallback bits (host memory, same layout and size as
 * cool_surrogate_mask; bits past the last cell are ignored).  A set bit
 * sends every cell whose sub-cycle lands in that table cell to the table. */
cool_status cool_surrogate_set_mask(cool_surrogate* s, const uint32_t* host_bits, long long words);

/* The step of cool_step (explicit mode with the limiter, FP32 fields, FP32
 * table) with the synchrotron channel read from the surrogate instead of
 * the table: each sub-cycle evaluates the network on tiles of 128 cells
 * (two tensor-core products) at the cell's (H, B, n_e, T_e), except where
 * the cell's 4-D table cell carries a fallback bit, which reads the table
 * as cool_step does.  Brems, Coulomb, the bridge (Eq. 11), the limiter and
 * the update are those of cool_step.  t must be the table s was fitted to
 * (same node counts and box, else COOL_EINVAL); implicit mode, fp64_critical
 * and 16-bit tables give COOL_EUNSUPPORTED.  Arguments, aliasing and
 * invalid-cell handling as cool_step; counters->n_fallback counts cells that
 * used the table in some sub-cycle.  Device pointers, asynchronous on stream. */
cool_status cool_surrogate_infer(const cool_surrogate* s, const cool_table* t, const cool_params* p,
                                 long long n_cells, const float* rho, const float* B, const float* H,
                                 const float* u_e_in, const float* u_i_in, float* u_e_out, float* u_i_out,
                                 float* q_cool_out, float* q_cc_out, cool_counters* counters, void* stream);

/* Check entry of the tensor-core GEMM primitive the surrogate is built on
 * (5th-generation tensor cores, tcgen05.mma kind::f16, FP32 accumulation in
 * tensor memory): C[M x N] = A[M x K] B[N x K]^T with A, B bf16 row-major
 * device arrays (16-byte aligned) and C fp32 row-major.  M % 128 == 0,
 * 16 <= N <= 128 and K <= 128, both multiples of 16.  err (nullable device
 * word) gets bit 0 set if the tensor core did not signal completion within
 * the kernel's bounded wait.  Asynchronous on stream. */
cool_status cool_debug_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, unsigned* err,
                                 void* stream);

/* Check entry of the kernels' bounded waits: one thread polls an mbarrier
 * that nothing completes, `polls` times (1 <= polls <= 2^20; each poll is
 * itself time-bounded by the hardware), then sets bit 0 of *err (a device
 * word) and returns -- the failure path that the TMA-staged step and the
 * tensor-core kernels take, reporting through their error words, when a
 * bulk copy or a tcgen05.mma never signals completion; the context stays
 * usable.  Errors: COOL_ENULL (err NULL), COOL_EINVAL (polls out of range).
 * Asynchronous on stream. */
cool_status cool_debug_wait_timeout(int polls, unsigned* err, void* stream);

/* Error word of the TMA_SMEM step path on the current device, read
 * synchronously into *err_out (host): bit 0 is set when a bulk copy of a
 * field tile never signalled completion within the kernel's bounded wait;
 * that warp then wrote none of its remaining tiles' outputs.  clear = 1
 * zeroes the word after reading it.  Errors: COOL_ENULL (err_out NULL),
 * COOL_EINVAL (clear not 0 or 1), COOL_ECUDA. */
cool_status cool_tma_error(unsigned* err_out, int clear);

/* Free the scratch the library keeps for the deferral lists of cool_step,
 * cool_step_disk and cool_step_bwd (implicit mode, fp64_critical) on the
 * current device: one buffer per stream that ran such a step, 4 bytes per
 * cell of its largest call, plus any it outgrew.  Waits for the device
 * (cudaDeviceSynchronize) first, so no launch can still use them; call it
 * while no other host thread is inside a step call on this device.  The
 * next call that needs a list allocates again.  Not part of the paper's
 * method.
 * COOL_ECUDA if the device cannot be synchronised. */
cool_status cool_release_scratch(void);

/* Index/weight selection of the table interpolation on one axis, for FP32
 * keys in the axis' physical unit (device arrays of n).  axis 0..4 (H, B,
 * n_e, T_e, Coulomb T), the exact rule: idx = the largest j in [0, N-2]
 * with node32[j] <= key (0 below the first node), w = log2(key / x_j) / dl
 * clamped to [0, 1].  axis 5..9: the same selection as the step computes
 * it on axes 0..4 (a guess from log2, confirmed by the weight, exact node
 * compares near a node): the same idx and w.  Asynchronous on stream. */
cool_status cool_debug_lookup(const cool_table* t, int axis, long long n, const float* keys,
                              int* idx, float* w, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* COOL_H */
