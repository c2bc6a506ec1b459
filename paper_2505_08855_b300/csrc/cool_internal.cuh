// cool_internal.cuh -- shared definitions of libcool's CUDA sources.
//
// Physical constants (cgs, CODATA 2018), the device-side table layout and
// the kernel parameter blocks.  This is the product path: it shares nothing
// with the CPU oracle used by the tests.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cool.h"

namespace cool {

// ---- constants (cgs) -------------------------------------------------------
constexpr double kC = 2.99792458e10;        // speed of light
constexpr double kKB = 1.380649e-16;        // Boltzmann
constexpr double kME = 9.1093837015e-28;    // electron mass
constexpr double kMP = 1.67262192369e-24;   // proton mass
constexpr double kQE = 4.80320471e-10;      // elementary charge (esu)
constexpr double kHP = 6.62607015e-27;      // Planck
constexpr double kSigT = 6.6524587321e-25;  // Thomson cross section
constexpr double kSigSB = 5.670374419e-5;   // Stefan-Boltzmann
constexpr double kG = 6.6743e-8;            // gravitational constant
constexpr double kMsun = 1.98847e33;        // solar mass
constexpr double kPi = 3.141592653589793238;

constexpr int kMaxAxis = 512;
constexpr int kMaxTc = 128;

// ---- the table --------------------------------------------------------------
// Axis data on the device, per axis a (0 H, 1 B, 2 n_e, 3 T_e, 4 Coulomb T):
//   x32[j]  FP32 node (index selection compares keys against it exactly)
//   rx32[j] FP32 of 1/x_j (weight: log2(key * rx_j) = log2(key/x_j))
//   lx32[j] FP32 of l_j = log2 x_j
// stored as axis_off[a] + {0, n, 2n} inside one float array.
struct DevTable {
    int n[5];
    int axis_off[5];
    float inv_dl[5];        // 1/dl, dl = node spacing in log2
    double dl64[5];
    double l0_64[5];
    const float* axes;      // concatenated axis arrays (x, rx, lx per axis)
    const double* axes64;   // concatenated FP64 axis arrays (x, lx per axis)
    const float* lb;        // [n_Te]       log2(Q_brem / n_e^2)
    // log2(eta Q_syn) packed in 32-byte blocks along T_e: row r = (h nB + b) nN + n
    // holds nblk blocks; block k covers nodes S k .. S k + W - 1 (clamped to nT - 1)
    // and serves the intervals S k .. S k + S - 1 (S = W - 1):
    //   fmt 0 (FP32):          8 floats                     W = 8,  S = 7
    //   fmt 1/2 (BF16/FP16):   16 16-bit values              W = 16, S = 15
    //   fmt 3/4 (BF16/FP16 block-scaled): float off, float scale, 12 16-bit
    //                          residuals r, value = off + scale r,   W = 12, S = 11
    const uint32_t* lsb;
    // the paper's layout (COOL_PATH_QTOTAL, made on first use): log2 Q_total
    // on the same grid, packed as fmt 0 blocks in the same row order
    const uint32_t* lst;
    int fmt;
    int blk_stride;         // S
    int nblk;               // ceil((nT - 1) / S)
    const float* lc;        // [nTc nTc]    log2 C
    const double* lb64;     // FP64 copies (FP64 step path, export)
    const double* ls64;
    const double* lc64;
};

}  // namespace cool

// The opaque handle of the C ABI.
struct cool_table {
    uint32_t magic;             // kTableMagic while alive
    int device;
    cool_table_spec spec;
    cool::DevTable dev;
    void* d_axes;               // device allocations owned by the table
    void* d_axes64;
    void* d_lb; void* d_ls; void* d_lc;
    void* d_lb64; void* d_ls64; void* d_lc64;
    double* h_lb64;             // host FP64 copies of the channels (export / save)
    double* h_ls64;
    double* h_lc64;
    float* h_axes;              // host copy of the FP32 axis arrays
    size_t ls_bytes;
    int l2_persist;             // cool_table_l2_persist on: step launches carry the L2 window
    int l2_raised;              // this table raised the context's persisting-L2 limit ...
    size_t l2_prev_limit;       // ... from this value
    // texture comparison paths (created on first use): the FP32 4-D channel
    // as a 3-D CUDA array (x = T_e, y = n_e, z = h n_B + b) and two texture
    // objects on it, point sampling and hardware linear filtering
    cudaArray_t tex_arr;
    unsigned long long tex_point, tex_linear;
    // the paper's-layout channel (COOL_PATH_QTOTAL): FP64 natural layout and
    // packed FP32 blocks, made on first use
    void* d_lt64;
    void* d_lst;
};

constexpr uint32_t kTableMagic = 0xC0011AB1u;

namespace cool {

// Host helpers shared by the .cu files of the library.
// The step's tile counter for the current device and stream `st`: created
// on first use (8 bytes of device memory kept for the life of the process),
// one per (device, stream) so that steps on different streams never share
// one; nullptr if it cannot be created (first use inside stream capture, or
// an allocation failure), and the step then takes its static tile order.
unsigned long long* sched_counter(cudaStream_t st);
// Scratch for a deferral list of `words` 32-bit words, kept per (device,
// stream) between calls and grown as needed; nullptr inside a stream
// capture (*capturing set: allocate stream-ordered scratch in the graph
// instead) or on an allocation failure (step without the list).
unsigned* list_scratch(cudaStream_t st, size_t words, bool* capturing);
// The deferral list of one call over n cells (n + 1 words: the count,
// zeroed on `st`, then the indices): the per-stream scratch, or inside a
// capture stream-ordered scratch the caller frees with cudaFreeAsync after
// its launches (*owned).  nullptr: no list (*err set if the zeroing failed).
unsigned* list_for_call(cudaStream_t st, long long n, bool* owned, cudaError_t* err);
cool_status set_cuda_error(cudaError_t e);
bool table_ok(const cool_table* t);
long long syn_count(const cool_table_spec& s);

// Builder entry (cool_build.cu): evaluates the FP64 channels on the device.
cool_status build_channels_fp64(const cool_table_spec& s, const double* d_axes64,
                                const int* axis_off64, double* d_lb64, double* d_ls64,
                                double* d_lc64, cudaStream_t st);
// The paper's layout: log2 Q_total on the 4-D grid from the FP64 brems and
// synchrotron channels (synchronous on st).
cool_status build_qtotal_fp64(const cool_table_spec& s, const double* d_axes64, const int* axis_off64,
                              const double* d_lb64, const double* d_ls64, double* d_lt64, cudaStream_t st);
// Build (once, synchronously) and pack the paper's-layout channel of an FP32
// table: t->d_lt64 (FP64, natural layout) and t->dev.lst (packed blocks).
cool_status table_qtotal(cool_table* t);

// Surrogate training samples (cool_build.cu): x [n][4] normalised coordinates,
// y [n] log2(eta Q_syn) from the formulas; even samples sit on table nodes.
cool_status fit_samples_fp64(const cool_table_spec& s, long long n, unsigned long long seed, float* x, double* y,
                             cudaStream_t st);

// Step launches (cool_step.cu).
cool_status launch_step_f32(const cool_table* t, const cool_params* p, long long n,
                            const float* rho, const float* B, const float* H,
                            const float* ue, const float* ui, float* ue_o, float* ui_o,
                            float* qc, float* qx, cool_counters* cnt, cudaStream_t st,
                            const cool_disk* disk = nullptr, const float* r = nullptr);
// Step kernels of the 16-bit table formats (cool_step_f16.cu: fmt 1, 2;
// cool_step_f16s.cu: fmt 3, 4) for launch_step_f32: var = implicit |
// fp64_critical << 1 | counters << 2; nullptr outside their formats.
const void* step_kernel_f16(int fmt, bool vec, int var);
const void* step_kernel_f16s(int fmt, bool vec, int var);
cool_status launch_step_f64(const cool_table* t, const cool_params* p, long long n,
                            const double* rho, const double* B, const double* H,
                            const double* ue, const double* ui, double* ue_o, double* ui_o,
                            double* qc, double* qx, cool_counters* cnt, cudaStream_t st);
cool_status launch_step_bwd_f32(const cool_table* t, const cool_params* p, long long n, const float* rho,
                                const float* B, const float* H, const float* ue, const float* ui,
                                const float* gue, const float* gui, float* g_rho, float* g_B, float* g_H,
                                float* g_ue, float* g_ui, float* g_lb, float* g_ls, float* g_lc, cudaStream_t st);
cool_status launch_step_fwd_jac_f32(const cool_table* t, const cool_params* p, long long n, const float* rho,
                                    const float* B, const float* H, const float* ue, const float* ui, float* ue_out,
                                    float* ui_out, float* jac, cudaStream_t st);
cool_status launch_jac_contract_f32(long long n, const float* jac, const float* gue, const float* gui, float* g_rho,
                                    float* g_B, float* g_H, float* g_ue, float* g_ui, cudaStream_t st);
cool_status validate_params(const cool_params* p);
cool_status table_textures(cool_table* t);
cool_status launch_step_tma(const cool_table* t, const cool_params* p, long long n, const float* rho,
                            const float* B, const float* H, const float* ue, const float* ui, float* ue_o,
                            float* ui_o, float* qc, float* qx, cool_counters* cnt, cudaStream_t st);
cool_status launch_step_direct(const cool_table_spec& phys, const cool_params* p, long long n, const double* rho,
                               const double* B, const double* H, const double* ue, const double* ui, double* ue_o,
                               double* ui_o, double* qc, double* qx, cool_counters* cnt, cudaStream_t st);
cool_status launch_step_tex(const cool_table* t, const cool_params* p, long long n, const float* rho,
                            const float* B, const float* H, const float* ue, const float* ui, float* ue_o,
                            float* ui_o, float* qc, float* qx, cool_counters* cnt, cudaStream_t st);
cool_status launch_step_surrogate(const cool_surrogate* sg, const cool_table* t, const cool_params* p, long long n,
                                  const float* rho, const float* B, const float* H, const float* ue,
                                  const float* ui, float* ue_o, float* ui_o, float* qc, float* qx,
                                  cool_counters* cnt, cudaStream_t st);
cool_status launch_debug_lookup(const cool_table* t, int axis, long long n, const float* keys,
                                int* idx, float* w, cudaStream_t st);

}  // namespace cool
