// cool_api.cu -- host side of the libcool C ABI (include/cool.h): argument
// validation, table construction/packing/persistence, and kernel dispatch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>
#include <utility>

#include "cool_internal.cuh"

namespace cool {

static thread_local int g_last_cuda_error = 0;

cool_status set_cuda_error(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return COOL_ECUDA;
}

// Live tables: a handle is valid only while registered, so a freed (or
// never created) handle is rejected without reading its memory.
static std::mutex g_tables_mu;
static std::unordered_set<const cool_table*>& live_tables() {
    static std::unordered_set<const cool_table*> s;
    return s;
}
static void register_table(const cool_table* t) {
    std::lock_guard<std::mutex> g(g_tables_mu);
    live_tables().insert(t);
}
static bool unregister_table(const cool_table* t) {
    std::lock_guard<std::mutex> g(g_tables_mu);
    return live_tables().erase(t) == 1;
}

// Tile counter of the dynamic tile order, one per (device, stream id).  The
// stream's unique id, not its handle, is the key: cudaStreamPerThread (and
// the legacy stream under per-thread default streams) is one handle value
// for many streams.  Inside a stream capture no counter is used (nullptr:
// the static tile order), so a captured launch replayed on another stream
// never shares a counter with a launch running at the same time; a counter
// is only ever used by launches on its own stream, which run in order.
unsigned long long* sched_counter(cudaStream_t st) {
    static std::mutex mu;
    static std::map<std::pair<int, unsigned long long>, unsigned long long*> counters;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = 0;
    unsigned long long sid = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetId(st, &sid) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    auto it = counters.find({dev, sid});
    if (it != counters.end()) return it->second;
    unsigned long long* p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    counters[{dev, sid}] = p;
    return p;
}

// Scratch of the deferral lists (the flagged cells of the implicit mode and
// of fp64_critical, stepped by the list kernels): at least `words` 32-bit
// words, one buffer per (device, stream id), kept between calls so that a
// caller who synchronises after every step does not hand the memory back
// and map it again on every call.  A call that needs more grows it to at
// least twice its size; the superseded buffer is kept (a launch another
// host thread already enqueued on the same stream may still read it) until
// cool_release_scratch.  Inside a stream capture: nullptr with *capturing
// set (the caller allocates stream-ordered scratch inside the graph, which
// a replay on any stream owns alone); nullptr on an allocation failure.
namespace {
struct ListBuf {
    unsigned* p = nullptr;
    size_t words = 0;
};
std::mutex g_list_mu;
std::map<std::pair<int, unsigned long long>, ListBuf>& list_bufs() {
    static std::map<std::pair<int, unsigned long long>, ListBuf> m;
    return m;
}
std::vector<std::pair<int, unsigned*>>& list_superseded() {
    static std::vector<std::pair<int, unsigned*>> v;
    return v;
}
}  // namespace

unsigned* list_scratch(cudaStream_t st, size_t words, bool* capturing) {
    *capturing = false;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cap != cudaStreamCaptureStatusNone) {
        *capturing = true;
        return nullptr;
    }
    int dev = 0;
    unsigned long long sid = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetId(st, &sid) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_list_mu);
    ListBuf& b = list_bufs()[{dev, sid}];
    if (b.words >= words) return b.p;
    const size_t want = words > 2 * b.words ? words : 2 * b.words;
    unsigned* p = nullptr;
    if (cudaMalloc(&p, want * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.p) list_superseded().push_back({dev, b.p});
    b.p = p;
    b.words = want;
    return p;
}

unsigned* list_for_call(cudaStream_t st, long long n, bool* owned, cudaError_t* err) {
    *owned = false;
    *err = cudaSuccess;
    bool cap = false;
    unsigned* p = list_scratch(st, (size_t)n + 1, &cap);
    if (!p && cap) {
        if (cudaMallocAsync(&p, sizeof(unsigned) * ((size_t)n + 1), st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        *owned = true;
    }
    if (!p) return nullptr;
    const cudaError_t e = cudaMemsetAsync(p, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) {
        if (*owned) cudaFreeAsync(p, st);
        *owned = false;
        *err = e;
        return nullptr;
    }
    return p;
}

bool table_ok(const cool_table* t) {
    if (t == nullptr) return false;
    std::lock_guard<std::mutex> g(g_tables_mu);
    return live_tables().count(t) == 1 && t->magic == kTableMagic;
}

long long syn_count(const cool_table_spec& s) {
    return (long long)s.n_H * s.n_B * s.n_ne * s.n_Te;
}

cool_status validate_params(const cool_params* p) {
    if (!p) return COOL_ENULL;
    if (!(p->rho_scale > 0.0) || !isfinite(p->rho_scale)) return COOL_EINVAL;
    if (!(p->M_bh_msun > 0.0) || !isfinite(p->M_bh_msun)) return COOL_EINVAL;
    if (!(p->gamma_e > 1.0) || !(p->gamma_i > 1.0) || !isfinite(p->gamma_e) || !isfinite(p->gamma_i))
        return COOL_EINVAL;
    if (!(p->dt >= 0.0) || !isfinite(p->dt)) return COOL_EINVAL;
    if (p->n_sub < 1 || p->n_sub > 64) return COOL_EINVAL;
    if (p->mode != COOL_EXPLICIT_LIMITED && p->mode != COOL_IMPLICIT_STIFF) return COOL_EINVAL;
    if (!(p->limiter_frac > 0.0 && p->limiter_frac <= 1.0)) return COOL_EINVAL;
    if (!(p->eq_band >= 0.0 && p->eq_band < 1.0)) return COOL_EINVAL;
    if (!(p->coulomb_clamp > 0.0 && p->coulomb_clamp <= 1.0)) return COOL_EINVAL;
    if (p->implicit_iters < 1 || p->implicit_iters > 200) return COOL_EINVAL;
    if (p->path != COOL_PATH_L2WINDOW && p->path != COOL_PATH_TMA_SMEM && p->path != COOL_PATH_TEXTURE_POINT &&
        p->path != COOL_PATH_TEXTURE_HWLERP && p->path != COOL_PATH_QTOTAL)
        return COOL_EUNSUPPORTED;
    if ((p->path == COOL_PATH_TEXTURE_POINT || p->path == COOL_PATH_TEXTURE_HWLERP ||
         p->path == COOL_PATH_QTOTAL) &&
        (p->mode != COOL_EXPLICIT_LIMITED || p->fp64_critical != 0))
        return COOL_EUNSUPPORTED;   // the texture and paper's-layout paths are explicit FP32 only
    if (p->fp64_critical != 0 && p->fp64_critical != 1) return COOL_EINVAL;
    return COOL_OK;
}

namespace {
__global__ void k_f64_to_f32(const double* src, float* dst, long long n) {
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (float)src[i];
}
std::mutex g_tex_mu;
}  // namespace

// The texture comparison paths' 3-D array (FP32 log2 values of the 4-D
// channel, x = T_e, y = n_e, z = h n_B + b) and texture objects, made once
// per table (synchronous).  Limits: the device's 3-D texture extents.
cool_status table_textures(cool_table* t) {
    std::lock_guard<std::mutex> g(g_tex_mu);
    if (t->tex_arr) return COOL_OK;
    const cool_table_spec& s = t->spec;
    int wmax = 0, hmax = 0, dmax = 0;
    cudaDeviceGetAttribute(&wmax, cudaDevAttrMaxTexture3DWidth, t->device);
    cudaDeviceGetAttribute(&hmax, cudaDevAttrMaxTexture3DHeight, t->device);
    cudaDeviceGetAttribute(&dmax, cudaDevAttrMaxTexture3DDepth, t->device);
    const long long depth = (long long)s.n_H * s.n_B;
    if (s.n_Te > wmax || s.n_ne > hmax || depth > dmax) return COOL_EUNSUPPORTED;
    const long long cnt = syn_count(s);
    float* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(float) * cnt);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? COOL_ENOMEM : set_cuda_error(e);
    k_f64_to_f32<<<1184, 256>>>((const double*)t->d_ls64, tmp, cnt);
    cudaArray_t arr = nullptr;
    cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
    const cudaExtent ext = make_cudaExtent(s.n_Te, s.n_ne, depth);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMalloc3DArray(&arr, &fd, ext, 0);
    if (e == cudaSuccess) {
        cudaMemcpy3DParms cp;
        memset(&cp, 0, sizeof(cp));
        cp.srcPtr = make_cudaPitchedPtr(tmp, sizeof(float) * s.n_Te, s.n_Te, s.n_ne);
        cp.dstArray = arr;
        cp.extent = ext;
        cp.kind = cudaMemcpyDeviceToDevice;
        e = cudaMemcpy3D(&cp);
    }
    cudaTextureObject_t to[2] = {0, 0};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        cudaResourceDesc rd;
        memset(&rd, 0, sizeof(rd));
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td;
        memset(&td, 0, sizeof(td));
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = k == 0 ? cudaFilterModePoint : cudaFilterModeLinear;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&to[k], &rd, &td, nullptr);
    }
    cudaError_t e2 = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        for (int k = 0; k < 2; ++k)
            if (to[k]) cudaDestroyTextureObject(to[k]);
        if (arr) cudaFreeArray(arr);
        return e == cudaErrorMemoryAllocation ? COOL_ENOMEM : set_cuda_error(e);
    }
    t->tex_point = (unsigned long long)to[0];
    t->tex_linear = (unsigned long long)to[1];
    t->tex_arr = arr;
    return COOL_OK;
}


namespace {

__global__ void k_pack_f32(const double* src, float* dst, long long n) {
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (float)src[i];
}

// 16-bit codes: FP64 -> FP32 (round to nearest even) -> BF16 or FP16 (RNE).
__device__ __forceinline__ uint32_t code16(double v, int f16) {
    float f = (float)v;
    if (f16) return (uint32_t)__half_as_ushort(__float2half_rn(f));
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// FP64 [rows][nT] -> 32-byte blocks [rows][nblk] of the table format (see
// DevTable): one thread per block.
__global__ void k_pack_blocks(const double* src, uint32_t* dst, long long rows, int nT, int nblk, int fmt) {
    long long total = rows * nblk;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        int k = (int)(i % nblk);
        long long r = i / nblk;
        const double* row = src + r * nT;
        uint32_t* out = dst + i * 8;
        if (fmt == 0) {
            for (int o = 0; o < 8; ++o) {
                int node = min(7 * k + o, nT - 1);
                out[o] = __float_as_uint((float)row[node]);
            }
        } else if (fmt == 1 || fmt == 2) {
            int f16 = fmt == 2;
            for (int o = 0; o < 8; ++o) {
                int n0 = min(15 * k + 2 * o, nT - 1), n1 = min(15 * k + 2 * o + 1, nT - 1);
                out[o] = code16(row[n0], f16) | (code16(row[n1], f16) << 16);
            }
        } else {
            int f16 = fmt == 4;
            double lo = row[min(11 * k, nT - 1)], hi = lo;
            for (int o = 1; o < 12; ++o) {
                double v = row[min(11 * k + o, nT - 1)];
                lo = fmin(lo, v);
                hi = fmax(hi, v);
            }
            float off = (float)(0.5 * (hi + lo));
            float sc = (float)(0.5 * (hi - lo));
            out[0] = __float_as_uint(off);
            out[1] = __float_as_uint(sc);
            for (int o = 0; o < 6; ++o) {
                int n0 = min(11 * k + 2 * o, nT - 1), n1 = min(11 * k + 2 * o + 1, nT - 1);
                double r0 = sc > 0.f ? (row[n0] - (double)off) / (double)sc : 0.0;
                double r1 = sc > 0.f ? (row[n1] - (double)off) / (double)sc : 0.0;
                out[2 + o] = code16(r0, f16) | (code16(r1, f16) << 16);
            }
        }
    }
}


cool_status validate_spec(const cool_table_spec* s) {
    if (!s) return COOL_ENULL;
    int n[5] = {s->n_H, s->n_B, s->n_ne, s->n_Te, s->n_Tc};
    for (int a = 0; a < 5; ++a)
        if (n[a] < 2 || n[a] > kMaxAxis) return COOL_EINVAL;
    if (s->n_Tc > kMaxTc) return COOL_EINVAL;
    double lo[4] = {s->H_min, s->B_min, s->ne_min, s->T_min};
    double hi[4] = {s->H_max, s->B_max, s->ne_max, s->T_max};
    for (int a = 0; a < 4; ++a)
        if (!(lo[a] > 0.0) || !(hi[a] > lo[a]) || !isfinite(hi[a])) return COOL_EINVAL;
    if (s->dtype != COOL_F32 && s->dtype != COOL_BF16 && s->dtype != COOL_F16) return COOL_EUNSUPPORTED;
    if (s->row_scaled != 0 && s->row_scaled != 1) return COOL_EINVAL;
    if (s->dtype == COOL_F32 && s->row_scaled) return COOL_EUNSUPPORTED;
    // the step addresses the packed 4-D channel with 32-bit word offsets
    long long rows = (long long)s->n_H * s->n_B * s->n_ne;
    if (rows * 8LL * ((s->n_Te - 1 + 6) / 7) >= (1LL << 31)) return COOL_EINVAL;
    if (!(s->k2_switch_T >= 0.0) || !(s->lnLambda > 0.0)) return COOL_EINVAL;
    if ((s->theta_i_uses_mp != 0 && s->theta_i_uses_mp != 1) ||
        (s->compton_literal != 0 && s->compton_literal != 1))
        return COOL_EINVAL;
    return COOL_OK;
}


// Node arrays of one axis: l_j = log2(min) + j dl, x_j = 2^l_j.
void axis_nodes(double lo, double hi, int n, double* x64, double* l64) {
    double l0 = log2(lo);
    double dl = (log2(hi) - l0) / (n - 1);
    for (int j = 0; j < n; ++j) {
        l64[j] = l0 + j * dl;
        x64[j] = exp2(l64[j]);
    }
}

void free_table_memory(cool_table* t) {
    if (t->tex_point) cudaDestroyTextureObject((cudaTextureObject_t)t->tex_point);
    if (t->tex_linear) cudaDestroyTextureObject((cudaTextureObject_t)t->tex_linear);
    if (t->tex_arr) cudaFreeArray(t->tex_arr);
    void* dptrs[] = {t->d_axes, t->d_axes64, t->d_lb, t->d_ls, t->d_lc, t->d_lb64, t->d_ls64, t->d_lc64,
                     t->d_lt64, t->d_lst};
    for (void* p : dptrs)
        if (p) cudaFree(p);
    free(t->h_lb64);
    free(t->h_ls64);
    free(t->h_lc64);
    free(t->h_axes);
}

// Allocate a table, fill its node arrays; channels left to the caller.
cool_status table_alloc(const cool_table_spec& s, cool_table** out) {
    cool_table* t = new (std::nothrow) cool_table;
    if (!t) return COOL_ENOMEM;
    memset(t, 0, sizeof(*t));
    t->spec = s;
    cudaGetDevice(&t->device);
    int n[5] = {s.n_H, s.n_B, s.n_ne, s.n_Te, s.n_Tc};
    double lo[5] = {s.H_min, s.B_min, s.ne_min, s.T_min, s.T_min};
    double hi[5] = {s.H_max, s.B_max, s.ne_max, s.T_max, s.T_max};
    int na = 0, na64 = 0;
    int off64[5];
    for (int a = 0; a < 5; ++a) {
        t->dev.n[a] = n[a];
        t->dev.axis_off[a] = na;
        off64[a] = na64;
        na += 3 * n[a];
        na64 += 2 * n[a];
    }
    t->h_axes = (float*)malloc(sizeof(float) * na);
    double* h64 = (double*)malloc(sizeof(double) * na64);
    long long nls = syn_count(s);
    t->h_lb64 = (double*)malloc(sizeof(double) * s.n_Te);
    t->h_ls64 = (double*)malloc(sizeof(double) * nls);
    t->h_lc64 = (double*)malloc(sizeof(double) * s.n_Tc * s.n_Tc);
    if (!t->h_axes || !h64 || !t->h_lb64 || !t->h_ls64 || !t->h_lc64) {
        free(h64);
        free_table_memory(t);
        delete t;
        return COOL_ENOMEM;
    }
    for (int a = 0; a < 5; ++a) {
        double* x64 = h64 + off64[a];
        double* l64 = x64 + n[a];
        axis_nodes(lo[a], hi[a], n[a], x64, l64);
        float* x = t->h_axes + t->dev.axis_off[a];
        for (int j = 0; j < n[a]; ++j) {
            x[j] = (float)x64[j];
            x[n[a] + j] = (float)(1.0 / x64[j]);
            x[2 * n[a] + j] = (float)l64[j];
        }
        double dl = (log2(hi[a]) - log2(lo[a])) / (n[a] - 1);
        t->dev.dl64[a] = dl;
        t->dev.l0_64[a] = log2(lo[a]);
        t->dev.inv_dl[a] = (float)(1.0 / dl);
    }
    cudaError_t e = cudaSuccess;
    int fmt = s.dtype == COOL_F32 ? 0 : (s.row_scaled ? (s.dtype == COOL_BF16 ? 3 : 4)
                                                       : (s.dtype == COOL_BF16 ? 1 : 2));
    t->dev.fmt = fmt;
    t->dev.blk_stride = fmt == 0 ? 7 : (fmt <= 2 ? 15 : 11);
    t->dev.nblk = (s.n_Te - 1 + t->dev.blk_stride - 1) / t->dev.blk_stride;
    size_t lsb = 32 * (size_t)t->dev.nblk * (size_t)(nls / s.n_Te);
    t->ls_bytes = lsb;
    if (e == cudaSuccess) e = cudaMalloc(&t->d_axes, sizeof(float) * na);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_axes64, sizeof(double) * na64);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_lb, sizeof(float) * s.n_Te);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_ls, lsb);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_lc, sizeof(float) * s.n_Tc * s.n_Tc);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_lb64, sizeof(double) * s.n_Te);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_ls64, sizeof(double) * nls);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_lc64, sizeof(double) * s.n_Tc * s.n_Tc);
    if (e == cudaSuccess) e = cudaMemcpy(t->d_axes, t->h_axes, sizeof(float) * na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->d_axes64, h64, sizeof(double) * na64, cudaMemcpyHostToDevice);
    free(h64);
    if (e != cudaSuccess) {
        free_table_memory(t);
        delete t;
        return e == cudaErrorMemoryAllocation ? COOL_ENOMEM : set_cuda_error(e);
    }
    t->dev.axes = (const float*)t->d_axes;
    t->dev.axes64 = (const double*)t->d_axes64;
    t->dev.lb = (const float*)t->d_lb;
    t->dev.lsb = (const uint32_t*)t->d_ls;
    t->dev.lc = (const float*)t->d_lc;
    t->dev.lb64 = (const double*)t->d_lb64;
    t->dev.ls64 = (const double*)t->d_ls64;
    t->dev.lc64 = (const double*)t->d_lc64;
    t->magic = kTableMagic;
    *out = t;
    return COOL_OK;
}

// FP64 device channels -> FP32 packed device channels; FP64 host copies.
cool_status table_finish(cool_table* t, cudaStream_t st, bool copy_host) {
    const cool_table_spec& s = t->spec;
    long long nls = syn_count(s);
    struct { const void* src; void* dst; long long n; } parts[2] = {
        {t->d_lb64, t->d_lb, s.n_Te}, {t->d_lc64, t->d_lc, (long long)s.n_Tc * s.n_Tc}};
    for (auto& pt : parts) {
        long long blocks = (pt.n + 255) / 256;
        if (blocks > 8192) blocks = 8192;
        k_pack_f32<<<(int)blocks, 256, 0, st>>>((const double*)pt.src, (float*)pt.dst, pt.n);
    }
    {
        long long rows = nls / s.n_Te;
        long long total = rows * t->dev.nblk;
        long long blocks = (total + 255) / 256;
        if (blocks > 8192) blocks = 8192;
        k_pack_blocks<<<(int)blocks, 256, 0, st>>>((const double*)t->d_ls64, (uint32_t*)t->d_ls, rows, s.n_Te,
                                                   t->dev.nblk, t->dev.fmt);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && copy_host) {
        e = cudaMemcpyAsync(t->h_lb64, t->d_lb64, sizeof(double) * s.n_Te, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t->h_ls64, t->d_ls64, sizeof(double) * nls, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t->h_lc64, t->d_lc64, sizeof(double) * s.n_Tc * s.n_Tc,
                                cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

// Turn the table's persisting-L2 reservation off: persisting lines back to
// normal, and the context limit back to what it was if this table raised it.
static cool_status l2_persist_off(cool_table* t) {
    cudaError_t e = cudaSuccess;
    if (t->l2_persist) e = cudaCtxResetPersistingL2Cache();
    if (e == cudaSuccess && t->l2_raised) e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, t->l2_prev_limit);
    t->l2_persist = 0;
    t->l2_raised = 0;
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

const char kFileMagic[8] = {'C', 'O', 'O', 'L', 'T', 'A', 'B', '1'};

}  // namespace

// The paper's layout channel (COOL_PATH_QTOTAL) of an FP32 table, made once
// (synchronous): log2 Q_total in FP64 on the device from the table's FP64
// brems and synchrotron channels, then packed into FP32 blocks like the
// synchrotron channel.
cool_status table_qtotal(cool_table* t) {
    std::lock_guard<std::mutex> g(g_tex_mu);
    if (t->d_lst) return COOL_OK;
    if (t->dev.fmt != 0) return COOL_EUNSUPPORTED;
    const cool_table_spec& s = t->spec;
    const long long cnt = syn_count(s);
    double* lt = nullptr;
    void* packed = nullptr;
    cudaError_t e = cudaMalloc(&lt, sizeof(double) * cnt);
    if (e == cudaSuccess) e = cudaMalloc(&packed, t->ls_bytes);
    if (e != cudaSuccess) {
        cudaFree(lt);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? COOL_ENOMEM : set_cuda_error(e);
    }
    int off64[5], o = 0;
    for (int a = 0; a < 5; ++a) { off64[a] = o; o += 2 * t->dev.n[a]; }
    cool_status st = build_qtotal_fp64(s, (const double*)t->d_axes64, off64, (const double*)t->d_lb64,
                                       (const double*)t->d_ls64, lt, 0);
    if (st == COOL_OK) {
        const long long rows = cnt / s.n_Te;
        const long long total = rows * t->dev.nblk;
        long long blocks = (total + 255) / 256;
        if (blocks > 8192) blocks = 8192;
        k_pack_blocks<<<(int)blocks, 256>>>(lt, (uint32_t*)packed, rows, s.n_Te, t->dev.nblk, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = set_cuda_error(e);
    }
    if (st != COOL_OK) {
        cudaFree(lt);
        cudaFree(packed);
        return st;
    }
    t->d_lt64 = lt;
    t->d_lst = packed;
    t->dev.lst = (const uint32_t*)packed;
    return COOL_OK;
}

}  // namespace cool

using namespace cool;

extern "C" {

cool_status cool_release_scratch(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_cuda_error(e);
    std::lock_guard<std::mutex> g(g_list_mu);
    auto& m = list_bufs();
    for (auto it = m.begin(); it != m.end();) {
        if (it->first.first == dev) {
            if (it->second.p) cudaFree(it->second.p);
            it = m.erase(it);
        } else {
            ++it;
        }
    }
    auto& v = list_superseded();
    for (size_t k = 0; k < v.size();) {
        if (v[k].first == dev) {
            cudaFree(v[k].second);
            v[k] = v.back();
            v.pop_back();
        } else {
            ++k;
        }
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
}

const char* cool_strerror(cool_status s) {
    switch (s) {
    case COOL_OK: return "ok";
    case COOL_EINVAL: return "invalid argument";
    case COOL_ENULL: return "null pointer";
    case COOL_EALIGN: return "misaligned pointer";
    case COOL_ECUDA: return "CUDA error";
    case COOL_ENOMEM: return "out of memory";
    case COOL_ESTATE: return "invalid object state";
    case COOL_EUNSUPPORTED: return "unsupported option";
    case COOL_EIO: return "I/O error";
    }
    return "unknown status";
}

int cool_last_cuda_error(void) { return g_last_cuda_error; }

cool_status cool_table_spec_default(cool_table_spec* s) {
    if (!s) return COOL_ENULL;
    memset(s, 0, sizeof(*s));
    s->n_H = s->n_B = s->n_ne = s->n_Te = s->n_Tc = 64;
    s->H_min = 1e3; s->H_max = 1e12;
    s->B_min = 1.0; s->B_max = 1e10;
    s->ne_min = 1e2; s->ne_max = 1e25;
    s->T_min = 1e2; s->T_max = 1e15;
    s->dtype = COOL_F32;
    s->row_scaled = 0;
    s->k2_switch_T = 1e8;
    s->lnLambda = 20.0;
    s->theta_i_uses_mp = 1;
    s->compton_literal = 0;
    return COOL_OK;
}

cool_status cool_params_default(cool_params* p) {
    if (!p) return COOL_ENULL;
    memset(p, 0, sizeof(*p));
    p->rho_scale = 3e-7;
    p->M_bh_msun = 10.0;
    p->gamma_e = 5.0 / 3.0;
    p->gamma_i = 5.0 / 3.0;
    p->dt = 1e-2;
    p->n_sub = 8;
    p->mode = COOL_EXPLICIT_LIMITED;
    p->limiter_frac = 0.3;
    p->eq_band = 0.1;
    p->coulomb_clamp = 1.0;
    p->implicit_iters = 60;
    p->path = COOL_PATH_L2WINDOW;
    p->fp64_critical = 0;
    return COOL_OK;
}

cool_status cool_build_table(const cool_table_spec* spec, void* stream, cool_table** out) {
    if (!out) return COOL_ENULL;
    *out = nullptr;
    cool_status st = validate_spec(spec);
    if (st != COOL_OK) return st;
    cool_table* t = nullptr;
    st = table_alloc(*spec, &t);
    if (st != COOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int off64[5], o = 0;
    for (int a = 0; a < 5; ++a) { off64[a] = o; o += 2 * t->dev.n[a]; }
    st = build_channels_fp64(*spec, (const double*)t->d_axes64, off64, (double*)t->d_lb64,
                             (double*)t->d_ls64, (double*)t->d_lc64, s);
    if (st == COOL_OK) st = table_finish(t, s, true);
    if (st != COOL_OK) {
        t->magic = 0;
        free_table_memory(t);
        delete t;
        return st;
    }
    register_table(t);
    *out = t;
    return COOL_OK;
}

cool_status cool_table_l2_persist(cool_table* t, int on) {
    if (!t) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    if (on != 0 && on != 1) return COOL_EINVAL;
    if (!on) return l2_persist_off(t);
    if (t->l2_persist) return COOL_OK;
    int maxp = 0;
    cudaError_t e = cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, t->device);
    size_t cur = 0;
    if (e == cudaSuccess) e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    if (e != cudaSuccess) return set_cuda_error(e);
    const size_t want = t->ls_bytes < (size_t)maxp ? t->ls_bytes : (size_t)maxp;
    if (want > cur) {
        e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
        if (e != cudaSuccess) return set_cuda_error(e);
        t->l2_raised = 1;
        t->l2_prev_limit = cur;
    }
    t->l2_persist = 1;
    return COOL_OK;
}

cool_status cool_table_free(cool_table* t) {
    if (!t) return COOL_OK;
    if (!unregister_table(t)) return COOL_ESTATE;
    l2_persist_off(t);   // best effort: the table goes regardless
    t->magic = 0;
    free_table_memory(t);
    delete t;
    return COOL_OK;
}

cool_status cool_table_get_spec(const cool_table* t, cool_table_spec* spec) {
    if (!t || !spec) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    *spec = t->spec;
    return COOL_OK;
}

cool_status cool_table_export(const cool_table* t, int channel, double* host_out, long long count) {
    if (!t || !host_out) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    const double* src;
    long long n;
    switch (channel) {
    case 0: src = t->h_lb64; n = t->spec.n_Te; break;
    case 1: src = t->h_ls64; n = syn_count(t->spec); break;
    case 2: src = t->h_lc64; n = (long long)t->spec.n_Tc * t->spec.n_Tc; break;
    case 3: {
        // the paper's layout (made on first use), copied from the device
        n = syn_count(t->spec);
        if (count != n) return COOL_EINVAL;
        cool_status st = table_qtotal(const_cast<cool_table*>(t));
        if (st != COOL_OK) return st;
        cudaError_t e = cudaMemcpy(host_out, t->d_lt64, sizeof(double) * n, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? COOL_OK : set_cuda_error(e);
    }
    default: return COOL_EINVAL;
    }
    if (count != n) return COOL_EINVAL;
    memcpy(host_out, src, sizeof(double) * n);
    return COOL_OK;
}

cool_status cool_table_export_packed(const cool_table* t, void* host_out, long long bytes) {
    if (!t || !host_out) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    if (bytes != (long long)t->ls_bytes) return COOL_EINVAL;
    cudaError_t e = cudaMemcpy(host_out, t->d_ls, t->ls_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e);
    return COOL_OK;
}

cool_status cool_table_packed_bytes(const cool_table* t, long long* bytes) {
    if (!t || !bytes) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    *bytes = (long long)t->ls_bytes;
    return COOL_OK;
}

cool_status cool_table_nodes(const cool_table* t, int axis, float* host_out, int n) {
    if (!t || !host_out) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    if (axis < 0 || axis > 4 || n != t->dev.n[axis]) return COOL_EINVAL;
    memcpy(host_out, t->h_axes + t->dev.axis_off[axis], sizeof(float) * n);
    return COOL_OK;
}

cool_status cool_table_save(const cool_table* t, const char* path) {
    if (!t || !path) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    FILE* f = fopen(path, "wb");
    if (!f) return COOL_EIO;
    const cool_table_spec& s = t->spec;
    long long n[3] = {s.n_Te, syn_count(s), (long long)s.n_Tc * s.n_Tc};
    const double* d[3] = {t->h_lb64, t->h_ls64, t->h_lc64};
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(&s, sizeof(s), h);
    for (int c = 0; c < 3; ++c) h = fnv1a(d[c], sizeof(double) * n[c], h);
    uint32_t ver = 1, sz = (uint32_t)sizeof(s);
    bool ok = fwrite(kFileMagic, 1, 8, f) == 8 && fwrite(&ver, 4, 1, f) == 1 && fwrite(&sz, 4, 1, f) == 1 &&
              fwrite(&s, sizeof(s), 1, f) == 1;
    for (int c = 0; c < 3 && ok; ++c) ok = fwrite(d[c], sizeof(double), n[c], f) == (size_t)n[c];
    ok = ok && fwrite(&h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? COOL_OK : COOL_EIO;
}

cool_status cool_table_load(const char* path, void* stream, cool_table** out) {
    if (!path || !out) return COOL_ENULL;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return COOL_EIO;
    char magic[8];
    uint32_t ver = 0, sz = 0;
    cool_table_spec s;
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kFileMagic, 8) != 0 || fread(&ver, 4, 1, f) != 1 ||
        ver != 1 || fread(&sz, 4, 1, f) != 1 || sz != sizeof(s) || fread(&s, sizeof(s), 1, f) != 1) {
        fclose(f);
        return COOL_EIO;
    }
    cool_status st = validate_spec(&s);
    if (st != COOL_OK) { fclose(f); return COOL_EIO; }
    cool_table* t = nullptr;
    st = table_alloc(s, &t);
    if (st != COOL_OK) { fclose(f); return st; }
    long long n[3] = {s.n_Te, syn_count(s), (long long)s.n_Tc * s.n_Tc};
    double* d[3] = {t->h_lb64, t->h_ls64, t->h_lc64};
    bool ok = true;
    for (int c = 0; c < 3 && ok; ++c) ok = fread(d[c], sizeof(double), n[c], f) == (size_t)n[c];
    uint64_t hf = 0;
    ok = ok && fread(&hf, 8, 1, f) == 1;
    fclose(f);
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(&s, sizeof(s), h);
    for (int c = 0; c < 3 && ok; ++c) h = fnv1a(d[c], sizeof(double) * n[c], h);
    if (!ok || h != hf) {
        t->magic = 0;
        free_table_memory(t);
        delete t;
        return COOL_EIO;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    void* dd[3] = {t->d_lb64, t->d_ls64, t->d_lc64};
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(dd[c], d[c], sizeof(double) * n[c], cudaMemcpyHostToDevice, cs);
    st = e == cudaSuccess ? table_finish(t, cs, false) : set_cuda_error(e);
    if (st != COOL_OK) {
        t->magic = 0;
        free_table_memory(t);
        delete t;
        return st;
    }
    register_table(t);
    *out = t;
    return COOL_OK;
}

cool_status cool_step(const cool_table* t, const cool_params* p, long long n_cells, cool_dtype field_dtype,
                      const void* rho, const void* B, const void* H, const void* u_e_in, const void* u_i_in,
                      void* u_e_out, void* u_i_out, void* q_cool_out, void* q_cc_out,
                      cool_counters* counters, void* stream) {
    if (!t || !p) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    cool_status st = validate_params(p);
    if (st != COOL_OK) return st;
    if (n_cells < 0) return COOL_EINVAL;
    if (field_dtype != COOL_F32 && field_dtype != COOL_F64) return COOL_EUNSUPPORTED;
    if (n_cells == 0) return COOL_OK;
    if (!rho || !B || !H || !u_e_in || !u_i_in || !u_e_out || !u_i_out) return COOL_ENULL;
    size_t esz = field_dtype == COOL_F32 ? 4 : 8;
    const void* ptrs[] = {rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, q_cool_out, q_cc_out};
    for (const void* q : ptrs)
        if ((uintptr_t)q % esz != 0) return COOL_EALIGN;
    if ((uintptr_t)counters % 8 != 0) return COOL_EALIGN;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return COOL_ESTATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->path == COOL_PATH_TMA_SMEM) {
        if (field_dtype != COOL_F32) return COOL_EUNSUPPORTED;
        return launch_step_tma(t, p, n_cells, (const float*)rho, (const float*)B, (const float*)H,
                               (const float*)u_e_in, (const float*)u_i_in, (float*)u_e_out, (float*)u_i_out,
                               (float*)q_cool_out, (float*)q_cc_out, counters, s);
    }
    if (p->path == COOL_PATH_TEXTURE_POINT || p->path == COOL_PATH_TEXTURE_HWLERP) {
        if (field_dtype != COOL_F32 || t->spec.dtype != COOL_F32) return COOL_EUNSUPPORTED;
        st = table_textures(const_cast<cool_table*>(t));
        if (st != COOL_OK) return st;
        return launch_step_tex(t, p, n_cells, (const float*)rho, (const float*)B, (const float*)H,
                               (const float*)u_e_in, (const float*)u_i_in, (float*)u_e_out, (float*)u_i_out,
                               (float*)q_cool_out, (float*)q_cc_out, counters, s);
    }
    if (p->path == COOL_PATH_QTOTAL) {
        if (field_dtype != COOL_F32 || t->spec.dtype != COOL_F32) return COOL_EUNSUPPORTED;
        st = table_qtotal(const_cast<cool_table*>(t));
        if (st != COOL_OK) return st;
    }
    if (field_dtype == COOL_F32)
        return launch_step_f32(t, p, n_cells, (const float*)rho, (const float*)B, (const float*)H,
                               (const float*)u_e_in, (const float*)u_i_in, (float*)u_e_out,
                               (float*)u_i_out, (float*)q_cool_out, (float*)q_cc_out, counters, s);
    return launch_step_f64(t, p, n_cells, (const double*)rho, (const double*)B, (const double*)H,
                           (const double*)u_e_in, (const double*)u_i_in, (double*)u_e_out,
                           (double*)u_i_out, (double*)q_cool_out, (double*)q_cc_out, counters, s);
}

}  // extern "C"

namespace cool {
namespace {
// Two copy/compute streams per device for the host-buffer step (created once).
constexpr int kMaxDevices = 64;
cudaStream_t g_pipe[kMaxDevices][2];
std::mutex g_pipe_mu;

cool_status pipe_streams(int dev, cudaStream_t (&out)[2]) {
    if (dev < 0 || dev >= kMaxDevices) return COOL_EUNSUPPORTED;
    std::lock_guard<std::mutex> g(g_pipe_mu);
    for (int k = 0; k < 2; ++k) {
        if (!g_pipe[dev][k]) {
            cudaError_t e = cudaStreamCreateWithFlags(&g_pipe[dev][k], cudaStreamNonBlocking);
            if (e != cudaSuccess) return set_cuda_error(e);
        }
        out[k] = g_pipe[dev][k];
    }
    return COOL_OK;
}
}  // namespace
}  // namespace cool

extern "C" {

cool_status cool_step_host(const cool_table* t, const cool_params* p, long long n_cells, const float* rho,
                           const float* B, const float* H, const float* u_e_in, const float* u_i_in,
                           float* u_e_out, float* u_i_out, long long chunk_cells, cool_counters* counters,
                           void* stream) {
    if (!t || !p) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    cool_status st = validate_params(p);
    if (st != COOL_OK) return st;
    if (p->path != COOL_PATH_L2WINDOW) return COOL_EUNSUPPORTED;
    if (n_cells < 0 || chunk_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    if (!rho || !B || !H || !u_e_in || !u_i_in || !u_e_out || !u_i_out) return COOL_ENULL;
    if ((uintptr_t)counters % 8 != 0) return COOL_EALIGN;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return COOL_ESTATE;
    cudaStream_t ps[2];
    st = pipe_streams(dev, ps);
    if (st != COOL_OK) return st;
    // chunks: a multiple of 128 cells (every staged array stays 16-byte
    // aligned); by default 12 of them: fewer expose more of the pipeline's
    // fill (the first chunk's copies in) and drain (the last chunk's step and
    // copies out), more pay more per-chunk costs (measured on 16.8 M cells:
    // 8 chunks 7.80 ms, 12 7.67 ms, 32 8.20 ms per step)
    long long chunk = chunk_cells > 0 ? chunk_cells : (n_cells + 11) / 12;
    if (chunk < (1 << 16)) chunk = 1 << 16;
    chunk = (chunk + 127) / 128 * 128;
    if (chunk > n_cells) chunk = (n_cells + 127) / 128 * 128;
    const long long nchunks = (n_cells + chunk - 1) / chunk;
    cudaStream_t cs = (cudaStream_t)stream;
    // staging: two sets (one per stream) of 7 arrays of `chunk` floats
    float* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, sizeof(float) * 14 * (size_t)chunk, cs);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? COOL_ENOMEM : set_cuda_error(e);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], cs);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ps[k], ev[0], 0);
    const float* in[5] = {rho, B, H, u_e_in, u_i_in};
    float* out[2] = {u_e_out, u_i_out};
    for (long long c = 0; c < nchunks && e == cudaSuccess && st == COOL_OK; ++c) {
        const int k = (int)(c & 1);
        float* d = buf + (size_t)k * 7 * chunk;
        const long long first = c * chunk;
        const long long m = n_cells - first < chunk ? n_cells - first : chunk;
        for (int a = 0; a < 5 && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(d + (size_t)a * chunk, in[a] + first, sizeof(float) * m, cudaMemcpyHostToDevice,
                                ps[k]);
        if (e != cudaSuccess) break;
        st = launch_step_f32(t, p, m, d, d + chunk, d + 2 * chunk, d + 3 * chunk, d + 4 * chunk, d + 5 * chunk,
                             d + 6 * chunk, nullptr, nullptr, counters, ps[k]);
        for (int a = 0; a < 2 && e == cudaSuccess && st == COOL_OK; ++a)
            e = cudaMemcpyAsync(out[a] + first, d + (size_t)(5 + a) * chunk, sizeof(float) * m,
                                cudaMemcpyDeviceToHost, ps[k]);
    }
    // the caller's stream continues after both pipeline streams, then frees
    cudaError_t e2 = cudaSuccess;
    for (int k = 0; k < 2; ++k) {
        if (ev[1 + k]) {
            cudaError_t a = cudaEventRecord(ev[1 + k], ps[k]);
            if (a == cudaSuccess) a = cudaStreamWaitEvent(cs, ev[1 + k], 0);
            if (a != cudaSuccess) e2 = a;
        }
    }
    cudaFreeAsync(buf, cs);
    for (int k = 0; k < 3; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (st != COOL_OK) return st;
    if (e2 != cudaSuccess) return set_cuda_error(e2);
    return COOL_OK;
}

cool_status cool_step_disk(const cool_table* t, const cool_params* p, const cool_disk* disk, long long n_cells,
                           const float* rho, const float* B, const float* H, const float* u_e_in,
                           const float* u_i_in, const float* r, float* u_e_out, float* u_i_out,
                           float* q_cool_out, float* q_cc_out, cool_counters* counters, void* stream) {
    if (!t || !p || !disk) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    cool_status st = validate_params(p);
    if (st != COOL_OK) return st;
    if (p->path != COOL_PATH_L2WINDOW || t->spec.dtype != COOL_F32) return COOL_EUNSUPPORTED;
    if (!isfinite(disk->spin) || !(disk->h_floor >= 0.0) || !isfinite(disk->h_floor) ||
        (disk->h_from_state != 0 && disk->h_from_state != 1))
        return COOL_EINVAL;
    if (n_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    if (!rho || !B || !u_e_in || !u_i_in || !r || !u_e_out || !u_i_out) return COOL_ENULL;
    if (!H && !disk->h_from_state) return COOL_ENULL;
    const float* Hs = H ? H : r;   // with h_from_state the H values are not used
    const void* ptrs[] = {rho, B, Hs, u_e_in, u_i_in, r, u_e_out, u_i_out, q_cool_out, q_cc_out};
    for (const void* q : ptrs)
        if ((uintptr_t)q % 4 != 0) return COOL_EALIGN;
    if ((uintptr_t)counters % 8 != 0) return COOL_EALIGN;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return COOL_ESTATE;
    return launch_step_f32(t, p, n_cells, rho, B, Hs, u_e_in, u_i_in, u_e_out, u_i_out, q_cool_out, q_cc_out,
                           counters, (cudaStream_t)stream, disk, r);
}

cool_status cool_step_direct(const cool_table_spec* physics, const cool_params* p, long long n_cells,
                             const double* rho, const double* B, const double* H, const double* u_e_in,
                             const double* u_i_in, double* u_e_out, double* u_i_out, double* q_cool_out,
                             double* q_cc_out, cool_counters* counters, void* stream) {
    if (!physics || !p) return COOL_ENULL;
    cool_status st = validate_params(p);
    if (st != COOL_OK) return st;
    if (p->path != COOL_PATH_L2WINDOW || p->fp64_critical) return COOL_EUNSUPPORTED;
    if (!(physics->k2_switch_T > 0.0) || !(physics->lnLambda > 0.0) ||
        (physics->theta_i_uses_mp != 0 && physics->theta_i_uses_mp != 1) ||
        (physics->compton_literal != 0 && physics->compton_literal != 1))
        return COOL_EINVAL;
    if (n_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    if (!rho || !B || !H || !u_e_in || !u_i_in || !u_e_out || !u_i_out) return COOL_ENULL;
    const void* ptrs[] = {rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, q_cool_out, q_cc_out};
    for (const void* q : ptrs)
        if ((uintptr_t)q % 8 != 0) return COOL_EALIGN;
    if ((uintptr_t)counters % 8 != 0) return COOL_EALIGN;
    return launch_step_direct(*physics, p, n_cells, rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, q_cool_out,
                              q_cc_out, counters, (cudaStream_t)stream);
}

cool_status cool_step_bwd(const cool_table* t, const cool_params* p, long long n_cells, const float* rho,
                          const float* B, const float* H, const float* u_e_in, const float* u_i_in,
                          const float* g_u_e_out, const float* g_u_i_out, float* g_rho, float* g_B, float* g_H,
                          float* g_u_e_in, float* g_u_i_in, float* g_lb, float* g_ls, float* g_lc, void* stream) {
    if (!t || !p) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    cool_status st = validate_params(p);
    if (st != COOL_OK) return st;
    if (p->path != COOL_PATH_L2WINDOW) return COOL_EUNSUPPORTED;
    if (n_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    const void* req[] = {rho, B, H, u_e_in, u_i_in, g_u_e_out, g_u_i_out, g_rho, g_B, g_H, g_u_e_in, g_u_i_in};
    for (const void* q : req)
        if (!q) return COOL_ENULL;
    for (const void* q : req)
        if ((uintptr_t)q % 4 != 0) return COOL_EALIGN;
    const void* opt[] = {g_lb, g_ls, g_lc};
    for (const void* q : opt)
        if ((uintptr_t)q % 4 != 0) return COOL_EALIGN;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return COOL_ESTATE;
    return launch_step_bwd_f32(t, p, n_cells, rho, B, H, u_e_in, u_i_in, g_u_e_out, g_u_i_out, g_rho, g_B, g_H,
                               g_u_e_in, g_u_i_in, g_lb, g_ls, g_lc, (cudaStream_t)stream);
}

cool_status cool_step_fwd_jac(const cool_table* t, const cool_params* p, long long n_cells, const float* rho,
                              const float* B, const float* H, const float* u_e_in, const float* u_i_in,
                              float* u_e_out, float* u_i_out, float* jac, void* stream) {
    if (!t || !p) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    cool_status st = validate_params(p);
    if (st != COOL_OK) return st;
    if (p->path != COOL_PATH_L2WINDOW) return COOL_EUNSUPPORTED;
    if (n_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    const void* req[] = {rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, jac};
    for (const void* q : req)
        if (!q) return COOL_ENULL;
    for (const void* q : req)
        if ((uintptr_t)q % 4 != 0) return COOL_EALIGN;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return COOL_ESTATE;
    return launch_step_fwd_jac_f32(t, p, n_cells, rho, B, H, u_e_in, u_i_in, u_e_out, u_i_out, jac,
                                   (cudaStream_t)stream);
}

cool_status cool_step_bwd_jac(long long n_cells, const float* jac, const float* g_u_e_out, const float* g_u_i_out,
                              float* g_rho, float* g_B, float* g_H, float* g_u_e_in, float* g_u_i_in, void* stream) {
    if (n_cells < 0) return COOL_EINVAL;
    if (n_cells == 0) return COOL_OK;
    const void* req[] = {jac, g_u_e_out, g_u_i_out, g_rho, g_B, g_H, g_u_e_in, g_u_i_in};
    for (const void* q : req)
        if (!q) return COOL_ENULL;
    for (const void* q : req)
        if ((uintptr_t)q % 4 != 0) return COOL_EALIGN;
    return launch_jac_contract_f32(n_cells, jac, g_u_e_out, g_u_i_out, g_rho, g_B, g_H, g_u_e_in, g_u_i_in,
                                   (cudaStream_t)stream);
}

cool_status cool_debug_lookup(const cool_table* t, int axis, long long n, const float* keys, int* idx,
                              float* w, void* stream) {
    if (!t) return COOL_ENULL;
    if (!table_ok(t)) return COOL_ESTATE;
    if (axis < 0 || axis > 9 || n < 0) return COOL_EINVAL;
    if (n == 0) return COOL_OK;
    if (!keys || !idx || !w) return COOL_ENULL;
    return launch_debug_lookup(t, axis, n, keys, idx, w, (cudaStream_t)stream);
}

}  // extern "C"
