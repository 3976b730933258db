// Internal definitions shared by the MDC library's translation units.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/mdc.h"

namespace mdc {

// ------------------------------------------------------------------ small helpers
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Dynamic shared-memory limit of one kernel, raised once per device.  The attribute belongs to the
// device that is current when it is set, so a process driving several devices sets it on each; only
// a successful call is remembered, and concurrent first calls are serialised.  A failure leaves the
// error for the launch that follows (which then fails and is reported by the caller).
struct SmemLimit {
    std::atomic<uint64_t> done{0};
    std::mutex m;
    template <typename F> void ensure(F* func, int bytes) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0;
        if (bit && (done.load(std::memory_order_acquire) & bit)) return;
        std::lock_guard<std::mutex> g(m);
        if (bit && (done.load(std::memory_order_acquire) & bit)) return;
        if (cudaFuncSetAttribute(reinterpret_cast<const void*>(func), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes) == cudaSuccess)
            done.fetch_or(bit, std::memory_order_release);
    }
};

// Bounds checks of the debug build (compiled with MDC_CHECK_BOUNDS into a library of its own):
// every instrumented global access checks that elements [off, off + span) lie inside its buffer of
// n elements.  A miss records MDC_BOUNDS_CODE + site in the handle's error flag (the first miss
// wins; mdc_device_status then reports MDC_ERR_BOUNDS) and the access goes to a small dummy buffer
// instead, so nothing outside any buffer is read or written.  Release builds expand MDC_AT to the
// plain pointer arithmetic.
constexpr int MDC_BOUNDS_CODE = 1000;
#ifdef MDC_CHECK_BOUNDS
static __device__ __align__(16) unsigned char mdc_bounds_dummy[64];
template <typename T>
__device__ __forceinline__ T* mdc_checked(T* p, long long off, long long span, long long n, int* err, int site) {
    if (p != nullptr && off >= 0 && off + span <= n) return p + off;
    if (err) atomicCAS(err, 0, MDC_BOUNDS_CODE + site);
    return reinterpret_cast<T*>(mdc_bounds_dummy);
}
#define MDC_AT(p, off, span, n, err, site) \
    mdc::mdc_checked((p), (long long)(off), (long long)(span), (long long)(n), (err), (site))
// Guard form for accesses kept verbatim: `if (MDC_INB(...)) access;` (a miss is recorded and the
// access skipped); release builds reduce the guard to the constant true.
__device__ __forceinline__ bool mdc_ok(long long off, long long span, long long n, int* err, int site) {
    if (off >= 0 && off + span <= n) return true;
    if (err) atomicCAS(err, 0, MDC_BOUNDS_CODE + site);
    return false;
}
#define MDC_INB(off, span, n, err, site) \
    mdc::mdc_ok((long long)(off), (long long)(span), (long long)(n), (err), (site))
#else
#define MDC_AT(p, off, span, n, err, site) ((p) + (off))
#define MDC_INB(off, span, n, err, site) true
#endif
// Status of a device error flag value: 0, a bounded wait that gave up, or a bounds miss.
inline int device_flag_status(int v) {
    return v == 0 ? MDC_OK : (v >= MDC_BOUNDS_CODE ? MDC_ERR_BOUNDS : MDC_ERR_TIMEOUT);
}

inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// A scalar coefficient used by fused epilogues: value = h * (*d) when d is set, else h.
struct Coef {
    float h;
    const double* d;
};
__device__ inline float coef(Coef c) { return c.d ? (float)((double)c.h * (*c.d)) : c.h; }
inline Coef C1(float v) { return Coef{v, nullptr}; }
inline Coef CD(float v, const double* d) { return Coef{v, d}; }

// Pad of the kernel's row pitch (complex elements) so every row starts 512-byte aligned
// in complex64 storage and whole 16-byte vectors never straddle a row end.
constexpr int G_PITCH_ALIGN = 64;

// ------------------------------------------------------------------ plan
struct EventPair { cudaEvent_t a, b; };

// Product variant chosen by the autotuner for column counts up to `ncol`.
// PATH_GEMV_GROUPS: GEMV passes over groups of up to 4 columns (one kernel read per group)
enum ProductPath { PATH_AUTO = 0, PATH_GEMV = 1, PATH_SIMT = 2, PATH_TC = 3, PATH_GEMV_GROUPS = 4 };
struct ProductChoice {
    int ncol;
    int path;
    int bn;     // tensor-core column tile (PATH_TC)
};

struct TimingState {
    bool on = false;
    std::vector<EventPair> pool;
    std::vector<int> used_class;   // class of each used pair
    size_t used = 0;
    int64_t launches[MDC_KC_COUNT] = {};
    int64_t recorded[MDC_KC_COUNT] = {};
};

}  // namespace mdc

struct mdc_plan {
    int nf, nr, ns, nt, logn;
    // Frequency shard: this handle holds bins k0 .. k0 + nf - 1 of the nt-point transform (k0 = 0
    // and no hook for an ordinary handle).  With a reduction hook every inverse transform writes
    // its partial signal to red_buf, the hook sums it over all shards, and the epilogue runs on
    // the sum.
    int k0 = 0;
    bool shard = false;
    mdc_allreduce_fn red_fn = nullptr;
    void* red_ctx = nullptr;
    float* red_buf = nullptr;
    int64_t red_cap = 0;        // floats in red_buf
    int host_error = 0;         // first failure inside a pass (allocation, hook), taken by the entry point
    double dt, dr;
    int storage;
    int64_t ldg;                // row pitch of the kernel copy, in complex elements
    void* G = nullptr;          // library-owned kernel [nf][nr][ldg] in `storage` format
    float* gscale = nullptr;    // [nf][nr] per-row scales (reduced storage), else null
    float2* tw = nullptr;       // [nt/2] e^{-2 pi i j/nt}, then [nt/2] e^{-2 pi i m/(nt/2)} and [nt/2] its
                                // conjugate (half-length transforms), from host float64
    // scratch spectra, sized for nv_cap columns
    int nv_cap = 0;
    float2* specA = nullptr;    // [nf][max(nr,ns)][nv_cap]
    float2* specB = nullptr;
    // tensor-core path (FP16/BF16 storage): prepared B operand and its column scales
    void* tcB = nullptr;        // [nf][rows_pad][max(2*ldg, nr8)] 16-bit
    float* tcSigma = nullptr;   // [nf][tc_cap]
    int tc_cap = 0;
    int* err_flag = nullptr;    // device int: non-zero after a bounded device wait gave up
    unsigned long long wait_ns = 2000000000ull;   // bound on each tensor-core pipeline wait
    int64_t tc_fallbacks = 0;   // products the tensor-core rule chose that ran on another path
    bool force_tc = false;      // FP16/BF16: tensor-core products for every column count
    bool graphs = false;        // capture repeated solves into CUDA graphs (mdc_set_option)
    std::vector<mdc::ProductChoice> tune[2];   // autotuned variants [forward, adjoint], ascending ncol
    std::vector<void*> graph_cache;   // solver workspaces with their instantiated graphs
    cudaStream_t graph_stream = nullptr;   // private stream for capture and replay
    cudaEvent_t graph_ev[2] = {nullptr, nullptr};
    void (*graph_free)(void*) = nullptr;
    int64_t launch_count = 0;
    mdc::TimingState timing;
};

namespace mdc {

// ------------------------------------------------------------------ launch bookkeeping
struct LaunchScope {
    mdc_plan* p; cudaStream_t s; int cls; EventPair* ev = nullptr;
    LaunchScope(mdc_plan* p_, cudaStream_t s_, int cls_);
    ~LaunchScope();
};

// ------------------------------------------------------------------ kernels (launchers)
struct RfftArgs {
    const float* x;        // [nt][C]
    const float* x2;       // optional second input added to x (same layout), or null
    int C, S, nv;          // C = S * nv real columns
    int nt, logn, nf;
    int k0;                // first bin kept: X[j] holds bin k0 + j, j < nf (a frequency slab)
    const int* cut;        // Theta cut-offs [C] applied to the input, or null
    Coef scale;            // multiplies the input
    int conj;              // conjugate the output spectrum (time reversal of the input)
    float2* X;             // [nf][S][ldv]
    int ldv, voff;
    const float2* tw;
    const int* active;     // if non-null and *active == 0 the kernel does nothing
    int vec4;              // set by the launcher: x (and x2) 16-byte aligned rows, C % 4 == 0
    int* err;              // set by the launcher: the plan's device error flag (bounds checks)
};
struct IrfftArgs {
    const float2* Y;       // [nf][S][ldv]
    int ldv, voff;
    int C, S, nv, nt, logn, nf;
    int k0;                // Y[j] holds bin k0 + j (j < nf); every other bin is zero
    int conj_in;           // conjugate the input spectrum before the inverse transform
    float scale;           // multiplies the inverse transform (1/nt and dt*dr folded in)
    float* out;            // [nt][C]
    // epilogue: out = a_mdc * Theta * ifft + a_base * base + a_prev * out_old
    Coef a_mdc, a_base, a_prev;
    const float* base;
    const int* cut;        // Theta on the transform term, or null
    int reverse_out;       // write at (-t) mod nt
    double* colsum;        // per-column sum of squares of out, or null
    const float2* tw;
    const int* active;
    int vec4;              // set by the launcher: aligned 4-column output path
    // An LSQR step applied with the previous output v = out (before it is overwritten), same layout:
    //   xw_x <- xw_x + kx * xw_w,   xw_w <- ia * v + kw * xw_w     (kx, kw, ia: device doubles)
    // xw_w null: no step.  Needs the previous-output term and no time reversal.
    float* xw_x;
    float* xw_w;
    const double* xw_kx;
    const double* xw_kw;
    const double* xw_ia;
    // The forward transform of the final output (times the window fwd_cut if set, unscaled,
    // conjugated if fwd_conj) into the spectrum fwd_X [nf][S][ldv] at column offset fwd_voff: fused
    // into the kernel's epilogue where its tile holds the whole output, else launched after it.
    // fwd_X null: none.
    float2* fwd_X;
    const int* fwd_cut;
    int fwd_conj, fwd_voff;
    int* err;              // set by the launcher: the plan's device error flag (bounds checks)
};
void launch_rfft(mdc_plan* p, const RfftArgs& a, cudaStream_t s);
// The inverse transform; on a frequency shard with a reduction hook: the partial transform, the
// hook's sum over shards, then the epilogue (failures go to p->host_error).
void launch_irfft(mdc_plan* p, const IrfftArgs& a, cudaStream_t s);
// Status of the plan's last failure inside a pass (MDC_OK if none), cleared.
inline int take_host_error(mdc_plan* p) {
    const int e = p->host_error;
    p->host_error = 0;
    return e;
}

// Per-frequency products on the library layout.
//   forward: Y[k][r][voff_o + j] = sum_s G[k][r][s] X[k][s][voff_i + j], j < ncol
//   adjoint: X[k][s][voff_o + j] = sum_r conj(G[k][r][s]) Y[k][r][voff_i + j]
void launch_product(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i,
                    float2* out, int ldo, int voff_o, int ncol, cudaStream_t s,
                    const int* active);

// Tensor-core products (tc_gemm.cu).
bool tc_supported(const mdc_plan* p, int ncol);
// scoped: time the B-operand preparation (MDC_KC_TC_PREP) and the GEMM (product class) separately
bool launch_tc_product(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                       int voff_o, int ncol, cudaStream_t s, const int* active, int bn_override = 0,
                       bool scoped = false);
// One product with an explicit variant (autotuner); returns false if the variant cannot run.
bool launch_product_variant(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i, float2* out,
                            int ldo, int voff_o, int ncol, cudaStream_t s, int path, int bn);
size_t tc_scratch_elems(const mdc_plan* p, int ncol);

// Quantise a complex64 kernel [nf][nr][ns] into the plan's reduced-storage copy and row scales.
void launch_quantize(mdc_plan* p, const float2* G, const float* w, cudaStream_t s);
void launch_quantize_rows(mdc_plan* p, const float2* G, const float* w, int64_t row0, int64_t nrows, cudaStream_t s);

// Bytes of one stored complex value (MDC_C32S: 4 in each of its two planes).
inline int storage_bytes(int storage) {
    return (storage == MDC_C64 || storage == MDC_C32S) ? 8 : (storage == MDC_CE4M3 ? 2 : 4);
}
// Storage the tensor-core path can consume: 16-bit halves, or E4M3 bytes that the GEMM widens to
// FP16 in shared memory.
inline bool storage_tc(int storage) {
    return storage == MDC_C16F || storage == MDC_CBF16 || storage == MDC_C32S || storage == MDC_CE4M3;
}

void set_cuda_error(cudaError_t e);

}  // namespace mdc
