// C ABI: plan construction, MDC forward/adjoint (Eq. 3), instrumentation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace mdc {

static thread_local int g_last_cuda_error = 0;
void set_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

// NVTX range names of the kernel classes (host ranges around each launch; free without a tool)
static const char* const kClassRange[MDC_KC_COUNT] = {"mdc rfft", "mdc product forward", "mdc product adjoint",
                                                      "mdc irfft", "mdc solver", "mdc tensor-core operand"};

LaunchScope::LaunchScope(mdc_plan* p_, cudaStream_t s_, int cls_) : p(p_), s(s_), cls(cls_) {
    nvtxRangePushA(kClassRange[cls]);
    p->launch_count++;
    p->timing.launches[cls]++;
    if (p->timing.on && p->timing.used < p->timing.pool.size()) {
        ev = &p->timing.pool[p->timing.used];
        p->timing.used_class[p->timing.used] = cls;
        p->timing.recorded[cls]++;
        p->timing.used++;
        cudaEventRecord(ev->a, s);
    }
}
LaunchScope::~LaunchScope() {
    if (ev) cudaEventRecord(ev->b, s);
    nvtxRangePop();
}

int ensure_scratch(mdc_plan* p, int ncols);

}  // namespace mdc

using namespace mdc;

#define MDC_CUDA_TRY(expr)                              \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) {                        \
            set_cuda_error(_e);                         \
            return _e == cudaErrorMemoryAllocation ? MDC_ERR_OOM : MDC_ERR_CUDA; \
        }                                               \
    } while (0)

static bool valid_nt(int nt) { return nt >= 64 && nt <= 4096 && (nt & (nt - 1)) == 0; }

extern "C" int64_t mdc_kernel_bytes(int nfmax, int nr, int ns, int storage) {
    if (nfmax < 1 || nr < 1 || ns < 1) return -1;
    const int64_t ldg = round_up(ns, G_PITCH_ALIGN);
    const int64_t n = (int64_t)nfmax * nr * ldg;
    switch (storage) {
        case MDC_C64: return n * 8;
        case MDC_C16F:
        case MDC_CBF16: return n * 4 + (int64_t)nfmax * nr * 4;
        case MDC_CE4M3: return n * 2 + (int64_t)nfmax * nr * 4;
        case MDC_C32S: return n * 8 + (int64_t)nfmax * nr * 4;
        default: return -1;
    }
}

extern "C" const char* mdc_strerror(int status) {
    switch (status) {
        case MDC_OK: return "ok";
        case MDC_ERR_ARG: return "invalid argument";
        case MDC_ERR_OOM: return "device allocation failed";
        case MDC_ERR_CUDA: return "CUDA runtime error";
        case MDC_ERR_TIMEOUT: return "bounded device wait timed out";
        case MDC_ERR_NUMERIC: return "non-finite value in solver recurrence";
        case MDC_ERR_BUDGET: return "request exceeds memory budget";
        case MDC_ERR_STATE: return "call not valid in current state";
        case MDC_ERR_BOUNDS: return "kernel index outside its buffer (debug build)";
        default: return "unknown status";
    }
}

extern "C" int mdc_last_cuda_error(void) { return g_last_cuda_error; }

static void free_plan(mdc_plan* p) {
    if (!p) return;
    if (p->graph_free)
        for (void* g : p->graph_cache) p->graph_free(g);
    if (p->graph_stream) cudaStreamDestroy(p->graph_stream);
    for (cudaEvent_t e : p->graph_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(p->G);
    cudaFree(p->gscale);
    cudaFree(p->tw);
    cudaFree(p->specA);
    cudaFree(p->specB);
    cudaFree(p->tcB);
    cudaFree(p->tcSigma);
    cudaFree(p->err_flag);
    cudaFree(p->red_buf);
    for (auto& e : p->timing.pool) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete p;
}

// Column weights (receiver integration areas) multiply the library's copy of the kernel.
__global__ void scale_columns(float2* __restrict__ G, int ns, size_t ldg, const float* __restrict__ w) {
    float2* g = G + (size_t)blockIdx.x * ldg;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const float2 v = g[s];
        g[s] = make_float2(v.x * w[s], v.y * w[s]);
    }
}

static int create_plan(mdc_handle* out, const void* G, const double* weights, int nfmax, int nr, int ns, int nt,
                       double dt, double dr, int storage, void* stream, int k0 = 0, bool shard = false) {
    if (!out) return MDC_ERR_ARG;
    *out = nullptr;
    // G == nullptr: an empty (zero) kernel copy, filled later by mdc_load_slab
    if (nr < 1 || ns < 1 || !valid_nt(nt) || nfmax < 1 || k0 < 0 || k0 + nfmax > nt / 2 + 1) return MDC_ERR_ARG;
    if (!(dt > 0.0) || !(dr > 0.0) || !std::isfinite(dt) || !std::isfinite(dr)) return MDC_ERR_ARG;
    if (storage < MDC_C64 || storage > MDC_C32S) return MDC_ERR_ARG;
    if ((int64_t)nr * nfmax > (int64_t)1 << 31) return MDC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    mdc_plan* p = new (std::nothrow) mdc_plan();
    if (!p) return MDC_ERR_OOM;
    p->nf = nfmax; p->nr = nr; p->ns = ns; p->nt = nt; p->logn = ilog2(nt);
    p->k0 = k0; p->shard = shard;
    p->dt = dt; p->dr = dr; p->storage = storage;
    p->ldg = round_up(ns, G_PITCH_ALIGN);
    const size_t rowbytes = (size_t)p->ldg * storage_bytes(storage);
    cudaError_t e = cudaMalloc(&p->G, rowbytes * nr * nfmax);
    float* w_d = nullptr;
    if (weights && e == cudaSuccess) {
        std::vector<float> wf(ns);
        for (int i = 0; i < ns; ++i) wf[i] = (float)weights[i];
        e = cudaMalloc(&w_d, sizeof(float) * ns);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w_d, wf.data(), sizeof(float) * ns, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // wf is a host temporary
    }
    if (!G) {
        if (e == cudaSuccess) e = cudaMemsetAsync(p->G, 0, rowbytes * nr * nfmax, s);
        if (e == cudaSuccess && storage != MDC_C64) e = cudaMalloc(&p->gscale, sizeof(float) * (size_t)nr * nfmax);
        if (e == cudaSuccess && storage != MDC_C64)
            e = cudaMemsetAsync(p->gscale, 0, sizeof(float) * (size_t)nr * nfmax, s);
    } else if (storage == MDC_C64) {
        if (e == cudaSuccess) e = cudaMemcpy2DAsync(p->G, rowbytes, G, (size_t)ns * sizeof(float2),
                                                    (size_t)ns * sizeof(float2), (size_t)nr * nfmax,
                                                    cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && p->ldg > ns)
            e = cudaMemset2DAsync((char*)p->G + (size_t)ns * sizeof(float2), rowbytes, 0,
                                  (size_t)(p->ldg - ns) * sizeof(float2), (size_t)nr * nfmax, s);
        if (e == cudaSuccess && w_d) {
            scale_columns<<<(unsigned)((int64_t)nr * nfmax), 256, 0, s>>>(static_cast<float2*>(p->G), ns, p->ldg, w_d);
            e = cudaGetLastError();
        }
    } else {
        if (e == cudaSuccess) e = cudaMalloc(&p->gscale, sizeof(float) * (size_t)nr * nfmax);
        if (e == cudaSuccess) {
            launch_quantize(p, static_cast<const float2*>(G), w_d, s);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->err_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->err_flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        // W_nt^j for j < nt/2, then W_{nt/2}^m and its conjugate for m < nt/2 (half-length transforms)
        const int h = nt / 2;
        std::vector<float2> tw(3 * (size_t)h);
        for (int j = 0; j < h; ++j) {
            const double ang = -2.0 * M_PI * (double)j / (double)nt;
            tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            const double angh = -2.0 * M_PI * (double)j / (double)h;
            tw[h + j] = make_float2((float)std::cos(angh), (float)std::sin(angh));
            tw[2 * h + j] = make_float2((float)std::cos(angh), -(float)std::sin(angh));
        }
        e = cudaMalloc(&p->tw, sizeof(float2) * tw.size());
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->tw, tw.data(), sizeof(float2) * tw.size(),
                                                  cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (w_d) cudaFree(w_d);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        free_plan(p);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? MDC_ERR_OOM : MDC_ERR_CUDA;
    }
    *out = p;
    return MDC_OK;
}

extern "C" int mdc_create(mdc_handle* out, const void* G, int nfmax, int nr, int ns, int nt,
                          double dt, double dr, int storage, void* stream) {
    if (!G) return MDC_ERR_ARG;
    return create_plan(out, G, nullptr, nfmax, nr, ns, nt, dt, dr, storage, stream);
}

extern "C" int mdc_create_empty(mdc_handle* out, int nfmax, int nr, int ns, int nt, double dt, double dr,
                                int storage, void* stream) {
    return create_plan(out, nullptr, nullptr, nfmax, nr, ns, nt, dt, dr, storage, stream);
}

extern "C" int mdc_create_shard(mdc_handle* out, const void* G, int k0, int nk, int nr, int ns, int nt, double dt,
                                double dr, int storage, void* stream) {
    return create_plan(out, G, nullptr, nk, nr, ns, nt, dt, dr, storage, stream, k0, true);
}

extern "C" int mdc_set_allreduce(mdc_handle h, mdc_allreduce_fn fn, void* ctx) {
    if (!h || !h->shard) return MDC_ERR_ARG;
    h->red_fn = fn;
    h->red_ctx = fn ? ctx : nullptr;
    return MDC_OK;
}

extern "C" int mdc_load_slab(mdc_handle h, const void* G_slab, int k0, int nk, void* stream) {
    if (!h || !G_slab || k0 < 0 || nk < 1 || k0 + nk > h->nf) return MDC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    mdc_plan* p = h;
    const int64_t row0 = (int64_t)k0 * p->nr, nrows = (int64_t)nk * p->nr;
    cudaError_t e = cudaSuccess;
    if (p->storage == MDC_C64) {
        const size_t rowbytes = (size_t)p->ldg * sizeof(float2);
        char* dst = static_cast<char*>(p->G) + (size_t)row0 * rowbytes;
        e = cudaMemcpy2DAsync(dst, rowbytes, G_slab, (size_t)p->ns * sizeof(float2), (size_t)p->ns * sizeof(float2),
                              (size_t)nrows, cudaMemcpyDeviceToDevice, s);
    } else {
        launch_quantize_rows(p, static_cast<const float2*>(G_slab), nullptr, row0, nrows, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);       // the caller may reuse the slab buffer
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    return MDC_OK;
}

extern "C" int mdc_create_weighted(mdc_handle* out, const void* G, const double* weights, int nfmax, int nr,
                                   int ns, int nt, double dt, double dr, int storage, void* stream) {
    if (!G || !weights) return MDC_ERR_ARG;
    for (int i = 0; i < ns; ++i)
        if (!std::isfinite(weights[i]) || weights[i] < 0.0) return MDC_ERR_ARG;
    return create_plan(out, G, weights, nfmax, nr, ns, nt, dt, dr, storage, stream);
}

int mdc::ensure_scratch(mdc_plan* p, int ncols) {
    if (ncols > p->nv_cap) {
        const size_t n = (size_t)p->nf * (size_t)(p->nr > p->ns ? p->nr : p->ns) * ncols;
        float2 *a = nullptr, *b = nullptr;
        cudaError_t e = cudaMalloc(&a, n * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&b, n * sizeof(float2));
        if (e != cudaSuccess) {
            cudaFree(a);
            cudaGetLastError();
            set_cuda_error(e);
            return MDC_ERR_OOM;
        }
        cudaFree(p->specA);
        cudaFree(p->specB);
        p->specA = a;
        p->specB = b;
        p->nv_cap = ncols;
    }
    // tensor-core operand for the FP16/BF16/E4M3 copies (used from 8 columns on)
    if (storage_tc(p->storage) && ncols > p->tc_cap) {
        void* b = nullptr;
        float* sg = nullptr;
        cudaError_t e = cudaMalloc(&b, tc_scratch_elems(p, ncols) * 2 * (p->storage == MDC_C32S ? 2 : 1));
        if (e == cudaSuccess) e = cudaMalloc(&sg, (size_t)p->nf * ncols * sizeof(float));
        if (e != cudaSuccess) {
            cudaFree(b);
            cudaGetLastError();
            set_cuda_error(e);
            return MDC_ERR_OOM;
        }
        cudaFree(p->tcB);
        cudaFree(p->tcSigma);
        p->tcB = b;
        p->tcSigma = sg;
        p->tc_cap = ncols;
    }
    return MDC_OK;
}

extern "C" int mdc_reserve(mdc_handle h, int nv_max) {
    if (!h || nv_max < 1) return MDC_ERR_ARG;
    return ensure_scratch(h, nv_max);
}

// One MDC pass: rFFT of `in` (S_in spatial points), per-frequency product, irFFT to `out`.
static int mdc_pass(mdc_plan* p, bool adjoint, const float* in, float* outp, int nv, unsigned flags,
                    cudaStream_t s) {
    if (!in || !outp || nv < 1) return MDC_ERR_ARG;
    int st = ensure_scratch(p, nv);
    if (st != MDC_OK) return st;
    const int S_in = adjoint ? p->nr : p->ns;
    const int S_out = adjoint ? p->ns : p->nr;
    const int conj = (flags & MDC_CONJ_KERNEL) ? 1 : 0;
    RfftArgs ra{};
    ra.x = in; ra.x2 = nullptr; ra.C = S_in * nv; ra.S = S_in; ra.nv = nv;
    ra.nt = p->nt; ra.logn = p->logn; ra.nf = p->nf; ra.k0 = p->k0; ra.cut = nullptr; ra.scale = C1(1.f);
    ra.conj = conj; ra.X = p->specA; ra.ldv = nv; ra.voff = 0; ra.tw = p->tw; ra.active = nullptr;
    launch_rfft(p, ra, s);
    launch_product(p, adjoint, p->specA, nv, 0, p->specB, nv, 0, nv, s, nullptr);
    IrfftArgs ia{};
    ia.Y = p->specB; ia.ldv = nv; ia.voff = 0; ia.C = S_out * nv; ia.S = S_out; ia.nv = nv;
    ia.nt = p->nt; ia.logn = p->logn; ia.nf = p->nf; ia.k0 = p->k0; ia.conj_in = conj;
    ia.scale = (float)(p->dt * p->dr / (double)p->nt);
    ia.out = outp; ia.a_mdc = C1(1.f); ia.a_base = C1(0.f); ia.a_prev = C1(0.f);
    ia.base = nullptr; ia.cut = nullptr; ia.reverse_out = 0; ia.colsum = nullptr; ia.tw = p->tw;
    ia.active = nullptr;
    launch_irfft(p, ia, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(e); return MDC_ERR_CUDA; }
    return take_host_error(p);
}

extern "C" int mdc_forward(mdc_handle h, const float* x, float* y, int nv, unsigned flags, void* stream) {
    if (!h || (flags & ~MDC_CONJ_KERNEL)) return MDC_ERR_ARG;
    return mdc_pass(h, false, x, y, nv, flags, (cudaStream_t)stream);
}

extern "C" int mdc_adjoint(mdc_handle h, const float* y, float* x, int nv, unsigned flags, void* stream) {
    if (!h || (flags & ~MDC_CONJ_KERNEL)) return MDC_ERR_ARG;
    return mdc_pass(h, true, y, x, nv, flags, (cudaStream_t)stream);
}

extern "C" int mdc_destroy(mdc_handle h) {
    if (!h) return MDC_ERR_ARG;
    cudaDeviceSynchronize();
    free_plan(h);
    return MDC_OK;
}

extern "C" int mdc_timing(mdc_handle h, int enable) {
    if (!h) return MDC_ERR_ARG;
    TimingState& t = h->timing;
    if (enable) {
        if (t.pool.empty()) {
            t.pool.resize(16384);
            t.used_class.resize(t.pool.size());
            for (auto& e : t.pool) {
                MDC_CUDA_TRY(cudaEventCreate(&e.a));
                MDC_CUDA_TRY(cudaEventCreate(&e.b));
            }
        }
        t.used = 0;
        for (int i = 0; i < MDC_KC_COUNT; ++i) t.launches[i] = t.recorded[i] = 0;
    }
    t.on = enable != 0;
    return MDC_OK;
}

extern "C" int mdc_timing_read(mdc_handle h, int cls, double* total_ms, int64_t* launches) {
    if (!h || cls < 0 || cls >= MDC_KC_COUNT) return MDC_ERR_ARG;
    TimingState& t = h->timing;
    double tot = 0.0;
    for (size_t i = 0; i < t.used; ++i) {
        if (t.used_class[i] != cls) continue;
        MDC_CUDA_TRY(cudaEventSynchronize(t.pool[i].b));
        float ms = 0.f;
        MDC_CUDA_TRY(cudaEventElapsedTime(&ms, t.pool[i].a, t.pool[i].b));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = t.recorded[cls];
    return MDC_OK;
}

extern "C" int64_t mdc_launch_count(mdc_handle h) { return h ? h->launch_count : -1; }

namespace mdc {
int autotune(mdc_plan* p, int ncol_max, cudaStream_t s);
}

extern "C" int mdc_autotune(mdc_handle h, int ncol_max, void* stream) {
    if (!h || ncol_max < 1) return MDC_ERR_ARG;
    return mdc::autotune(h, ncol_max, (cudaStream_t)stream);
}

extern "C" int mdc_autotune_choice(mdc_handle h, int adjoint, int ncol, int* path, int* bn) {
    if (!h || ncol < 1 || !path || !bn) return MDC_ERR_ARG;
    *path = 0;
    *bn = 0;
    for (const ProductChoice& c : h->tune[adjoint ? 1 : 0])
        if (ncol <= c.ncol) {
            *path = c.path;
            *bn = c.bn;
            break;
        }
    return MDC_OK;
}

extern "C" int mdc_set_option(mdc_handle h, int option, int value) {
    if (!h) return MDC_ERR_ARG;
    switch (option) {
        case MDC_OPT_GRAPHS:
            h->graphs = value != 0;
            if (!h->graphs && h->graph_free) {
                cudaDeviceSynchronize();
                for (void* g : h->graph_cache) h->graph_free(g);
                h->graph_cache.clear();
            }
            return MDC_OK;
        case MDC_OPT_WAIT_LIMIT_US:
            if (value < 0) return MDC_ERR_ARG;
            h->wait_ns = value == 0 ? 2000000000ull : (unsigned long long)value * 1000ull;
            return MDC_OK;
        default:
            return MDC_ERR_ARG;
    }
}

extern "C" int64_t mdc_tc_fallback_count(mdc_handle h) { return h ? h->tc_fallbacks : -1; }

extern "C" int mdc_device_status(mdc_handle h, void* stream) {
    if (!h) return MDC_ERR_ARG;
    int v = 0;
    MDC_CUDA_TRY(cudaMemcpyAsync(&v, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    MDC_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (v != 0) {
        MDC_CUDA_TRY(cudaMemsetAsync(h->err_flag, 0, sizeof(int), (cudaStream_t)stream));
        MDC_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        return mdc::device_flag_status(v);
    }
    return MDC_OK;
}
