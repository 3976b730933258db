// mdc_forward_static_scratch: the MDC forward pass with its frequency-domain
// scratch in a fixed, file-scope device array instead of handle-owned cudaMalloc
// memory.  It exists for callers that must not allocate device memory at call
// time (see include/mdc.h); the paper has no counterpart.
//
// The array below is a module-scope __device__ variable: the CUDA runtime
// reserves it on every device that loads this module and keeps it until the
// process exits.  Host code cannot use its name as a device address, so the
// first call on each device asks the runtime for the address
// (cudaGetSymbolAddress) with that device current and caches it.
#include <mutex>

#include "common.cuh"

namespace mdc {
namespace {

// Two spectra of up to MDC_STATIC_SCRATCH_COMPLEX complex64 values each (32 MiB in total).
constexpr size_t kSpectrumCapacity = (size_t)MDC_STATIC_SCRATCH_COMPLEX;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_static_scratch[2 * kSpectrumCapacity];

std::mutex g_addr_mutex;
float2* g_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set-up on first use).
int scratch_address(float2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_cuda_error(e); return MDC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return MDC_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_cuda_error(e);
            return MDC_ERR_CUDA;
        }
        g_addr[dev] = static_cast<float2*>(p);
    }
    *out = g_addr[dev];
    return MDC_OK;
}

}  // namespace
}  // namespace mdc

using namespace mdc;

extern "C" int mdc_forward_static_scratch(mdc_handle h, const float* x, float* y, int nv, unsigned flags,
                                          void* stream) {
    if (!h || !x || !y || nv < 1 || (flags & ~MDC_CONJ_KERNEL)) return MDC_ERR_ARG;
    if (h->red_fn) return MDC_ERR_STATE;       // the sum over shards would need a reduction buffer
    const size_t nspace = (size_t)(h->nr > h->ns ? h->nr : h->ns);
    if ((size_t)h->nf * nspace * (size_t)nv > kSpectrumCapacity) return MDC_ERR_BUDGET;
    float2* base = nullptr;
    int st = scratch_address(&base);
    if (st != MDC_OK) return st;
    float2* specX = base;                       // rFFT of x:          [nf][ns][nv]
    float2* specY = base + kSpectrumCapacity;   // product output:     [nf][nr][nv]
    cudaStream_t s = (cudaStream_t)stream;
    const int conj = (flags & MDC_CONJ_KERNEL) ? 1 : 0;

    RfftArgs ra{};
    ra.x = x; ra.x2 = nullptr; ra.C = h->ns * nv; ra.S = h->ns; ra.nv = nv;
    ra.nt = h->nt; ra.logn = h->logn; ra.nf = h->nf; ra.k0 = h->k0; ra.cut = nullptr; ra.scale = C1(1.f);
    ra.conj = conj; ra.X = specX; ra.ldv = nv; ra.voff = 0; ra.tw = h->tw; ra.active = nullptr;
    launch_rfft(h, ra, s);
    launch_product(h, false, specX, nv, 0, specY, nv, 0, nv, s, nullptr);
    IrfftArgs ia{};
    ia.Y = specY; ia.ldv = nv; ia.voff = 0; ia.C = h->nr * nv; ia.S = h->nr; ia.nv = nv;
    ia.nt = h->nt; ia.logn = h->logn; ia.nf = h->nf; ia.k0 = h->k0; ia.conj_in = conj;
    ia.scale = (float)(h->dt * h->dr / (double)h->nt);
    ia.out = y; ia.a_mdc = C1(1.f); ia.a_base = C1(0.f); ia.a_prev = C1(0.f);
    ia.base = nullptr; ia.cut = nullptr; ia.reverse_out = 0; ia.colsum = nullptr; ia.tw = h->tw;
    ia.active = nullptr;
    launch_irfft(h, ia, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(e); return MDC_ERR_CUDA; }
    return MDC_OK;
}
