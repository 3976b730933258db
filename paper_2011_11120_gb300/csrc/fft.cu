// Real FFT along the slow time axis, truncated to the kept band (F and I_wmax of
// Eq. 3), and the zero-padded inverse (I_wmax^H and F^H of Eq. 3).
//
// Layout: time-domain arrays are [nt][C] float32 with C = n_space * nv columns,
// so the transform runs down a column with stride C.  One CTA owns a tile of CT
// adjacent columns for the whole time axis: the tile is read row by row (CT
// consecutive floats per time sample, coalesced), held in shared memory, and two
// real columns are packed into one complex sequence (real part = even column,
// imaginary part = odd column) so that a complex radix-2 FFT transforms two
// columns at once.  The first nf bins of each column are then separated from the
// packed spectrum with the conjugate-symmetry identities
//     A[k] = (Z[k] + conj Z[-k]) / 2,   B[k] = (Z[k] - conj Z[-k]) / (2i).
// The inverse builds the Hermitian spectrum of two columns (bins >= nf are zero,
// the DC and Nyquist bins keep only their real part) as Z = A + iB, transforms
// back, and reads column A from the real and column B from the imaginary part.
//
// Twiddles come from a float64 host table rounded once to float32.
#include "common.cuh"

namespace mdc {
namespace {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ int bitrev(int v, int logn) { return (int)(__brev((unsigned)v) >> (32 - logn)); }

// In-place radix-2 decimation-in-time over P packed sequences stored as rows of
// RS floats ([t][2P] interleaved complex), input already in bit-reversed order.
__device__ __forceinline__ void fft_dit(float* zf, const float2* tw, int logn, int logP, int RS) {
    const int nt = 1 << logn;
    const int P = 1 << logP;
    const int nb = (nt >> 1) << logP;
    for (int l = 1; l <= logn; ++l) {
        const int half = 1 << (l - 1);
        for (int bi = threadIdx.x; bi < nb; bi += FFT_THREADS) {
            const int j = bi & (P - 1);
            const int b = bi >> logP;
            const int pos = b & (half - 1);
            const int i0 = ((b >> (l - 1)) << l) + pos;
            const int i1 = i0 + half;
            const float2 w = tw[pos << (logn - l)];
            float2* p0 = reinterpret_cast<float2*>(zf + i0 * RS) + j;
            float2* p1 = reinterpret_cast<float2*>(zf + i1 * RS) + j;
            const float2 u = *p0;
            const float2 v = cmul(*p1, w);
            *p0 = cadd(u, v);
            *p1 = csub(u, v);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(FFT_THREADS) rfft_kernel(RfftArgs a, int logCT) {
    if (a.active && *a.active == 0) return;
    extern __shared__ __align__(16) float smem[];
    const int CT = 1 << logCT, RS = CT + 2;
    const int nt = a.nt, logn = a.logn;
    float2* tw = reinterpret_cast<float2*>(smem);
    float* zf = smem + nt;                          // [nt][RS]
    const int c0 = blockIdx.x * CT;

    for (int i = threadIdx.x; i < nt / 2; i += FFT_THREADS) tw[i] = a.tw[i];
    const float sc = coef(a.scale);
    for (int idx = threadIdx.x; idx < (nt << logCT); idx += FFT_THREADS) {
        const int t = idx >> logCT, cl = idx & (CT - 1), c = c0 + cl;
        float v = 0.f;
        if (c < a.C) {
            const size_t off = (size_t)t * a.C + c;
            v = a.x[off];
            if (a.x2) v += a.x2[off];
            if (a.cut) {
                const int tau = t < (nt >> 1) ? t : nt - t;
                if (tau >= a.cut[c]) v = 0.f;
            }
            v *= sc;
        }
        zf[bitrev(t, logn) * RS + cl] = v;
    }
    __syncthreads();
    fft_dit(zf, tw, logn, logCT - 1, RS);

    for (int idx = threadIdx.x; idx < (a.nf << logCT); idx += FFT_THREADS) {
        const int k = idx >> logCT, cl = idx & (CT - 1), c = c0 + cl;
        if (c >= a.C) continue;
        const int j = cl >> 1;
        const float2 Z = reinterpret_cast<const float2*>(zf + k * RS)[j];
        const float2 Zm = reinterpret_cast<const float2*>(zf + ((nt - k) & (nt - 1)) * RS)[j];
        float2 r;
        if ((cl & 1) == 0) r = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
        else               r = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
        if (a.conj) r.y = -r.y;
        const int s = c / a.nv, v = c - s * a.nv;
        a.X[((size_t)k * a.S + s) * a.ldv + a.voff + v] = r;
    }
}

__device__ __forceinline__ float2 load_bin(const IrfftArgs& a, int k, int c) {
    const int s = c / a.nv, v = c - s * a.nv;
    return a.Y[((size_t)k * a.S + s) * a.ldv + a.voff + v];
}

__global__ void __launch_bounds__(FFT_THREADS) irfft_kernel(IrfftArgs a, int logCT) {
    if (a.active && *a.active == 0) return;
    extern __shared__ __align__(16) float smem[];
    const int CT = 1 << logCT, RS = CT + 2, logP = logCT - 1, P = CT >> 1;
    const int nt = a.nt, logn = a.logn;
    float2* tw = reinterpret_cast<float2*>(smem);
    float* zf = smem + nt;                                         // [nt][RS]
    double* red = reinterpret_cast<double*>(zf + (size_t)nt * RS); // [FFT_THREADS]
    const int c0 = blockIdx.x * CT;

    for (int i = threadIdx.x; i < nt / 2; i += FFT_THREADS) tw[i] = cconj(a.tw[i]);
    for (int idx = threadIdx.x; idx < (nt << logP); idx += FFT_THREADS) {
        const int j = idx & (P - 1), k = idx >> logP;
        const int kk = k <= (nt >> 1) ? k : nt - k;
        float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
        if (kk < a.nf) {
            const int ca = c0 + 2 * j;
            if (ca < a.C) A = load_bin(a, kk, ca);
            if (ca + 1 < a.C) B = load_bin(a, kk, ca + 1);
            if (a.conj_in) { A.y = -A.y; B.y = -B.y; }
            if (kk == 0 || 2 * kk == nt) { A.y = 0.f; B.y = 0.f; }
            if (k > (nt >> 1)) { A.y = -A.y; B.y = -B.y; }
        }
        reinterpret_cast<float2*>(zf + bitrev(k, logn) * RS)[j] = make_float2(A.x - B.y, A.y + B.x);
    }
    __syncthreads();
    fft_dit(zf, tw, logn, logP, RS);

    const float am = coef(a.a_mdc), ab = coef(a.a_base), ap = coef(a.a_prev);
    const bool has_prev = (a.a_prev.h != 0.f) || (a.a_prev.d != nullptr);
    const int cl = threadIdx.x & (CT - 1), c = c0 + cl;
    double ss = 0.0;
    if (c < a.C) {
        const int cut = a.cut ? a.cut[c] : 0x7fffffff;
        for (int t = threadIdx.x >> logCT; t < nt; t += FFT_THREADS >> logCT) {
            const float2 zz = reinterpret_cast<const float2*>(zf + t * RS)[cl >> 1];
            float val = ((cl & 1) ? zz.y : zz.x) * a.scale;
            const int tau = t < (nt >> 1) ? t : nt - t;
            if (tau >= cut) val = 0.f;
            float r = am * val;
            if (a.base) r += ab * a.base[(size_t)t * a.C + c];
            const int to = a.reverse_out ? ((nt - t) & (nt - 1)) : t;
            const size_t o = (size_t)to * a.C + c;
            if (has_prev) r += ap * a.out[o];
            a.out[o] = r;
            ss += (double)r * (double)r;
        }
    }
    if (a.colsum) {
        red[threadIdx.x] = ss;
        __syncthreads();
        if (threadIdx.x < CT && c < a.C) {
            double tot = 0.0;
            for (int i = threadIdx.x; i < FFT_THREADS; i += CT) tot += red[i];
            a.colsum[c] = tot;
        }
    }
}

int tile_log_columns(int nt) {
    // CT * nt ~ 16K floats per CTA (64 KB), CT in [4, 64]
    int ct = 16384 / nt;
    if (ct > 64) ct = 64;
    if (ct < 4) ct = 4;
    return ilog2(ct);
}

size_t rfft_smem(int nt, int logCT) { return (size_t)nt * 4 + (size_t)nt * ((1 << logCT) + 2) * 4; }
size_t irfft_smem(int nt, int logCT) { return rfft_smem(nt, logCT) + FFT_THREADS * 8; }

}  // namespace

void launch_rfft(mdc_plan* p, const RfftArgs& a, cudaStream_t s) {
    const int logCT = tile_log_columns(a.nt);
    const size_t smem = rfft_smem(a.nt, logCT);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(rfft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int grid = (a.C + (1 << logCT) - 1) >> logCT;
    LaunchScope ls(p, s, MDC_KC_RFFT);
    rfft_kernel<<<grid, FFT_THREADS, smem, s>>>(a, logCT);
}

void launch_irfft(mdc_plan* p, const IrfftArgs& a, cudaStream_t s) {
    const int logCT = tile_log_columns(a.nt);
    const size_t smem = irfft_smem(a.nt, logCT);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(irfft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int grid = (a.C + (1 << logCT) - 1) >> logCT;
    LaunchScope ls(p, s, MDC_KC_IRFFT);
    irfft_kernel<<<grid, FFT_THREADS, smem, s>>>(a, logCT);
}

}  // namespace mdc
