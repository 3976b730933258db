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
            [[maybe_unused]] const long long nx = (long long)nt * a.C;
            v = *MDC_AT(a.x, off, 1, nx, a.err, 1);
            if (a.x2) v += *MDC_AT(a.x2, off, 1, nx, a.err, 2);
            if (a.cut) {
                const int tau = t < (nt >> 1) ? t : nt - t;
                if (tau >= *MDC_AT(a.cut, c, 1, a.C, a.err, 3)) v = 0.f;
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
        const int j = cl >> 1, kb = k + a.k0;                    // bin of the slab's k-th entry
        const float2 Z = reinterpret_cast<const float2*>(zf + kb * RS)[j];
        const float2 Zm = reinterpret_cast<const float2*>(zf + ((nt - kb) & (nt - 1)) * RS)[j];
        float2 r;
        if ((cl & 1) == 0) r = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
        else               r = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
        if (a.conj) r.y = -r.y;
        const int s = c / a.nv, v = c - s * a.nv;
        *MDC_AT(a.X, ((size_t)k * a.S + s) * a.ldv + a.voff + v, 1, (long long)a.nf * a.S * a.ldv, a.err, 4) = r;
    }
}

__device__ __forceinline__ float2 load_bin(const IrfftArgs& a, int k, int c) {
    const int s = c / a.nv, v = c - s * a.nv;
    return *MDC_AT(a.Y, ((size_t)k * a.S + s) * a.ldv + a.voff + v, 1, (long long)a.nf * a.S * a.ldv, a.err, 5);
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
        if (kk >= a.k0 && kk < a.k0 + a.nf) {
            const int ca = c0 + 2 * j;
            if (ca < a.C) A = load_bin(a, kk - a.k0, ca);
            if (ca + 1 < a.C) B = load_bin(a, kk - a.k0, ca + 1);
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
        const int cut = a.cut ? *MDC_AT(a.cut, c, 1, a.C, a.err, 6) : 0x7fffffff;
        [[maybe_unused]] const long long nx = (long long)nt * a.C;
        for (int t = threadIdx.x >> logCT; t < nt; t += FFT_THREADS >> logCT) {
            const float2 zz = reinterpret_cast<const float2*>(zf + t * RS)[cl >> 1];
            float val = ((cl & 1) ? zz.y : zz.x) * a.scale;
            const int tau = t < (nt >> 1) ? t : nt - t;
            if (tau >= cut) val = 0.f;
            float r = am * val;
            if (a.base) r += ab * *MDC_AT(a.base, (size_t)t * a.C + c, 1, nx, a.err, 7);
            const int to = a.reverse_out ? ((nt - t) & (nt - 1)) : t;
            const size_t o = (size_t)to * a.C + c;
            if (has_prev) r += ap * *MDC_AT(a.out, o, 1, nx, a.err, 8);
            *MDC_AT(a.out, o, 1, nx, a.err, 9) = r;
            ss += (double)r * (double)r;
        }
    }
    if (a.colsum) {
        red[threadIdx.x] = ss;
        __syncthreads();
        if (threadIdx.x < CT && c < a.C) {
            double tot = 0.0;
            for (int i = threadIdx.x; i < FFT_THREADS; i += CT) tot += red[i];
            *MDC_AT(a.colsum, c, 1, a.C, a.err, 10) = tot;
        }
    }
}

// ------------------------------------------------------------------ four-step kernels
// nt = N1 * N2 (N1, N2 in {8, 16, 32}).  Pass A: for each residue n2, an N1-point DFT in
// registers over t = n1 * N2 + n2, then the twiddle W_nt^(n2 k1); pass B: for each k1 an
// N2-point DFT over the N2 consecutive rows k1 * N2 + n2.  Result bin k = k1 + N1 * k2
// sits in row k1 * N2 + k2.  Four shared-memory sweeps per transform instead of
// 2 log2(nt) + 1 for radix 2.  Layout: row t of P complex sequences at
// t * RS + (t / N2) * BP, RS = P + 1 and BP chosen so that both passes spread a warp's
// 8-byte accesses over distinct bank pairs.

__host__ __device__ constexpr int brev_bits(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int clog2(int n) { return n <= 1 ? 0 : 1 + clog2(n / 2); }

// Roots of unity as compile-time constants: cos and sin of 2*pi/R from the half-angle identities
// (cos(t/2) = sqrt((1 + cos t) / 2), sin(t/2) = sin t / (2 cos(t/2))) starting at t = pi/2, then
// powers by angle addition, all in double precision and rounded once to float.
struct Rot {
    double c, s;
};
constexpr double newton_sqrt(double x) {
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
    return r;
}
constexpr Rot unit_root(int R, int m) {   // exp(+2 pi i m / R)
    Rot b{0.0, 1.0};
    if (R == 1) b = Rot{1.0, 0.0};
    if (R == 2) b = Rot{-1.0, 0.0};
    for (int r = 4; r < R; r *= 2) {
        const double c = newton_sqrt(0.5 * (1.0 + b.c));
        b = Rot{c, b.s / (2.0 * c)};
    }
    Rot w{1.0, 0.0};
    for (int i = 0; i < m; ++i) w = Rot{w.c * b.c - w.s * b.s, w.s * b.c + w.c * b.s};
    return w;
}

// exp(-2 pi i m / 32) for m < 16: every twiddle of the in-register DFTs (R <= 32) is one of
// these; as constant-bank operands they need no load.
#define MDC_ROOT32(m) float2{(float)unit_root(32, m).c, -(float)unit_root(32, m).s}
__constant__ float2 kRoot32[16] = {
    MDC_ROOT32(0),  MDC_ROOT32(1),  MDC_ROOT32(2),  MDC_ROOT32(3),  MDC_ROOT32(4),  MDC_ROOT32(5),
    MDC_ROOT32(6),  MDC_ROOT32(7),  MDC_ROOT32(8),  MDC_ROOT32(9),  MDC_ROOT32(10), MDC_ROOT32(11),
    MDC_ROOT32(12), MDC_ROOT32(13), MDC_ROOT32(14), MDC_ROOT32(15)};
#undef MDC_ROOT32

// Complex add and subtract as one packed two-lane float32 instruction (sm_100 and later);
// each lane rounds to nearest like the scalar operation.
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// Length-R DFT (R <= 32) of a register array, forward sign exp(-2 pi i n k / R) or, with INV,
// the inverse sign (unscaled): decimation in frequency (natural order in, bit-reversed order
// out), then a compile-time permutation back to natural order.  After unrolling every index
// and twiddle choice is a constant: quarter turns are a swap, eighth turns take the
// equal-magnitude short form, the rest multiply by a table constant.
template <int R, bool INV>
__device__ __forceinline__ void reg_fft(float2 (&a)[R]) {
    static_assert(R <= 32, "register DFT length");
    constexpr int L = clog2(R);
    constexpr float h8 = (float)unit_root(8, 1).c;
#pragma unroll
    for (int st = 0; st < L; ++st) {
        const int h = R >> (st + 1);          // half span of this stage
#pragma unroll
        for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const float2 u = a[g + j], v = a[g + j + h];
                a[g + j] = padd(u, v);
                float2 d = psub(u, v);
                const int m = j << st;       // twiddle exp(-+2 pi i m / R)
                if (m == 0) {
                } else if (4 * m == R) {
                    d = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
                } else if (8 * m == R) {
                    d = INV ? make_float2(h8 * (d.x - d.y), h8 * (d.x + d.y))
                            : make_float2(h8 * (d.x + d.y), h8 * (d.y - d.x));
                } else if (8 * m == 3 * R) {
                    d = INV ? make_float2(-h8 * (d.x + d.y), h8 * (d.x - d.y))
                            : make_float2(h8 * (d.y - d.x), -h8 * (d.x + d.y));
                } else {
                    const float2 w = kRoot32[m * (32 / R)];
                    d = cmul(d, INV ? cconj(w) : w);
                }
                a[g + j + h] = d;
            }
        }
    }
    float2 b[R];
#pragma unroll
    for (int i = 0; i < R; ++i) b[i] = a[brev_bits(i, L)];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = b[i];
}

// PP: complex sequences per CTA, or 0 for the default of about 8192 complex values per tile (the
// few-column variant PP = max(1024 / NT, 2) spreads small batches over more CTAs).
template <int N1, int N2, int PP = 0> struct FourStep {
    static constexpr int NT = N1 * N2;
    static constexpr int P0 = 8192 / NT;
    static constexpr int P = PP ? PP : (P0 > 32 ? 32 : (P0 < 8 ? 8 : P0));   // complex sequences per CTA
    static constexpr int CT = 2 * P;                                  // real columns per CTA
    // Rows of P complex values, unpadded, plus BP slots after every block of N2 rows: with P = 8
    // two consecutive rows (or blocks, in pass B) then fill all 16 bank pairs, and rows stay
    // 16-byte aligned for vector accesses.
    static constexpr int RS = P;
    static constexpr int BP = P == 8 ? 8 : 0;
    static constexpr int ZSIZE = NT * RS + N1 * BP;                  // float2 elements
    // twiddle table and tile; the inverse transform's column-sum reduction reuses the tile
    static constexpr size_t smem = (size_t)(NT / 2 + ZSIZE) * sizeof(float2);
    static constexpr size_t smem_full = (size_t)(NT + ZSIZE) * sizeof(float2);   // full-period twiddles
    static_assert(ZSIZE * sizeof(float2) >= FFT_THREADS * 4 * sizeof(double), "reduction fits the tile");
    __device__ static __forceinline__ int zi(int t, int j) { return t * RS + (t / N2) * BP + j; }
};

__device__ __forceinline__ float2 tw_full(const float2* tw, int m, int nt) {
    return m < (nt >> 1) ? tw[m] : make_float2(-tw[m - (nt >> 1)].x, -tw[m - (nt >> 1)].y);
}

// Second pass of the four-step transform: the length-N2 DFTs over n2 of every block k1, in
// place; ends with a barrier.
template <int N1, int N2, bool INV, int PP = 0>
__device__ __forceinline__ void four_step_pass_b(float2* z) {
    using F = FourStep<N1, N2, PP>;
    constexpr int P = F::P;
    for (int task = threadIdx.x; task < P * N1; task += FFT_THREADS) {
        const int j = task % P, k1 = task / P;
        float2 r[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) r[n2] = z[F::zi(k1 * N2 + n2, j)];
        reg_fft<N2, INV>(r);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) z[F::zi(k1 * N2 + k2, j)] = r[k2];
    }
    __syncthreads();
}

// tw: the twiddle table W_NT^m of the transform's sign (conjugated for INV), m < NT/2, or with
// FULL the whole period m < NT (no sign select per twiddle).
template <int N1, int N2, bool INV, bool FULL = false, int PP = 0>
__device__ __forceinline__ void four_step(float2* z, const float2* tw) {
    using F = FourStep<N1, N2, PP>;
    constexpr int P = F::P;
    for (int task = threadIdx.x; task < P * N2; task += FFT_THREADS) {
        const int j = task % P, n2 = task / P;
        float2 r[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) r[n1] = z[F::zi(n1 * N2 + n2, j)];
        reg_fft<N1, INV>(r);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            const float2 v = k1 == 0 ? r[0] : cmul(r[k1], FULL ? tw[n2 * k1] : tw_full(tw, n2 * k1, F::NT));
            z[F::zi(k1 * N2 + n2, j)] = v;
        }
    }
    __syncthreads();
    four_step_pass_b<N1, N2, INV, PP>(z);
}

// Row holding bin (or time sample) q after four_step.
template <int N1, int N2>
__device__ __forceinline__ int out_row(int q) { return (q % N1) * N2 + q / N1; }

// WIN: the window Theta multiplies the input; X2: a second input is added.  The input scale is
// applied to the separated spectrum (the transform is linear), together with its factor 1/2.
template <int N1, int N2, bool WIN, bool X2, int PP>
__global__ void __launch_bounds__(FFT_THREADS, 2) rfft4_kernel(RfftArgs a) {
    using F = FourStep<N1, N2, PP>;
    constexpr int NT = F::NT, CT = F::CT;
    if (a.active && *a.active == 0) return;
    extern __shared__ __align__(16) float2 sm2[];
    float2* tw = sm2;                  // W_NT^m for the whole period m < NT
    float2* z = sm2 + NT;
    const int c0 = blockIdx.x * CT;
    for (int i = threadIdx.x; i < NT / 2; i += FFT_THREADS) {
        const float2 w = a.tw[i];
        tw[i] = w;
        tw[i + NT / 2] = make_float2(-w.x, -w.y);
    }
    // Load the [NT][CT] tile with many independent loads in flight per thread.
    auto put = [&](int t, int cl, float v) {
        if constexpr (WIN) {
            const int tau = t < (NT >> 1) ? t : NT - t;
            if (tau >= *MDC_AT(a.cut, c0 + cl, 1, a.C, a.err, 11)) v = 0.f;
        }
        reinterpret_cast<float*>(z + F::zi(t, cl >> 1))[cl & 1] = v;
    };
    if (a.vec4 && c0 + CT <= a.C) {
        // First pass straight from global memory: task (j, n2) loads the column pair
        // (c0 + 2j, c0 + 2j + 1) at rows n1 * N2 + n2 (a warp reads whole 64- or 128-byte row
        // segments), applies window and scale, transforms over n1 in registers, twiddles, and
        // writes the tile; only the second pass goes through shared memory.
        __syncthreads();                                  // twiddle table
        constexpr int P = F::P;
        const size_t rstride = (size_t)N2 * a.C;          // floats between the rows n1 and n1 + 1
        for (int task = threadIdx.x; task < P * N2; task += FFT_THREADS) {
            const int j = task % P, n2 = task / P, c = c0 + 2 * j;
            const size_t xo = c + (size_t)n2 * a.C;
            float2 r[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1)
                r[n1] = *reinterpret_cast<const float2*>(MDC_AT(a.x, xo + n1 * rstride, 2, (long long)NT * a.C, a.err, 12));
            if constexpr (X2) {
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) {
                    const float2 w = *reinterpret_cast<const float2*>(MDC_AT(a.x2, xo + n1 * rstride, 2, (long long)NT * a.C, a.err, 13));
                    r[n1].x += w.x;
                    r[n1].y += w.y;
                }
            }
            if constexpr (WIN) {
                const int cut0 = *MDC_AT(a.cut, c, 1, a.C, a.err, 14), cut1 = *MDC_AT(a.cut, c + 1, 1, a.C, a.err, 14);
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) {
                    const int t = n1 * N2 + n2;
                    const int tau = t < (NT >> 1) ? t : NT - t;
                    if (tau >= cut0) r[n1].x = 0.f;
                    if (tau >= cut1) r[n1].y = 0.f;
                }
            }
            reg_fft<N1, false>(r);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1)
                z[F::zi(k1 * N2 + n2, j)] = k1 == 0 ? r[0] : cmul(r[k1], tw[n2 * k1]);
        }
        __syncthreads();
        four_step_pass_b<N1, N2, false, PP>(z);
    } else {
        constexpr int PER = NT * CT / FFT_THREADS, B = PER < 16 ? PER : 16;
#pragma unroll 1
        for (int b0 = 0; b0 < PER; b0 += B) {
            float v[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int idx = threadIdx.x + (b0 + u) * FFT_THREADS;
                const int t = idx / CT, c = c0 + idx % CT;
                v[u] = 0.f;
                if (c < a.C) {
                    const size_t off = (size_t)t * a.C + c;
                    v[u] = *MDC_AT(a.x, off, 1, (long long)NT * a.C, a.err, 15);
                    if constexpr (X2) v[u] += *MDC_AT(a.x2, off, 1, (long long)NT * a.C, a.err, 16);
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int idx = threadIdx.x + (b0 + u) * FFT_THREADS;
                const int t = idx / CT, cl = idx % CT;
                if (c0 + cl < a.C) put(t, cl, v[u]);
                else reinterpret_cast<float*>(z + F::zi(t, cl >> 1))[cl & 1] = 0.f;
            }
        }
        __syncthreads();
        four_step<N1, N2, false, true, PP>(z, tw);
    }
    const float hs = 0.5f * coef(a.scale);
    // Bin k = k1 + N1 * k2 sits in row k1 * N2 + k2, its mirror NT - k in row
    // ((-k1) mod N1) * N2 + (NT/N1 - k2 - [k1 > 0]) (k > 0).  A thread keeps one column and walks
    // the bins of every G-th block k1; the G threads of a column cover all N1 blocks, and the
    // CT threads of one row write CT adjacent columns.
    constexpr int G = FFT_THREADS / CT;
    const int cl = threadIdx.x % CT, g = threadIdx.x / CT, c = c0 + cl;
    if (c < a.C) {
        int s, v;
        if ((a.nv % CT) == 0) {               // every column of the tile has the same spatial index
            s = c0 / a.nv;
            v = c0 - s * a.nv + cl;
        } else {
            s = c / a.nv;
            v = c - s * a.nv;
        }
        const size_t dsto = (size_t)s * a.ldv + a.voff + v;
        const size_t kstride = (size_t)a.S * a.ldv;
        const int j = cl >> 1;
        const bool odd = (cl & 1) != 0;
        const int kend = a.k0 + a.nf;                              // bins [k0, kend) are written
        for (int k1 = g; k1 < N1 && k1 < kend; k1 += G) {
            const int mk1 = (N1 - k1) & (N1 - 1);
            const float2* zr = z + F::zi(k1 * N2, j);              // rows k1 * N2 + k2
            const float2* zm = z + F::zi(mk1 * N2, j);             // rows mk1 * N2 + (...)
            int mrow2 = NT / N1 - (k1 > 0 ? 1 : 0);                // second index of the mirror row
            for (int k = k1, k2 = 0; k < kend; k += N1, ++k2, --mrow2) {
                if (k < a.k0) continue;
                const float2 Z = zr[k2 * F::RS];
                const float2 Zm = k == 0 ? Z : zm[(mrow2 & (N2 - 1)) * F::RS];
                float2 r = odd ? make_float2(hs * (Z.y + Zm.y), hs * (Zm.x - Z.x))
                               : make_float2(hs * (Z.x + Zm.x), hs * (Z.y - Zm.y));
                if (a.conj) r.y = -r.y;
                *MDC_AT(a.X, dsto + (size_t)(k - a.k0) * kstride, 1, (long long)a.nf * a.S * a.ldv, a.err, 17) = r;
            }
        }
    }
}

// Forward transform of the tile the inverse kernel leaves behind: storage row rho = t1 * N2 + t2
// holds time t = t1 + N1 t2 of P packed column pairs.  With k = k2 + N2 k1,
//   X[k] = sum_t1 W_N1^(t1 k1) [ W_NT^(t1 k2) sum_t2 W_N2^(t2 k2) x[t1 + N1 t2] ],
// so N2-point DFTs in each block t1, the twiddle, then N1-point DFTs over t1 leave bin k in row
// k1 * N2 + k2 = k (natural order).  The two columns of each pair are then separated as in the
// forward kernels (scale 1/2, optional conjugation) and bins [k0, k0 + nf) stored into fwd_X.
// tw: the inverse transform's half-period table, conjugated here.
template <int N1, int N2, int PP>
__device__ __forceinline__ void fused_forward(const IrfftArgs& a, float2* z, const float2* tw, int c0) {
    using F = FourStep<N1, N2, PP>;
    constexpr int NT = F::NT, CT = F::CT, P = F::P;
    for (int task = threadIdx.x; task < P * N1; task += FFT_THREADS) {
        const int j = task % P, t1 = task / P;
        float2 r[N2];
#pragma unroll
        for (int t2 = 0; t2 < N2; ++t2) r[t2] = z[F::zi(t1 * N2 + t2, j)];
        reg_fft<N2, false>(r);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2)
            z[F::zi(t1 * N2 + k2, j)] = k2 == 0 ? r[0] : cmul(r[k2], cconj(tw_full(tw, t1 * k2, NT)));
    }
    __syncthreads();
    for (int task = threadIdx.x; task < P * N2; task += FFT_THREADS) {
        const int j = task % P, k2 = task / P;
        float2 r[N1];
#pragma unroll
        for (int t1 = 0; t1 < N1; ++t1) r[t1] = z[F::zi(t1 * N2 + k2, j)];
        reg_fft<N1, false>(r);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) z[F::zi(k1 * N2 + k2, j)] = r[k1];
    }
    __syncthreads();
    constexpr int G = FFT_THREADS / CT;
    const int cl = threadIdx.x % CT, g = threadIdx.x / CT, c = c0 + cl;
    if (c >= a.C) return;
    int s, v;
    if ((a.nv % CT) == 0) {
        s = c0 / a.nv;
        v = c0 - s * a.nv + cl;
    } else {
        s = c / a.nv;
        v = c - s * a.nv;
    }
    const size_t dsto = (size_t)s * a.ldv + a.fwd_voff + v;
    const size_t kstride = (size_t)a.S * a.ldv;
    const int j = cl >> 1;
    const bool odd = (cl & 1) != 0;
    for (int kk = g; kk < a.nf; kk += G) {
        const int k = a.k0 + kk;
        const float2 Z = z[F::zi(k, j)];
        const float2 Zm = k == 0 ? Z : z[F::zi(NT - k, j)];
        float2 r = odd ? make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x))
                       : make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
        if (a.fwd_conj) r.y = -r.y;
        *MDC_AT(a.fwd_X, dsto + (size_t)kk * kstride, 1, (long long)a.nf * a.S * a.ldv, a.err, 18) = r;
    }
}

// MODE 1 (plain): the output is the transform alone (no window, base or previous-output terms,
// column sums or time reversal, a_mdc = 1); MODE 0: the general epilogue; MODE 2: the general
// epilogue with the LSQR x/w step of IrfftArgs fused in.  The inverse scale multiplies the
// spectrum as it is loaded.  FUSE (aligned path, MODES 0 and 2): the epilogue also keeps its
// outputs (windowed by fwd_cut) in the tile, and the kernel ends with their forward transform into
// fwd_X -- the transform the next product of an LSQR iteration needs, without reading the output
// back from memory.
template <int N1, int N2, int MODE, int PP, bool FUSE = false>
__global__ void __launch_bounds__(FFT_THREADS, MODE == 2 ? 2 : 3) irfft4_kernel(IrfftArgs a) {
    constexpr bool PLAIN = MODE == 1, XW = MODE == 2;
    static_assert(!(FUSE && PLAIN), "the fused forward transform follows the general epilogue");
    using F = FourStep<N1, N2, PP>;
    constexpr int NT = F::NT, CT = F::CT, P = F::P;
    if (a.active && *a.active == 0) return;
    extern __shared__ __align__(16) float2 sm2[];
    float2* tw = sm2;
    float2* z = sm2 + NT / 2;
    // column-sum reduction: on the consumed tile, or (FUSE: the tile is transformed again) after it
    double* red = reinterpret_cast<double*>(FUSE ? z + F::ZSIZE : z);
    const int c0 = blockIdx.x * CT;
    for (int i = threadIdx.x; i < NT / 2; i += FFT_THREADS) tw[i] = cconj(a.tw[i]);
    // rows no bin of the slab [k0, k0 + nf) reaches are zero (16-byte stores, P is even)
    const int kend = a.k0 + a.nf;
    for (int idx = threadIdx.x; idx < NT * (P / 2); idx += FFT_THREADS) {
        const int k = idx / (P / 2);
        const bool hit = (k >= a.k0 && k < kend) || (NT - k >= a.k0 && NT - k < kend);
        if (!hit) *reinterpret_cast<float4*>(z + F::zi(k, 2 * (idx % (P / 2)))) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float isc = a.scale;
    // Each loaded entry kk < nf (bin kb = k0 + kk) of the two columns fills Z[kb] and its
    // Hermitian mirror Z[NT - kb].  Every thread keeps one column pair j (FFT_THREADS is a
    // multiple of P), so its two spectrum columns are located once.
    {
        const int j = threadIdx.x % P, ca = c0 + 2 * j;
        const size_t kstride = (size_t)a.S * a.ldv;
        const float2* pa = nullptr;
        const float2* pb = nullptr;
        size_t paoff = 0, pboff = 0;
        if (ca < a.C) {
            const int sa = ca / a.nv, va = ca - sa * a.nv;
            paoff = (size_t)sa * a.ldv + a.voff + va;
            pa = a.Y + paoff;
            if (ca + 1 < a.C) {
                const int sb = (ca + 1) / a.nv, vb = ca + 1 - sb * a.nv;
                pboff = (size_t)sb * a.ldv + a.voff + vb;
                pb = a.Y + pboff;
            }
        }
        // both columns as one 16-byte load when they are adjacent and every row keeps the alignment
        const bool pair16 = pb == pa + 1 && ((uintptr_t)pa & 15) == 0 && (kstride & 1) == 0;
        constexpr int B = 4, STEP = FFT_THREADS / P;
#pragma unroll 1
        for (int kk0 = threadIdx.x / P; kk0 < a.nf; kk0 += B * STEP) {
            float2 A[B], Bv[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int kk = kk0 + u * STEP;
                A[u] = make_float2(0.f, 0.f);
                Bv[u] = A[u];
                if (kk < a.nf && pa) {
                    const size_t o = (size_t)kk * kstride;
                    if (pair16) {
                        const float4 q = *reinterpret_cast<const float4*>(MDC_AT(a.Y, paoff + o, 2, (long long)a.nf * a.S * a.ldv, a.err, 20));
                        A[u] = make_float2(q.x, q.y);
                        Bv[u] = make_float2(q.z, q.w);
                    } else {
                        A[u] = *MDC_AT(a.Y, paoff + o, 1, (long long)a.nf * a.S * a.ldv, a.err, 21);
                        if (pb) Bv[u] = *MDC_AT(a.Y, pboff + o, 1, (long long)a.nf * a.S * a.ldv, a.err, 22);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int kk = kk0 + u * STEP;
                if (kk >= a.nf) continue;
                const int kb = kk + a.k0;
                float2 Av = make_float2(isc * A[u].x, isc * A[u].y), Bw = make_float2(isc * Bv[u].x, isc * Bv[u].y);
                if (a.conj_in) { Av.y = -Av.y; Bw.y = -Bw.y; }
                if (kb == 0 || 2 * kb == NT) { Av.y = 0.f; Bw.y = 0.f; }
                z[F::zi(kb, j)] = make_float2(Av.x - Bw.y, Av.y + Bw.x);
                if (kb > 0 && 2 * kb < NT) z[F::zi(NT - kb, j)] = make_float2(Av.x + Bw.y, Bw.x - Av.y);
            }
        }
    }
    __syncthreads();
    four_step<N1, N2, true, false, PP>(z, tw);

    if constexpr (PLAIN) {
        // storage row rho holds time sample t = (rho % N2) * N1 + rho / N2
        if (a.vec4) {
            constexpr int Q = CT / 4, TS = FFT_THREADS / Q;
            const int q = threadIdx.x % Q, cq = c0 + 4 * q;
            if (cq < a.C) {
#pragma unroll 4
                for (int rho = threadIdx.x / Q; rho < NT; rho += TS) {
                    const int t = (rho % N2) * N1 + rho / N2;
                    *reinterpret_cast<float4*>(MDC_AT(a.out, (size_t)t * a.C + cq, 4, (long long)NT * a.C, a.err, 23)) =
                        *reinterpret_cast<const float4*>(z + F::zi(rho, 2 * q));
                }
            }
        } else {
            const int cl = threadIdx.x % CT, c = c0 + cl;
            if (c < a.C) {
                for (int rho = threadIdx.x / CT; rho < NT; rho += FFT_THREADS / CT) {
                    const int t = (rho % N2) * N1 + rho / N2;
                    const float2 zz = z[F::zi(rho, cl >> 1)];
                    *MDC_AT(a.out, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 24) = (cl & 1) ? zz.y : zz.x;
                }
            }
        }
        return;
    }
    const float am = coef(a.a_mdc), ab = coef(a.a_base), ap = coef(a.a_prev);
    const bool has_prev = (a.a_prev.h != 0.f) || (a.a_prev.d != nullptr);
    float xkx = 0.f, xkw = 0.f, xia = 0.f;
    if constexpr (XW) {
        xkx = (float)*a.xw_kx;
        xkw = (float)*a.xw_kw;
        xia = (float)*a.xw_ia;
    }
    if (a.vec4) {
        // four adjacent columns per thread: 16-byte loads and stores
        constexpr int Q = CT / 4, TS = FFT_THREADS / Q, PER = NT / TS, BB = XW ? 2 : 4, B = PER < BB ? PER : BB;
        const int q = threadIdx.x % Q, t0 = threadIdx.x / Q, cq = c0 + 4 * q;
        const bool want_ss = a.colsum != nullptr;
        float ss[4] = {0.f, 0.f, 0.f, 0.f};   // per-thread partial sums of squares (<= 16 terms)
        if (cq < a.C) {
            int cut[4], fcut[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                cut[i] = a.cut ? *MDC_AT(a.cut, cq + i, 1, a.C, a.err, 25) : 0x7fffffff;
                fcut[i] = (FUSE && a.fwd_cut) ? *MDC_AT(a.fwd_cut, cq + i, 1, a.C, a.err, 26) : 0x7fffffff;
            }
#pragma unroll 1
            for (int b0 = 0; b0 < PER; b0 += B) {
                // storage row rho holds time sample t = (rho % N2) * N1 + rho / N2
                float4 bv[B], pv[B], wv[XW ? B : 1], xv[XW ? B : 1];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int rho = t0 + (b0 + u) * TS;
                    const size_t o = (size_t)((rho % N2) * N1 + rho / N2) * a.C + cq;
                    bv[u] = a.base ? *reinterpret_cast<const float4*>(MDC_AT(a.base, o, 4, (long long)NT * a.C, a.err, 27))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    pv[u] = has_prev ? *reinterpret_cast<const float4*>(MDC_AT(a.out, o, 4, (long long)NT * a.C, a.err, 28))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                    if constexpr (XW) {
                        wv[u] = *reinterpret_cast<const float4*>(MDC_AT(a.xw_w, o, 4, (long long)NT * a.C, a.err, 29));
                        xv[u] = *reinterpret_cast<const float4*>(MDC_AT(a.xw_x, o, 4, (long long)NT * a.C, a.err, 30));
                    }
                }
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int rho = t0 + (b0 + u) * TS;
                    const int t = (rho % N2) * N1 + rho / N2;
                    const float4 zz = *reinterpret_cast<const float4*>(z + F::zi(rho, 2 * q));
                    const float2 z0 = make_float2(zz.x, zz.y), z1 = make_float2(zz.z, zz.w);
                    const int tau = t < (NT >> 1) ? t : NT - t;
                    float v[4] = {z0.x, z0.y, z1.x, z1.y};
                    const float bb[4] = {bv[u].x, bv[u].y, bv[u].z, bv[u].w};
                    const float pp[4] = {pv[u].x, pv[u].y, pv[u].z, pv[u].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float val = tau >= cut[i] ? 0.f : v[i];          // scale applied at load
                        v[i] = am * val + ab * bb[i] + ap * pp[i];
                        if (want_ss) ss[i] = fmaf(v[i], v[i], ss[i]);
                    }
                    const size_t o = (size_t)t * a.C + cq;
                    *reinterpret_cast<float4*>(MDC_AT(a.out, o, 4, (long long)NT * a.C, a.err, 31)) = make_float4(v[0], v[1], v[2], v[3]);
                    if constexpr (FUSE) {
                        // the same tile slot, windowed for the forward transform
                        *reinterpret_cast<float4*>(z + F::zi(rho, 2 * q)) =
                            make_float4(tau >= fcut[0] ? 0.f : v[0], tau >= fcut[1] ? 0.f : v[1],
                                        tau >= fcut[2] ? 0.f : v[2], tau >= fcut[3] ? 0.f : v[3]);
                    }
                    if constexpr (XW) {
                        const float ww[4] = {wv[u].x, wv[u].y, wv[u].z, wv[u].w};
                        const float xx[4] = {xv[u].x, xv[u].y, xv[u].z, xv[u].w};
                        float nw[4], nx[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            nx[i] = fmaf(xkx, ww[i], xx[i]);
                            nw[i] = fmaf(xkw, ww[i], xia * pp[i]);
                        }
                        *reinterpret_cast<float4*>(MDC_AT(a.xw_x, o, 4, (long long)NT * a.C, a.err, 32)) = make_float4(nx[0], nx[1], nx[2], nx[3]);
                        *reinterpret_cast<float4*>(MDC_AT(a.xw_w, o, 4, (long long)NT * a.C, a.err, 33)) = make_float4(nw[0], nw[1], nw[2], nw[3]);
                    }
                }
            }
        }
        if (a.colsum) {
            __syncthreads();                             // every thread is done reading the tile
#pragma unroll
            for (int i = 0; i < 4; ++i) red[4 * threadIdx.x + i] = (double)ss[i];
            __syncthreads();
            if (threadIdx.x < CT && c0 + (int)threadIdx.x < a.C) {
                const int qq = threadIdx.x / 4, ii = threadIdx.x % 4;
                double tot = 0.0;
                for (int tt = qq; tt < FFT_THREADS; tt += Q) tot += red[4 * tt + ii];
                *MDC_AT(a.colsum, c0 + threadIdx.x, 1, a.C, a.err, 34) = tot;
            }
        }
        if constexpr (FUSE) {
            __syncthreads();                             // every output is in the tile
            fused_forward<N1, N2, PP>(a, z, tw, c0);
        }
        return;
    }
    const int cl = threadIdx.x % CT, c = c0 + cl;
    const bool want_ss = a.colsum != nullptr;
    float ss = 0.f;   // per-thread partial sum of squares (<= 64 terms)
    if (c < a.C) {
        const int cut = a.cut ? *MDC_AT(a.cut, c, 1, a.C, a.err, 35) : 0x7fffffff;
        constexpr int TS = FFT_THREADS / CT, PER = NT / TS, B = PER < 8 ? PER : 8;
        const int t0 = threadIdx.x / CT;
#pragma unroll 1
        for (int b0 = 0; b0 < PER; b0 += B) {
            float bv[B], pv[B], wv[XW ? B : 1], xv[XW ? B : 1];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int rho = t0 + (b0 + u) * TS;
                const int t = (rho % N2) * N1 + rho / N2;
                const int to = a.reverse_out ? ((NT - t) & (NT - 1)) : t;
                bv[u] = a.base ? *MDC_AT(a.base, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 36) : 0.f;
                pv[u] = has_prev ? *MDC_AT(a.out, (size_t)to * a.C + c, 1, (long long)NT * a.C, a.err, 37) : 0.f;
                if constexpr (XW) {
                    wv[u] = *MDC_AT(a.xw_w, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 38);
                    xv[u] = *MDC_AT(a.xw_x, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 39);
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int rho = t0 + (b0 + u) * TS;
                const int t = (rho % N2) * N1 + rho / N2;
                const float2 zz = z[F::zi(rho, cl >> 1)];
                float val = (cl & 1) ? zz.y : zz.x;                      // scale applied at load
                const int tau = t < (NT >> 1) ? t : NT - t;
                if (tau >= cut) val = 0.f;
                const float r = am * val + ab * bv[u] + ap * pv[u];
                const int to = a.reverse_out ? ((NT - t) & (NT - 1)) : t;
                *MDC_AT(a.out, (size_t)to * a.C + c, 1, (long long)NT * a.C, a.err, 40) = r;
                if (want_ss) ss = fmaf(r, r, ss);
                if constexpr (XW) {
                    *MDC_AT(a.xw_x, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 41) = fmaf(xkx, wv[u], xv[u]);
                    *MDC_AT(a.xw_w, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 42) = fmaf(xkw, wv[u], xia * pv[u]);
                }
            }
        }
    }
    if (a.colsum) {
        __syncthreads();                                 // every thread is done reading the tile
        red[threadIdx.x] = (double)ss;
        __syncthreads();
        if (threadIdx.x < CT && c < a.C) {
            double tot = 0.0;
            for (int i = threadIdx.x; i < FFT_THREADS; i += CT) tot += red[i];
            *MDC_AT(a.colsum, c, 1, a.C, a.err, 10) = tot;
        }
    }
}

// ------------------------------------------------------------------ half-length real transforms
// nt = 2 * N1 * N2 (2048 with N1 = N2 = 32): one real column x per complex sequence
// z[n] = x[2n] + i x[2n+1] of length NC = nt / 2, transformed by the four-step DFT above.
// With E and O the spectra of the even and odd samples (period NC),
//   Z[k] = E[k] + i O[k],  E[k] = (Z[k] + conj Z[NC-k]) / 2,  O[k] = (Z[k] - conj Z[NC-k]) / (2i),
//   X[k] = E[k] + W_nt^k O[k]  (k < NC),   X[NC] = E[0] - O[0];
// the inverse builds Z[k] = (X[k] + conj X[NC-k]) + i (X[k] - conj X[NC-k]) W_nt^-k and takes the
// unnormalised inverse DFT of length NC, whose real and imaginary parts are nt times the even and
// odd samples.  A CTA holds P columns; the tile is the same as the nt = NC four-step kernels'.

template <int N1, int N2>
struct HalfStep {
    using F = FourStep<N1, N2>;
    static constexpr int NC = F::NT;               // complex length
    static constexpr int NT = 2 * NC;              // real length
    static constexpr int P = F::P;                 // columns per CTA
    // the tile only: the twiddles W_NC^m come from the plan's table (a.tw + NC, conjugates at
    // a.tw + 2 NC), read through L1
    static constexpr size_t smem = (size_t)F::ZSIZE * sizeof(float2);
};

template <int N1, int N2, bool WIN, bool X2>
__global__ void __launch_bounds__(FFT_THREADS, 2) rfft_half_kernel(RfftArgs a) {
    using H = HalfStep<N1, N2>;
    using F = typename H::F;
    constexpr int NC = H::NC, NT = H::NT, P = H::P;
    if (a.active && *a.active == 0) return;
    extern __shared__ __align__(16) float2 z[];
    const float2* __restrict__ twc = a.tw + NC;       // W_NC^m, m < NC
    const int c0 = blockIdx.x * P;
    // Pass A straight from global memory: task (j, n2) reads samples 2n and 2n + 1 of column
    // c0 + j for n = n1 * N2 + n2, applies the window, and transforms over n1 (the input scale
    // multiplies the split spectrum).
    for (int task = threadIdx.x; task < P * N2; task += FFT_THREADS) {
        const int j = task % P, n2 = task / P, c = c0 + j;
        float2 r[N1];
        if (c < a.C) {
            const size_t rstride = (size_t)2 * N2 * a.C;       // floats between n1 and n1 + 1
            const size_t xo = c + (size_t)2 * n2 * a.C;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1)
                r[n1] = make_float2(*MDC_AT(a.x, xo + n1 * rstride, 1, (long long)NT * a.C, a.err, 50),
                                    *MDC_AT(a.x, xo + n1 * rstride + a.C, 1, (long long)NT * a.C, a.err, 50));
            if constexpr (X2) {
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) {
                    r[n1].x += *MDC_AT(a.x2, xo + n1 * rstride, 1, (long long)NT * a.C, a.err, 51);
                    r[n1].y += *MDC_AT(a.x2, xo + n1 * rstride + a.C, 1, (long long)NT * a.C, a.err, 51);
                }
            }
            if constexpr (WIN) {
                const int cut = *MDC_AT(a.cut, c, 1, a.C, a.err, 52);
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) {
                    const int t = 2 * (n1 * N2 + n2);
                    const int tau0 = t < NC ? t : NT - t, tau1 = t + 1 < NC ? t + 1 : NT - t - 1;
                    if (tau0 >= cut) r[n1].x = 0.f;
                    if (tau1 >= cut) r[n1].y = 0.f;
                }
            }
        } else {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) r[n1] = make_float2(0.f, 0.f);
        }
        reg_fft<N1, false>(r);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) z[F::zi(k1 * N2 + n2, j)] = k1 == 0 ? r[0] : cmul(r[k1], twc[n2 * k1]);
    }
    __syncthreads();
    four_step_pass_b<N1, N2, false>(z);
    // Z[k] sits in row (k % N1) * N2 + k / N1.  Thread (cl, g) writes the bins k = k1 + N1 * k2 of
    // column c0 + cl for k1 = g, g + G, ...
    constexpr int G = FFT_THREADS / P;
    const int cl = threadIdx.x % P, g = threadIdx.x / P, c = c0 + cl;
    if (c >= a.C) return;
    const int s = c / a.nv, v = c - s * a.nv;
    const size_t dsto = (size_t)s * a.ldv + a.voff + v;
    const size_t kstride = (size_t)a.S * a.ldv;
    const float sc = coef(a.scale), hs = 0.5f * sc;
    const int kend = a.k0 + a.nf;                                  // bins [k0, kend) are written
    for (int k1 = g; k1 < N1 && k1 < kend; k1 += G) {
        for (int k = k1, k2 = 0; k < kend; k += N1, ++k2) {
            if (k < a.k0) continue;
            float2 X;
            if (k >= NC) {                                     // Nyquist bin k = NC
                const float2 Z0 = z[F::zi(0, cl)];
                X = make_float2(sc * (Z0.x - Z0.y), 0.f);
            } else {
                const float2 Z = z[F::zi(k1 * N2 + k2, cl)];
                const int km = (NC - k) & (NC - 1);
                const float2 Zm = z[F::zi((km % N1) * N2 + km / N1, cl)];
                const float2 E = make_float2(hs * (Z.x + Zm.x), hs * (Z.y - Zm.y));
                const float2 O = make_float2(hs * (Z.y + Zm.y), hs * (Zm.x - Z.x));
                X = cadd(E, cmul(O, a.tw[k]));
            }
            if (a.conj) X.y = -X.y;
            *MDC_AT(a.X, dsto + (size_t)(k - a.k0) * kstride, 1, (long long)a.nf * a.S * a.ldv, a.err, 53) = X;
        }
    }
}

// Forward half-length transform of the tile the inverse kernel leaves behind: row rho = t1 * N2 + t2
// holds z[n] = x[2n] + i x[2n+1], n = t1 + N1 t2, of column j.  The NC-point DFT in the order of
// fused_forward (N2-point DFTs, twiddle W_NC^(t1 k2), N1-point DFTs) leaves Z[k] in row k; the
// even/odd split then gives X[k] = E[k] + W_nt^k O[k] (k < NC), X[NC] = E[0] - O[0], as in
// rfft_half_kernel (unscaled, optional conjugation), stored into fwd_X for bins [k0, k0 + nf).
template <int N1, int N2>
__device__ __forceinline__ void fused_forward_half(const IrfftArgs& a, float2* z, int c0) {
    using H = HalfStep<N1, N2>;
    using F = typename H::F;
    constexpr int NC = H::NC, P = H::P;
    const float2* __restrict__ twc = a.tw + NC;           // W_NC^m, m < NC
    for (int task = threadIdx.x; task < P * N1; task += FFT_THREADS) {
        const int j = task % P, t1 = task / P;
        float2 r[N2];
#pragma unroll
        for (int t2 = 0; t2 < N2; ++t2) r[t2] = z[F::zi(t1 * N2 + t2, j)];
        reg_fft<N2, false>(r);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) z[F::zi(t1 * N2 + k2, j)] = k2 == 0 ? r[0] : cmul(r[k2], twc[t1 * k2]);
    }
    __syncthreads();
    for (int task = threadIdx.x; task < P * N2; task += FFT_THREADS) {
        const int j = task % P, k2 = task / P;
        float2 r[N1];
#pragma unroll
        for (int t1 = 0; t1 < N1; ++t1) r[t1] = z[F::zi(t1 * N2 + k2, j)];
        reg_fft<N1, false>(r);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) z[F::zi(k1 * N2 + k2, j)] = r[k1];
    }
    __syncthreads();
    constexpr int G = FFT_THREADS / P;
    const int cl = threadIdx.x % P, g = threadIdx.x / P, c = c0 + cl;
    if (c >= a.C) return;
    const int s = c / a.nv, v = c - s * a.nv;
    const size_t dsto = (size_t)s * a.ldv + a.fwd_voff + v;
    const size_t kstride = (size_t)a.S * a.ldv;
    for (int kk = g; kk < a.nf; kk += G) {
        const int k = a.k0 + kk;
        float2 X;
        if (k >= NC) {                                        // Nyquist bin k = NC
            const float2 Z0 = z[F::zi(0, cl)];
            X = make_float2(Z0.x - Z0.y, 0.f);
        } else {
            const float2 Z = z[F::zi(k, cl)];
            const float2 Zm = z[F::zi((NC - k) & (NC - 1), cl)];
            const float2 E = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
            const float2 O = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
            X = cadd(E, cmul(O, a.tw[k]));
        }
        if (a.fwd_conj) X.y = -X.y;
        *MDC_AT(a.fwd_X, dsto + (size_t)kk * kstride, 1, (long long)a.nf * a.S * a.ldv, a.err, 54) = X;
    }
}

// FUSE (aligned general path): the epilogue keeps its outputs (windowed by fwd_cut) in the tile as
// z[n] = x[2n] + i x[2n+1], and the kernel ends with their forward half-length transform into fwd_X.
template <int N1, int N2, bool PLAIN, bool FUSE = false>
__global__ void __launch_bounds__(FFT_THREADS, PLAIN ? 3 : 2) irfft_half_kernel(IrfftArgs a) {
    static_assert(!(FUSE && PLAIN), "the fused forward transform follows the general epilogue");
    using H = HalfStep<N1, N2>;
    using F = typename H::F;
    constexpr int NC = H::NC, NT = H::NT, P = H::P;
    if (a.active && *a.active == 0) return;
    extern __shared__ __align__(16) float2 z[];
    // column-sum reduction: on the consumed tile, or (FUSE: the tile is transformed again) after it
    double* red = reinterpret_cast<double*>(FUSE ? z + F::ZSIZE : z);
    const float2* __restrict__ twc = a.tw + 2 * NC;   // conj W_NC^m, m < NC
    const int c0 = blockIdx.x * P;
    // Item (kk, j), kk <= NC / 2, reads X[kk] and X[NC - kk] of column c0 + j and writes Z[kk]
    // and Z[NC - kk]; bins outside the band are zero, DC and Nyquist lose their imaginary parts.
    // Every thread keeps one column j (FFT_THREADS is a multiple of P).
    {
        constexpr int KK = NC / 2 + 1, BL = 4, STEP = FFT_THREADS / P;
        const size_t kstride = (size_t)a.S * a.ldv;
        const int j = threadIdx.x % P, c = c0 + j, kend = a.k0 + a.nf;
        const float2* col = nullptr;
        size_t colo = 0;
        if (c < a.C) {
            const int sp = c / a.nv, vp = c - sp * a.nv;
            colo = (size_t)sp * a.ldv + a.voff + vp;
            col = a.Y + colo;
        }
#pragma unroll 1
        for (int kk0 = threadIdx.x / P; kk0 < KK; kk0 += BL * STEP) {
          float2 Al[BL], Bl[BL];
#pragma unroll
          for (int u = 0; u < BL; ++u) {                 // loads first, BL items in flight
            const int kk = kk0 + u * STEP;
            Al[u] = make_float2(0.f, 0.f);
            Bl[u] = Al[u];
            if (kk < KK && col) {
                if (kk >= a.k0 && kk < kend) Al[u] = *MDC_AT(a.Y, colo + (size_t)(kk - a.k0) * kstride, 1, (long long)a.nf * a.S * a.ldv, a.err, 55);
                if (NC - kk >= a.k0 && NC - kk < kend)
                    Bl[u] = *MDC_AT(a.Y, colo + (size_t)(NC - kk - a.k0) * kstride, 1, (long long)a.nf * a.S * a.ldv, a.err, 56);
            }
          }
#pragma unroll
          for (int u = 0; u < BL; ++u) {
            const int kk = kk0 + u * STEP;
            if (kk >= KK) continue;
            float2 A = make_float2(a.scale * Al[u].x, a.scale * Al[u].y);      // inverse scale at load
            float2 B = make_float2(a.scale * Bl[u].x, a.scale * Bl[u].y);
            if (a.conj_in) { A.y = -A.y; B.y = -B.y; }
            if (kk == 0) { A.y = 0.f; B.y = 0.f; }
            // E = A + conj B, O = (A - conj B) W_nt^-kk; the mirror NC - kk has E' = conj E and
            // O' = (conj A - B) W_nt^-(NC-kk) = (A - conj B)^* W_nt^kk.  Z goes in natural order.
            const float2 w = a.tw[kk < NC ? kk : 0];
            const float2 E = make_float2(A.x + B.x, A.y - B.y);
            const float2 D = make_float2(A.x - B.x, A.y + B.y);
            const float2 O = cmul(D, cconj(w));
            z[F::zi(kk, j)] = make_float2(E.x - O.y, E.y + O.x);
            if (kk > 0 && 2 * kk < NC) {
                const float2 Om = cmul(make_float2(D.x, -D.y), w);
                z[F::zi(NC - kk, j)] = make_float2(E.x - Om.y, -E.y + Om.x);
            }
          }
        }
    }
    __syncthreads();
    four_step<N1, N2, true, true>(z, twc);

    // Row rho holds complex sample n = (rho % N2) * N1 + rho / N2, i.e. real samples 2n (real
    // part) and 2n + 1 (imaginary part).
    if constexpr (PLAIN) {
        if (a.vec4) {
            constexpr int Q = P / 4, TSQ = FFT_THREADS / Q;
            const int q = threadIdx.x % Q, cq = c0 + 4 * q;
            if (cq < a.C) {
#pragma unroll 4
                for (int rho = threadIdx.x / Q; rho < NC; rho += TSQ) {
                    const int n = (rho % N2) * N1 + rho / N2;
                    const float4 z01 = *reinterpret_cast<const float4*>(z + F::zi(rho, 4 * q));
                    const float4 z23 = *reinterpret_cast<const float4*>(z + F::zi(rho, 4 * q + 2));
                    *reinterpret_cast<float4*>(MDC_AT(a.out, (size_t)(2 * n) * a.C + cq, 4, (long long)NT * a.C, a.err, 57)) =
                        make_float4(z01.x, z01.z, z23.x, z23.z);
                    *reinterpret_cast<float4*>(MDC_AT(a.out, (size_t)(2 * n + 1) * a.C + cq, 4, (long long)NT * a.C, a.err, 57)) =
                        make_float4(z01.y, z01.w, z23.y, z23.w);
                }
            }
        } else {
            const int cl = threadIdx.x % P, c = c0 + cl;
            if (c < a.C) {
                for (int rho = threadIdx.x / P; rho < NC; rho += FFT_THREADS / P) {
                    const int n = (rho % N2) * N1 + rho / N2;
                    const float2 zz = z[F::zi(rho, cl)];
                    *MDC_AT(a.out, (size_t)(2 * n) * a.C + c, 1, (long long)NT * a.C, a.err, 58) = zz.x;
                    *MDC_AT(a.out, (size_t)(2 * n + 1) * a.C + c, 1, (long long)NT * a.C, a.err, 58) = zz.y;
                }
            }
        }
        return;
    }
    const float am = coef(a.a_mdc), ab = coef(a.a_base), ap = coef(a.a_prev);
    const bool has_prev = (a.a_prev.h != 0.f) || (a.a_prev.d != nullptr);
    const bool want_ss = a.colsum != nullptr;
    if (a.vec4) {
        // four adjacent columns per thread (16-byte loads and stores), BQ rows of samples in flight
        constexpr int Q = P / 4, TSQ = FFT_THREADS / Q, PERQ = NC / TSQ, BQ = PERQ < 4 ? PERQ : 4;
        const int q = threadIdx.x % Q, t0 = threadIdx.x / Q, cq = c0 + 4 * q;
        float ss[4] = {0.f, 0.f, 0.f, 0.f};
        if (cq < a.C) {
            int cut[4], fcut[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                cut[i] = a.cut ? *MDC_AT(a.cut, cq + i, 1, a.C, a.err, 25) : 0x7fffffff;
                fcut[i] = (FUSE && a.fwd_cut) ? *MDC_AT(a.fwd_cut, cq + i, 1, a.C, a.err, 26) : 0x7fffffff;
            }
#pragma unroll 1
            for (int b0 = 0; b0 < PERQ; b0 += BQ) {
                float4 bv[BQ][2], pv[BQ][2];
#pragma unroll
                for (int u = 0; u < BQ; ++u) {
                    const int rho = t0 + (b0 + u) * TSQ;
                    const int n = (rho % N2) * N1 + rho / N2;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const size_t o = (size_t)(2 * n + h) * a.C + cq;
                        bv[u][h] = a.base ? *reinterpret_cast<const float4*>(MDC_AT(a.base, o, 4, (long long)NT * a.C, a.err, 59))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                        pv[u][h] = has_prev ? *reinterpret_cast<const float4*>(MDC_AT(a.out, o, 4, (long long)NT * a.C, a.err, 60))
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < BQ; ++u) {
                    const int rho = t0 + (b0 + u) * TSQ;
                    const int n = (rho % N2) * N1 + rho / N2;
                    const float4 z01 = *reinterpret_cast<const float4*>(z + F::zi(rho, 4 * q));
                    const float4 z23 = *reinterpret_cast<const float4*>(z + F::zi(rho, 4 * q + 2));
                    const float re[4] = {z01.x, z01.z, z23.x, z23.z}, im[4] = {z01.y, z01.w, z23.y, z23.w};
                    float vw[2][4];                  // (FUSE) the outputs, windowed for the forward transform
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = 2 * n + h;
                        const int tau = t < NC ? t : NT - t;
                        const float bb[4] = {bv[u][h].x, bv[u][h].y, bv[u][h].z, bv[u][h].w};
                        const float pp[4] = {pv[u][h].x, pv[u][h].y, pv[u][h].z, pv[u][h].w};
                        float v[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float val = tau >= cut[i] ? 0.f : (h ? im[i] : re[i]);
                            v[i] = am * val + ab * bb[i] + ap * pp[i];
                            if (want_ss) ss[i] = fmaf(v[i], v[i], ss[i]);
                            vw[h][i] = tau >= fcut[i] ? 0.f : v[i];
                        }
                        *reinterpret_cast<float4*>(MDC_AT(a.out, (size_t)t * a.C + cq, 4, (long long)NT * a.C, a.err, 61)) =
                            make_float4(v[0], v[1], v[2], v[3]);
                    }
                    if constexpr (FUSE) {
                        *reinterpret_cast<float4*>(z + F::zi(rho, 4 * q)) =
                            make_float4(vw[0][0], vw[1][0], vw[0][1], vw[1][1]);
                        *reinterpret_cast<float4*>(z + F::zi(rho, 4 * q + 2)) =
                            make_float4(vw[0][2], vw[1][2], vw[0][3], vw[1][3]);
                    }
                }
            }
        }
        if (a.colsum) {
            __syncthreads();                             // every thread is done reading the tile
#pragma unroll
            for (int i = 0; i < 4; ++i) red[4 * threadIdx.x + i] = (double)ss[i];
            __syncthreads();
            if (threadIdx.x < P && c0 + (int)threadIdx.x < a.C) {
                const int qq = threadIdx.x / 4, ii = threadIdx.x % 4;
                double tot = 0.0;
                for (int tt = qq; tt < FFT_THREADS; tt += Q) tot += red[4 * tt + ii];
                *MDC_AT(a.colsum, c0 + threadIdx.x, 1, a.C, a.err, 34) = tot;
            }
        }
        if constexpr (FUSE) {
            __syncthreads();                             // every output is in the tile
            fused_forward_half<N1, N2>(a, z, c0);
        }
        return;
    }
    constexpr int TS = FFT_THREADS / P, PER = NC / TS, BS = PER < 8 ? PER : 8;
    const int cl = threadIdx.x % P, t0 = threadIdx.x / P, c = c0 + cl;
    float ss = 0.f;
    if (c < a.C) {
        const int cut = a.cut ? *MDC_AT(a.cut, c, 1, a.C, a.err, 62) : 0x7fffffff;
#pragma unroll 1
        for (int b0 = 0; b0 < PER; b0 += BS) {
            float bv[BS][2], pv[BS][2];
#pragma unroll
            for (int u = 0; u < BS; ++u) {
                const int rho = t0 + (b0 + u) * TS;
                const int n = (rho % N2) * N1 + rho / N2;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t = 2 * n + h;
                    const int to = a.reverse_out ? ((NT - t) & (NT - 1)) : t;
                    bv[u][h] = a.base ? *MDC_AT(a.base, (size_t)t * a.C + c, 1, (long long)NT * a.C, a.err, 63) : 0.f;
                    pv[u][h] = has_prev ? *MDC_AT(a.out, (size_t)to * a.C + c, 1, (long long)NT * a.C, a.err, 64) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < BS; ++u) {
                const int rho = t0 + (b0 + u) * TS;
                const int n = (rho % N2) * N1 + rho / N2;
                const float2 zz = z[F::zi(rho, cl)];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t = 2 * n + h;
                    const int tau = t < NC ? t : NT - t;
                    float val = h ? zz.y : zz.x;
                    if (tau >= cut) val = 0.f;
                    const int to = a.reverse_out ? ((NT - t) & (NT - 1)) : t;
                    const float r = am * val + ab * bv[u][h] + ap * pv[u][h];
                    *MDC_AT(a.out, (size_t)to * a.C + c, 1, (long long)NT * a.C, a.err, 65) = r;
                    if (want_ss) ss = fmaf(r, r, ss);
                }
            }
        }
    }
    if (a.colsum) {
        __syncthreads();                                 // every thread is done reading the tile
        red[threadIdx.x] = (double)ss;
        __syncthreads();
        if (threadIdx.x < P && c < a.C) {
            double tot = 0.0;
            for (int i = threadIdx.x; i < FFT_THREADS; i += P) tot += red[i];
            *MDC_AT(a.colsum, c, 1, a.C, a.err, 66) = tot;
        }
    }
}

// The transform alone: no window, base or previous-output terms, column sums or reversal.
inline bool irfft_plain(const IrfftArgs& a) {
    return !a.cut && !a.base && !a.colsum && !a.reverse_out && a.a_mdc.h == 1.f && !a.a_mdc.d &&
           a.a_prev.h == 0.f && !a.a_prev.d && !a.xw_w && !a.fwd_X;
}

template <int N1, int N2, bool WIN, bool X2>
void rfft_half_go(mdc_plan* p, const RfftArgs& a, cudaStream_t s) {
    using H = HalfStep<N1, N2>;
    static SmemLimit attr;
    attr.ensure(rfft_half_kernel<N1, N2, WIN, X2>, (int)H::smem);
    LaunchScope ls(p, s, MDC_KC_RFFT);
    rfft_half_kernel<N1, N2, WIN, X2><<<(a.C + H::P - 1) / H::P, FFT_THREADS, H::smem, s>>>(a);
}

template <int N1, int N2, bool PLAIN, bool FUSE = false>
void irfft_half_go(mdc_plan* p, const IrfftArgs& a, cudaStream_t s) {
    using H = HalfStep<N1, N2>;
    // FUSE: the column-sum reduction buffer follows the tile
    constexpr size_t smem = H::smem + (FUSE ? (size_t)FFT_THREADS * 4 * sizeof(double) : 0);
    static SmemLimit attr;
    attr.ensure(irfft_half_kernel<N1, N2, PLAIN, FUSE>, (int)smem);
    LaunchScope ls(p, s, MDC_KC_IRFFT);
    irfft_half_kernel<N1, N2, PLAIN, FUSE><<<(a.C + H::P - 1) / H::P, FFT_THREADS, smem, s>>>(a);
}

template <int N1, int N2>
void rfft_half_launch(mdc_plan* p, const RfftArgs& a, cudaStream_t s) {
    if (a.cut) {
        if (a.x2) rfft_half_go<N1, N2, true, true>(p, a, s);
        else rfft_half_go<N1, N2, true, false>(p, a, s);
    } else {
        if (a.x2) rfft_half_go<N1, N2, false, true>(p, a, s);
        else rfft_half_go<N1, N2, false, false>(p, a, s);
    }
}

// Returns true if the kernel also made the forward transform of IrfftArgs::fwd_X.
template <int N1, int N2>
bool irfft_half_launch(mdc_plan* p, const IrfftArgs& a0, cudaStream_t s) {
    IrfftArgs a = a0;
    a.vec4 = (a.C % 4 == 0) && !a.reverse_out && ((uintptr_t)a.out % 16 == 0) &&
             (!a.base || (uintptr_t)a.base % 16 == 0);
    const bool fuse = a.fwd_X && a.vec4;
    if (irfft_plain(a)) irfft_half_go<N1, N2, true>(p, a, s);
    else if (fuse) irfft_half_go<N1, N2, false, true>(p, a, s);
    else irfft_half_go<N1, N2, false>(p, a, s);
    return fuse;
}

template <int N1, int N2, bool WIN, bool X2, int PP>
void rfft4_go(mdc_plan* p, const RfftArgs& a, cudaStream_t s) {
    using F = FourStep<N1, N2, PP>;
    static SmemLimit attr;
    attr.ensure(rfft4_kernel<N1, N2, WIN, X2, PP>, (int)F::smem_full);
    LaunchScope ls(p, s, MDC_KC_RFFT);
    rfft4_kernel<N1, N2, WIN, X2, PP><<<(a.C + F::CT - 1) / F::CT, FFT_THREADS, F::smem_full, s>>>(a);
}

// Few columns: the default tile would leave most SMs idle (fewer CTAs than half the SMs); smaller
// tiles then shorten each CTA's work.  (With one or more default CTAs per SM the smaller tiles only
// add waves: measured slower at 3721 columns of 1024 samples.)
template <int N1, int N2>
constexpr int few_cols_p() { return 1024 / (N1 * N2) > 2 ? 1024 / (N1 * N2) : 2; }
inline bool few_columns(int C, int ct) { return (C + ct - 1) / ct < 148 / 2; }

template <int N1, int N2>
void rfft4_launch(mdc_plan* p, const RfftArgs& a0, cudaStream_t s) {
    RfftArgs a = a0;
    a.vec4 = (a.C % 4 == 0) && ((uintptr_t)a.x % 16 == 0) && (!a.x2 || (uintptr_t)a.x2 % 16 == 0);
    constexpr int PS = few_cols_p<N1, N2>();
    const bool few = few_columns(a.C, FourStep<N1, N2>::CT) && PS < FourStep<N1, N2>::P;
    if (a.cut) {
        if (a.x2) rfft4_go<N1, N2, true, true, 0>(p, a, s);
        else rfft4_go<N1, N2, true, false, 0>(p, a, s);
    } else if (a.x2) {
        rfft4_go<N1, N2, false, true, 0>(p, a, s);
    } else if (few) {
        rfft4_go<N1, N2, false, false, PS>(p, a, s);
    } else {
        rfft4_go<N1, N2, false, false, 0>(p, a, s);
    }
}

template <int N1, int N2, int MODE, int PP, bool FUSE = false>
void irfft4_go(mdc_plan* p, const IrfftArgs& a, cudaStream_t s) {
    using F = FourStep<N1, N2, PP>;
    // FUSE: the column-sum reduction buffer follows the tile
    constexpr size_t smem = F::smem + (FUSE ? (size_t)FFT_THREADS * 4 * sizeof(double) : 0);
    static SmemLimit attr;
    attr.ensure(irfft4_kernel<N1, N2, MODE, PP, FUSE>, (int)smem);
    LaunchScope ls(p, s, MDC_KC_IRFFT);
    irfft4_kernel<N1, N2, MODE, PP, FUSE><<<(a.C + F::CT - 1) / F::CT, FFT_THREADS, smem, s>>>(a);
}

// Returns true if the kernel also made the forward transform of IrfftArgs::fwd_X.
template <int N1, int N2>
bool irfft4_launch(mdc_plan* p, const IrfftArgs& a0, cudaStream_t s) {
    IrfftArgs a = a0;
    a.vec4 = (a.C % 4 == 0) && !a.reverse_out && ((uintptr_t)a.out % 16 == 0) &&
             (!a.base || (uintptr_t)a.base % 16 == 0) &&
             (!a.xw_w || ((uintptr_t)a.xw_w % 16 == 0 && (uintptr_t)a.xw_x % 16 == 0));
    constexpr int PS = few_cols_p<N1, N2>();
    const bool few = few_columns(a.C, FourStep<N1, N2>::CT) && PS < FourStep<N1, N2>::P;
    const bool fuse = a.fwd_X && a.vec4 && !a.reverse_out;
    if (irfft_plain(a)) {
        if (few) irfft4_go<N1, N2, 1, PS>(p, a, s);
        else irfft4_go<N1, N2, 1, 0>(p, a, s);
    } else if (a.xw_w) {
        if (fuse) irfft4_go<N1, N2, 2, 0, true>(p, a, s);
        else irfft4_go<N1, N2, 2, 0>(p, a, s);
    } else {
        if (fuse) irfft4_go<N1, N2, 0, 0, true>(p, a, s);
        else irfft4_go<N1, N2, 0, 0>(p, a, s);
    }
    return fuse;
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

void launch_rfft(mdc_plan* p, const RfftArgs& a0, cudaStream_t s) {
    RfftArgs a = a0;
    a.err = p->err_flag;
    switch (a.nt) {
        case 64: rfft4_launch<8, 8>(p, a, s); return;
        case 128: rfft4_launch<16, 8>(p, a, s); return;
        case 256: rfft4_launch<16, 16>(p, a, s); return;
        case 512: rfft4_launch<32, 16>(p, a, s); return;
        case 1024: rfft4_launch<32, 32>(p, a, s); return;
        case 2048: rfft_half_launch<32, 32>(p, a, s); return;
        default: break;
    }
    const int logCT = tile_log_columns(a.nt);
    const size_t smem = rfft_smem(a.nt, logCT);
    static SmemLimit attr_set;
    attr_set.ensure(rfft_kernel, 200 * 1024);
    const int grid = (a.C + (1 << logCT) - 1) >> logCT;
    LaunchScope ls(p, s, MDC_KC_RFFT);
    rfft_kernel<<<grid, FFT_THREADS, smem, s>>>(a, logCT);
}

namespace {

bool launch_irfft_local(mdc_plan* p, const IrfftArgs& a, cudaStream_t s);

// The forward transform IrfftArgs::fwd_X asks for, as its own launch on the finished output.
void forward_of_output(mdc_plan* p, const IrfftArgs& a, cudaStream_t s) {
    RfftArgs r{};
    r.x = a.out;
    r.C = a.C; r.S = a.S; r.nv = a.nv; r.nt = a.nt; r.logn = a.logn; r.nf = a.nf; r.k0 = a.k0;
    r.cut = a.fwd_cut; r.scale = C1(1.f); r.conj = a.fwd_conj;
    r.X = a.fwd_X; r.ldv = a.ldv; r.voff = a.fwd_voff;
    r.tw = a.tw; r.active = a.active;
    launch_rfft(p, r, s);
}

// Epilogue of a frequency shard's inverse transform, run on T = the partial transforms summed over
// every shard (so the same signal on every shard): out = a_mdc Theta T + a_base base + a_prev out,
// optionally written time-reversed, with per-column sums of squares -- the terms the local
// kernels fuse into their own epilogue, which cannot be applied to a partial sum.
__global__ void __launch_bounds__(256) shard_epilogue(IrfftArgs a, const float* __restrict__ T) {
    if (a.active && *a.active == 0) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const float am = coef(a.a_mdc), ab = coef(a.a_base), ap = coef(a.a_prev);
    const bool has_prev = (a.a_prev.h != 0.f) || (a.a_prev.d != nullptr);
    double ss = 0.0;
    if (c < a.C) {
        const int cut = a.cut ? *MDC_AT(a.cut, c, 1, a.C, a.err, 70) : 0x7fffffff;
        [[maybe_unused]] const long long nx = (long long)a.nt * a.C;
        for (int t = ty; t < a.nt; t += 8) {
            const int tau = t < (a.nt >> 1) ? t : a.nt - t;
            const float val = tau >= cut ? 0.f : *MDC_AT(T, (size_t)t * a.C + c, 1, nx, a.err, 71);
            float r = am * val;
            if (a.base) r += ab * *MDC_AT(a.base, (size_t)t * a.C + c, 1, nx, a.err, 72);
            const int to = a.reverse_out ? ((a.nt - t) & (a.nt - 1)) : t;
            const size_t o = (size_t)to * a.C + c;
            if (has_prev) r += ap * *MDC_AT(a.out, o, 1, nx, a.err, 73);
            *MDC_AT(a.out, o, 1, nx, a.err, 74) = r;
            ss += (double)r * (double)r;
        }
    }
    if (a.colsum) {
        __shared__ double red[256];
        red[threadIdx.x] = ss;
        __syncthreads();
        if (ty == 0 && c < a.C) {
            double tot = 0.0;
            for (int i = 0; i < 8; ++i) tot += red[32 * i + tx];
            *MDC_AT(a.colsum, c, 1, a.C, a.err, 75) = tot;
        }
    }
}

}  // namespace

namespace {
// The LSQR x/w step of IrfftArgs on its own, for the transforms that do not fuse it: run before the
// transform overwrites its previous output v.  Same rounding as the fused form.
__global__ void xw_step(int64_t n, float* __restrict__ x, float* __restrict__ w, const float* __restrict__ v,
                        const double* kx, const double* kw, const double* ia, const int* active) {
    if (active && *active == 0) return;
    const float fx = (float)*kx, fw = (float)*kw, fa = (float)*ia;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float wo = w[i];
        x[i] = fmaf(fx, wo, x[i]);
        w[i] = fmaf(fw, wo, fa * v[i]);
    }
}

// The inverse transforms that fuse the LSQR x/w step: the four-step kernels (nt <= 1024).
inline bool irfft_fuses_xw(const IrfftArgs& a) { return a.nt <= 1024 && !a.reverse_out; }
}  // namespace

void launch_irfft(mdc_plan* p, const IrfftArgs& a0, cudaStream_t s) {
    IrfftArgs a = a0;
    a.err = p->err_flag;
    if (a.xw_w && (p->red_fn || !irfft_fuses_xw(a))) {
        const int64_t n = (int64_t)a.nt * a.C;
        int64_t g = (n + 255) / 256;
        if (g > 152 * 16) g = 152 * 16;
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        xw_step<<<(unsigned)g, 256, 0, s>>>(n, a.xw_x, a.xw_w, a.out, a.xw_kx, a.xw_kw, a.xw_ia, a.active);
        a.xw_x = a.xw_w = nullptr;
    }
    if (!p->red_fn) {
        if (!launch_irfft_local(p, a, s) && a.fwd_X) forward_of_output(p, a, s);
        return;
    }
    const int64_t count = (int64_t)a.nt * a.C;
    if (count > p->red_cap) {
        float* b = nullptr;
        const cudaError_t e = cudaMalloc(&b, (size_t)count * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_cuda_error(e);
            if (!p->host_error) p->host_error = MDC_ERR_OOM;
            return;
        }
        cudaStreamSynchronize(s);            // nothing in flight still uses the old buffer
        cudaFree(p->red_buf);
        p->red_buf = b;
        p->red_cap = count;
    }
    IrfftArgs part = a;                      // this shard's bins only, no epilogue terms
    part.out = p->red_buf;
    part.a_mdc = C1(1.f);
    part.a_base = C1(0.f);
    part.a_prev = C1(0.f);
    part.base = nullptr;
    part.cut = nullptr;
    part.reverse_out = 0;
    part.colsum = nullptr;
    part.fwd_X = nullptr;
    launch_irfft_local(p, part, s);
    const int st = p->red_fn(p->red_buf, count, (void*)s, p->red_ctx);
    if (st != MDC_OK && !p->host_error) p->host_error = st < 0 ? st : MDC_ERR_STATE;
    {
        LaunchScope ls(p, s, MDC_KC_IRFFT);
        shard_epilogue<<<(unsigned)((a.C + 31) / 32), 256, 0, s>>>(a, p->red_buf);
    }
    if (a.fwd_X) forward_of_output(p, a, s);
}

namespace {

bool launch_irfft_local(mdc_plan* p, const IrfftArgs& a, cudaStream_t s) {
    switch (a.nt) {
        case 64: return irfft4_launch<8, 8>(p, a, s);
        case 128: return irfft4_launch<16, 8>(p, a, s);
        case 256: return irfft4_launch<16, 16>(p, a, s);
        case 512: return irfft4_launch<32, 16>(p, a, s);
        case 1024: return irfft4_launch<32, 32>(p, a, s);
        case 2048: return irfft_half_launch<32, 32>(p, a, s);
        default: break;
    }
    const int logCT = tile_log_columns(a.nt);
    const size_t smem = irfft_smem(a.nt, logCT);
    static SmemLimit attr_set;
    attr_set.ensure(irfft_kernel, 200 * 1024);
    const int grid = (a.C + (1 << logCT) - 1) >> logCT;
    LaunchScope ls(p, s, MDC_KC_IRFFT);
    irfft_kernel<<<grid, FFT_THREADS, smem, s>>>(a, logCT);
    return false;
}

}  // namespace

}  // namespace mdc
