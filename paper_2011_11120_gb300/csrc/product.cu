// Per-frequency products with the kernel: K-hat and K-hat^H of Eq. 3, the batch of
// dense frequency slices of Eq. 4.  The kernel copy is [nf][nr][ldg] complex64 with
// ldg a multiple of 64 (zero padded), so every row is 512-byte aligned and read as
// whole 16-byte vectors (two complex numbers).
//
// Few columns (GEMV regime, bound by streaming G from HBM):
//   forward  one warp per kernel row; lanes stride the row with 16-byte loads and
//            the dot products are finished with warp shuffles.  X(w) sits in shared
//            memory for the whole CTA.
//   adjoint  the same buffer read transposed: a CTA owns 64 adjacent columns s of
//            one frequency, each warp walks a subset of rows r reading the 512-byte
//            row segment, and the per-warp partial sums meet in shared memory.
//            No atomics, no second copy of G.
// Many columns (GEMM regime): a tiled FP32 complex GEMM (64x64 complex tile per
// CTA, 4x4 per thread), the adjoint tile loader conjugating and transposing.
#include "common.cuh"
#include <cstdlib>

namespace mdc {

// Largest column count served by the GEMV kernels.
int gemv_max_columns() { return 4; }

namespace {

constexpr int GEMV_THREADS = 256;
constexpr int FWD_ROWS_PER_CTA = 64;

// Storage formats of the kernel copy: complex values per 16-byte vector and decoding.
template <int FMT> struct Fmt;
template <> struct Fmt<MDC_C64> { static constexpr int CPV = 2; };
template <> struct Fmt<MDC_C16F> { static constexpr int CPV = 4; };
template <> struct Fmt<MDC_CBF16> { static constexpr int CPV = 4; };
template <> struct Fmt<MDC_CE4M3> { static constexpr int CPV = 8; };
template <> struct Fmt<MDC_C32S> { static constexpr int CPV = 4; };   // per plane (hi, lo)

__device__ __forceinline__ float2 dec_h2(unsigned w) {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
}
__device__ __forceinline__ float2 dec_b2(unsigned w) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
    return __bfloat1622float2(h);
}
__device__ __forceinline__ float2 dec_e4m3x2(unsigned short w) {
    __half2_raw r = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)w, __NV_E4M3);
    return __half22float2(__half2(r));
}

// Decode one 16-byte vector into CPV complex values (in storage units; row scale applied elsewhere).
// MDC_C32S decodes each plane like MDC_C16F; the caller adds the lo plane (decode2).
template <int FMT>
__device__ __forceinline__ void decode(const uint4& v, float2* c) {
    if constexpr (FMT == MDC_C64) {
        c[0] = make_float2(__uint_as_float(v.x), __uint_as_float(v.y));
        c[1] = make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
    } else if constexpr (FMT == MDC_C16F || FMT == MDC_C32S) {
        c[0] = dec_h2(v.x); c[1] = dec_h2(v.y); c[2] = dec_h2(v.z); c[3] = dec_h2(v.w);
    } else if constexpr (FMT == MDC_CBF16) {
        c[0] = dec_b2(v.x); c[1] = dec_b2(v.y); c[2] = dec_b2(v.z); c[3] = dec_b2(v.w);
    } else {
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            c[2 * q] = dec_e4m3x2((unsigned short)(w[q] & 0xffffu));
            c[2 * q + 1] = dec_e4m3x2((unsigned short)(w[q] >> 16));
        }
    }
}

__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcs(p); }

// Load and decode the vector at g[i]; for the split format add its lo plane at g[i + lo].
template <int FMT>
__device__ __forceinline__ void load_decode(const uint4* g, size_t i, int64_t lo, float2* c) {
    decode<FMT>(ld_stream(g + i), c);
    if constexpr (FMT == MDC_C32S) {
        float2 l[4];
        decode<FMT>(ld_stream(g + i + lo), l);
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = cadd(c[j], l[j]);
    }
}

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}

__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

// ---- complex64 GEMV kernels (begin)
// complex64 specialisations: one warp per row, X(w) interleaved in shared memory (C64 keeps
// two complex values per vector, so lanes already read distinct words).
template <int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_fwd_c64(
    const float4* __restrict__ G, int ldg, int nr, int ns,
    const float2* __restrict__ X, int ldi, int voff_i,
    float2* __restrict__ Y, int ldo, int voff_o, const int* active, int* err) {
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 xs[];   // [ldg][NVC]
    const int k = blockIdx.y;
    const float2* Xk = X + (size_t)k * ns * ldi + voff_i;
    for (int i = threadIdx.x; i < ldg * NVC; i += GEMV_THREADS) {
        const int s = i / NVC, v = i - s * NVC;
        xs[i] = s < ns && MDC_INB((size_t)k * ns * ldi + voff_i + (size_t)s * ldi + v, 1, (long long)gridDim.y * ns * ldi, err, 100)
                    ? Xk[(size_t)s * ldi + v] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg >> 1;
    const int r0 = blockIdx.x * FWD_ROWS_PER_CTA;
    const int r1 = min(r0 + FWD_ROWS_PER_CTA, nr);
    for (int r = r0 + warp; r < r1; r += GEMV_THREADS / 32) {
        if (!MDC_INB(((size_t)k * nr + r) * nvec, nvec, (long long)gridDim.y * nr * nvec, err, 101)) continue;
        const float4* g = G + ((size_t)k * nr + r) * nvec;
        float2 acc[NVC];
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[v] = make_float2(0.f, 0.f);
        int i = lane;
        for (; i + 96 < nvec; i += 128) {
            float4 gv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) gv[u] = ld_stream(g + i + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s = 2 * (i + 32 * u);
#pragma unroll
                for (int v = 0; v < NVC; ++v) {
                    cfma(acc[v], make_float2(gv[u].x, gv[u].y), xs[s * NVC + v]);
                    cfma(acc[v], make_float2(gv[u].z, gv[u].w), xs[(s + 1) * NVC + v]);
                }
            }
        }
        for (; i < nvec; i += 32) {
            const float4 gv = ld_stream(g + i);
            const int s = 2 * i;
#pragma unroll
            for (int v = 0; v < NVC; ++v) {
                cfma(acc[v], make_float2(gv.x, gv.y), xs[s * NVC + v]);
                cfma(acc[v], make_float2(gv.z, gv.w), xs[(s + 1) * NVC + v]);
            }
        }
#pragma unroll
        for (int v = 0; v < NVC; ++v) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc[v].x += __shfl_xor_sync(0xffffffffu, acc[v].x, off);
                acc[v].y += __shfl_xor_sync(0xffffffffu, acc[v].y, off);
            }
        }
        if (lane == 0 && MDC_INB(((size_t)k * nr + r) * ldo + voff_o, NVC, (long long)gridDim.y * nr * ldo, err, 102)) {
            float2* y = Y + ((size_t)k * nr + r) * ldo + voff_o;
#pragma unroll
            for (int v = 0; v < NVC; ++v) y[v] = acc[v];
        }
    }
}

constexpr int ADJ_TILE = 64;   // complex columns per CTA (one 512-byte row segment)

template <int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_adj_c64(
    const float4* __restrict__ G, int ldg, int nr, int ns,
    const float2* __restrict__ Yin, int ldi, int voff_i,
    float2* __restrict__ Xout, int ldo, int voff_o, const int* active, int* err) {
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 ys[];   // [nr][NVC], then reduction space
    const int k = blockIdx.y;
    const int s0 = blockIdx.x * ADJ_TILE;
    const float2* Yk = Yin + (size_t)k * nr * ldi + voff_i;
    for (int i = threadIdx.x; i < nr * NVC; i += GEMV_THREADS) {
        const int r = i / NVC, v = i - r * NVC;
        ys[i] = MDC_INB((size_t)k * nr * ldi + voff_i + (size_t)r * ldi + v, 1, (long long)gridDim.y * nr * ldi, err, 103)
                    ? Yk[(size_t)r * ldi + v] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg >> 1;
    const float4* g = G + (size_t)k * nr * nvec + (s0 >> 1) + lane;
    float2 a0[NVC], a1[NVC];
#pragma unroll
    for (int v = 0; v < NVC; ++v) { a0[v] = make_float2(0.f, 0.f); a1[v] = make_float2(0.f, 0.f); }
    constexpr int W = GEMV_THREADS / 32;
    // this lane's column of vectors: rows 0 .. nr - 1, nvec apart
    const bool gok = MDC_INB((size_t)k * nr * nvec + (s0 >> 1) + lane, (size_t)(nr - 1) * nvec + 1,
                             (long long)gridDim.y * nr * nvec, err, 104);
    int r = gok ? warp : nr;
    for (; r + 3 * W < nr; r += 4 * W) {
        float4 gv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) gv[u] = ld_stream(g + (size_t)(r + u * W) * nvec);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int v = 0; v < NVC; ++v) {
                const float2 y = ys[(r + u * W) * NVC + v];
                cfma_conj(a0[v], make_float2(gv[u].x, gv[u].y), y);
                cfma_conj(a1[v], make_float2(gv[u].z, gv[u].w), y);
            }
        }
    }
    for (; r < nr; r += W) {
        const float4 gv = ld_stream(g + (size_t)r * nvec);
#pragma unroll
        for (int v = 0; v < NVC; ++v) {
            const float2 y = ys[r * NVC + v];
            cfma_conj(a0[v], make_float2(gv.x, gv.y), y);
            cfma_conj(a1[v], make_float2(gv.z, gv.w), y);
        }
    }
    // reduce the W warps' partial sums: red[w][64 columns][NVC]
    __syncthreads();
    float2* red = ys;   // reuse (needs W * 64 * NVC float2 <= smem, ensured by the launcher)
#pragma unroll
    for (int v = 0; v < NVC; ++v) {
        red[(warp * ADJ_TILE + 2 * lane) * NVC + v] = a0[v];
        red[(warp * ADJ_TILE + 2 * lane + 1) * NVC + v] = a1[v];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ADJ_TILE * NVC; i += GEMV_THREADS) {
        const int sl = i / NVC, v = i - sl * NVC;
        const int s = s0 + sl;
        float2 tot = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < W; ++w) tot = cadd(tot, red[(w * ADJ_TILE + sl) * NVC + v]);
        if (s < ns && MDC_INB(((size_t)k * ns + s) * ldo + voff_o + v, 1, (long long)gridDim.y * ns * ldo, err, 105))
            Xout[((size_t)k * ns + s) * ldo + voff_o + v] = tot;
    }
}

// ---- complex64 GEMV kernels (end)

// Forward GEMV.  X(w) is staged de-interleaved by vector lane position:
// xs[(j * nvec + i) * NVC + v] = X[CPV * i + j][v], so the 32 lanes of a warp, which
// hold vectors i..i+31, read consecutive shared-memory words for every j.
template <int FMT, int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_fwd(
    const uint4* __restrict__ G, int ldg, int nr, int ns, const float* __restrict__ gscale,
    const float2* __restrict__ X, int ldi, int voff_i,
    float2* __restrict__ Y, int ldo, int voff_o, const int* active, int64_t lo, int* err) {
    constexpr int CPV = Fmt<FMT>::CPV;
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 xs[];
    const int k = blockIdx.y;
    const int nvec = ldg / CPV;
    const float2* Xk = X + (size_t)k * ns * ldi + voff_i;
    for (int e = threadIdx.x; e < ldg * NVC; e += GEMV_THREADS) {
        const int s = e / NVC, v = e - s * NVC;
        const int i = s / CPV, j = s - i * CPV;
        xs[(j * nvec + i) * NVC + v] =
            s < ns && MDC_INB((size_t)k * ns * ldi + voff_i + (size_t)s * ldi + v, 1, (long long)gridDim.y * ns * ldi, err, 106)
                ? Xk[(size_t)s * ldi + v] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * FWD_ROWS_PER_CTA;
    const int r1 = min(r0 + FWD_ROWS_PER_CTA, nr);
    for (int r = r0 + warp; r < r1; r += GEMV_THREADS / 32) {
        if (!MDC_INB(((size_t)k * nr + r) * nvec, nvec, (long long)gridDim.y * nr * nvec, err, 107)) continue;
        const uint4* g = G + ((size_t)k * nr + r) * nvec;
        float2 acc[NVC];
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[v] = make_float2(0.f, 0.f);
        int i = lane;
        for (; i + 96 < nvec; i += 128) {
            float2 c4[4][CPV];
#pragma unroll
            for (int u = 0; u < 4; ++u) load_decode<FMT>(g, i + 32 * u, lo, c4[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int j = 0; j < CPV; ++j)
#pragma unroll
                    for (int v = 0; v < NVC; ++v) cfma(acc[v], c4[u][j], xs[(j * nvec + i + 32 * u) * NVC + v]);
            }
        }
        for (; i < nvec; i += 32) {
            float2 c[CPV];
            load_decode<FMT>(g, i, lo, c);
#pragma unroll
            for (int j = 0; j < CPV; ++j)
#pragma unroll
                for (int v = 0; v < NVC; ++v) cfma(acc[v], c[j], xs[(j * nvec + i) * NVC + v]);
        }
#pragma unroll
        for (int v = 0; v < NVC; ++v) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc[v].x += __shfl_xor_sync(0xffffffffu, acc[v].x, off);
                acc[v].y += __shfl_xor_sync(0xffffffffu, acc[v].y, off);
            }
        }
        if (lane == 0 && MDC_INB(((size_t)k * nr + r) * ldo + voff_o, NVC, (long long)gridDim.y * nr * ldo, err, 109)) {
            const float sc = (FMT == MDC_C64) ? 1.f : gscale[(size_t)k * nr + r];
            float2* y = Y + ((size_t)k * nr + r) * ldo + voff_o;
#pragma unroll
            for (int v = 0; v < NVC; ++v) y[v] = make_float2(acc[v].x * sc, acc[v].y * sc);
        }
    }
}

// Adjoint GEMV: a CTA owns TILE = 32 * CPV adjacent columns s of one frequency (one 512-byte
// segment of every row); warp w walks rows r = w, w + 8, ...; the row scale is folded into Y.
template <int FMT, int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_adj(
    const uint4* __restrict__ G, int ldg, int nr, int ns, const float* __restrict__ gscale,
    const float2* __restrict__ Yin, int ldi, int voff_i,
    float2* __restrict__ Xout, int ldo, int voff_o, const int* active, int64_t lo, int* err) {
    constexpr int CPV = Fmt<FMT>::CPV;
    constexpr int TILE = 32 * CPV;
    constexpr int W = GEMV_THREADS / 32;
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 ys[];   // [nr][NVC], then reduction space
    const int k = blockIdx.y;
    const int s0 = blockIdx.x * TILE;
    const float2* Yk = Yin + (size_t)k * nr * ldi + voff_i;
    for (int e = threadIdx.x; e < nr * NVC; e += GEMV_THREADS) {
        const int r = e / NVC, v = e - r * NVC;
        float2 y = MDC_INB((size_t)k * nr * ldi + voff_i + (size_t)r * ldi + v, 1, (long long)gridDim.y * nr * ldi, err, 110)
                       ? Yk[(size_t)r * ldi + v] : make_float2(0.f, 0.f);
        if (FMT != MDC_C64) {
            const float sc = gscale[(size_t)k * nr + r];
            y.x *= sc;
            y.y *= sc;
        }
        ys[e] = y;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg / CPV;
    // live lanes walk their column of vectors: rows 0 .. nr - 1, nvec apart
    const bool live = s0 + CPV * lane < ldg &&
                      MDC_INB((size_t)k * nr * nvec + (s0 / CPV) + lane, (size_t)(nr - 1) * nvec + 1,
                              (long long)gridDim.y * nr * nvec, err, 112);
    const uint4* g = G + (size_t)k * nr * nvec + (s0 / CPV) + lane;
    float2 acc[CPV][NVC];
#pragma unroll
    for (int j = 0; j < CPV; ++j)
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[j][v] = make_float2(0.f, 0.f);
    if (live) {
        int r = warp;
        for (; r + 3 * W < nr; r += 4 * W) {
            float2 c4[4][CPV];
#pragma unroll
            for (int u = 0; u < 4; ++u) load_decode<FMT>(g, (size_t)(r + u * W) * nvec, lo, c4[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int v = 0; v < NVC; ++v) {
                    const float2 y = ys[(r + u * W) * NVC + v];
#pragma unroll
                    for (int j = 0; j < CPV; ++j) cfma_conj(acc[j][v], c4[u][j], y);
                }
            }
        }
        for (; r < nr; r += W) {
            float2 c[CPV];
            load_decode<FMT>(g, (size_t)r * nvec, lo, c);
#pragma unroll
            for (int v = 0; v < NVC; ++v) {
                const float2 y = ys[r * NVC + v];
#pragma unroll
                for (int j = 0; j < CPV; ++j) cfma_conj(acc[j][v], c[j], y);
            }
        }
    }
    __syncthreads();
    float2* red = ys;   // reuse: W * TILE * NVC float2 (the launcher sizes shared memory for it)
#pragma unroll
    for (int j = 0; j < CPV; ++j)
#pragma unroll
        for (int v = 0; v < NVC; ++v) red[(warp * TILE + CPV * lane + j) * NVC + v] = acc[j][v];
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * NVC; e += GEMV_THREADS) {
        const int sl = e / NVC, v = e - sl * NVC;
        const int s = s0 + sl;
        float2 tot = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < W; ++w) tot = cadd(tot, red[(w * TILE + sl) * NVC + v]);
        if (s < ns && MDC_INB(((size_t)k * ns + s) * ldo + voff_o + v, 1, (long long)gridDim.y * ns * ldo, err, 113))
            Xout[((size_t)k * ns + s) * ldo + voff_o + v] = tot;
    }
}

// ---- chunked GEMV for long rows or columns
// When X(w) (forward) or Y(w) (adjoint) would take more than GEMV_STAGE_MAX bytes of shared
// memory -- e.g. 9801 x 9801 kernels, where a whole complex row is 78 KB per column and only one
// or two CTAs would fit on an SM, too few loads in flight to stream HBM -- it is staged in
// chunks of GEMV_CHUNK_BYTES instead.  Each lane still visits its vectors (forward) or rows
// (adjoint) in ascending order and the warp and CTA reductions are unchanged, so the chunked
// kernels give the same bits as the kernels above.
constexpr int GEMV_STAGE_MAX = 48 * 1024;
constexpr int GEMV_CHUNK_BYTES = 32 * 1024;
constexpr int FWD_CHUNK_ROWS = 32;     // rows per CTA of the chunked forward (4 per warp, in registers)

// Forward chunk: CHV vectors of every row (a multiple of 128, the 4-way unrolled lane stride).
template <int FMT, int NVC>
struct FwdChunk {
    static constexpr int CHV = ((GEMV_CHUNK_BYTES / (8 * NVC * Fmt<FMT>::CPV)) / 128) * 128;
    static_assert(CHV >= 128, "forward chunk too small");
};
// Adjoint chunk: CHR rows (a multiple of 4 * 8 warps, the unrolled row stride).
template <int NVC>
struct AdjChunk {
    static constexpr int CHR = ((GEMV_CHUNK_BYTES / (8 * NVC)) / 32) * 32;
};

// Forward: the CTA's 32 rows, warp w owning rows r0 + w + 8 q (q < 4) with their partial sums
// held in registers across chunks.
template <int FMT, int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_fwd_chunked(
    const uint4* __restrict__ G, int ldg, int nr, int ns, const float* __restrict__ gscale,
    const float2* __restrict__ X, int ldi, int voff_i,
    float2* __restrict__ Y, int ldo, int voff_o, const int* active, int64_t lo, int* err) {
    constexpr int CPV = Fmt<FMT>::CPV;
    constexpr int CHV = FwdChunk<FMT, NVC>::CHV;
    constexpr int W = GEMV_THREADS / 32;
    constexpr int RPW = FWD_CHUNK_ROWS / W;
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 xs[];   // [CPV][CHV][NVC]
    const int k = blockIdx.y;
    const int nvec = ldg / CPV;
    const float2* Xk = X + (size_t)k * ns * ldi + voff_i;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rw = blockIdx.x * FWD_CHUNK_ROWS + warp;
    float2 acc[RPW][NVC];
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[q][v] = make_float2(0.f, 0.f);
    for (int c0 = 0; c0 < nvec; c0 += CHV) {
        const int c1 = min(c0 + CHV, nvec);
        __syncthreads();                               // the previous chunk has been consumed
        for (int e = threadIdx.x; e < (c1 - c0) * CPV * NVC; e += GEMV_THREADS) {
            const int sl = e / NVC, v = e - sl * NVC;
            const int i = sl / CPV, j = sl - i * CPV;
            const int s = c0 * CPV + sl;
            xs[(j * CHV + i) * NVC + v] =
                s < ns && MDC_INB((size_t)k * ns * ldi + voff_i + (size_t)s * ldi + v, 1, (long long)gridDim.y * ns * ldi, err, 114)
                    ? Xk[(size_t)s * ldi + v] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int r = rw + W * q;
            if (r >= nr) break;                        // warp-uniform
            if (!MDC_INB(((size_t)k * nr + r) * nvec, nvec, (long long)gridDim.y * nr * nvec, err, 115)) continue;
            const uint4* g = G + ((size_t)k * nr + r) * nvec;
            int i = c0 + lane;
            for (; i + 96 < c1; i += 128) {
                float2 c4[4][CPV];
#pragma unroll
                for (int u = 0; u < 4; ++u) load_decode<FMT>(g, i + 32 * u, lo, c4[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int j = 0; j < CPV; ++j)
#pragma unroll
                        for (int v = 0; v < NVC; ++v)
                            cfma(acc[q][v], c4[u][j], xs[(j * CHV + i - c0 + 32 * u) * NVC + v]);
                }
            }
            for (; i < c1; i += 32) {
                float2 c[CPV];
                load_decode<FMT>(g, i, lo, c);
#pragma unroll
                for (int j = 0; j < CPV; ++j)
#pragma unroll
                    for (int v = 0; v < NVC; ++v) cfma(acc[q][v], c[j], xs[(j * CHV + i - c0) * NVC + v]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        const int r = rw + W * q;
        if (r >= nr) break;
#pragma unroll
        for (int v = 0; v < NVC; ++v) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc[q][v].x += __shfl_xor_sync(0xffffffffu, acc[q][v].x, off);
                acc[q][v].y += __shfl_xor_sync(0xffffffffu, acc[q][v].y, off);
            }
        }
        if (lane == 0 && MDC_INB(((size_t)k * nr + r) * ldo + voff_o, NVC, (long long)gridDim.y * nr * ldo, err, 117)) {
            const float sc = (FMT == MDC_C64) ? 1.f : gscale[(size_t)k * nr + r];
            float2* y = Y + ((size_t)k * nr + r) * ldo + voff_o;
#pragma unroll
            for (int v = 0; v < NVC; ++v) y[v] = make_float2(acc[q][v].x * sc, acc[q][v].y * sc);
        }
    }
}

// Adjoint: Y(w) (row scales folded in) staged CHR rows at a time; per-lane column sums persist
// across chunks.
template <int FMT, int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_adj_chunked(
    const uint4* __restrict__ G, int ldg, int nr, int ns, const float* __restrict__ gscale,
    const float2* __restrict__ Yin, int ldi, int voff_i,
    float2* __restrict__ Xout, int ldo, int voff_o, const int* active, int64_t lo, int* err) {
    constexpr int CPV = Fmt<FMT>::CPV;
    constexpr int TILE = 32 * CPV;
    constexpr int W = GEMV_THREADS / 32;
    constexpr int CHR = AdjChunk<NVC>::CHR;
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 ys[];   // [CHR][NVC], then reduction space
    const int k = blockIdx.y;
    const int s0 = blockIdx.x * TILE;
    const float2* Yk = Yin + (size_t)k * nr * ldi + voff_i;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg / CPV;
    // live lanes walk their column of vectors: rows 0 .. nr - 1, nvec apart
    const bool live = s0 + CPV * lane < ldg &&
                      MDC_INB((size_t)k * nr * nvec + (s0 / CPV) + lane, (size_t)(nr - 1) * nvec + 1,
                              (long long)gridDim.y * nr * nvec, err, 112);
    const uint4* g = G + (size_t)k * nr * nvec + (s0 / CPV) + lane;
    float2 acc[CPV][NVC];
#pragma unroll
    for (int j = 0; j < CPV; ++j)
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[j][v] = make_float2(0.f, 0.f);
    for (int c0 = 0; c0 < nr; c0 += CHR) {
        const int c1 = min(c0 + CHR, nr);
        __syncthreads();                               // the previous chunk has been consumed
        for (int e = threadIdx.x; e < (c1 - c0) * NVC; e += GEMV_THREADS) {
            const int rl = e / NVC, v = e - rl * NVC;
            const int r = c0 + rl;
            float2 y = MDC_INB((size_t)k * nr * ldi + voff_i + (size_t)r * ldi + v, 1, (long long)gridDim.y * nr * ldi, err, 118)
                           ? Yk[(size_t)r * ldi + v] : make_float2(0.f, 0.f);
            if (FMT != MDC_C64) {
                const float sc = gscale[(size_t)k * nr + r];
                y.x *= sc;
                y.y *= sc;
            }
            ys[e] = y;
        }
        __syncthreads();
        if (live) {
            int r = c0 + warp;
            for (; r + 3 * W < c1; r += 4 * W) {
                float2 c4[4][CPV];
#pragma unroll
                for (int u = 0; u < 4; ++u) load_decode<FMT>(g, (size_t)(r + u * W) * nvec, lo, c4[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int v = 0; v < NVC; ++v) {
                        const float2 y = ys[(r - c0 + u * W) * NVC + v];
#pragma unroll
                        for (int j = 0; j < CPV; ++j) cfma_conj(acc[j][v], c4[u][j], y);
                    }
                }
            }
            for (; r < c1; r += W) {
                float2 c[CPV];
                load_decode<FMT>(g, (size_t)r * nvec, lo, c);
#pragma unroll
                for (int v = 0; v < NVC; ++v) {
                    const float2 y = ys[(r - c0) * NVC + v];
#pragma unroll
                    for (int j = 0; j < CPV; ++j) cfma_conj(acc[j][v], c[j], y);
                }
            }
        }
    }
    __syncthreads();
    float2* red = ys;   // reuse: W * TILE * NVC float2 (the launcher sizes shared memory for it)
#pragma unroll
    for (int j = 0; j < CPV; ++j)
#pragma unroll
        for (int v = 0; v < NVC; ++v) red[(warp * TILE + CPV * lane + j) * NVC + v] = acc[j][v];
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * NVC; e += GEMV_THREADS) {
        const int sl = e / NVC, v = e - sl * NVC;
        const int s = s0 + sl;
        float2 tot = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < W; ++w) tot = cadd(tot, red[(w * TILE + sl) * NVC + v]);
        if (s < ns && MDC_INB(((size_t)k * ns + s) * ldo + voff_o + v, 1, (long long)gridDim.y * ns * ldo, err, 113))
            Xout[((size_t)k * ns + s) * ldo + voff_o + v] = tot;
    }
}

// MDC_GEMV_CHUNK=0 in the environment stages whole rows whenever they fit (for comparisons).
bool gemv_chunk_allowed() {
    static int env = -1;
    if (env < 0) {
        const char* e = getenv("MDC_GEMV_CHUNK");
        env = (e && e[0] == '0') ? 0 : 1;
    }
    return env == 1;
}

// ------------------------------------------------------------------ SIMT complex GEMM
constexpr int GBM = 64, GBN = 64, GBK = 8;
constexpr int GCHUNK = 16;                 // reduction tiles per partial sum (128 terms)
// Narrow tile for few columns: 128 rows x 32 columns (each thread still 4 x 4 outputs), so a
// 20-column product leaves 38 % of the tile idle instead of 69 %.
constexpr int GBM_N = 128, GBN_N = 32;

template <int FMT> struct Bytes;
template <> struct Bytes<MDC_C64> { static constexpr int v = 8; };
template <> struct Bytes<MDC_C16F> { static constexpr int v = 4; };
template <> struct Bytes<MDC_CBF16> { static constexpr int v = 4; };
template <> struct Bytes<MDC_CE4M3> { static constexpr int v = 2; };
template <> struct Bytes<MDC_C32S> { static constexpr int v = 4; };   // per plane

// Two consecutive complex values starting at (even) element e of a kernel row.
template <int FMT>
__device__ __forceinline__ void load2(const unsigned char* row, int e, float2& c0, float2& c1, size_t lo = 0) {
    if constexpr (FMT == MDC_C64) {
        const float4 v = *reinterpret_cast<const float4*>(row + (size_t)e * 8);
        c0 = make_float2(v.x, v.y);
        c1 = make_float2(v.z, v.w);
    } else if constexpr (FMT == MDC_C16F || FMT == MDC_CBF16 || FMT == MDC_C32S) {
        const uint2 v = *reinterpret_cast<const uint2*>(row + (size_t)e * 4);
        if constexpr (FMT == MDC_CBF16) { c0 = dec_b2(v.x); c1 = dec_b2(v.y); }
        else { c0 = dec_h2(v.x); c1 = dec_h2(v.y); }
        if constexpr (FMT == MDC_C32S) {
            const uint2 l = *reinterpret_cast<const uint2*>(row + lo + (size_t)e * 4);
            c0 = cadd(c0, dec_h2(l.x));
            c1 = cadd(c1, dec_h2(l.y));
        }
    } else {
        const unsigned v = *reinterpret_cast<const unsigned*>(row + (size_t)e * 2);
        c0 = dec_e4m3x2((unsigned short)(v & 0xffffu));
        c1 = dec_e4m3x2((unsigned short)(v >> 16));
    }
}

template <int FMT, bool ADJ, bool NARROW = false>
__global__ void __launch_bounds__(256) cgemm_simt(
    const unsigned char* __restrict__ G, int ldg, int nr, int ns, const float* __restrict__ gscale,
    const float2* __restrict__ B, int ldb, int voff_b,
    float2* __restrict__ Cm, int ldc, int voff_c, int N, const int* active, size_t lo, int* err) {
    if (active && *active == 0) return;
    constexpr int BPC = Bytes<FMT>::v;
    constexpr int TBM = NARROW ? GBM_N : GBM, TBN = NARROW ? GBN_N : GBN;
    constexpr int TXN = TBN / 4;                   // threads along the columns (4 columns each)
    const int M = ADJ ? ns : nr;
    const int K = ADJ ? nr : ns;
    const int k = blockIdx.z;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    __shared__ __align__(16) float2 As[GBK][TBM];
    __shared__ __align__(16) float2 Bs[GBK][TBN];
    const unsigned char* Gk = G + (size_t)k * nr * ldg * BPC;
    const float* sck = gscale + (size_t)k * nr;
    const float2* Bk = B + (size_t)k * K * ldb + voff_b;
    const int tid = threadIdx.x, tx = tid % TXN, ty = tid / TXN;
    // Two-level sums: each chunk of GCHUNK reduction tiles accumulates in part (registers), which is
    // then added to the thread's running totals (shared memory, one slot per output and thread, so the
    // registers stay at one accumulator set), so a float32 sum over K terms carries about
    // (GCHUNK * GBK + K / (GCHUNK * GBK)) roundings per output instead of K.
    __shared__ float2 tot[16][256];
    float2 part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            part[i][j] = make_float2(0.f, 0.f);
            tot[4 * i + j][tid] = make_float2(0.f, 0.f);
        }

    for (int kt = 0; kt < K; kt += GBK) {
        // A tile: GBK x TBM complex values, 64 rows (forward) or 64 columns (adjoint) per round
#pragma unroll
        for (int r = 0; r < TBM / 64; ++r) {
            if (!ADJ) {
                const int m = (tid >> 2) + 64 * r, kq = (tid & 3) * 2;
                float2 c0 = make_float2(0.f, 0.f), c1 = c0;
                if (m0 + m < M && MDC_INB(((size_t)k * nr + m0 + m) * ldg * BPC + (size_t)(kt + kq) * BPC, 2 * BPC,
                                          (long long)gridDim.z * nr * ldg * BPC, err, 120))
                    load2<FMT>(Gk + (size_t)(m0 + m) * ldg * BPC, kt + kq, c0, c1, lo);
                As[kq][m] = c0;
                As[kq + 1][m] = c1;
            } else {
                const int kk = tid >> 5, mq = (tid & 31) * 2 + 64 * r;
                float2 c0 = make_float2(0.f, 0.f), c1 = c0;
                // a 128-column tile may reach past the padded row (ldg is a multiple of 64 only)
                if (kt + kk < K && m0 + mq < ldg &&
                    MDC_INB(((size_t)k * nr + kt + kk) * ldg * BPC + (size_t)(m0 + mq) * BPC, 2 * BPC,
                            (long long)gridDim.z * nr * ldg * BPC, err, 121)) {
                    load2<FMT>(Gk + (size_t)(kt + kk) * ldg * BPC, m0 + mq, c0, c1, lo);
                    const float sc = (FMT == MDC_C64) ? 1.f : sck[kt + kk];
                    c0 = make_float2(c0.x * sc, -c0.y * sc);
                    c1 = make_float2(c1.x * sc, -c1.y * sc);
                }
                As[kk][mq] = c0;
                As[kk][mq + 1] = c1;
            }
        }
        // B tile: GBK x TBN complex values, two per thread (the narrow tile uses half the threads)
        if (tid < GBK * TBN / 2) {
            const int kk = tid / (TBN / 2), nq = (tid % (TBN / 2)) * 2;
            float2 b0 = make_float2(0.f, 0.f), b1 = make_float2(0.f, 0.f);
            if (kt + kk < K) {
                const float2* row = Bk + (size_t)(kt + kk) * ldb + n0 + nq;
                [[maybe_unused]] const size_t ro = (size_t)k * K * ldb + voff_b + (size_t)(kt + kk) * ldb + n0 + nq;
                if (n0 + nq < N && MDC_INB(ro, 1, (long long)gridDim.z * K * ldb, err, 123)) b0 = row[0];
                if (n0 + nq + 1 < N && MDC_INB(ro + 1, 1, (long long)gridDim.z * K * ldb, err, 123)) b1 = row[1];
            }
            Bs[kk][nq] = b0;
            Bs[kk][nq + 1] = b1;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + (TBM / 4) * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + TXN * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(part[i][j], a[i], b[j]);
        }
        __syncthreads();
        if ((kt / GBK) % GCHUNK == GCHUNK - 1 || kt + GBK >= K) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    tot[4 * i + j][tid] = cadd(tot[4 * i + j][tid], part[i][j]);
                    part[i][j] = make_float2(0.f, 0.f);
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + (TBM / 4) * i;
        if (m >= M) continue;
        const float sc = (FMT == MDC_C64 || ADJ) ? 1.f : sck[m];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + TXN * j;
            if (n < N && MDC_INB(((size_t)k * M + m) * ldc + voff_c + n, 1, (long long)gridDim.z * M * ldc, err, 125))
                Cm[((size_t)k * M + m) * ldc + voff_c + n] = make_float2(tot[4 * i + j][tid].x * sc, tot[4 * i + j][tid].y * sc);
        }
    }
}

// Offset of the split format's lo plane (bytes, and 16-byte vectors); 0 for other formats.
size_t lo_plane_bytes(const mdc_plan* p) {
    return p->storage == MDC_C32S ? (size_t)p->nf * p->nr * p->ldg * 4 : 0;
}
int64_t lo_plane_vec(const mdc_plan* p) { return (int64_t)(lo_plane_bytes(p) / 16); }

template <int FMT, int NVC>
void gemv_fwd_launch(mdc_plan* p, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                     int voff_o, cudaStream_t s, const int* active) {
    const size_t smem = (size_t)p->ldg * NVC * sizeof(float2);
    if (smem > (size_t)GEMV_STAGE_MAX && gemv_chunk_allowed()) {
        constexpr size_t csmem = (size_t)Fmt<FMT>::CPV * FwdChunk<FMT, NVC>::CHV * NVC * sizeof(float2);
        dim3 grid((p->nr + FWD_CHUNK_ROWS - 1) / FWD_CHUNK_ROWS, p->nf);
        gemv_fwd_chunked<FMT, NVC><<<grid, GEMV_THREADS, csmem, s>>>(
            reinterpret_cast<const uint4*>(p->G), (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi, voff_i, out,
            ldo, voff_o, active, lo_plane_vec(p), p->err_flag);
        return;
    }
    static SmemLimit attr;
    attr.ensure(gemv_fwd<FMT, NVC>, 220 * 1024);
    dim3 grid((p->nr + FWD_ROWS_PER_CTA - 1) / FWD_ROWS_PER_CTA, p->nf);
    if constexpr (FMT == MDC_C64) {
        static SmemLimit attr64;
        attr64.ensure(gemv_fwd_c64<NVC>, 220 * 1024);
        gemv_fwd_c64<NVC><<<grid, GEMV_THREADS, smem, s>>>(
            reinterpret_cast<const float4*>(p->G), (int)p->ldg, p->nr, p->ns, in, ldi, voff_i, out, ldo,
            voff_o, active, p->err_flag);
        return;
    }
    gemv_fwd<FMT, NVC><<<grid, GEMV_THREADS, smem, s>>>(
        reinterpret_cast<const uint4*>(p->G), (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi, voff_i, out,
        ldo, voff_o, active, lo_plane_vec(p), p->err_flag);
}

template <int FMT, int NVC>
void gemv_adj_launch(mdc_plan* p, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                     int voff_o, cudaStream_t s, const int* active) {
    constexpr int TILE = 32 * Fmt<FMT>::CPV;
    size_t smem = (size_t)p->nr * NVC * sizeof(float2);
    const size_t red = (size_t)(GEMV_THREADS / 32) * TILE * NVC * sizeof(float2);
    if (smem > (size_t)GEMV_STAGE_MAX && gemv_chunk_allowed()) {
        size_t csmem = (size_t)AdjChunk<NVC>::CHR * NVC * sizeof(float2);
        if (csmem < red) csmem = red;
        static SmemLimit cattr;
        cattr.ensure(gemv_adj_chunked<FMT, NVC>, 220 * 1024);
        dim3 grid((unsigned)((p->ldg + TILE - 1) / TILE), p->nf);
        gemv_adj_chunked<FMT, NVC><<<grid, GEMV_THREADS, csmem, s>>>(
            reinterpret_cast<const uint4*>(p->G), (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi, voff_i, out,
            ldo, voff_o, active, lo_plane_vec(p), p->err_flag);
        return;
    }
    if (smem < red) smem = red;
    static SmemLimit attr;
    attr.ensure(gemv_adj<FMT, NVC>, 220 * 1024);
    dim3 grid((unsigned)((p->ldg + TILE - 1) / TILE), p->nf);
    if constexpr (FMT == MDC_C64) {
        static SmemLimit attr64;
        attr64.ensure(gemv_adj_c64<NVC>, 220 * 1024);
        gemv_adj_c64<NVC><<<grid, GEMV_THREADS, smem, s>>>(
            reinterpret_cast<const float4*>(p->G), (int)p->ldg, p->nr, p->ns, in, ldi, voff_i, out, ldo,
            voff_o, active, p->err_flag);
        return;
    }
    gemv_adj<FMT, NVC><<<grid, GEMV_THREADS, smem, s>>>(
        reinterpret_cast<const uint4*>(p->G), (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi, voff_i, out,
        ldo, voff_o, active, lo_plane_vec(p), p->err_flag);
}

bool gemv_fits(const mdc_plan* p, bool adjoint, int ncol, int cpv) {
    const int64_t stage = (int64_t)(adjoint ? p->nr : p->ldg) * ncol * (int64_t)sizeof(float2);
    const int64_t red = (int64_t)(GEMV_THREADS / 32) * 32 * cpv * ncol * (int64_t)sizeof(float2);
    const bool staged = stage <= 200 * 1024 || (stage > GEMV_STAGE_MAX && gemv_chunk_allowed());
    return ncol <= gemv_max_columns() && staged && red <= 200 * 1024;
}

// Default rule for column counts above the GEMV width: up to GEMV_GROUP_MAX_FWD (forward) or
// GEMV_GROUP_MAX_ADJ (adjoint) columns the GEMV runs in passes over groups of 4, each streaming the
// kernel near the HBM rate; above, the FP32 SIMT GEMM (128 x 32 tiles up to 32 columns).  The
// crossover depends on the shape (measured on 8281^2, 3721 x 841 and 1681^2 complex64 kernels:
// groups win at 8 columns forward, at 8 and 16 adjoint, except the 3721 x 841 forward at 8);
// mdc_autotune measures it per handle.
constexpr int GEMV_GROUP_MAX_FWD = 8;
constexpr int GEMV_GROUP_MAX_ADJ = 16;

// path: PATH_GEMV, PATH_GEMV_GROUPS or PATH_SIMT (PATH_AUTO: GEMV when it fits, GEMV groups up to
// GEMV_GROUP_MAX_FWD or _ADJ columns, else SIMT)
template <int FMT>
bool product_fmt(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                 int voff_o, int ncol, cudaStream_t s, const int* active, int path) {
    const int gw = gemv_max_columns();
    const bool fits = gemv_fits(p, adjoint, ncol, Fmt<FMT>::CPV);
    const bool group_fits = ncol > gw && gemv_fits(p, adjoint, gw, Fmt<FMT>::CPV);
    if (path == PATH_GEMV && !fits) return false;
    if (path == PATH_GEMV_GROUPS && !group_fits) return false;
    const int gmax = adjoint ? GEMV_GROUP_MAX_ADJ : GEMV_GROUP_MAX_FWD;
    const bool groups = group_fits && (path == PATH_GEMV_GROUPS || (path == PATH_AUTO && ncol <= gmax));
    if ((fits && path != PATH_SIMT && path != PATH_GEMV_GROUPS) || groups) {
        for (int c0 = 0; c0 < ncol; c0 += gw) {
            const int nc = ncol - c0 < gw ? ncol - c0 : gw;
#define MDC_GEMV_CASE(n)                                                                                       \
    case n:                                                                                                    \
        if (adjoint) gemv_adj_launch<FMT, n>(p, in, ldi, voff_i + c0, out, ldo, voff_o + c0, s, active);      \
        else gemv_fwd_launch<FMT, n>(p, in, ldi, voff_i + c0, out, ldo, voff_o + c0, s, active);              \
        break;
            switch (nc) {
                MDC_GEMV_CASE(1)
                MDC_GEMV_CASE(2)
                MDC_GEMV_CASE(3)
                MDC_GEMV_CASE(4)
            }
#undef MDC_GEMV_CASE
        }
        return true;
    }
    const int M = adjoint ? p->ns : p->nr;
    const unsigned char* G = reinterpret_cast<const unsigned char*>(p->G);
    if (ncol <= GBN_N) {        // few columns: the 128 x 32 tile
        dim3 grid((ncol + GBN_N - 1) / GBN_N, (M + GBM_N - 1) / GBM_N, p->nf);
        if (adjoint)
            cgemm_simt<FMT, true, true><<<grid, 256, 0, s>>>(G, (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi,
                                                             voff_i, out, ldo, voff_o, ncol, active, lo_plane_bytes(p), p->err_flag);
        else
            cgemm_simt<FMT, false, true><<<grid, 256, 0, s>>>(G, (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi,
                                                              voff_i, out, ldo, voff_o, ncol, active, lo_plane_bytes(p), p->err_flag);
        return true;
    }
    dim3 grid((ncol + GBN - 1) / GBN, (M + GBM - 1) / GBM, p->nf);
    if (adjoint)
        cgemm_simt<FMT, true><<<grid, 256, 0, s>>>(G, (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi, voff_i,
                                                   out, ldo, voff_o, ncol, active, lo_plane_bytes(p), p->err_flag);
    else
        cgemm_simt<FMT, false><<<grid, 256, 0, s>>>(G, (int)p->ldg, p->nr, p->ns, p->gscale, in, ldi, voff_i,
                                                    out, ldo, voff_o, ncol, active, lo_plane_bytes(p), p->err_flag);
    return true;
}

bool product_simt_or_gemv(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                          int voff_o, int ncol, cudaStream_t s, const int* active, int path) {
    switch (p->storage) {
        case MDC_C64: return product_fmt<MDC_C64>(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, path);
        case MDC_C16F: return product_fmt<MDC_C16F>(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, path);
        case MDC_CBF16: return product_fmt<MDC_CBF16>(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, path);
        case MDC_C32S: return product_fmt<MDC_C32S>(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, path);
        default: return product_fmt<MDC_CE4M3>(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, path);
    }
}

}  // namespace

bool launch_product_variant(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i, float2* out,
                            int ldo, int voff_o, int ncol, cudaStream_t s, int path, int bn) {
    if (path == PATH_TC)
        return storage_tc(p->storage) && p->tcB && ncol <= p->tc_cap &&
               launch_tc_product(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, nullptr, bn);
    return product_simt_or_gemv(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, nullptr, path);
}

void launch_product(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i,
                    float2* out, int ldo, int voff_o, int ncol, cudaStream_t s,
                    const int* active) {
    int path = PATH_AUTO, bn = 0;
    if (!p->force_tc) {
        // autotuned variant of the smallest tuned bucket holding ncol columns
        for (const ProductChoice& c : p->tune[adjoint ? 1 : 0])
            if (ncol <= c.ncol) {
                path = c.path;
                bn = c.bn;
                break;
            }
    }
    // the tensor-core rule wants this product on tensor cores (a tuned choice, or the default rule
    // for tensor-core storage); when the operand buffers are missing (no mdc_reserve for this many
    // columns) or the launch cannot be made, it runs on the SIMT/GEMV path and is counted
    const bool tc_wanted =
        path == PATH_TC || (path == PATH_AUTO && storage_tc(p->storage) && (ncol >= 8 || p->force_tc));
    if (path == PATH_TC || (path == PATH_AUTO && tc_supported(p, ncol))) {
        if (storage_tc(p->storage) && p->tcB && ncol <= p->tc_cap &&
            launch_tc_product(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, bn, true))
            return;
        path = PATH_AUTO;
    }
    if (tc_wanted) ++p->tc_fallbacks;
    LaunchScope ls(p, s, adjoint ? MDC_KC_PRODUCT_ADJ : MDC_KC_PRODUCT_FWD);
    if (!product_simt_or_gemv(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, path))
        product_simt_or_gemv(p, adjoint, in, ldi, voff_i, out, ldo, voff_o, ncol, s, active, PATH_AUTO);
}

// ------------------------------------------------------------------ quantiser
// One CTA per kernel row (k, r): scale = max_s max(|Re|, |Im|) / QMAX, q = RNE(G / scale),
// saturating for E4M3.  QMAX = 32768 (FP16: keeps the row far from subnormals), 1 (BF16),
// 448 (E4M3 largest finite).  Padding columns s >= ns are written as zeros.
template <int FMT>
__global__ void __launch_bounds__(256) quantize_rows(const float2* __restrict__ G, int ns, int ldg,
                                                     unsigned char* __restrict__ Q, float* __restrict__ scale,
                                                     const float* __restrict__ w, size_t lo_plane) {
    constexpr float QMAX = (FMT == MDC_C16F || FMT == MDC_C32S) ? 32768.f : (FMT == MDC_CBF16 ? 1.f : 448.f);
    const size_t row = blockIdx.x;
    const float2* g = G + row * ns;
    float m = 0.f;
    // optional column weights multiply the kernel before it is quantised
    auto at = [&](int s) {
        const float2 v = g[s];
        return w ? make_float2(v.x * w[s], v.y * w[s]) : v;
    };
    for (int s = threadIdx.x; s < ns; s += 256) {
        const float2 v = at(s);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    __shared__ float red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const float rowmax = red[0];
    const float sc = rowmax > 0.f ? rowmax / QMAX : 0.f;
    const float inv = rowmax > 0.f ? QMAX / rowmax : 0.f;
    if (threadIdx.x == 0) scale[row] = sc;
    for (int s = threadIdx.x; s < ldg; s += 256) {
        float2 v = s < ns ? at(s) : make_float2(0.f, 0.f);
        v.x *= inv;
        v.y *= inv;
        if constexpr (FMT == MDC_C16F) {
            reinterpret_cast<__half2*>(Q)[row * ldg + s] = __floats2half2_rn(v.x, v.y);
        } else if constexpr (FMT == MDC_C32S) {
            // hi = RNE(v), lo = RNE(v - hi): the pair carries about 22 significant bits
            const __half2 hi = __floats2half2_rn(v.x, v.y);
            const float2 h = __half22float2(hi);
            reinterpret_cast<__half2*>(Q)[row * ldg + s] = hi;
            reinterpret_cast<__half2*>(Q)[lo_plane + row * ldg + s] = __floats2half2_rn(v.x - h.x, v.y - h.y);
        } else if constexpr (FMT == MDC_CBF16) {
            reinterpret_cast<__nv_bfloat162*>(Q)[row * ldg + s] = __floats2bfloat162_rn(v.x, v.y);
        } else {
            reinterpret_cast<__nv_fp8x2_storage_t*>(Q)[row * ldg + s] =
                __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// Quantise kernel rows [row0, row0 + nrows) of the [nf * nr] rows from G (which holds exactly
// those rows); the split format's lo plane sits one full plane (nf * nr * ldg values) above hi.
void launch_quantize_rows(mdc_plan* p, const float2* G, const float* w, int64_t row0, int64_t nrows, cudaStream_t s) {
    const size_t vb = p->storage == MDC_CE4M3 ? 2 : 4;        // bytes per stored complex value (one plane)
    unsigned char* Q = reinterpret_cast<unsigned char*>(p->G) + (size_t)row0 * p->ldg * vb;
    float* sc = p->gscale + row0;
    const size_t lo = (size_t)p->nf * p->nr * p->ldg;
    const unsigned rows = (unsigned)nrows;
    switch (p->storage) {
        case MDC_C16F: quantize_rows<MDC_C16F><<<rows, 256, 0, s>>>(G, p->ns, (int)p->ldg, Q, sc, w, lo); break;
        case MDC_CBF16: quantize_rows<MDC_CBF16><<<rows, 256, 0, s>>>(G, p->ns, (int)p->ldg, Q, sc, w, lo); break;
        case MDC_CE4M3: quantize_rows<MDC_CE4M3><<<rows, 256, 0, s>>>(G, p->ns, (int)p->ldg, Q, sc, w, lo); break;
        case MDC_C32S: quantize_rows<MDC_C32S><<<rows, 256, 0, s>>>(G, p->ns, (int)p->ldg, Q, sc, w, lo); break;
        default: break;
    }
}

void launch_quantize(mdc_plan* p, const float2* G, const float* w, cudaStream_t s) {
    launch_quantize_rows(p, G, w, 0, (int64_t)p->nf * p->nr, s);
}

}  // namespace mdc

// ------------------------------------------------------------------ autotuner
// For each direction and each column-count bucket (1, 2, 4, ..., up to ncol_max) time every
// variant that can run -- GEMV (<= 4 columns), SIMT GEMM, and for 16-bit storage the tensor-core
// GEMM with column tiles of 32, 64, 128 and 256 -- on the handle's own spectra with CUDA events
// (one warm-up, median of three), and keep the fastest.  The table maps ncol to the variant of
// the smallest bucket >= ncol.  With MDC_AUTOTUNE_CACHE set, tables are read from / appended to
// that file (one JSON object per line) keyed by device name, shape and storage.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

namespace mdc {

int ensure_scratch(mdc_plan* p, int ncols);

static std::string tune_key(const mdc_plan* p) {
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|nf=%d|nr=%d|ns=%d|nt=%d|storage=%d", prop.name, p->nf, p->nr, p->ns, p->nt,
             p->storage);
    for (char* c = buf; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    return buf;
}

static bool tune_load(mdc_plan* p, const std::string& key, int ncol_max) {
    const char* path = getenv("MDC_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    std::string want = "\"key\": \"" + key + "\"";
    char line[1 << 16];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        if (!strstr(line, want.c_str())) continue;
        int cmax = 0;
        const char* q = strstr(line, "\"ncol_max\": ");
        if (!q || sscanf(q + 12, "%d", &cmax) != 1 || cmax < ncol_max) continue;
        q = strstr(line, "\"choices\": [");
        if (!q) continue;
        q += 12;
        std::vector<ProductChoice> t[2];
        int d, n, pa, bn, used;
        while (sscanf(q, " [%d, %d, %d, %d]%n", &d, &n, &pa, &bn, &used) == 4 && (d == 0 || d == 1)) {
            t[d].push_back(ProductChoice{n, pa, bn});
            q += used;
            while (*q == ',' || *q == ' ') ++q;
        }
        if (!t[0].empty() && !t[1].empty()) {
            p->tune[0] = t[0];
            p->tune[1] = t[1];
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void tune_store(const mdc_plan* p, const std::string& key, int ncol_max) {
    const char* path = getenv("MDC_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"ncol_max\": %d, \"choices\": [", key.c_str(), ncol_max);
    bool first = true;
    for (int d = 0; d < 2; ++d)
        for (const ProductChoice& c : p->tune[d]) {
            fprintf(f, "%s[%d, %d, %d, %d]", first ? "" : ", ", d, c.ncol, c.path, c.bn);
            first = false;
        }
    fprintf(f, "]}\n");
    fclose(f);
}

int autotune(mdc_plan* p, int ncol_max, cudaStream_t s) {
    const std::string key = tune_key(p);
    if (tune_load(p, key, ncol_max)) return MDC_OK;
    int st = ensure_scratch(p, ncol_max);
    if (st != MDC_OK) return st;
    const size_t nspace = (size_t)(p->nr > p->ns ? p->nr : p->ns);
    cudaMemsetAsync(p->specA, 0, (size_t)p->nf * nspace * p->nv_cap * sizeof(float2), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    p->tune[0].clear();
    p->tune[1].clear();
    for (int d = 0; d < 2; ++d) {
        const bool adj = d == 1;
        for (int n = 1;; n *= 2) {
            const int ncol = n < ncol_max ? n : ncol_max;
            struct Cand { int path, bn; };
            std::vector<Cand> cands;
            if (ncol <= gemv_max_columns()) cands.push_back({PATH_GEMV, 0});
            else if (ncol <= 64) cands.push_back({PATH_GEMV_GROUPS, 0});
            cands.push_back({PATH_SIMT, 0});
            if (storage_tc(p->storage) && p->tcB)
                for (int bn = 32; bn <= 256; bn *= 2)
                    if (bn / 2 <= 2 * ncol || bn == 32) cands.push_back({PATH_TC, bn});
            float best = 1e30f;
            ProductChoice pick{ncol, PATH_AUTO, 0};
            for (const Cand& c : cands) {
                if (!launch_product_variant(p, adj, p->specA, ncol, 0, p->specB, ncol, 0, ncol, s, c.path, c.bn))
                    continue;
                float t[3];
                for (int r = 0; r < 3; ++r) {
                    cudaEventRecord(e0, s);
                    launch_product_variant(p, adj, p->specA, ncol, 0, p->specB, ncol, 0, ncol, s, c.path, c.bn);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&t[r], e0, e1);
                }
                const float med = t[0] < t[1] ? (t[1] < t[2] ? t[1] : (t[0] < t[2] ? t[2] : t[0]))
                                              : (t[0] < t[2] ? t[0] : (t[1] < t[2] ? t[2] : t[1]));
                if (med < best) {
                    best = med;
                    pick = ProductChoice{ncol, c.path, c.bn};
                }
            }
            p->tune[d].push_back(pick);
            if (ncol >= ncol_max) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        p->tune[0].clear();
        p->tune[1].clear();
        return MDC_ERR_CUDA;
    }
    tune_store(p, key, ncol_max);
    return MDC_OK;
}

}  // namespace mdc
