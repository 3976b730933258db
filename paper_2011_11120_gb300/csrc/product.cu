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

namespace mdc {
namespace {

constexpr int GEMV_THREADS = 256;
constexpr int FWD_ROWS_PER_CTA = 64;

__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

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

template <int NVC>
__global__ void __launch_bounds__(GEMV_THREADS) gemv_fwd_c64(
    const float4* __restrict__ G, int ldg, int nr, int ns,
    const float2* __restrict__ X, int ldi, int voff_i,
    float2* __restrict__ Y, int ldo, int voff_o, const int* active) {
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 xs[];   // [ldg][NVC]
    const int k = blockIdx.y;
    const float2* Xk = X + (size_t)k * ns * ldi + voff_i;
    for (int i = threadIdx.x; i < ldg * NVC; i += GEMV_THREADS) {
        const int s = i / NVC, v = i - s * NVC;
        xs[i] = s < ns ? Xk[(size_t)s * ldi + v] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg >> 1;
    const int r0 = blockIdx.x * FWD_ROWS_PER_CTA;
    const int r1 = min(r0 + FWD_ROWS_PER_CTA, nr);
    for (int r = r0 + warp; r < r1; r += GEMV_THREADS / 32) {
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
        if (lane == 0) {
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
    float2* __restrict__ Xout, int ldo, int voff_o, const int* active) {
    if (active && *active == 0) return;
    extern __shared__ __align__(16) float2 ys[];   // [nr][NVC], then reduction space
    const int k = blockIdx.y;
    const int s0 = blockIdx.x * ADJ_TILE;
    const float2* Yk = Yin + (size_t)k * nr * ldi + voff_i;
    for (int i = threadIdx.x; i < nr * NVC; i += GEMV_THREADS) {
        const int r = i / NVC, v = i - r * NVC;
        ys[i] = Yk[(size_t)r * ldi + v];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg >> 1;
    const float4* g = G + (size_t)k * nr * nvec + (s0 >> 1) + lane;
    float2 a0[NVC], a1[NVC];
#pragma unroll
    for (int v = 0; v < NVC; ++v) { a0[v] = make_float2(0.f, 0.f); a1[v] = make_float2(0.f, 0.f); }
    constexpr int W = GEMV_THREADS / 32;
    int r = warp;
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
        if (s < ns) Xout[((size_t)k * ns + s) * ldo + voff_o + v] = tot;
    }
}

// ------------------------------------------------------------------ SIMT complex GEMM
constexpr int GBM = 64, GBN = 64, GBK = 8;

template <bool ADJ>
__global__ void __launch_bounds__(256) cgemm_simt(
    const float2* __restrict__ G, int ldg, int nr, int ns,
    const float2* __restrict__ B, int ldb, int voff_b,
    float2* __restrict__ Cm, int ldc, int voff_c, int N, const int* active) {
    if (active && *active == 0) return;
    const int M = ADJ ? ns : nr;
    const int K = ADJ ? nr : ns;
    const int k = blockIdx.z;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    __shared__ __align__(16) float2 As[GBK][GBM];
    __shared__ __align__(16) float2 Bs[GBK][GBN];
    const float2* Gk = G + (size_t)k * nr * ldg;
    const float2* Bk = B + (size_t)k * K * ldb + voff_b;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int kt = 0; kt < K; kt += GBK) {
        // A tile -> As[kk][m]
        if (!ADJ) {
            const int m = tid >> 2, kq = (tid & 3) * 2;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m0 + m < M) v = *reinterpret_cast<const float4*>(Gk + (size_t)(m0 + m) * ldg + kt + kq);
            As[kq][m] = make_float2(v.x, v.y);
            As[kq + 1][m] = make_float2(v.z, v.w);
        } else {
            const int kk = tid >> 5, mq = (tid & 31) * 2;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kt + kk < K) v = *reinterpret_cast<const float4*>(Gk + (size_t)(kt + kk) * ldg + m0 + mq);
            As[kk][mq] = make_float2(v.x, -v.y);
            As[kk][mq + 1] = make_float2(v.z, -v.w);
        }
        {
            const int kk = tid >> 5, nq = (tid & 31) * 2;
            float2 b0 = make_float2(0.f, 0.f), b1 = make_float2(0.f, 0.f);
            if (kt + kk < K) {
                const float2* row = Bk + (size_t)(kt + kk) * ldb + n0 + nq;
                if (n0 + nq < N) b0 = row[0];
                if (n0 + nq + 1 < N) b1 = row[1];
            }
            Bs[kk][nq] = b0;
            Bs[kk][nq + 1] = b1;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n < N) Cm[((size_t)k * M + m) * ldc + voff_c + n] = acc[i][j];
        }
    }
}

template <int NVC>
void gemv_fwd_launch(mdc_plan* p, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                     int voff_o, cudaStream_t s, const int* active) {
    const size_t smem = (size_t)p->ldg * NVC * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemv_fwd_c64<NVC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    dim3 grid((p->nr + FWD_ROWS_PER_CTA - 1) / FWD_ROWS_PER_CTA, p->nf);
    gemv_fwd_c64<NVC><<<grid, GEMV_THREADS, smem, s>>>(
        reinterpret_cast<const float4*>(p->G), (int)p->ldg, p->nr, p->ns, in, ldi, voff_i, out, ldo,
        voff_o, active);
}

template <int NVC>
void gemv_adj_launch(mdc_plan* p, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                     int voff_o, cudaStream_t s, const int* active) {
    size_t smem = (size_t)p->nr * NVC * sizeof(float2);
    const size_t red = (size_t)(GEMV_THREADS / 32) * ADJ_TILE * NVC * sizeof(float2);
    if (smem < red) smem = red;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemv_adj_c64<NVC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    dim3 grid((unsigned)(p->ldg / ADJ_TILE), p->nf);
    gemv_adj_c64<NVC><<<grid, GEMV_THREADS, smem, s>>>(
        reinterpret_cast<const float4*>(p->G), (int)p->ldg, p->nr, p->ns, in, ldi, voff_i, out, ldo,
        voff_o, active);
}

}  // namespace

// Largest column count served by the GEMV kernels (shared memory holds ldg * NVC complex).
int gemv_max_columns() { return 4; }

void launch_product(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i,
                    float2* out, int ldo, int voff_o, int ncol, cudaStream_t s,
                    const int* active) {
    LaunchScope ls(p, s, adjoint ? MDC_KC_PRODUCT_ADJ : MDC_KC_PRODUCT_FWD);
    // the GEMV stages one frequency's input block (ldg or nr rows x ncol) in shared memory
    const int64_t stage = (int64_t)(adjoint ? p->nr : p->ldg) * ncol * (int64_t)sizeof(float2);
    if (ncol <= gemv_max_columns() && stage <= 200 * 1024) {
#define MDC_GEMV_CASE(n)                                                                  \
    case n:                                                                               \
        if (adjoint) gemv_adj_launch<n>(p, in, ldi, voff_i, out, ldo, voff_o, s, active); \
        else gemv_fwd_launch<n>(p, in, ldi, voff_i, out, ldo, voff_o, s, active);         \
        break;
        switch (ncol) {
            MDC_GEMV_CASE(1)
            MDC_GEMV_CASE(2)
            MDC_GEMV_CASE(3)
            MDC_GEMV_CASE(4)
        }
#undef MDC_GEMV_CASE
        return;
    }
    const int M = adjoint ? p->ns : p->nr;
    dim3 grid((ncol + GBN - 1) / GBN, (M + GBM - 1) / GBM, p->nf);
    const float2* G = reinterpret_cast<const float2*>(p->G);
    if (adjoint)
        cgemm_simt<true><<<grid, 256, 0, s>>>(G, (int)p->ldg, p->nr, p->ns, in, ldi, voff_i, out, ldo,
                                              voff_o, ncol, active);
    else
        cgemm_simt<false><<<grid, 256, 0, s>>>(G, (int)p->ldg, p->nr, p->ns, in, ldi, voff_i, out, ldo,
                                               voff_o, ncol, active);
}

}  // namespace mdc
