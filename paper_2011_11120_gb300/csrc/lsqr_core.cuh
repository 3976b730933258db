// LSQR building blocks shared by the Marchenko (Eq. 5) and multi-dimensional deconvolution
// (Eq. 8) solvers: the float64 scalar recurrences of Paige and Saunders (1982), run on the
// device by one CTA with fixed-order sums, and the float32 vector updates.  Each translation
// unit that includes this header gets its own copies (internal linkage).
#pragma once

#include <cmath>

#include "common.cuh"

namespace mdc {
namespace {

enum Slot {
    S_ALPHA, S_BETA, S_RHO, S_RHOBAR, S_PHI, S_PHIBAR, S_C, S_S, S_THETA, S_BETA1,
    S_INV_ALPHA, S_INV_BETA, S_U_PREV, S_V_PREV, S_KX, S_KW, S_STATUS, S_COUNT
};

constexpr int RED_THREADS = 1024;

// Sum of v[0..n) by one CTA in a fixed order (deterministic): each thread keeps eight partial sums
// (eight loads in flight), combined pairwise, then a tree over the threads.
__device__ double block_sum(const double* v, int n) {
    __shared__ double red[RED_THREADS];
    constexpr int U = 8;
    double a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = 0.0;
    int i = threadIdx.x;
    for (; i + (U - 1) * RED_THREADS < n; i += U * RED_THREADS) {
        double t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) t[u] = v[i + u * RED_THREADS];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] += t[u];
    }
    for (; i < n; i += RED_THREADS) a[0] += v[i];
    const double acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Sums of squares are reduced in two fixed-order steps: colsum_partials writes PART_CTAS partial
// sums of contiguous chunks of the per-column sums (all SMs reading), then the one-CTA scalar
// kernel below sums the partials.  Skips its work when *act == 0 (act may be null).
constexpr int PART_CTAS = 304;
__global__ void __launch_bounds__(256) colsum_partials(const double* __restrict__ cs, int n,
                                                       double* __restrict__ part, const int* act) {
    if (act && *act == 0) return;
    __shared__ double red[256];
    const int chunk = (n + PART_CTAS - 1) / PART_CTAS;
    const int b0 = blockIdx.x * chunk, b1 = b0 + chunk < n ? b0 + chunk : n;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    int i = b0 + threadIdx.x;
    for (; i + 3 * 256 < b1; i += 4 * 256) {
        const double t0 = cs[i], t1 = cs[i + 256], t2 = cs[i + 512], t3 = cs[i + 768];
        a[0] += t0; a[1] += t1; a[2] += t2; a[3] += t3;
    }
    for (; i < b1; i += 256) a[0] += cs[i];
    red[threadIdx.x] = (a[0] + a[1]) + (a[2] + a[3]);
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// beta_1 = ||d||, u_1 = d / beta_1 (Paige-Saunders initialisation).
__global__ void __launch_bounds__(RED_THREADS) lsqr_init_beta(double* sc, const double* cs, int n,
                                                              double* resid, int* act1) {
    const double b = sqrt(block_sum(cs, n));
    if (threadIdx.x == 0) {
        sc[S_BETA] = b;
        sc[S_BETA1] = b;
        sc[S_PHIBAR] = b;
        sc[S_INV_BETA] = b > 0.0 ? 1.0 / b : 0.0;
        sc[S_V_PREV] = 0.0;
        sc[S_STATUS] = isfinite(b) ? 0.0 : 1.0;
        resid[0] = b;
        *act1 = (b > 0.0 && isfinite(b)) ? 1 : 0;
    }
}

// alpha_1 v_1 = M^H u_1, w_1 = v_1, rhobar_1 = alpha_1.
__global__ void __launch_bounds__(RED_THREADS) lsqr_init_alpha(double* sc, const double* cs, int n,
                                                               int* act1) {
    if (*act1 == 0) return;
    const double a = sqrt(block_sum(cs, n));
    if (threadIdx.x == 0) {
        sc[S_ALPHA] = a;
        sc[S_RHOBAR] = a;
        sc[S_INV_ALPHA] = a > 0.0 ? 1.0 / a : 0.0;
        sc[S_U_PREV] = a > 0.0 ? -a * sc[S_INV_BETA] : 0.0;
        if (!isfinite(a)) { sc[S_STATUS] = 1.0; *act1 = 0; }
        if (a == 0.0) *act1 = 0;   // M^H d = 0: x = 0 is a least-squares solution
    }
}

// After u-hat = M v - alpha u: beta = ||u-hat||, coefficients for the M^H step.
__global__ void __launch_bounds__(RED_THREADS) lsqr_beta(double* sc, const double* cs, int n,
                                                         const int* act) {
    if (*act == 0) return;
    const double b = sqrt(block_sum(cs, n));
    if (threadIdx.x == 0) {
        sc[S_BETA] = b;
        sc[S_INV_BETA] = b > 0.0 ? 1.0 / b : 0.0;
        sc[S_V_PREV] = -b * sc[S_INV_ALPHA];
        if (!isfinite(b)) sc[S_STATUS] = 1.0;
    }
}

// After v-hat = M^H u - beta v: alpha, the plane rotation, and the x/w coefficients.
__global__ void __launch_bounds__(RED_THREADS) lsqr_alpha_rotate(double* sc, const double* cs, int n,
                                                                 const int* act, int* act_next,
                                                                 double* resid, int* iters, int it,
                                                                 int niter, double tol) {
    if (*act == 0) return;
    double a = sqrt(block_sum(cs, n));
    if (threadIdx.x == 0) {
        const double b = sc[S_BETA];
        if (b == 0.0) a = 0.0;
        sc[S_ALPHA] = a;
        sc[S_INV_ALPHA] = a > 0.0 ? 1.0 / a : 0.0;
        const double rhobar = sc[S_RHOBAR], phibar = sc[S_PHIBAR];
        const double rho = hypot(rhobar, b);
        const double c = rhobar / rho, s = b / rho;
        const double theta = s * a;
        sc[S_RHO] = rho; sc[S_C] = c; sc[S_S] = s; sc[S_THETA] = theta;
        sc[S_RHOBAR] = -c * a;
        sc[S_PHI] = c * phibar;
        sc[S_PHIBAR] = s * phibar;
        sc[S_KX] = sc[S_PHI] / rho;
        sc[S_KW] = -theta / rho;
        sc[S_U_PREV] = -a * sc[S_INV_BETA];
        resid[it] = sc[S_PHIBAR];
        *iters = it;
        bool bad = !isfinite(a) || !isfinite(rho) || sc[S_STATUS] != 0.0;
        if (bad) sc[S_STATUS] = 1.0;
        const bool stop = bad || a == 0.0 || b == 0.0 || it >= niter ||
                          (tol > 0.0 && sc[S_PHIBAR] <= tol * sc[S_BETA1]);
        *act_next = stop ? 0 : 1;
    }
}

// The x and w updates with one rounding order for the scalar and the vector kernels.
__device__ __forceinline__ float xw_x(float x, float w, float kx) { return fmaf(kx, w, x); }
__device__ __forceinline__ float xw_w(float v, float w, float ia, float kw) { return fmaf(kw, w, ia * v); }

// The pending x step of the last plane rotation, x += (phi/rho) w, over both blocks: the w step of a
// rotation is applied with the next iteration's adjoint transform, which also applies the x step,
// so the last rotation's x step is left for the end of the solve.
__global__ void lsqr_x_flush(int64_t n, float* __restrict__ x1, float* __restrict__ x2, const float* __restrict__ w1,
                             const float* __restrict__ w2, const double* sc) {
    const float kx = (float)sc[S_KX];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x1[i] = xw_x(x1[i], w1[i], kx);
        x2[i] = xw_x(x2[i], w2[i], kx);
    }
}

// w_1 = v_1 = v-hat / alpha_1, x_0 = 0.
__global__ void lsqr_xw_init(int64_t n, float* __restrict__ x1, float* __restrict__ x2,
                             float* __restrict__ w1, float* __restrict__ w2,
                             const float* __restrict__ v1, const float* __restrict__ v2,
                             const double* sc) {
    const float ia = (float)sc[S_INV_ALPHA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x1[i] = 0.f;
        x2[i] = 0.f;
        w1[i] = ia * v1[i];
        w2[i] = ia * v2[i];
    }
}

__global__ void vec_add(int64_t n, const float* a, const float* b, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

__global__ void fill_d(double* p, int n, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

inline bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

int elementwise_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

// sqrt(sum of column sums) / reference norm, written to out (the FP64 residual check).
__global__ void __launch_bounds__(RED_THREADS) norm_ratio(const double* cs, int n, const double* ref, double* out) {
    const double v = sqrt(block_sum(cs, n));
    if (threadIdx.x == 0) *out = (*ref > 0.0) ? v / *ref : v;
}
__global__ void __launch_bounds__(RED_THREADS) norm_store(const double* cs, int n, double* out) {
    const double v = sqrt(block_sum(cs, n));
    if (threadIdx.x == 0) *out = v;
}

__global__ void copy_f(int64_t n, const float* a, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i];
}

// w_1 = v_1 = v-hat / alpha_1; x is kept (refinement continues from the current solution).
__global__ void lsqr_w_init(int64_t n, float* __restrict__ w1, float* __restrict__ w2,
                            const float* __restrict__ v1, const float* __restrict__ v2, const double* sc) {
    const float ia = (float)sc[S_INV_ALPHA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        w1[i] = ia * v1[i];
        w2[i] = ia * v2[i];
    }
}

enum Extra { X_DNORM, X_FINAL, X_COUNT };

}  // namespace
}  // namespace mdc
