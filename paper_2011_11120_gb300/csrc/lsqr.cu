// Marchenko redatuming by LSQR (Eq. 5) and Green's-function evaluation (Eq. 6).
//
// The block operator M = [[I, -Theta R], [-Theta R*, I]] is applied in ONE pass
// over the kernel with 2nv columns: R* x has spectrum conj(G conj(X)), so the
// conjugated spectrum of f^- rides along the columns of f_m^+ through the same
// forward product (row layout), and (R*)^H y = conj(G^H conj(Y)) rides along
// R^H in the adjoint product (column layout).  The Theta window, the identity
// term, the LSQR "minus alpha u" / "minus beta v" terms and the sum of squares
// of the result are fused into the inverse-FFT epilogue.
//
// LSQR follows Paige and Saunders (1982), x0 = 0.  Vectors u and v are stored
// unnormalised (u-hat = beta u, v-hat = alpha v) and the normalisations travel
// as device-resident float64 coefficients, so no pass exists only to rescale.
// The scalar recurrences (alpha, beta, rho, rhobar, c, s, theta, phi, phibar)
// run on the device in float64 with one CTA, summing the per-column sums of
// squares in a fixed order (results do not depend on scheduling).  Each
// iteration reads a device flag; once the recurrence decides to stop (niter,
// tolerance or breakdown) the remaining launches return immediately, so the
// host never waits inside the loop.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mdc {

int ensure_scratch(mdc_plan* p, int ncols);

namespace {

enum Slot {
    S_ALPHA, S_BETA, S_RHO, S_RHOBAR, S_PHI, S_PHIBAR, S_C, S_S, S_THETA, S_BETA1,
    S_INV_ALPHA, S_INV_BETA, S_U_PREV, S_V_PREV, S_KX, S_KW, S_STATUS, S_COUNT
};

constexpr int RED_THREADS = 1024;

__device__ double block_sum(const double* v, int n) {
    __shared__ double red[RED_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += RED_THREADS) acc += v[i];
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

// x += (phi/rho) w ;  w = v-hat / alpha - (theta/rho) w, over both blocks.
__global__ void lsqr_xw(int64_t n, float* __restrict__ x1, float* __restrict__ x2,
                        float* __restrict__ w1, float* __restrict__ w2,
                        const float* __restrict__ v1, const float* __restrict__ v2,
                        const double* sc, const int* act) {
    if (*act == 0) return;
    const float kx = (float)sc[S_KX], kw = (float)sc[S_KW], ia = (float)sc[S_INV_ALPHA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float w = w1[i];
        x1[i] += kx * w;
        w1[i] = ia * v1[i] + kw * w;
        w = w2[i];
        x2[i] += kx * w;
        w2[i] = ia * v2[i] + kw * w;
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

int elementwise_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

struct Buffers {
    float* blk[6] = {};        // U1 U2 V1 V2 W1 W2
    double* csU = nullptr;     // [2C]
    double* csV = nullptr;
    double* sc = nullptr;      // [S_COUNT]
    double* resid = nullptr;   // [niter+1]
    int* act = nullptr;        // [niter+2]
    int* iters = nullptr;
    ~Buffers() {
        for (float* b : blk) cudaFree(b);
        cudaFree(csU); cudaFree(csV); cudaFree(sc); cudaFree(resid); cudaFree(act); cudaFree(iters);
    }
};

}  // namespace

int run_marchenko_lsqr(mdc_plan* p, const int* cut, const float* fd, int nv, int niter, double tol,
                       float* fm, float* fmp, float* gm, float* gp, double* resid_h, int* iters_h,
                       cudaStream_t s) {
    const int n = p->ns;
    const int C = n * nv;
    const int64_t B = (int64_t)p->nt * C;
    int st = ensure_scratch(p, 2 * nv);
    if (st != MDC_OK) return st;
    Buffers b;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc(&b.blk[i], B * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.csU, 2 * C * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.csV, 2 * C * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.sc, S_COUNT * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.resid, (niter + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.act, (niter + 2) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b.iters, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_cuda_error(e);
        return MDC_ERR_OOM;
    }
    float *U1 = b.blk[0], *U2 = b.blk[1], *V1 = b.blk[2], *V2 = b.blk[3], *W1 = b.blk[4], *W2 = b.blk[5];
    const double* sc = b.sc;
    const int eg = elementwise_grid(B);

    cudaMemsetAsync(b.sc, 0, S_COUNT * sizeof(double), s);
    cudaMemsetAsync(b.act, 0, (niter + 2) * sizeof(int), s);
    cudaMemsetAsync(b.iters, 0, sizeof(int), s);
    {
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        fill_d<<<1, 256, 0, s>>>(b.resid, niter + 1, -1.0);
    }

    const float irscale = (float)(p->dt * p->dr / (double)p->nt);
    auto rfft = [&](const float* x, const float* x2, const int* cutp, Coef scale, int conj, int voff,
                    const int* active) {
        RfftArgs a{};
        a.x = x; a.x2 = x2; a.C = C; a.S = n; a.nv = nv; a.nt = p->nt; a.logn = p->logn; a.nf = p->nf;
        a.cut = cutp; a.scale = scale; a.conj = conj; a.X = p->specA; a.ldv = 2 * nv; a.voff = voff;
        a.tw = p->tw; a.active = active;
        launch_rfft(p, a, s);
    };
    auto irfft = [&](int voff, int conj_in, float* out, Coef a_mdc, const int* cutp, const float* base,
                     Coef a_base, Coef a_prev, double* colsum, int reverse, const int* active) {
        IrfftArgs a{};
        a.Y = p->specB; a.ldv = 2 * nv; a.voff = voff; a.C = C; a.S = n; a.nv = nv; a.nt = p->nt;
        a.logn = p->logn; a.nf = p->nf; a.conj_in = conj_in; a.scale = irscale; a.out = out;
        a.a_mdc = a_mdc; a.a_base = a_base; a.a_prev = a_prev; a.base = base; a.cut = cutp;
        a.reverse_out = reverse; a.colsum = colsum; a.tw = p->tw; a.active = active;
        launch_irfft(p, a, s);
    };
    const Coef zero = C1(0.f);

    // d = [Theta R f_d+ ; 0] -> u-hat, beta_1
    rfft(fd, nullptr, nullptr, C1(1.f), 0, 0, nullptr);
    launch_product(p, false, p->specA, 2 * nv, 0, p->specB, 2 * nv, 0, nv, s, nullptr);
    irfft(0, 0, U1, C1(1.f), cut, nullptr, zero, zero, b.csU, 0, nullptr);
    cudaMemsetAsync(U2, 0, B * sizeof(float), s);
    cudaMemsetAsync(b.csU + C, 0, C * sizeof(double), s);
    {
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        lsqr_init_beta<<<1, RED_THREADS, 0, s>>>(b.sc, b.csU, 2 * C, b.resid, b.act + 1);
    }
    // alpha_1 v_1 = M^H u_1 :  M^H [a; b] = [a - (R*)^H Theta b ; b - R^H Theta a]
    auto apply_MH = [&](const int* active, Coef vprev) {
        rfft(U1, nullptr, cut, CD(1.f, sc + S_INV_BETA), 0, 0, active);
        rfft(U2, nullptr, cut, CD(1.f, sc + S_INV_BETA), 1, nv, active);
        launch_product(p, true, p->specA, 2 * nv, 0, p->specB, 2 * nv, 0, 2 * nv, s, active);
        irfft(nv, 1, V1, C1(-1.f), nullptr, U1, CD(1.f, sc + S_INV_BETA), vprev, b.csV, 0, active);
        irfft(0, 0, V2, C1(-1.f), nullptr, U2, CD(1.f, sc + S_INV_BETA), vprev, b.csV + C, 0, active);
    };
    apply_MH(b.act + 1, zero);
    {
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        lsqr_init_alpha<<<1, RED_THREADS, 0, s>>>(b.sc, b.csV, 2 * C, b.act + 1);
    }
    {
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        lsqr_xw_init<<<eg, 256, 0, s>>>(B, fm, fmp, W1, W2, V1, V2, sc);
    }

    for (int it = 1; it <= niter; ++it) {
        const int* act = b.act + it;
        // u-hat <- M v - alpha u,  v = v-hat / alpha,  u = u-hat / beta
        //   M [a; b] = [a - Theta R b ; b - Theta R* a]
        rfft(V2, nullptr, nullptr, CD(1.f, sc + S_INV_ALPHA), 0, 0, act);
        rfft(V1, nullptr, nullptr, CD(1.f, sc + S_INV_ALPHA), 1, nv, act);
        launch_product(p, false, p->specA, 2 * nv, 0, p->specB, 2 * nv, 0, 2 * nv, s, act);
        irfft(0, 0, U1, C1(-1.f), cut, V1, CD(1.f, sc + S_INV_ALPHA), CD(1.f, sc + S_U_PREV), b.csU, 0, act);
        irfft(nv, 1, U2, C1(-1.f), cut, V2, CD(1.f, sc + S_INV_ALPHA), CD(1.f, sc + S_U_PREV), b.csU + C, 0,
              act);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            lsqr_beta<<<1, RED_THREADS, 0, s>>>(b.sc, b.csU, 2 * C, act);
        }
        // v-hat <- M^H u - beta v
        apply_MH(act, CD(1.f, sc + S_V_PREV));
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            lsqr_alpha_rotate<<<1, RED_THREADS, 0, s>>>(b.sc, b.csV, 2 * C, act, b.act + it + 1, b.resid,
                                                        b.iters, it, niter, tol);
        }
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            lsqr_xw<<<eg, 256, 0, s>>>(B, fm, fmp, W1, W2, V1, V2, sc, act);
        }
    }

    // Eq. 6: g- = R f+ - f-,  g+* = f+ - R* f-,  f+ = f_d+ + f_m+ ; g+ = time reversal of g+*
    if (gm || gp) {
        float* fplus = W1;   // w is no longer needed
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            vec_add<<<eg, 256, 0, s>>>(B, fd, fmp, fplus);
        }
        rfft(fplus, nullptr, nullptr, C1(1.f), 0, 0, nullptr);
        rfft(fm, nullptr, nullptr, C1(1.f), 1, nv, nullptr);
        launch_product(p, false, p->specA, 2 * nv, 0, p->specB, 2 * nv, 0, 2 * nv, s, nullptr);
        if (gm) irfft(0, 0, gm, C1(1.f), nullptr, fm, C1(-1.f), zero, nullptr, 0, nullptr);
        if (gp) irfft(nv, 1, gp, C1(-1.f), nullptr, fplus, C1(1.f), zero, nullptr, 1, nullptr);
    }

    std::vector<double> sch(S_COUNT);
    std::vector<double> rh(niter + 1);
    int ih = 0;
    e = cudaMemcpyAsync(sch.data(), b.sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rh.data(), b.resid, (niter + 1) * sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ih, b.iters, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    if (resid_h) for (int i = 0; i <= niter; ++i) resid_h[i] = rh[i];
    if (iters_h) *iters_h = ih;
    return sch[S_STATUS] != 0.0 ? MDC_ERR_NUMERIC : MDC_OK;
}

}  // namespace mdc

extern "C" int marchenko_lsqr(mdc_handle R, const int* window, const float* fd_plus, int nv, int niter,
                              double tol, float* f_minus, float* f_mplus, float* g_minus, float* g_plus,
                              double* resid, int* iters_done, void* stream) {
    if (!R || !window || !fd_plus || !f_minus || !f_mplus || nv < 1 || niter < 1) return MDC_ERR_ARG;
    if (R->nr != R->ns) return MDC_ERR_ARG;
    if (!std::isfinite(tol)) return MDC_ERR_ARG;
    return mdc::run_marchenko_lsqr(R, window, fd_plus, nv, niter, tol, f_minus, f_mplus, g_minus, g_plus,
                                   resid, iters_done, (cudaStream_t)stream);
}
