// Multi-dimensional deconvolution (Eq. 8): the local reflectivity r solves g- = G+ r, a
// Fredholm equation of the first kind with the MDC operator of the down-going Green's function
// G+(omega, x_S, x_F) as its kernel (Section "Source-side redatuming via Multi-dimensional
// deconvolution").  No Neumann expansion applies, so it is solved by LSQR (x0 = 0), one batch
// of nv virtual sources x_F' per call; each iteration costs one forward and one adjoint MDC.
//
// Layout: kernel [nf][nr][ns] with nr = n(x_S) rows and ns = n(x_F) columns (rectangular
// allowed), data g- [nt][nr][nv], reflectivity r [nt][ns][nv].  The LSQR state follows the
// Marchenko solver: u and v unnormalised, the normalisations as device float64 coefficients
// applied by the FFT prologue, the "minus alpha u" / "minus beta v" terms and the sums of
// squares fused into the inverse-FFT epilogue, scalars on the device, a device flag per
// iteration so the host never waits inside the loop.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "lsqr_core.cuh"

namespace mdc {

int ensure_scratch(mdc_plan* p, int ncols);

namespace {

// x += (phi/rho) w ;  w = v-hat / alpha - (theta/rho) w  (one block).
__global__ void lsqr_xw_one(int64_t n, float* __restrict__ x, float* __restrict__ w, const float* __restrict__ v,
                            const double* sc, const int* act) {
    if (*act == 0) return;
    const float kx = (float)sc[S_KX], kw = (float)sc[S_KW], ia = (float)sc[S_INV_ALPHA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float wi = w[i];
        x[i] += kx * wi;
        w[i] = ia * v[i] + kw * wi;
    }
}

// x_0 = 0, w_1 = v_1 = v-hat / alpha_1.
__global__ void lsqr_xw_one_init(int64_t n, float* __restrict__ x, float* __restrict__ w,
                                 const float* __restrict__ v, const double* sc) {
    const float ia = (float)sc[S_INV_ALPHA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = 0.f;
        w[i] = ia * v[i];
    }
}

// u-hat = d and the float64 sum of squares of each of its columns (fixed order over t).
__global__ void copy_colsum(int nt, int C, const float* __restrict__ d, float* __restrict__ u,
                           double* __restrict__ cs) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double acc = 0.0;
    for (int t = 0; t < nt; ++t) {
        const float v = d[(size_t)t * C + c];
        u[(size_t)t * C + c] = v;
        acc += (double)v * (double)v;
    }
    cs[c] = acc;
}

struct MddSolver {
    mdc_plan* p = nullptr;
    cudaStream_t s = nullptr;
    int nv = 0, Cu = 0, Cv = 0;   // columns of the data (nr * nv) and model (ns * nv) spaces
    int64_t Bu = 0, Bv = 0;       // elements of one data / model vector
    float *U = nullptr, *V = nullptr, *W = nullptr;
    double *csU = nullptr, *csV = nullptr, *part = nullptr, *sc = nullptr, *resid = nullptr;
    int *act = nullptr, *iters = nullptr;

    ~MddSolver() {
        for (void* q : {(void*)U, (void*)V, (void*)W, (void*)csU, (void*)csV, (void*)part, (void*)sc, (void*)resid, (void*)act,
                        (void*)iters})
            if (q) cudaFree(q);
    }
    int alloc(int niter) {
        cudaError_t e = cudaMalloc(&U, Bu * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&V, Bv * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&W, Bv * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&csU, (size_t)Cu * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&csV, (size_t)Cv * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&part, PART_CTAS * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&sc, S_COUNT * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&resid, (size_t)(niter + 1) * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&act, (size_t)(niter + 2) * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&iters, sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_cuda_error(e);
            return MDC_ERR_OOM;
        }
        cudaMemsetAsync(sc, 0, S_COUNT * sizeof(double), s);
        cudaMemsetAsync(act, 0, (size_t)(niter + 2) * sizeof(int), s);
        cudaMemsetAsync(iters, 0, sizeof(int), s);
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        fill_d<<<1, 256, 0, s>>>(resid, niter + 1, -1.0);
        return MDC_OK;
    }

    // spectrum of in/scale ([nt][S][nv], S = nr for the data space, ns for the model space)
    void rfft(const float* in, int S, Coef scale, const int* active) {
        RfftArgs a{};
        a.x = in; a.x2 = nullptr; a.C = S * nv; a.S = S; a.nv = nv; a.nt = p->nt; a.logn = p->logn; a.nf = p->nf;
        a.k0 = p->k0;
        a.cut = nullptr; a.scale = scale; a.conj = 0; a.X = p->specA; a.ldv = nv; a.voff = 0; a.tw = p->tw;
        a.active = active;
        launch_rfft(p, a, s);
    }
    // out = a_mdc (operator result) + a_prev * out, with the column sums of squares of the new out,
    // and the unscaled spectrum of the new out into specA: the next product's input (the forward
    // transform fused into the inverse kernel where it can be)
    void irfft(float* out, int S, Coef a_mdc, Coef a_prev, double* colsum, const int* active) {
        IrfftArgs a{};
        a.Y = p->specB; a.ldv = nv; a.voff = 0; a.C = S * nv; a.S = S; a.nv = nv; a.nt = p->nt; a.logn = p->logn;
        a.nf = p->nf; a.k0 = p->k0; a.conj_in = 0; a.scale = (float)(p->dt * p->dr / (double)p->nt); a.out = out;
        a.a_mdc = a_mdc; a.a_base = C1(0.f); a.a_prev = a_prev; a.base = nullptr; a.cut = nullptr;
        a.reverse_out = 0; a.colsum = colsum; a.tw = p->tw; a.active = active;
        a.fwd_X = p->specA; a.fwd_voff = 0; a.fwd_cut = nullptr; a.fwd_conj = 0;
        launch_irfft(p, a, s);
    }
    void product(bool adjoint, const int* active) {
        launch_product(p, adjoint, p->specA, nv, 0, p->specB, nv, 0, nv, s, active);
    }

    void solve(const float* d, float* x, int niter, double tol) {
        const int eg = elementwise_grid(Bv);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            copy_colsum<<<(Cu + 255) / 256, 256, 0, s>>>(p->nt, Cu, d, U, csU);
            colsum_partials<<<PART_CTAS, 256, 0, s>>>(csU, Cu, part, nullptr);
            lsqr_init_beta<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, resid, act + 1);
        }
        // alpha_1 v_1 = G+^H u_1.  Each product's input is the unscaled spectrum the inverse
        // transform before it leaves (of v-hat, of u-hat); 1 / alpha and 1 / beta, which normalise
        // v and u, are applied by the inverse transform after the product.
        rfft(U, p->nr, CD(1.f, sc + S_INV_BETA), act + 1);
        product(true, act + 1);
        irfft(V, p->ns, C1(1.f), C1(0.f), csV, act + 1);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            colsum_partials<<<PART_CTAS, 256, 0, s>>>(csV, Cv, part, act + 1);
            lsqr_init_alpha<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, act + 1);
            lsqr_xw_one_init<<<eg, 256, 0, s>>>(Bv, x, W, V, sc);
        }
        for (int it = 1; it <= niter; ++it) {
            const int* a = act + it;
            // u-hat <- G+ v - alpha u
            product(false, a);
            irfft(U, p->nr, CD(1.f, sc + S_INV_ALPHA), CD(1.f, sc + S_U_PREV), csU, a);
            {
                LaunchScope ls(p, s, MDC_KC_SOLVER);
                colsum_partials<<<PART_CTAS, 256, 0, s>>>(csU, Cu, part, a);
                lsqr_beta<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, a);
            }
            // v-hat <- G+^H u - beta v
            product(true, a);
            irfft(V, p->ns, CD(1.f, sc + S_INV_BETA), CD(1.f, sc + S_V_PREV), csV, a);
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            colsum_partials<<<PART_CTAS, 256, 0, s>>>(csV, Cv, part, a);
            lsqr_alpha_rotate<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, a, act + it + 1, resid, iters, it, niter,
                                                        tol);
            lsqr_xw_one<<<eg, 256, 0, s>>>(Bv, x, W, V, sc, a);
        }
    }
};

}  // namespace
}  // namespace mdc

using namespace mdc;

extern "C" int mdd_lsqr(mdc_handle Gplus, const float* g_minus, int nv, int niter, double tol, float* r,
                        double* resid, int* iters_done, void* stream) {
    if (!Gplus || !g_minus || !r || nv < 1 || niter < 1 || !std::isfinite(tol)) return MDC_ERR_ARG;
    mdc_plan* p = Gplus;
    if (p->shard && !p->red_fn) return MDC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int st = ensure_scratch(p, nv);
    if (st != MDC_OK) return st;
    MddSolver S;
    S.p = p;
    S.s = s;
    S.nv = nv;
    S.Cu = p->nr * nv;
    S.Cv = p->ns * nv;
    S.Bu = (int64_t)p->nt * S.Cu;
    S.Bv = (int64_t)p->nt * S.Cv;
    st = S.alloc(niter);
    if (st != MDC_OK) return st;
    S.solve(g_minus, r, niter, tol);
    std::vector<double> rh(niter + 1), sch(S_COUNT);
    int it = 0;
    cudaError_t e = cudaMemcpyAsync(rh.data(), S.resid, (niter + 1) * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sch.data(), S.sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&it, S.iters, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    if (resid)
        for (int i = 0; i <= niter; ++i) resid[i] = rh[i];
    if (iters_done) *iters_done = it;
    int err = 0;
    cudaMemcpy(&err, p->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return mdc::device_flag_status(err);
    const int he = take_host_error(p);
    if (he != MDC_OK) return he;
    return sch[S_STATUS] != 0.0 ? MDC_ERR_NUMERIC : MDC_OK;
}
