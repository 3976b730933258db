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
#include "lsqr_core.cuh"

namespace mdc {

int ensure_scratch(mdc_plan* p, int ncols);

namespace {

// Work state of one Marchenko solve (Eq. 5) on one GPU stream.
struct Solver {
    mdc_plan* p = nullptr;     // operator used inside LSQR (any storage)
    mdc_plan* pr = nullptr;    // operator for data, residuals and Green's functions (FP32 path)
    int nv = 0, n = 0, C = 0;
    int64_t B = 0;
    cudaStream_t s = nullptr;
    const int* cut = nullptr;
    float* blk[7] = {};        // U1 U2 V1 V2 W1 W2 D1
    double* csU = nullptr;
    double* csV = nullptr;
    double* part = nullptr;    // [PART_CTAS] partial sums of csU or csV
    double* sc = nullptr;      // [S_COUNT] LSQR scalars
    double* xs = nullptr;      // [X_COUNT] data norm, final residual ratio
    double* resid = nullptr;   // [nresid]
    int* act = nullptr;        // [nact]
    int* iters = nullptr;      // [nsolves]
    int nresid = 0, nact = 0, nsolves = 0;
    int ldv = 0, voff0 = 0;    // spectrum layout: columns per point and this system's first column
    bool async_alloc = false;  // stream-ordered allocation (serving)
    // The inverse transforms that produce v-hat also leave its spectra for the next forward product.
    // Off for served jobs: the stacked spectrum layout changes between iterations.
    bool fuse_v = true;

    void release(void* q) {
        if (!q) return;
        if (async_alloc) cudaFreeAsync(q, s);
        else cudaFree(q);
    }
    ~Solver() {
        for (float* b : blk) release(b);
        release(csU); release(csV); release(part); release(sc); release(xs); release(resid); release(act); release(iters);
    }
    template <typename T> cudaError_t get(T** q, size_t bytes) {
        return async_alloc ? cudaMallocAsync((void**)q, bytes, s) : cudaMalloc((void**)q, bytes);
    }
    void layout(int ld, int off) { ldv = ld; voff0 = off; }
    int LD() const { return ldv ? ldv : 2 * nv; }
    float* U1() { return blk[0]; } float* U2() { return blk[1]; }
    float* V1() { return blk[2]; } float* V2() { return blk[3]; }
    float* W1() { return blk[4]; } float* W2() { return blk[5]; }
    float* D1() { return blk[6]; }

    int alloc(bool keep_data) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < (keep_data ? 7 : 6) && e == cudaSuccess; ++i) e = get(&blk[i], B * sizeof(float));
        if (e == cudaSuccess) e = get(&csU, 2 * (size_t)C * sizeof(double));
        if (e == cudaSuccess) e = get(&csV, 2 * (size_t)C * sizeof(double));
        if (e == cudaSuccess) e = get(&part, PART_CTAS * sizeof(double));
        if (e == cudaSuccess) e = get(&sc, S_COUNT * sizeof(double));
        if (e == cudaSuccess) e = get(&xs, X_COUNT * sizeof(double));
        if (e == cudaSuccess) e = get(&resid, nresid * sizeof(double));
        if (e == cudaSuccess) e = get(&act, nact * sizeof(int));
        if (e == cudaSuccess) e = get(&iters, nsolves * sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_cuda_error(e);
            return MDC_ERR_OOM;
        }
        reset();
        return MDC_OK;
    }
    // Per-solve initial state (stream-ordered; part of a captured graph when graphs are on).
    void reset() {
        cudaMemsetAsync(xs, 0, X_COUNT * sizeof(double), s);
        cudaMemsetAsync(act, 0, nact * sizeof(int), s);
        cudaMemsetAsync(iters, 0, nsolves * sizeof(int), s);
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        fill_d<<<1, 256, 0, s>>>(resid, nresid, -1.0);
    }

    void rfft(mdc_plan* q, const float* x, const float* x2, const int* cutp, Coef scale, int conj, int voff,
              const int* active) {
        RfftArgs a{};
        a.x = x; a.x2 = x2; a.C = C; a.S = n; a.nv = nv; a.nt = q->nt; a.logn = q->logn; a.nf = q->nf; a.k0 = q->k0;
        a.cut = cutp; a.scale = scale; a.conj = conj; a.X = q->specA; a.ldv = LD(); a.voff = voff0 + voff;
        a.tw = q->tw; a.active = active;
        launch_rfft(q, a, s);
    }
    // fwd_voff >= 0: also the forward transform of the output (times the window fwd_cut if set,
    // unscaled, conjugated if fwd_conj) into specA at column offset fwd_voff -- the next product's
    // input, fused into the inverse kernel where it can be.
    void irfft(mdc_plan* q, int voff, int conj_in, float* out, Coef a_mdc, const int* cutp, const float* base,
               Coef a_base, Coef a_prev, double* colsum, int reverse, const int* active, float* xw_x = nullptr,
               float* xw_w = nullptr, int fwd_voff = -1, const int* fwd_cut = nullptr, int fwd_conj = 0) {
        IrfftArgs a{};
        if (fwd_voff >= 0) {
            a.fwd_X = q->specA;
            a.fwd_voff = voff0 + fwd_voff;
            a.fwd_cut = fwd_cut;
            a.fwd_conj = fwd_conj;
        }
        if (xw_w) {                   // the pending LSQR x/w step, applied with the previous v-hat
            a.xw_x = xw_x; a.xw_w = xw_w;
            a.xw_kx = sc + S_KX; a.xw_kw = sc + S_KW; a.xw_ia = sc + S_INV_ALPHA;
        }
        a.Y = q->specB; a.ldv = LD(); a.voff = voff0 + voff; a.C = C; a.S = n; a.nv = nv; a.nt = q->nt;
        a.logn = q->logn; a.nf = q->nf; a.k0 = q->k0; a.conj_in = conj_in;
        a.scale = (float)(q->dt * q->dr / (double)q->nt);
        a.out = out; a.a_mdc = a_mdc; a.a_base = a_base; a.a_prev = a_prev; a.base = base; a.cut = cutp;
        a.reverse_out = reverse; a.colsum = colsum; a.tw = q->tw; a.active = active;
        launch_irfft(q, a, s);
    }

    // u-hat = d = [Theta R f_d+ ; 0] (kernel pr), column sums into csU; D1 keeps d for refinement.
    void data_pass(const float* fd) {
        const Coef zero = C1(0.f);
        rfft(pr, fd, nullptr, nullptr, C1(1.f), 0, 0, nullptr);
        launch_product(pr, false, pr->specA, LD(), voff0, pr->specB, LD(), voff0, nv, s, nullptr);
        irfft(pr, 0, 0, U1(), C1(1.f), cut, nullptr, zero, zero, csU, 0, nullptr);
        cudaMemsetAsync(U2(), 0, B * sizeof(float), s);
        cudaMemsetAsync(csU + C, 0, C * sizeof(double), s);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            colsum_partials<<<PART_CTAS, 256, 0, s>>>(csU, 2 * C, part, nullptr);
            norm_store<<<1, RED_THREADS, 0, s>>>(part, PART_CTAS, xs + X_DNORM);
        }
        if (D1()) {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            copy_f<<<elementwise_grid(B), 256, 0, s>>>(B, U1(), D1());
        }
    }

    // u-hat = d - M x with the kernel pr:  [D1 - x1 + Theta R x2 ; -x2 + Theta R* x1], sums into csU.
    void residual_pass(const float* x1, const float* x2) {
        rfft(pr, x2, nullptr, nullptr, C1(1.f), 0, 0, nullptr);
        rfft(pr, x1, nullptr, nullptr, C1(1.f), 1, nv, nullptr);
        launch_product(pr, false, pr->specA, LD(), voff0, pr->specB, LD(), voff0, 2 * nv, s, nullptr);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            copy_f<<<elementwise_grid(B), 256, 0, s>>>(B, D1(), U1());
        }
        irfft(pr, 0, 0, U1(), C1(1.f), cut, x1, C1(-1.f), C1(1.f), csU, 0, nullptr);
        irfft(pr, nv, 1, U2(), C1(1.f), cut, x2, C1(-1.f), C1(0.f), csU + C, 0, nullptr);
    }

    // M^H u with u = u-hat / beta:  v-hat <- [a - (R*)^H Theta b ; b - R^H Theta a] + vprev * v-hat;
    // the inverse transforms also leave the unscaled spectra of v-hat for the first forward product
    // (1 / alpha is applied after that product).
    void apply_MH(const int* active, Coef vprev) {
        rfft(p, U1(), nullptr, cut, CD(1.f, sc + S_INV_BETA), 0, 0, active);
        rfft(p, U2(), nullptr, cut, CD(1.f, sc + S_INV_BETA), 1, nv, active);
        launch_product(p, true, p->specA, LD(), voff0, p->specB, LD(), voff0, 2 * nv, s, active);
        irfft(p, nv, 1, V1(), C1(-1.f), nullptr, U1(), CD(1.f, sc + S_INV_BETA), vprev, csV, 0, active, nullptr,
              nullptr, fuse_v ? nv : -1, nullptr, 1);
        irfft(p, 0, 0, V2(), C1(-1.f), nullptr, U2(), CD(1.f, sc + S_INV_BETA), vprev, csV + C, 0, active, nullptr,
              nullptr, fuse_v ? 0 : -1, nullptr, 0);
    }

    // LSQR start on u-hat (holding the right-hand side and its column sums): beta_1, then
    // alpha_1 v_1 = M^H u_1, w_1 = v_1; x is zeroed or kept (refinement accumulates into it).
    void lsqr_init(float* x1, float* x2, bool zero_x, int* act0, double* resid0) {
        const Coef zero = C1(0.f);
        const int eg = elementwise_grid(B);
        cudaMemsetAsync(sc, 0, S_COUNT * sizeof(double), s);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            colsum_partials<<<PART_CTAS, 256, 0, s>>>(csU, 2 * C, part, nullptr);
            lsqr_init_beta<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, resid0, act0 + 1);
        }
        apply_MH(act0 + 1, zero);
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            colsum_partials<<<PART_CTAS, 256, 0, s>>>(csV, 2 * C, part, act0 + 1);
            lsqr_init_alpha<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, act0 + 1);
        }
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        if (zero_x) lsqr_xw_init<<<eg, 256, 0, s>>>(B, x1, x2, W1(), W2(), V1(), V2(), sc);
        else lsqr_w_init<<<eg, 256, 0, s>>>(B, W1(), W2(), V1(), V2(), sc);
    }
    // One LSQR iteration in four phases around the forward and adjoint products (so several
    // systems can share one product over their stacked columns).  The adjoint product's input
    // spectra come from the inverse transforms before it (the forward transform of their output,
    // fused): the spectra of Theta u-hat without the 1 / beta that normalises u, which the inverse
    // transform after the product applies instead.  With fuse_v the forward product's input is made
    // the same way (spectra of v-hat, 1 / alpha applied after the product).
    //   u-hat <- M v - alpha u:  M [a; b] = [a - Theta R b ; b - Theta R* a]
    void iter_fwd_pre(const int* a) {
        if (fuse_v) return;
        rfft(p, V2(), nullptr, nullptr, CD(1.f, sc + S_INV_ALPHA), 0, 0, a);
        rfft(p, V1(), nullptr, nullptr, CD(1.f, sc + S_INV_ALPHA), 1, nv, a);
    }
    void iter_fwd_post(const int* a) {
        const Coef am = fuse_v ? CD(-1.f, sc + S_INV_ALPHA) : C1(-1.f);
        irfft(p, 0, 0, U1(), am, cut, V1(), CD(1.f, sc + S_INV_ALPHA), CD(1.f, sc + S_U_PREV), csU, 0, a, nullptr,
              nullptr, 0, cut, 0);
        irfft(p, nv, 1, U2(), am, cut, V2(), CD(1.f, sc + S_INV_ALPHA), CD(1.f, sc + S_U_PREV), csU + C, 0, a,
              nullptr, nullptr, nv, cut, 1);
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        colsum_partials<<<PART_CTAS, 256, 0, s>>>(csU, 2 * C, part, a);
        lsqr_beta<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, a);
    }
    //   v-hat <- M^H u - beta v
    void iter_adj_pre(const int*) {}
    // The adjoint transforms also apply the previous rotation's x/w step (x += (phi/rho) w,
    // w = v / alpha + kw w) with the v-hat they overwrite; the last rotation's x step is applied by
    // xw_flush at the end of the solve.
    void iter_adj_post(int it, int niter, double tol, int* act0, double* resid0, int* itp, float* x1, float* x2) {
        const int* a = act0 + it;
        const Coef vprev = CD(1.f, sc + S_V_PREV);
        irfft(p, nv, 1, V1(), CD(-1.f, sc + S_INV_BETA), nullptr, U1(), CD(1.f, sc + S_INV_BETA), vprev, csV, 0, a,
              x1, W1(), fuse_v ? nv : -1, nullptr, 1);
        irfft(p, 0, 0, V2(), CD(-1.f, sc + S_INV_BETA), nullptr, U2(), CD(1.f, sc + S_INV_BETA), vprev, csV + C, 0,
              a, x2, W2(), fuse_v ? 0 : -1, nullptr, 0);
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        colsum_partials<<<PART_CTAS, 256, 0, s>>>(csV, 2 * C, part, a);
        lsqr_alpha_rotate<<<1, RED_THREADS, 0, s>>>(sc, part, PART_CTAS, a, act0 + it + 1, resid0, itp, it,
                                                    niter, tol);
    }
    // The last rotation's pending x step (once per solve, after its last iteration).
    void xw_flush(float* x1, float* x2) {
        LaunchScope ls(p, s, MDC_KC_SOLVER);
        lsqr_x_flush<<<elementwise_grid(B), 256, 0, s>>>(B, x1, x2, W1(), W2(), sc);
    }

    // LSQR on u-hat (already holding the right-hand side and its column sums); x accumulates.
    // act0: niter + 2 flags, resid0: niter + 1 entries, itp: iteration counter of this solve.
    void lsqr(float* x1, float* x2, int niter, double tol, bool zero_x, int* act0, double* resid0, int* itp) {
        lsqr_init(x1, x2, zero_x, act0, resid0);
        for (int it = 1; it <= niter; ++it) {
            const int* a = act0 + it;
            nvtxRangePushA("mdc lsqr iteration");
            iter_fwd_pre(a);
            launch_product(p, false, p->specA, LD(), voff0, p->specB, LD(), voff0, 2 * nv, s, a);
            iter_fwd_post(a);
            iter_adj_pre(a);
            launch_product(p, true, p->specA, LD(), voff0, p->specB, LD(), voff0, 2 * nv, s, a);
            iter_adj_post(it, niter, tol, act0, resid0, itp, x1, x2);
            nvtxRangePop();
        }
        xw_flush(x1, x2);
    }

    // Neumann series of Eq. 5 (forward passes only): x_k = d + N x_{k-1} from x_0 = 0, with
    // N [a; b] = [Theta R b ; Theta R* a] and d = [D1; 0] (data_pass with keep_data); after niter
    // passes x = sum_{j<niter} N^j d.  Both halves of N come from one forward product over 2nv
    // columns; the spectra are taken before x is overwritten, so the update is in place.
    void neumann(float* x1, float* x2, int niter) {
        const Coef zero = C1(0.f);
        if (niter == 0) {
            cudaMemsetAsync(x1, 0, B * sizeof(float), s);
            cudaMemsetAsync(x2, 0, B * sizeof(float), s);
            return;
        }
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            copy_f<<<elementwise_grid(B), 256, 0, s>>>(B, D1(), x1);
        }
        cudaMemsetAsync(x2, 0, B * sizeof(float), s);
        for (int k = 2; k <= niter; ++k) {
            rfft(p, x2, nullptr, nullptr, C1(1.f), 0, 0, nullptr);
            rfft(p, x1, nullptr, nullptr, C1(1.f), 1, nv, nullptr);
            launch_product(p, false, p->specA, LD(), voff0, p->specB, LD(), voff0, 2 * nv, s, nullptr);
            irfft(p, 0, 0, x1, C1(1.f), cut, D1(), C1(1.f), zero, nullptr, 0, nullptr);
            irfft(p, nv, 1, x2, C1(1.f), cut, nullptr, zero, zero, nullptr, 0, nullptr);
        }
    }

    // Eq. 6: g- = R f+ - f-,  g+* = f+ - R* f-,  f+ = f_d+ + f_m+ ; g+ = time reversal of g+*
    void greens(const float* fd, const float* fm, const float* fmp, float* gm, float* gp) {
        const Coef zero = C1(0.f);
        float* fplus = W1();
        {
            LaunchScope ls(p, s, MDC_KC_SOLVER);
            vec_add<<<elementwise_grid(B), 256, 0, s>>>(B, fd, fmp, fplus);
        }
        rfft(pr, fplus, nullptr, nullptr, C1(1.f), 0, 0, nullptr);
        rfft(pr, fm, nullptr, nullptr, C1(1.f), 1, nv, nullptr);
        launch_product(pr, false, pr->specA, LD(), voff0, pr->specB, LD(), voff0, 2 * nv, s, nullptr);
        if (gm) irfft(pr, 0, 0, gm, C1(1.f), nullptr, fm, C1(-1.f), zero, nullptr, 0, nullptr);
        if (gp) irfft(pr, nv, 1, gp, C1(-1.f), nullptr, fplus, C1(1.f), zero, nullptr, 1, nullptr);
    }
};

struct GraphEntry {
    // key
    mdc_plan* pr;
    const int* cut;
    const float* fd;
    float* out[4];
    int nv, niter, nref, niter_ref;
    double tol;
    bool want_final;
    // value
    Solver* S = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void free_graph_entry(void* q) {
    GraphEntry* g = static_cast<GraphEntry*>(q);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g->S;
    delete g;
}

// The device work of one solve: data vector, LSQR (and refinement solves), residual check, Eq. 6.
void solve_body(Solver& S, const float* fd, int niter, int nref, int niter_ref, double tol, float* fm, float* fmp,
                float* gm, float* gp, bool want_final) {
    S.data_pass(fd);
    S.lsqr(fm, fmp, niter, tol, true, S.act, S.resid, S.iters);
    int aoff = niter + 2, roff = niter + 1;
    for (int o = 0; o < nref; ++o) {
        S.residual_pass(fm, fmp);
        S.lsqr(fm, fmp, niter_ref, tol, false, S.act + aoff, S.resid + roff, S.iters + 1 + o);
        aoff += niter_ref + 2;
        roff += niter_ref + 1;
    }
    if (want_final) {
        S.residual_pass(fm, fmp);
        LaunchScope ls(S.p, S.s, MDC_KC_SOLVER);
        colsum_partials<<<PART_CTAS, 256, 0, S.s>>>(S.csU, 2 * S.C, S.part, nullptr);
        norm_ratio<<<1, RED_THREADS, 0, S.s>>>(S.part, PART_CTAS, S.xs + X_DNORM, S.xs + X_FINAL);
    }
    if (gm || gp) S.greens(fd, fm, fmp, gm, gp);
}

void init_solver(Solver& S, mdc_plan* p, mdc_plan* pr, const int* cut, int nv, int niter, int nref, int niter_ref,
                 cudaStream_t s) {
    S.p = p;
    S.pr = pr;
    S.nv = nv;
    S.n = p->ns;
    S.C = p->ns * nv;
    S.B = (int64_t)p->nt * S.C;
    S.s = s;
    S.cut = cut;
    S.nsolves = 1 + nref;
    S.nresid = (niter + 1) + nref * (niter_ref + 1);
    S.nact = (niter + 2) + nref * (niter_ref + 2);
}

}  // namespace

// Solve Eq. 5 with LSQR on kernel p; with a reference kernel pr != p, refine: each outer step
// recomputes u-hat = d - M_pr x in float32 and runs niter_ref further LSQR iterations on p
// from the current x (the correction accumulates into x).
int run_marchenko(mdc_plan* p, mdc_plan* pr, const int* cut, const float* fd, int nv, int niter, int nref,
                  int niter_ref, double tol, float* fm, float* fmp, float* gm, float* gp, double* resid_h,
                  double* final_h, int* iters_h, cudaStream_t s) {
    // a frequency shard solves in lock step with the others only through its sum over shards
    if ((p->shard && !p->red_fn) || (pr->shard && !pr->red_fn)) return MDC_ERR_STATE;
    if (pr->k0 != p->k0 || pr->shard != p->shard) return MDC_ERR_ARG;
    int st = ensure_scratch(p, 2 * nv);
    if (st == MDC_OK && pr != p) st = ensure_scratch(pr, 2 * nv);
    if (st != MDC_OK) return st;
    const bool keep_data = nref > 0 || final_h != nullptr;
    Solver local;
    Solver* S = &local;
    GraphEntry* ge = nullptr;
    cudaStream_t caller = s;
    if (p->graphs && !p->red_fn && !pr->red_fn) {
        // capture and replay on the handle's own stream (the legacy default stream cannot be
        // captured), ordered after and before the caller's stream with events
        if (!p->graph_stream) {
            if (cudaStreamCreateWithFlags(&p->graph_stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->graph_ev[0], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->graph_ev[1], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return MDC_ERR_CUDA;
            }
        }
        s = p->graph_stream;
        cudaEventRecord(p->graph_ev[0], caller);
        cudaStreamWaitEvent(s, p->graph_ev[0], 0);
        for (void* q : p->graph_cache) {
            GraphEntry* g = static_cast<GraphEntry*>(q);
            if (g->pr == pr && g->cut == cut && g->fd == fd && g->out[0] == fm && g->out[1] == fmp && g->out[2] == gm &&
                g->out[3] == gp && g->nv == nv && g->niter == niter && g->nref == nref && g->niter_ref == niter_ref &&
                g->tol == tol && g->want_final == (final_h != nullptr)) {
                ge = g;
                break;
            }
        }
        if (!ge) {
            ge = new GraphEntry{pr, cut, fd, {fm, fmp, gm, gp}, nv, niter, nref, niter_ref, tol, final_h != nullptr};
            ge->S = new Solver();
            init_solver(*ge->S, p, pr, cut, nv, niter, nref, niter_ref, s);
            st = ge->S->alloc(keep_data);
            cudaGraph_t graph = nullptr;
            cudaError_t e = st == MDC_OK ? cudaStreamSynchronize(s) : cudaErrorMemoryAllocation;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                ge->S->reset();
                solve_body(*ge->S, fd, niter, nref, niter_ref, tol, fm, fmp, gm, gp, final_h != nullptr);
                e = cudaStreamEndCapture(s, &graph);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess || st != MDC_OK) {
                cudaGetLastError();
                set_cuda_error(e);
                free_graph_entry(ge);
                return st != MDC_OK ? st : MDC_ERR_CUDA;
            }
            p->graph_free = free_graph_entry;
            if (p->graph_cache.size() >= 4) {
                cudaStreamSynchronize(s);
                free_graph_entry(p->graph_cache.front());
                p->graph_cache.erase(p->graph_cache.begin());
            }
            p->graph_cache.push_back(ge);
        }
        S = ge->S;
        cudaError_t e = cudaGraphLaunch(ge->exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(p->graph_ev[1], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, p->graph_ev[1], 0);
        if (e != cudaSuccess) {
            set_cuda_error(e);
            return MDC_ERR_CUDA;
        }
        s = caller;
    } else {
        init_solver(local, p, pr, cut, nv, niter, nref, niter_ref, s);
        st = local.alloc(keep_data);
        if (st != MDC_OK) return st;
        solve_body(local, fd, niter, nref, niter_ref, tol, fm, fmp, gm, gp, final_h != nullptr);
    }

    std::vector<double> sch(S_COUNT), rh(S->nresid), xh(X_COUNT);
    std::vector<int> ih(S->nsolves);
    cudaError_t e = cudaMemcpyAsync(sch.data(), S->sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rh.data(), S->resid, S->nresid * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(xh.data(), S->xs, X_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ih.data(), S->iters, S->nsolves * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    if (resid_h) for (int i = 0; i < S->nresid; ++i) resid_h[i] = rh[i];
    if (final_h) *final_h = xh[X_FINAL];
    if (iters_h) {
        int tot = 0;
        for (int v : ih) tot += v;
        *iters_h = tot;
    }
    int err = 0;
    cudaMemcpy(&err, p->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return mdc::device_flag_status(err);
    const int he = take_host_error(p), her = pr != p ? take_host_error(pr) : MDC_OK;
    if (he != MDC_OK) return he;
    if (her != MDC_OK) return her;
    return sch[S_STATUS] != 0.0 ? MDC_ERR_NUMERIC : MDC_OK;
}

}  // namespace mdc

extern "C" int marchenko_lsqr(mdc_handle R, const int* window, const float* fd_plus, int nv, int niter,
                              double tol, float* f_minus, float* f_mplus, float* g_minus, float* g_plus,
                              double* resid, int* iters_done, void* stream) {
    if (!R || !window || !fd_plus || !f_minus || !f_mplus || nv < 1 || niter < 1) return MDC_ERR_ARG;
    if (R->nr != R->ns) return MDC_ERR_ARG;
    if (!std::isfinite(tol)) return MDC_ERR_ARG;
    return mdc::run_marchenko(R, R, window, fd_plus, nv, niter, 0, 0, tol, f_minus, f_mplus, g_minus, g_plus,
                              resid, nullptr, iters_done, (cudaStream_t)stream);
}

extern "C" int marchenko_lsqr_refined(mdc_handle R, mdc_handle R_ref, const int* window, const float* fd_plus,
                                      int nv, int niter, int nrefine, int niter_refine, double tol, float* f_minus,
                                      float* f_mplus, float* g_minus, float* g_plus, double* resid,
                                      double* final_residual, int* iters_done, void* stream) {
    if (!R || !R_ref || !window || !fd_plus || !f_minus || !f_mplus || nv < 1 || niter < 1) return MDC_ERR_ARG;
    if (nrefine < 0 || (nrefine > 0 && niter_refine < 1)) return MDC_ERR_ARG;
    if (R->nr != R->ns || R_ref->nr != R->nr || R_ref->ns != R->ns || R_ref->nt != R->nt ||
        R_ref->nf != R->nf || (R_ref->storage != MDC_C64 && R_ref->storage != MDC_C32S))
        return MDC_ERR_ARG;
    if (!std::isfinite(tol)) return MDC_ERR_ARG;
    return mdc::run_marchenko(R, R_ref, window, fd_plus, nv, niter, nrefine, niter_refine, tol, f_minus, f_mplus,
                              g_minus, g_plus, resid, final_residual, iters_done, (cudaStream_t)stream);
}

extern "C" int marchenko_neumann(mdc_handle R, const int* window, const float* fd_plus, int nv, int niter,
                                 float* f_minus, float* f_mplus, float* g_minus, float* g_plus, void* stream) {
    if (!R || !window || !fd_plus || !f_minus || !f_mplus || nv < 1 || niter < 0) return MDC_ERR_ARG;
    if (R->nr != R->ns) return MDC_ERR_ARG;
    if (R->shard && !R->red_fn) return MDC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int st = mdc::ensure_scratch(R, 2 * nv);
    if (st != MDC_OK) return st;
    mdc::Solver S;
    mdc::init_solver(S, R, R, window, nv, 1, 0, 0, s);
    st = S.alloc(true);
    if (st != MDC_OK) return st;
    S.data_pass(fd_plus);
    S.neumann(f_minus, f_mplus, niter);
    if (g_minus || g_plus) S.greens(fd_plus, f_minus, f_mplus, g_minus, g_plus);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        mdc::set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    int err = 0;
    cudaMemcpy(&err, R->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return mdc::device_flag_status(err);
    return mdc::take_host_error(R);
}

// ======================================================================== serving
// Continuous batching of redatuming jobs (Eq. 5 systems for groups of focusing points).
// Each job keeps its own LSQR state (vectors and float64 scalars) resident on the device.
// srv_step admits queued jobs while the HBM budget and the column capacity allow (their
// data vector and LSQR start run as their own passes), then advances EVERY running job
// by one LSQR iteration with their columns stacked side by side in one spectrum: one
// forward and one adjoint product stream the kernel once for all jobs.  Jobs that finish
// a solve move to refinement (float32 residual on the reference kernel) or complete
// (Green's functions, results copied to the caller's host buffers).
#include <chrono>
#include <cstring>
#include <deque>
#include <unordered_map>

namespace mdc {
namespace {

enum JobState { JOB_QUEUED = 0, JOB_RUNNING = 1, JOB_DONE = 2, JOB_FAILED = 3 };

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeJob {
    int64_t id = 0;
    int nv = 0, niter = 0;
    double tol = 0.0;
    const int* cut_h = nullptr;  // caller host inputs [ns][ld] and [nt][ns][ld] (first nv columns used)
    const float* fd_h = nullptr;
    int ld = 0;
    float* out[4] = {};          // caller host buffers: f-, f_m+, g-, g+ (nullable), [nt][ns][nv]
    int state = JOB_QUEUED, status = MDC_OK;
    Solver* S = nullptr;
    int* cut_d = nullptr;
    float* fd_d = nullptr;
    float* x[4] = {};            // device f-, f_m+, g-, g+
    int solve = 0, it = 0, aoff = 0, roff = 0;
    int iters = 0;
    double final_resid = -1.0;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    int64_t bytes = 0;
    bool bound = true;           // false for a resumed job until srv_bind gives its outputs
    std::vector<int> cut_own;    // inputs held by the server (resumed queued jobs)
    std::vector<float> fd_own;
    std::vector<float> res_own[4];  // results kept by the server for outputs given as NULL
    bool keep = false;              // keep NULL outputs (server setting at submission)
};

}  // namespace
}  // namespace mdc

using mdc::ServeJob;

struct mdc_server {
    mdc_plan* p = nullptr;       // kernel used inside LSQR
    mdc_plan* pr = nullptr;      // float32 reference kernel (data, residuals, Green's functions)
    int64_t budget = 0, used = 0;
    int max_cols = 0, cols = 0;
    int nref = 0, niter_ref = 0;
    cudaStream_t s = nullptr;
    int64_t next_id = 1;
    std::deque<ServeJob*> queue;
    std::vector<ServeJob*> running;
    std::unordered_map<int64_t, ServeJob*> jobs;
    int* flags_h = nullptr;      // pinned
    int flags_cap = 0;
    bool keep_results = false;   // keep outputs given as NULL for srv_result
};

namespace mdc {
namespace {

int64_t job_bytes(const mdc_plan* p, int nv) {
    const int64_t C = (int64_t)p->ns * nv, B = (int64_t)p->nt * C;
    return 12 * B * 4 + 4 * C * 8 + C * 4 + (1 << 20);
}

void free_job_device(mdc_server* v, ServeJob* j) {
    delete j->S;
    j->S = nullptr;
    cudaFreeAsync(j->cut_d, v->s);
    cudaFreeAsync(j->fd_d, v->s);
    for (float*& q : j->x) {
        if (q) cudaFreeAsync(q, v->s);
        q = nullptr;
    }
    j->cut_d = nullptr;
    j->fd_d = nullptr;
}

int start_job(mdc_server* v, ServeJob* j) {
    mdc_plan* p = v->p;
    const int64_t C = (int64_t)p->ns * j->nv, B = (int64_t)p->nt * C;
    cudaError_t e = cudaMallocAsync((void**)&j->cut_d, C * sizeof(int), v->s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&j->fd_d, B * sizeof(float), v->s);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMallocAsync((void**)&j->x[i], B * sizeof(float), v->s);
    const size_t w = (size_t)j->nv;
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(j->cut_d, w * sizeof(int), j->cut_h, (size_t)j->ld * sizeof(int), w * sizeof(int),
                              (size_t)p->ns, cudaMemcpyHostToDevice, v->s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(j->fd_d, w * sizeof(float), j->fd_h, (size_t)j->ld * sizeof(float), w * sizeof(float),
                              (size_t)p->ns * p->nt, cudaMemcpyHostToDevice, v->s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_cuda_error(e);
        free_job_device(v, j);
        return MDC_ERR_OOM;
    }
    Solver* S = new Solver();
    S->p = p;
    S->pr = v->pr;
    S->nv = j->nv;
    S->n = p->ns;
    S->C = (int)C;
    S->B = B;
    S->s = v->s;
    S->cut = j->cut_d;
    S->async_alloc = true;
    S->fuse_v = false;
    S->nsolves = 1 + v->nref;
    S->nresid = (j->niter + 1) + v->nref * (v->niter_ref + 1);
    S->nact = (j->niter + 2) + v->nref * (v->niter_ref + 2);
    j->S = S;
    int st = S->alloc(true);
    if (st != MDC_OK) {
        free_job_device(v, j);
        return st;
    }
    S->layout(0, 0);
    S->data_pass(j->fd_d);
    S->lsqr_init(j->x[0], j->x[1], true, S->act, S->resid);
    j->solve = 0;
    j->it = 0;
    j->aoff = 0;
    j->roff = 0;
    return MDC_OK;
}

// ---------------------------------------------------------------- checkpoint format
// Native-endian, fixed-width records: a header, then per queued or running job a record, its
// inputs (window, f_d+) and, for a running job, every device array of its solver state.
struct CkptHeader {
    char magic[8];
    int32_t version, nf, nr, ns, nt, storage, ref_storage, nref, niter_ref, njobs;
    int64_t next_id;
};
struct CkptJob {
    int64_t id;
    int32_t nv, niter, state, solve, it, aoff, roff, nresid, nact, nsolves;
    double tol, age_submit, age_start;
};
constexpr char kCkptMagic[8] = {'M', 'D', 'C', 'S', 'R', 'V', 0, 1};
constexpr int kCkptVersion = 1;

// The device arrays of a running job, in checkpoint order: (pointer, bytes).
std::vector<std::pair<void*, size_t>> job_arrays(ServeJob* j) {
    Solver* S = j->S;
    const size_t fb = (size_t)S->B * sizeof(float);
    std::vector<std::pair<void*, size_t>> v;
    for (float* b : S->blk) v.emplace_back(b, fb);
    v.emplace_back(j->x[0], fb);
    v.emplace_back(j->x[1], fb);
    v.emplace_back(S->csU, 2 * (size_t)S->C * sizeof(double));
    v.emplace_back(S->csV, 2 * (size_t)S->C * sizeof(double));
    v.emplace_back(S->sc, S_COUNT * sizeof(double));
    v.emplace_back(S->xs, X_COUNT * sizeof(double));
    v.emplace_back(S->resid, (size_t)S->nresid * sizeof(double));
    v.emplace_back(S->act, (size_t)S->nact * sizeof(int));
    v.emplace_back(S->iters, (size_t)S->nsolves * sizeof(int));
    return v;
}

int64_t ckpt_job_bytes(const mdc_plan* p, const CkptJob& r) {
    const int64_t C = (int64_t)p->ns * r.nv, B = (int64_t)p->nt * C;
    int64_t n = (int64_t)sizeof(CkptJob) + C * 4 + B * 4;
    if (r.state == JOB_RUNNING)
        n += 9 * B * 4 + 4 * C * 8 + (S_COUNT + X_COUNT + r.nresid) * 8 + (int64_t)(r.nact + r.nsolves) * 4;
    return n;
}

CkptJob ckpt_record(ServeJob* j, double now) {
    CkptJob r{};
    r.id = j->id;
    r.nv = j->nv;
    r.niter = j->niter;
    r.state = j->state;
    r.solve = j->solve;
    r.it = j->it;
    r.aoff = j->aoff;
    r.roff = j->roff;
    r.nresid = j->S ? j->S->nresid : 0;
    r.nact = j->S ? j->S->nact : 0;
    r.nsolves = j->S ? j->S->nsolves : 0;
    r.tol = j->tol;
    r.age_submit = now - j->t_submit;
    r.age_start = j->state == JOB_RUNNING ? now - j->t_start : 0.0;
    return r;
}

// Device state of a resumed running job: buffers as start_job allocates them, contents from the
// checkpoint (cur points at the job's window).
int restore_job(mdc_server* v, ServeJob* j, const CkptJob& r, const unsigned char* cur) {
    mdc_plan* p = v->p;
    const int64_t C = (int64_t)p->ns * j->nv, B = (int64_t)p->nt * C;
    cudaError_t e = cudaMallocAsync((void**)&j->cut_d, C * sizeof(int), v->s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&j->fd_d, B * sizeof(float), v->s);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMallocAsync((void**)&j->x[i], B * sizeof(float), v->s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_cuda_error(e);
        free_job_device(v, j);
        return MDC_ERR_OOM;
    }
    Solver* S = new Solver();
    S->p = p;
    S->pr = v->pr;
    S->nv = j->nv;
    S->n = p->ns;
    S->C = (int)C;
    S->B = B;
    S->s = v->s;
    S->cut = j->cut_d;
    S->async_alloc = true;
    S->fuse_v = false;
    S->nsolves = r.nsolves;
    S->nresid = r.nresid;
    S->nact = r.nact;
    j->S = S;
    int st = S->alloc(true);
    if (st != MDC_OK) {
        free_job_device(v, j);
        return st;
    }
    S->layout(0, 0);
    e = cudaMemcpyAsync(j->cut_d, cur, C * sizeof(int), cudaMemcpyHostToDevice, v->s);
    cur += C * sizeof(int);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->fd_d, cur, B * sizeof(float), cudaMemcpyHostToDevice, v->s);
    cur += B * sizeof(float);
    for (auto& a : job_arrays(j)) {
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(a.first, cur, a.second, cudaMemcpyHostToDevice, v->s);
        cur += a.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->s);   // the checkpoint buffer may go after return
    if (e != cudaSuccess) {
        set_cuda_error(e);
        free_job_device(v, j);
        return MDC_ERR_CUDA;
    }
    return MDC_OK;
}

// Complete a finished job: float32 residual check, Green's functions, results to the host.
void finish_job(mdc_server* v, ServeJob* j) {
    Solver* S = j->S;
    S->layout(0, 0);
    S->residual_pass(j->x[0], j->x[1]);
    {
        LaunchScope ls(v->p, v->s, MDC_KC_SOLVER);
        colsum_partials<<<PART_CTAS, 256, 0, v->s>>>(S->csU, 2 * S->C, S->part, nullptr);
        norm_ratio<<<1, RED_THREADS, 0, v->s>>>(S->part, PART_CTAS, S->xs + X_DNORM, S->xs + X_FINAL);
    }
    S->greens(j->fd_d, j->x[0], j->x[1], j->x[2], j->x[3]);
    const size_t bytes = (size_t)S->B * sizeof(float);
    for (int i = 0; i < 4; ++i) {
        float* dst = j->out[i];
        if (!dst && !j->keep) continue;           // not wanted
        if (!dst) {                               // no caller buffer: keep it for srv_result
            j->res_own[i].resize((size_t)S->B);
            dst = j->res_own[i].data();
        }
        cudaMemcpyAsync(dst, j->x[i], bytes, cudaMemcpyDeviceToHost, v->s);
    }
}

}  // namespace
}  // namespace mdc

using namespace mdc;

extern "C" int srv_create(mdc_server** out, mdc_handle R, mdc_handle R_ref, int64_t hbm_budget_bytes, int max_cols,
                          int nrefine, int niter_refine, void* stream) {
    if (!out) return MDC_ERR_ARG;
    *out = nullptr;
    if (!R || hbm_budget_bytes <= 0 || max_cols < 2 || R->nr != R->ns || nrefine < 0) return MDC_ERR_ARG;
    if (R->shard || (R_ref && R_ref->shard)) return MDC_ERR_ARG;   // the server takes whole operators
    if (R_ref && ((R_ref->storage != MDC_C64 && R_ref->storage != MDC_C32S) || R_ref->nr != R->nr ||
                  R_ref->ns != R->ns || R_ref->nt != R->nt || R_ref->nf != R->nf))
        return MDC_ERR_ARG;
    if (nrefine > 0 && (!R_ref || niter_refine < 1)) return MDC_ERR_ARG;
    mdc_server* v = new (std::nothrow) mdc_server();
    if (!v) return MDC_ERR_OOM;
    v->p = R;
    v->pr = R_ref ? R_ref : R;
    v->budget = hbm_budget_bytes;
    v->max_cols = max_cols;
    v->nref = nrefine;
    v->niter_ref = niter_refine;
    v->s = (cudaStream_t)stream;
    // one product path for every batch composition: a job's columns see the same arithmetic
    // alone or in a mix
    R->force_tc = (R->storage == MDC_C16F || R->storage == MDC_CBF16 || R->storage == MDC_CE4M3);
    int st = ensure_scratch(R, max_cols);
    if (st == MDC_OK && v->pr != R) st = ensure_scratch(v->pr, max_cols);
    if (st != MDC_OK) {
        delete v;
        return st;
    }
    *out = v;
    return MDC_OK;
}

extern "C" int srv_submit(mdc_server* v, const int* window_host, const float* fd_plus_host, int nv, int ld,
                          int niter, double tol, float* f_minus_host, float* f_mplus_host, float* g_minus_host,
                          float* g_plus_host, int64_t* job_id) {
    if (!v || !window_host || !fd_plus_host || nv < 1 || ld < nv || niter < 1 || !job_id || !std::isfinite(tol))
        return MDC_ERR_ARG;
    if (2 * nv > v->max_cols) return MDC_ERR_BUDGET;
    if (job_bytes(v->p, nv) > v->budget) return MDC_ERR_BUDGET;
    ServeJob* j = new (std::nothrow) ServeJob();
    if (!j) return MDC_ERR_OOM;
    j->id = v->next_id++;
    j->nv = nv;
    j->niter = niter;
    j->tol = tol;
    j->cut_h = window_host;
    j->fd_h = fd_plus_host;
    j->ld = ld;
    j->out[0] = f_minus_host;
    j->out[1] = f_mplus_host;
    j->out[2] = g_minus_host;
    j->out[3] = g_plus_host;
    j->bytes = job_bytes(v->p, nv);
    j->t_submit = now_s();
    j->keep = v->keep_results;
    v->queue.push_back(j);
    v->jobs[j->id] = j;
    *job_id = j->id;
    return MDC_OK;
}

extern "C" int srv_step(mdc_server* v, int* completed) {
    if (!v) return MDC_ERR_ARG;
    for (ServeJob* j : v->queue)
        if (!j->bound) return MDC_ERR_STATE;
    for (ServeJob* j : v->running)
        if (!j->bound) return MDC_ERR_STATE;
    int ndone = 0;
    // 1. admission, in arrival order, while memory and columns allow
    while (!v->queue.empty()) {
        ServeJob* j = v->queue.front();
        if (v->used + j->bytes > v->budget || v->cols + 2 * j->nv > v->max_cols) break;
        v->queue.pop_front();
        j->t_start = now_s();
        const int st = start_job(v, j);
        if (st != MDC_OK) {
            j->state = JOB_FAILED;
            j->status = st;
            j->t_done = now_s();
            ++ndone;
            continue;
        }
        j->state = JOB_RUNNING;
        v->used += j->bytes;
        v->cols += 2 * j->nv;
        v->running.push_back(j);
    }
    // 2. one LSQR iteration for every running job, columns stacked in one spectrum
    const int nrun = (int)v->running.size();
    if (nrun > 0) {
        int L = 0;
        std::vector<int> off(nrun);
        for (int i = 0; i < nrun; ++i) {
            off[i] = L;
            L += 2 * v->running[i]->nv;
        }
        std::vector<const int*> act(nrun);
        for (int i = 0; i < nrun; ++i) {
            ServeJob* j = v->running[i];
            j->S->layout(L, off[i]);
            act[i] = j->S->act + j->aoff + j->it + 1;
            j->S->iter_fwd_pre(act[i]);
        }
        launch_product(v->p, false, v->p->specA, L, 0, v->p->specB, L, 0, L, v->s, nullptr);
        for (int i = 0; i < nrun; ++i) v->running[i]->S->iter_fwd_post(act[i]);
        for (int i = 0; i < nrun; ++i) v->running[i]->S->iter_adj_pre(act[i]);
        launch_product(v->p, true, v->p->specA, L, 0, v->p->specB, L, 0, L, v->s, nullptr);
        for (int i = 0; i < nrun; ++i) {
            ServeJob* j = v->running[i];
            const int niter = j->solve == 0 ? j->niter : v->niter_ref;
            j->S->iter_adj_post(j->it + 1, niter, j->tol, j->S->act + j->aoff, j->S->resid + j->roff,
                                j->S->iters + j->solve, j->x[0], j->x[1]);
            j->it += 1;
            j->S->layout(0, 0);
        }
        // 3. which jobs go on: read each job's continue flag for its next iteration
        if (v->flags_cap < nrun) {
            if (v->flags_h) cudaFreeHost(v->flags_h);
            v->flags_cap = nrun * 2;
            if (cudaMallocHost((void**)&v->flags_h, v->flags_cap * sizeof(int)) != cudaSuccess) {
                v->flags_h = nullptr;
                v->flags_cap = 0;
                return MDC_ERR_OOM;
            }
        }
        for (int i = 0; i < nrun; ++i) {
            ServeJob* j = v->running[i];
            cudaMemcpyAsync(v->flags_h + i, j->S->act + j->aoff + j->it + 1, sizeof(int), cudaMemcpyDeviceToHost,
                            v->s);
        }
        cudaError_t e = cudaStreamSynchronize(v->s);
        if (e != cudaSuccess) {
            set_cuda_error(e);
            return MDC_ERR_CUDA;
        }
        // 4. finished solves: refine or complete
        std::vector<ServeJob*> keep, fin;
        for (int i = 0; i < nrun; ++i) {
            ServeJob* j = v->running[i];
            if (v->flags_h[i]) {
                keep.push_back(j);
                continue;
            }
            j->S->xw_flush(j->x[0], j->x[1]);     // this solve's last x step
            if (j->solve < v->nref) {
                const int niter = j->solve == 0 ? j->niter : v->niter_ref;
                j->S->residual_pass(j->x[0], j->x[1]);
                j->aoff += niter + 2;
                j->roff += niter + 1;
                j->solve += 1;
                j->it = 0;
                j->S->lsqr_init(j->x[0], j->x[1], false, j->S->act + j->aoff, j->S->resid + j->roff);
                keep.push_back(j);
            } else {
                finish_job(v, j);
                fin.push_back(j);
            }
        }
        if (!fin.empty()) {
            std::vector<std::vector<int>> its(fin.size());
            std::vector<double> res(fin.size()), bad(fin.size());
            for (size_t q = 0; q < fin.size(); ++q) {
                its[q].resize(fin[q]->S->nsolves);
                cudaMemcpyAsync(its[q].data(), fin[q]->S->iters, its[q].size() * sizeof(int), cudaMemcpyDeviceToHost,
                                v->s);
                cudaMemcpyAsync(&res[q], fin[q]->S->xs + X_FINAL, sizeof(double), cudaMemcpyDeviceToHost, v->s);
                cudaMemcpyAsync(&bad[q], fin[q]->S->sc + S_STATUS, sizeof(double), cudaMemcpyDeviceToHost, v->s);
            }
            e = cudaStreamSynchronize(v->s);
            if (e != cudaSuccess) {
                set_cuda_error(e);
                return MDC_ERR_CUDA;
            }
            for (size_t q = 0; q < fin.size(); ++q) {
                ServeJob* j = fin[q];
                int tot = 0;
                for (int x : its[q]) tot += x;
                j->iters = tot;
                j->final_resid = res[q];
                j->t_done = now_s();
                // a non-finite alpha or beta retires this job alone: its batch mates' columns never mix with it
                j->state = (bad[q] != 0.0 || !std::isfinite(res[q])) ? JOB_FAILED : JOB_DONE;
                if (j->state == JOB_FAILED) j->status = MDC_ERR_NUMERIC;
                v->used -= j->bytes;
                v->cols -= 2 * j->nv;
                free_job_device(v, j);
                ++ndone;
            }
        }
        v->running.swap(keep);
    }
    if (completed) *completed = ndone;
    return MDC_OK;
}

extern "C" int srv_poll(mdc_server* v, int64_t id, int* state, int* iters, double* final_residual,
                        double* latency_s, double* queue_s) {
    if (!v) return MDC_ERR_ARG;
    auto it = v->jobs.find(id);
    if (it == v->jobs.end()) return MDC_ERR_ARG;
    ServeJob* j = it->second;
    if (state) *state = j->state;
    if (iters) *iters = j->iters;
    if (final_residual) *final_residual = j->final_resid;
    if (latency_s) *latency_s = j->state >= JOB_DONE ? j->t_done - j->t_submit : -1.0;
    if (queue_s) *queue_s = j->state >= JOB_RUNNING ? j->t_start - j->t_submit : -1.0;
    return j->state == JOB_FAILED ? j->status : MDC_OK;
}

extern "C" int srv_result(mdc_server* v, int64_t id, float* f_minus_host, float* f_mplus_host, float* g_minus_host,
                          float* g_plus_host) {
    if (!v) return MDC_ERR_ARG;
    auto it = v->jobs.find(id);
    if (it == v->jobs.end()) return MDC_ERR_ARG;
    ServeJob* j = it->second;
    if (j->state == JOB_FAILED) return j->status;
    if (j->state != JOB_DONE) return MDC_ERR_STATE;
    float* dst[4] = {f_minus_host, f_mplus_host, g_minus_host, g_plus_host};
    const size_t n = (size_t)v->p->nt * v->p->ns * j->nv;
    for (int i = 0; i < 4; ++i) {
        if (!dst[i]) continue;
        const float* src = j->out[i] ? j->out[i] : j->res_own[i].data();
        if (!j->out[i] && j->res_own[i].size() < n) return MDC_ERR_STATE;   // not kept
        if (src != dst[i]) std::memcpy(dst[i], src, n * sizeof(float));
    }
    return MDC_OK;
}

extern "C" int srv_keep_results(mdc_server* v, int keep) {
    if (!v) return MDC_ERR_ARG;
    v->keep_results = keep != 0;
    return MDC_OK;
}

extern "C" int srv_release(mdc_server* v, int64_t id) {
    if (!v) return MDC_ERR_ARG;
    auto it = v->jobs.find(id);
    if (it == v->jobs.end()) return MDC_ERR_ARG;
    if (it->second->state < JOB_DONE) return MDC_ERR_STATE;
    delete it->second;
    v->jobs.erase(it);
    return MDC_OK;
}

extern "C" int srv_stats(mdc_server* v, int* queued, int* running, int64_t* bytes_in_use, int* cols_in_use) {
    if (!v) return MDC_ERR_ARG;
    if (queued) *queued = (int)v->queue.size();
    if (running) *running = (int)v->running.size();
    if (bytes_in_use) *bytes_in_use = v->used;
    if (cols_in_use) *cols_in_use = v->cols;
    return MDC_OK;
}

extern "C" int srv_checkpoint(mdc_server* v, void* buf, int64_t cap, int64_t* bytes) {
    if (!v || !bytes) return MDC_ERR_ARG;
    std::vector<ServeJob*> js(v->running.begin(), v->running.end());
    js.insert(js.end(), v->queue.begin(), v->queue.end());
    const double now = now_s();
    int64_t need = (int64_t)sizeof(CkptHeader);
    for (ServeJob* j : js) need += ckpt_job_bytes(v->p, ckpt_record(j, now));
    *bytes = need;
    if (!buf) return MDC_OK;
    if (cap < need) return MDC_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(v->s);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    unsigned char* cur = static_cast<unsigned char*>(buf);
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.version = kCkptVersion;
    h.nf = v->p->nf;
    h.nr = v->p->nr;
    h.ns = v->p->ns;
    h.nt = v->p->nt;
    h.storage = v->p->storage;
    h.ref_storage = v->pr->storage;
    h.nref = v->nref;
    h.niter_ref = v->niter_ref;
    h.njobs = (int32_t)js.size();
    h.next_id = v->next_id;
    std::memcpy(cur, &h, sizeof h);
    cur += sizeof h;
    const int ns = v->p->ns, nt = v->p->nt;
    for (ServeJob* j : js) {
        const CkptJob r = ckpt_record(j, now);
        std::memcpy(cur, &r, sizeof r);
        cur += sizeof r;
        const size_t nv = (size_t)j->nv, C = (size_t)ns * nv, B = (size_t)nt * C;
        if (j->state == JOB_RUNNING) {
            e = cudaMemcpyAsync(cur, j->cut_d, C * sizeof(int), cudaMemcpyDeviceToHost, v->s);
            cur += C * sizeof(int);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cur, j->fd_d, B * sizeof(float), cudaMemcpyDeviceToHost, v->s);
            cur += B * sizeof(float);
            for (auto& a : job_arrays(j)) {
                if (e != cudaSuccess) break;
                e = cudaMemcpyAsync(cur, a.first, a.second, cudaMemcpyDeviceToHost, v->s);
                cur += a.second;
            }
            if (e != cudaSuccess) {
                set_cuda_error(e);
                return MDC_ERR_CUDA;
            }
        } else {
            // queued: the inputs still live in host memory, rows of ld values
            for (size_t i = 0; i < (size_t)ns; ++i) std::memcpy(cur + i * nv * 4, j->cut_h + i * j->ld, nv * 4);
            cur += C * sizeof(int);
            for (size_t i = 0; i < (size_t)ns * nt; ++i) std::memcpy(cur + i * nv * 4, j->fd_h + i * j->ld, nv * 4);
            cur += B * sizeof(float);
        }
    }
    e = cudaStreamSynchronize(v->s);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MDC_ERR_CUDA;
    }
    return MDC_OK;
}

extern "C" int srv_resume(mdc_server* v, const void* buf, int64_t bytes, int64_t* ids, int max_ids, int* n_jobs) {
    if (!v || !buf || bytes < (int64_t)sizeof(CkptHeader)) return MDC_ERR_ARG;
    if (!v->queue.empty() || !v->running.empty()) return MDC_ERR_STATE;
    const unsigned char* base = static_cast<const unsigned char*>(buf);
    CkptHeader h;
    std::memcpy(&h, base, sizeof h);
    if (std::memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0 || h.version != kCkptVersion || h.njobs < 0)
        return MDC_ERR_ARG;
    if (h.nf != v->p->nf || h.nr != v->p->nr || h.ns != v->p->ns || h.nt != v->p->nt ||
        h.storage != v->p->storage || h.ref_storage != v->pr->storage || h.nref != v->nref ||
        h.niter_ref != v->niter_ref)
        return MDC_ERR_ARG;
    if (ids && max_ids < h.njobs) return MDC_ERR_ARG;
    // pass 1: validate every record against the buffer, the budget and the ids in use
    std::vector<CkptJob> recs(h.njobs);
    std::vector<int64_t> offs(h.njobs);
    int64_t off = sizeof h, used = v->used;
    int cols = v->cols;
    for (int q = 0; q < h.njobs; ++q) {
        if (off + (int64_t)sizeof(CkptJob) > bytes) return MDC_ERR_ARG;
        std::memcpy(&recs[q], base + off, sizeof(CkptJob));
        const CkptJob& r = recs[q];
        if (r.nv < 1 || r.niter < 1 || (r.state != JOB_QUEUED && r.state != JOB_RUNNING) || v->jobs.count(r.id) ||
            r.id >= h.next_id)
            return r.id >= 0 && v->jobs.count(r.id) ? MDC_ERR_STATE : MDC_ERR_ARG;
        if (r.state == JOB_RUNNING) {
            if (r.nsolves != 1 + v->nref || r.nresid != (r.niter + 1) + v->nref * (v->niter_ref + 1) ||
                r.nact != (r.niter + 2) + v->nref * (v->niter_ref + 2) || r.solve < 0 || r.solve > v->nref)
                return MDC_ERR_ARG;
            used += job_bytes(v->p, r.nv);
            cols += 2 * r.nv;
        }
        offs[q] = off + (int64_t)sizeof(CkptJob);
        off += ckpt_job_bytes(v->p, r);
        if (off > bytes) return MDC_ERR_ARG;
    }
    if (used > v->budget || cols > v->max_cols) return MDC_ERR_BUDGET;
    // pass 2: rebuild the jobs (running ones with their device state), in checkpoint order
    const double now = now_s();
    std::vector<ServeJob*> made;
    int st = MDC_OK;
    for (int q = 0; q < h.njobs && st == MDC_OK; ++q) {
        const CkptJob& r = recs[q];
        ServeJob* j = new (std::nothrow) ServeJob();
        if (!j) {
            st = MDC_ERR_OOM;
            break;
        }
        j->id = r.id;
        j->nv = r.nv;
        j->niter = r.niter;
        j->tol = r.tol;
        j->ld = r.nv;
        j->bytes = job_bytes(v->p, r.nv);
        j->t_submit = now - r.age_submit;
        j->bound = false;
        const unsigned char* cur = base + offs[q];
        if (r.state == JOB_RUNNING) {
            j->t_start = now - r.age_start;
            j->solve = r.solve;
            j->it = r.it;
            j->aoff = r.aoff;
            j->roff = r.roff;
            st = restore_job(v, j, r, cur);
            if (st != MDC_OK) {
                delete j;
                break;
            }
            j->state = JOB_RUNNING;
        } else {
            const size_t C = (size_t)v->p->ns * r.nv, B = (size_t)v->p->nt * C;
            j->cut_own.resize(C);
            j->fd_own.resize(B);
            std::memcpy(j->cut_own.data(), cur, C * sizeof(int));
            std::memcpy(j->fd_own.data(), cur + C * sizeof(int), B * sizeof(float));
            j->cut_h = j->cut_own.data();
            j->fd_h = j->fd_own.data();
        }
        made.push_back(j);
    }
    if (st != MDC_OK) {
        for (ServeJob* j : made) {
            if (j->S) free_job_device(v, j);
            delete j;
        }
        cudaStreamSynchronize(v->s);
        return st;
    }
    for (ServeJob* j : made) {
        v->jobs[j->id] = j;
        if (j->state == JOB_RUNNING) {
            v->running.push_back(j);
            v->used += j->bytes;
            v->cols += 2 * j->nv;
        } else {
            v->queue.push_back(j);
        }
    }
    if (h.next_id > v->next_id) v->next_id = h.next_id;
    if (ids)
        for (int q = 0; q < h.njobs; ++q) ids[q] = made[q]->id;
    if (n_jobs) *n_jobs = h.njobs;
    return MDC_OK;
}

extern "C" int srv_bind(mdc_server* v, int64_t id, float* f_minus_host, float* f_mplus_host, float* g_minus_host,
                        float* g_plus_host) {
    if (!v) return MDC_ERR_ARG;
    auto it = v->jobs.find(id);
    if (it == v->jobs.end()) return MDC_ERR_ARG;
    ServeJob* j = it->second;
    if (j->state != JOB_QUEUED && j->state != JOB_RUNNING) return MDC_ERR_STATE;
    j->out[0] = f_minus_host;
    j->out[1] = f_mplus_host;
    j->out[2] = g_minus_host;
    j->out[3] = g_plus_host;
    j->bound = true;
    return MDC_OK;
}

extern "C" int srv_destroy(mdc_server* v) {
    if (!v) return MDC_ERR_ARG;
    cudaStreamSynchronize(v->s);
    for (auto& kv : v->jobs) {
        if (kv.second->S) free_job_device(v, kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(v->s);
    if (v->flags_h) cudaFreeHost(v->flags_h);
    v->p->force_tc = false;
    delete v;
    return MDC_OK;
}
