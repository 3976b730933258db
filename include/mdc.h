/*
 * mdc.h -- C ABI of the GB300 multi-dimensional convolution (MDC) library.
 *
 * The library applies the MDC operator of Ravasi & Vasconcelos (arXiv 2011.11120)
 * and solves the Marchenko redatuming system built on it, on one NVIDIA GB300
 * (sm_103a).  Every operation runs in hand-written CUDA kernels; there is no CPU
 * fallback.  Plain pointers and sizes only: no C++ or framework types cross it.
 *
 * Conventions shared by every call
 *   - Time-domain arrays are real float32, row-major [nt][n_space][nv] (nv fastest).
 *   - The kernel G is complex64 interleaved (re, im), row-major [nfmax][nr][ns]
 *     (s fastest): G[k][r][s] = K(w_k, x_r, x_s), w_k = 2 pi k / (nt dt).
 *   - "Device pointer" means memory the caller allocated on the current CUDA device;
 *     the caller keeps ownership.  The handle owns its copy of G and its scratch.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are stream-ordered and asynchronous unless documented as blocking.
 *   - Every call returns an mdc_status; no exception or abort crosses the ABI.
 *     A negative status leaves the handle usable unless it is MDC_ERR_CUDA, which
 *     reports a CUDA error (the context may then be unusable; see mdc_last_cuda_error).
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef MDC_GB300_H
#define MDC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdc_plan* mdc_handle;

typedef enum {
    MDC_OK = 0,
    MDC_ERR_ARG = -1,       /* invalid argument (null pointer, size out of range, ...) */
    MDC_ERR_OOM = -2,       /* device allocation failed */
    MDC_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    MDC_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up */
    MDC_ERR_NUMERIC = -5,   /* non-finite value met in a solver recurrence */
    MDC_ERR_BUDGET = -6,    /* request exceeds the configured memory budget */
    MDC_ERR_STATE = -7,     /* call not valid in the handle's current state */
    MDC_ERR_BOUNDS = -8     /* debug build only: a kernel index outside its buffer was caught (the
                               access was skipped); reported by mdc_device_status */
} mdc_status;

/* Storage format of the library-owned kernel copy (Section "Implementing the batch
 * matrix multiplication operator": the kernel streamed once per pass dominates cost). */
typedef enum {
    MDC_C64 = 0,    /* complex float32 (the paper's complex64 kernel, Table 1) */
    MDC_C16F = 1,   /* complex float16, one float32 scale per (frequency, row) */
    MDC_CBF16 = 2,  /* complex bfloat16, one float32 scale per (frequency, row) */
    MDC_CE4M3 = 3,  /* complex FP8 E4M3, one float32 scale per (frequency, row); tensor-core products
                       of at most 21 columns take the spectra as three E4M3 terms (about 12
                       significant bits), wider ones as FP16 */
    MDC_C32S = 4    /* complex as an FP16 pair hi + lo per component (about 22 significant bits,
                       float32-level accuracy), one float32 scale per (frequency, row); 8 bytes per
                       value like complex64, but products run on FP16 tensor cores */
} mdc_storage;

/* mdc_forward / mdc_adjoint flags */
#define MDC_CONJ_KERNEL 0x1u  /* use the conjugated kernel: R* (correlation) in Eq. 5 */

/* Kernel classes for the timing counters (mdc_timing_read). */
typedef enum {
    MDC_KC_RFFT = 0,        /* F and I_wmax of Eq. 3 (plus window and time reversal) */
    MDC_KC_PRODUCT_FWD = 1, /* K-hat of Eq. 3: per-frequency G(w) X(w) */
    MDC_KC_PRODUCT_ADJ = 2, /* K-hat^H of Eq. 3: per-frequency G(w)^H Y(w) */
    MDC_KC_IRFFT = 3,       /* I_wmax^H and F^H of Eq. 3 (plus fused epilogues) */
    MDC_KC_SOLVER = 4,      /* LSQR scalar recurrences and vector updates */
    MDC_KC_TC_PREP = 5,     /* tensor-core products: spectra to the 16-bit (or E4M3 three-term) operand
                               and column scales (the products' own time is in MDC_KC_PRODUCT_FWD / _ADJ) */
    MDC_KC_COUNT = 6
} mdc_kernel_class;

/*
 * mdc_create -- build an MDC operator C = F^H I^H K-hat I F (Eq. 3) for kernel G.
 *
 *   G        device pointer, complex64 interleaved [nfmax][nr][ns]: the first nfmax
 *            frequencies of the kernel (Eq. 2, truncated spectrum).  Read only; it is
 *            copied (and for reduced storage quantised) into a library-owned, padded
 *            layout, so the caller may free G when the call returns.
 *   nfmax    number of kept frequencies, 1 <= nfmax <= nt/2 + 1.
 *   nr, ns   output (receiver/row) and integration (source/column) sizes, >= 1.
 *   nt       number of time samples: a power of two in [64, 4096].
 *   dt, dr   time step and areal integration weight; the operator is scaled by dt*dr
 *            (the integration step multiplied into the kernel, Theory section).
 *   storage  an mdc_storage value.
 *   stream   stream for the copy kernels.
 * Blocking: allocates device memory and synchronises `stream` before returning.
 * Errors: MDC_ERR_ARG for bad sizes or a null pointer, MDC_ERR_OOM if the copy does
 * not fit; *out is set to NULL on failure.
 */
int mdc_create(mdc_handle* out, const void* G, int nfmax, int nr, int ns, int nt,
               double dt, double dr, int storage, void* stream);

/* mdc_create_weighted -- as mdc_create, with a per-column integration weight: the kernel's
 * column s (integration point x_R) is multiplied by weights[s] before it is copied or
 * quantised, so the operator integrates with dt * dr * weights[s].  This is the receiver-
 * dependent scaling for irregular geometries (areal extent of each receiver's Voronoi cell)
 * that the paper pre-multiplies into the kernel before the batched products (Theory section,
 * discretisation paragraph; irregular-geometry example).  weights: host double[ns], finite
 * and >= 0 (MDC_ERR_ARG otherwise), read during the call.  Pass dr = 1 for weights in m^2. */
int mdc_create_weighted(mdc_handle* out, const void* G, const double* weights, int nfmax, int nr, int ns, int nt,
                        double dt, double dr, int storage, void* stream);

/*
 * mdc_create_empty -- as mdc_create, but the library-owned kernel copy starts as zeros and
 * is filled one frequency slab at a time with mdc_load_slab.  This is for kernels larger
 * than the free device memory left beside a full complex64 staging copy (the paper's Full
 * geometry, Table 1: 300 frequencies of a 9801 x 9801 kernel, 230 GB in complex64, which
 * the paper keeps partitioned by frequency over its nodes, Section "Implementing the batch
 * matrix multiplication operator").  Same arguments and
 * errors as mdc_create without G; blocking.
 */
int mdc_create_empty(mdc_handle* out, int nfmax, int nr, int ns, int nt, double dt, double dr,
                     int storage, void* stream);

/*
 * mdc_load_slab -- copy (complex64 storage) or quantise (reduced storage, with the same
 * per-row scales mdc_create computes) frequencies k0 .. k0+nk-1 of the kernel into the
 * handle's copy.
 *   G_slab  device pointer, complex64 interleaved [nk][nr][ns]: kernel frequencies k0..k0+nk-1.
 *           Read only; the call synchronises `stream` before returning, so the caller may
 *           reuse or free the buffer afterwards.
 *   k0, nk  0 <= k0, nk >= 1, k0 + nk <= nfmax (MDC_ERR_ARG otherwise).
 * Loading every frequency once gives the same operator, bit for bit, as mdc_create on the
 * whole kernel; frequencies never loaded stay zero.  Not to be called while a product on
 * this handle is in flight on another stream.
 */
int mdc_load_slab(mdc_handle h, const void* G_slab, int k0, int nk, void* stream);

/*
 * mdc_forward -- y = C x (Eq. 3, left), or y = R* x with MDC_CONJ_KERNEL (Eq. 5).
 *   x  device float32 [nt][ns][nv] (input function f, integration axis ns).
 *   y  device float32 [nt][nr][nv] (output function g), fully overwritten.
 *   nv number of virtual points (columns), >= 1.
 * Stream-ordered.  Grows the handle's scratch on first use of a larger nv (which
 * allocates, so call mdc_reserve first when capturing into a CUDA graph).
 */
int mdc_forward(mdc_handle h, const float* x, float* y, int nv, unsigned flags, void* stream);

/*
 * mdc_adjoint -- x = C^H y (Eq. 3, right), or x = (R*)^H y with MDC_CONJ_KERNEL.
 *   y  device float32 [nt][nr][nv];  x  device float32 [nt][ns][nv], overwritten.
 * The same kernel buffer is read transposed; no second copy of G exists.
 */
int mdc_adjoint(mdc_handle h, const float* y, float* x, int nv, unsigned flags, void* stream);

/* mdc_reserve -- size the handle's scratch for up to nv_max columns per pass (blocking). */
int mdc_reserve(mdc_handle h, int nv_max);

/*
 * Frequency shards.  The method partitions the kernel along frequency with no communication
 * inside the per-frequency products (Section "Implementing the batch matrix multiplication
 * operator", Fig. 2): since the inverse transform is linear, the output of C is the sum over
 * disjoint bands of frequencies of each band's partial inverse transform.  A shard handle holds
 * bins k0 .. k0+nk-1 of the kernel; several of them (one per device or process) whose bands
 * tile 0 .. nfmax-1 make up the whole operator.
 *
 * mdc_create_shard -- as mdc_create for the kernel frequencies k0 .. k0+nk-1 only.
 *   G       device pointer, complex64 [nk][nr][ns] (bins k0 .. k0+nk-1), or NULL for a zero
 *           kernel to be filled with mdc_load_slab (its k0 then counts from the shard's first
 *           bin, 0 <= k0 + nk <= this shard's nk).
 *   k0, nk  0 <= k0, nk >= 1, k0 + nk <= nt/2 + 1 (MDC_ERR_ARG otherwise).
 * Without a reduction hook, mdc_forward / mdc_adjoint on a shard return the shard's partial
 * output (the inverse transform of its bins only, with the DC and Nyquist bins weighted once
 * and every other bin twice, as in the whole operator); the caller sums them.  Blocking.
 */
int mdc_create_shard(mdc_handle* out, const void* G, int k0, int nk, int nr, int ns, int nt, double dt, double dr,
                     int storage, void* stream);

/*
 * mdc_allreduce_fn -- the caller's sum over shards.  Called on the host thread of the library
 * call, in stream order: buf is a library-owned device array of `count` float32 values holding
 * this shard's partial signal; on return the work the function enqueued on `stream` (a
 * cudaStream_t as void*) must leave in buf the element-wise sum over all shards, or the
 * function must have synchronised `stream`, summed and copied back itself.  Every shard calls
 * it the same number of times with the same counts.  Returns MDC_OK or a negative status,
 * which the library call then returns.
 */
typedef int (*mdc_allreduce_fn)(float* buf, int64_t count, void* stream, void* ctx);

/*
 * mdc_set_allreduce -- give a shard handle its sum over shards (fn NULL removes it).  With a
 * hook, every inverse transform of the handle (mdc_forward, mdc_adjoint, marchenko_lsqr,
 * marchenko_lsqr_refined, marchenko_neumann, mdd_lsqr) writes its partial signal [nt][C] to a
 * handle-owned buffer (allocated on first use, grown as needed), calls fn on it, and applies
 * the remaining terms (window, identity and LSQR terms, norms) to the sum, so every shard
 * holds the complete result and identical LSQR scalars: the shards' solvers run in lock step,
 * one sum per pass, the LSQR vectors replicated.  Solves on a shard handle need a hook
 * (MDC_ERR_STATE otherwise); CUDA-graph replay is not used on hooked handles, and the serving
 * engine does not take shards.  MDC_ERR_ARG for a handle that is not a shard.
 */
int mdc_set_allreduce(mdc_handle h, mdc_allreduce_fn fn, void* ctx);

/*
 * mdc_forward_static_scratch -- y = C x (or R* x with MDC_CONJ_KERNEL) exactly as
 * mdc_forward, but without allocating anything: the two frequency-domain work
 * arrays live in one fixed device array compiled into the library instead of in
 * memory the handle obtains with cudaMalloc.  The paper has no counterpart; this
 * is a deployment variant of the forward pass.
 *
 * Who needs it: callers that cannot call cudaMalloc when they apply the operator:
 * services whose device memory is entirely pre-reserved by their own pool allocator
 * (a framework's caching allocator, a fixed per-tenant budget), so that a library
 * allocation would fail or break their accounting; and latency-critical loops that
 * cannot afford the device-wide synchronisation a cudaMalloc implies.  mdc_forward,
 * by contrast, allocates on its first call with a larger nv.
 *
 * Limit: nfmax * max(nr, ns) * nv <= MDC_STATIC_SCRATCH_COMPLEX (2^21 complex
 * values per work array; the fixed array is 32 MiB).  Larger requests return
 * MDC_ERR_BUDGET and launch nothing.  Every device that loads the library holds
 * the 32 MiB until the process exits.
 * Set-up: the first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it; make that first call before
 * any stream capture.  Later calls do no set-up.
 * Sharing: all calls on a device use the same array and it keeps the last call's
 * contents; every call overwrites all of it that it reads, so nothing needs
 * clearing.  Calls whose execution overlaps on the GPU (different streams without
 * ordering between them) race on the array and give wrong results: order them.
 * Overlapping calls on the same handle also share the handle's tensor-core operand
 * buffers, and race on those too.
 * Tensor cores: with 16-bit, split or E4M3 storage, products of 8 or more columns run
 * on tensor cores only if the handle's operand buffers were reserved beforehand
 * (mdc_reserve(h, nv), which allocates, so call it at set-up); otherwise the product
 * runs on the slower SIMT path (correct, and counted by mdc_tc_fallback_count).
 * Arguments, layout, ownership and errors are otherwise those of mdc_forward.
 */
#define MDC_STATIC_SCRATCH_COMPLEX (1 << 21)
int mdc_forward_static_scratch(mdc_handle h, const float* x, float* y, int nv, unsigned flags,
                               void* stream);

/*
 * marchenko_lsqr -- solve the Marchenko system of Eq. 5 by LSQR and evaluate Eq. 6.
 *
 *   d = M f,  M = [[I, -Theta R], [-Theta R*, I]],  d = [Theta R f_d+ ; 0],
 *   f = [f- ; f_m+],  then  g- = R f+ - f-,  g+* = f+ - R* f-,  f+ = f_d+ + f_m+.
 *
 *   R        handle whose kernel is the reflection response (requires nr == ns).
 *   window   device int32 [ns][nv]: Theta cut-offs; Theta[t][s][v] = 1 iff
 *            |tau(t)| < window[s][v], tau(t) = t for t < nt/2 and t - nt otherwise.
 *   fd_plus  device float32 [nt][ns][nv]: initial (direct) focusing function f_d+.
 *   nv       number of focusing points solved together as one system (one set of
 *            LSQR scalars for all nv columns).
 *   niter    maximum LSQR iterations (>= 1); tol > 0 also stops when the residual
 *            estimate falls to tol * ||d||, tol <= 0 runs exactly niter iterations.
 *   f_minus, f_mplus   device float32 [nt][ns][nv] outputs (the solution).
 *   g_minus, g_plus    device float32 [nt][ns][nv] outputs or NULL (skips Eq. 6);
 *            g_plus receives g+, the time reversal of the second row of Eq. 6.
 *   resid    host double[niter + 1] or NULL: ||d||, then the LSQR residual estimate
 *            after each iteration (unused tail entries set to -1).
 *   iters_done host int or NULL: iterations actually performed.
 * Blocking: synchronises `stream` before returning (host outputs).  Allocates its
 * work vectors (5 block vectors of 2*nt*ns*nv floats) for the duration of the call.
 * Errors: MDC_ERR_ARG (nr != ns, bad sizes, null required pointer), MDC_ERR_OOM,
 * MDC_ERR_NUMERIC (a non-finite alpha or beta).
 */
int marchenko_lsqr(mdc_handle R, const int* window, const float* fd_plus, int nv, int niter,
                   double tol, float* f_minus, float* f_mplus, float* g_minus, float* g_plus,
                   double* resid, int* iters_done, void* stream);

/*
 * marchenko_lsqr_refined -- marchenko_lsqr with a reduced-precision kernel copy inside LSQR
 * and float32-operator refinement (iterative refinement of the least-squares solution).
 *
 *   R        handle with any storage (typically MDC_C16F/MDC_CBF16) used inside LSQR.
 *   R_ref    float32-accurate handle (MDC_C64, or MDC_C32S whose products run on tensor cores)
 *            of the same kernel and shape: it computes the data vector d, the residuals
 *            d - M x, the Green's functions and the final check.
 *   niter    LSQR iterations of the first solve (from x = 0).
 *   nrefine  outer refinement steps: each recomputes r = d - M_ref x in float32 and runs
 *            niter_refine further LSQR iterations on R, adding the correction to x.
 *   resid    host double[(niter + 1) + nrefine * (niter_refine + 1)] or NULL: for each solve,
 *            its right-hand-side norm then its residual estimates (-1 where not reached).
 *   final_residual  host double or NULL: ||d - M_ref x|| / ||d||, accumulated in float64.
 * Other arguments as marchenko_lsqr.  Blocking.  MDC_ERR_ARG if R_ref is neither MDC_C64 nor
 * MDC_C32S or the shapes differ.
 */
int marchenko_lsqr_refined(mdc_handle R, mdc_handle R_ref, const int* window, const float* fd_plus,
                           int nv, int niter, int nrefine, int niter_refine, double tol,
                           float* f_minus, float* f_mplus, float* g_minus, float* g_plus,
                           double* resid, double* final_residual, int* iters_done, void* stream);

/* marchenko_neumann -- Eq. 5 by its Neumann series, the forward-only scheme of the solution
 * discussion in Section "Marchenko redatuming": with N = [[0, Theta R], [Theta R*, 0]] and
 * d = [Theta R f_d+; 0], x_k = d + N x_{k-1} from x_0 = 0, so the result is the partial sum
 * sum_{j<niter} N^j d (one forward pass of 2nv columns per term after the first).  It
 * converges only when the spectral radius of N is below 1.  niter = 0 gives f- = f_m+ = 0, for
 * which Eq. 6 yields the single-scattering Green's functions g0- = R f_d+ and g+ = P f_d+.
 * Arguments and layouts as marchenko_lsqr (g_minus, g_plus nullable); niter >= 0; nr == ns.
 * Blocking. */
int marchenko_neumann(mdc_handle R, const int* window, const float* fd_plus, int nv, int niter,
                      float* f_minus, float* f_mplus, float* g_minus, float* g_plus, void* stream);

/* mdd_lsqr -- multi-dimensional deconvolution, Eq. 8 (Section "Source-side redatuming via
 * Multi-dimensional deconvolution"): the local reflectivity r solving g- = G+ r by LSQR
 * (Paige-Saunders, x0 = 0, float64 scalars on the device, float32 vectors), one batch of nv
 * virtual sources per call.  Gplus: handle whose kernel is the down-going Green's function
 * G+[nf][nr][ns] (nr = receivers x_S, ns = focusing points x_F; rectangular allowed; any
 * storage).  g_minus: device float32 [nt][nr][nv] (data, caller-owned, not modified);
 * r: device float32 [nt][ns][nv] (output).  niter >= 1 iterations, or fewer when
 * ||r_k|| <= tol * ||g-|| (tol > 0).  resid: host double[niter + 1] (residual-norm estimates,
 * -1 after the stop; may be NULL); *iters_done: iterations performed (may be NULL).  Each
 * iteration is one forward and one adjoint MDC.  Blocking.  MDC_ERR_NUMERIC on a non-finite
 * recurrence. */
int mdd_lsqr(mdc_handle Gplus, const float* g_minus, int nv, int niter, double tol, float* r, double* resid,
             int* iters_done, void* stream);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of redatuming jobs (Eq. 5 for groups of focusing points,
 * the paper's embarrassingly parallel level of the Discussion, served on one GPU).
 *
 * Jobs arrive with srv_submit (host inputs, copied).  srv_step admits queued jobs in
 * arrival order while the device-memory budget and the column capacity allow, then
 * advances every running job by one LSQR iteration: all running jobs' columns are
 * stacked so ONE forward and ONE adjoint product stream the kernel for all of them.
 * Each job keeps its own float64 LSQR scalars, so its result does not depend on which
 * jobs share its steps (with an FP16/BF16 kernel the server routes every product through
 * the tensor-core path so the arithmetic per column is the same for any batch).  A job
 * that finishes its solve is refined (nrefine steps of niter_refine iterations against
 * the complex64 reference kernel), then its Green's functions (Eq. 6) and float64
 * residual check ||d - M_ref x|| / ||d|| are computed and its outputs copied to the host
 * buffers given at submission.
 * ------------------------------------------------------------------------------------ */
typedef struct mdc_server* mdc_server_handle;

enum { MDC_JOB_QUEUED = 0, MDC_JOB_RUNNING = 1, MDC_JOB_DONE = 2, MDC_JOB_FAILED = 3 };

/* srv_create -- R: kernel used inside LSQR (nr == ns); R_ref: float32-accurate reference of the
 * same kernel (MDC_C64 or MDC_C32S) or NULL (then R serves for data and Green's functions, and nrefine must be 0).
 * hbm_budget_bytes bounds the device memory of running jobs' state (about 48 bytes per
 * time sample per column); max_cols bounds the stacked columns (2 per virtual point).
 * The server owns R's scratch while it exists.  Allocates; blocking. */
int srv_create(mdc_server_handle* out, mdc_handle R, mdc_handle R_ref, int64_t hbm_budget_bytes,
               int max_cols, int nrefine, int niter_refine, void* stream);
/* srv_submit -- queue one job: window int32 [ns][ld] and fd_plus float32 [nt][ns][ld] in host
 * memory, of which the first nv columns are the job's (ld >= nv; pinned memory copies fastest).
 * The buffers are NOT copied at submission: they are read when the job is admitted, so the
 * caller keeps them unchanged until the job completes.  niter LSQR iterations (tol > 0: stop
 * earlier at tol * ||d||).  The four host output buffers [nt][ns][nv] are written when the job
 * completes; any of them may be NULL (that result is dropped, or kept for srv_result after
 * srv_keep_results(s, 1)).  MDC_ERR_BUDGET if the job can never fit the budget or the column
 * capacity.  *job_id receives the job's id. */
int srv_submit(mdc_server_handle s, const int* window_host, const float* fd_plus_host, int nv, int ld,
               int niter, double tol, float* f_minus_host, float* f_mplus_host, float* g_minus_host,
               float* g_plus_host, int64_t* job_id);
/* srv_step -- admit, advance every running job by one iteration, complete finished jobs
 * (their host outputs are written before return).  Blocking.  *completed = jobs completed. */
int srv_step(mdc_server_handle s, int* completed);
/* srv_poll -- state (MDC_JOB_*), iterations, final residual ratio, latency (submit to
 * completion, s) and queueing delay (submit to admission, s); -1 where not yet known.
 * Returns the job's error status if it failed. */
int srv_poll(mdc_server_handle s, int64_t job_id, int* state, int* iters, double* final_residual,
             double* latency_s, double* queue_s);
/* srv_keep_results -- keep = 1: jobs submitted from now on keep the results whose output
 * buffers are given as NULL in server-owned host memory until srv_release, for srv_result;
 * keep = 0 (the default): such results are dropped. */
int srv_keep_results(mdc_server_handle s, int keep);
/* srv_result -- copy a completed job's outputs [nt][ns][nv] into the given host buffers (each may
 * be NULL), from the buffers given at submission or from the server's kept copy.
 * MDC_ERR_STATE while the job is queued or running or if a requested result was neither given a
 * buffer nor kept; the job's error status if it failed. */
int srv_result(mdc_server_handle s, int64_t job_id, float* f_minus_host, float* f_mplus_host, float* g_minus_host,
               float* g_plus_host);
/* srv_release -- forget a completed or failed job (MDC_ERR_STATE while queued/running). */
int srv_release(mdc_server_handle s, int64_t job_id);
/* srv_stats -- queued and running job counts, bytes and columns in use. */
int srv_stats(mdc_server_handle s, int* queued, int* running, int64_t* bytes_in_use, int* cols_in_use);
/* srv_checkpoint -- serialise every queued and running job into host memory so that a server
 * built later (another process, after a failure) can carry on with srv_resume.  The record holds
 * each job's inputs and, for a running job, its whole solver state (LSQR vectors and float64
 * scalars, iterate, refinement stage), so the resumed solve continues bit for bit where it
 * stopped.  Completed jobs are not included (their outputs are already in the caller's
 * buffers).  buf == NULL: only *bytes is set (the size needed); otherwise cap >= *bytes
 * (MDC_ERR_ARG if smaller).  Call between srv_step calls; blocking.  The format is native-endian
 * with fixed-width fields, for the same library version.  The paper has no counterpart. */
int srv_checkpoint(mdc_server_handle s, void* buf, int64_t cap, int64_t* bytes);
/* srv_resume -- rebuild the jobs of a checkpoint on a server with no queued or running jobs,
 * created over kernels of the same shape and storage formats with the same refinement
 * settings (MDC_ERR_ARG otherwise; MDC_ERR_STATE if the server has live jobs or already knows
 * one of the ids; MDC_ERR_BUDGET if the running jobs do not fit its budget or column
 * capacity, in which case nothing changes).  Jobs keep their ids, order and progress; ids
 * (capacity max_ids, may be NULL) receives them in checkpoint order and *n_jobs their count.
 * The server keeps its own copy of queued jobs' inputs.  Resumed jobs have no output buffers:
 * srv_step returns MDC_ERR_STATE until srv_bind has been called for each.  Blocking. */
int srv_resume(mdc_server_handle s, const void* buf, int64_t bytes, int64_t* ids, int max_ids, int* n_jobs);
/* srv_bind -- give a queued or running job (normally a resumed one) its four host output
 * buffers [nt][ns][nv] (each may be NULL), as srv_submit does.  MDC_ERR_STATE for a job that
 * has completed. */
int srv_bind(mdc_server_handle s, int64_t job_id, float* f_minus_host, float* f_mplus_host, float* g_minus_host,
             float* g_plus_host);
/* srv_destroy -- drop all jobs and free the server (the handles stay valid). */
int srv_destroy(mdc_server_handle s);

/* mdc_destroy -- free the handle and everything it owns (synchronises the device). */
int mdc_destroy(mdc_handle h);

/* mdc_strerror -- static text for a status code. */
const char* mdc_strerror(int status);

/* mdc_last_cuda_error -- the cudaError_t value behind the last MDC_ERR_CUDA (per thread). */
int mdc_last_cuda_error(void);

/* mdc_kernel_bytes -- bytes the library-owned kernel copy of a given shape occupies
 * (padding and per-row scales included).  Host-only; no device needed. */
int64_t mdc_kernel_bytes(int nfmax, int nr, int ns, int storage);

/*
 * Instrumentation.  mdc_timing(h, 1) makes the handle bracket every kernel launch
 * with CUDA events on the launching stream; mdc_timing_read(h, cls, &ms, &n) then
 * synchronises and returns the summed device time and launch count of one kernel
 * class since the last mdc_timing(h, 1).  mdc_launch_count returns the number of
 * kernels the handle has launched since creation (timing on or off).
 */
int mdc_timing(mdc_handle h, int enable);
/*
 * mdc_autotune -- choose, per direction and per column count (buckets 1, 2, 4, ... up to
 * ncol_max), the fastest per-frequency product variant for this handle by timing every variant
 * that can run on the handle's own buffers: the GEMV (up to 4 columns, or in passes over groups of
 * 4 up to 64 columns), the SIMT GEMM, and, for 16-bit and E4M3 storage, the tensor-core GEMM with
 * each column-tile width (32, 64, 128, 256).  Later
 * products use the variant of the smallest bucket holding their column count (the serving
 * engine still forces tensor cores so a job's arithmetic does not depend on its batch).  With
 * the environment variable MDC_AUTOTUNE_CACHE naming a file, a stored table for the same device,
 * shape and storage is reused instead of timing, and new tables are appended (JSON lines).
 * Blocking; allocates scratch for ncol_max columns.  All variants compute the same operator.
 */
int mdc_autotune(mdc_handle h, int ncol_max, void* stream);
/* mdc_autotune_choice -- the variant selected for ncol columns: *path 0 = default rule, 1 = GEMV,
 * 2 = SIMT GEMM, 3 = tensor cores with column tile *bn, 4 = GEMV passes over groups of up to 4
 * columns. */
int mdc_autotune_choice(mdc_handle h, int adjoint, int ncol, int* path, int* bn);

/* mdc_set_option -- MDC_OPT_GRAPHS (value 1/0): when on, a marchenko_lsqr or
 * marchenko_lsqr_refined call whose arguments (sizes, iteration counts, tolerance and every
 * pointer) repeat an earlier call on this handle replays that call's CUDA graph: the whole solve
 * (data vector, all LSQR iterations, refinement, Green's functions) is captured on first use with
 * a workspace the handle keeps (up to 4 cached solves; turning the option off frees them). */
#define MDC_OPT_GRAPHS 1
/* MDC_OPT_WAIT_LIMIT_US (value >= 0): bound, in microseconds of wall time, on each wait inside the
 * tensor-core product kernel (TMA stages, MMA completion, accumulator hand-off); 0 restores the
 * default of 2 s.  A wait that runs out makes the kernel record MDC_ERR_TIMEOUT in the handle's
 * device flag (read by mdc_device_status), finish its copies and MMAs in flight, free its tensor
 * memory and exit; the product's output is then incomplete.  Negative values: MDC_ERR_ARG.
 * (Failure detection: a limit the pipeline cannot meet exercises that path.) */
#define MDC_OPT_WAIT_LIMIT_US 2
int mdc_set_option(mdc_handle h, int option, int value);
/* mdc_tc_fallback_count -- number of per-frequency products, since the handle was created, that
 * the tensor-core rule assigned to tensor cores (16-bit, split or E4M3 storage at 8 or more
 * columns, or an autotuned tensor-core choice) but that ran on the SIMT/GEMV path instead, because
 * the tensor-core operand buffers were not reserved for that many columns (mdc_reserve) or the
 * launch could not be set up.  Results are correct either way; the count exposes the slower
 * path.  -1 for a NULL handle.  Host-only. */
int64_t mdc_tc_fallback_count(mdc_handle h);
/* mdc_device_status -- synchronise `stream` and report MDC_ERR_TIMEOUT if a kernel of this
 * handle gave up a bounded device-side wait since the last check, or (bounds-checked build only)
 * MDC_ERR_BOUNDS if a kernel index fell outside its buffer; the flag is then cleared. */
int mdc_device_status(mdc_handle h, void* stream);
int mdc_timing_read(mdc_handle h, int kernel_class, double* total_ms, int64_t* launches);
int64_t mdc_launch_count(mdc_handle h);

#ifdef __cplusplus
}
#endif
#endif /* MDC_GB300_H */
