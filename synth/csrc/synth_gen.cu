// Device-side generator of the synthetic hyperbolic-event kernel (workload input,
// not part of the MDC library):
//     G[k][r][s] = scale * sum_e a_e W(f_k) exp(-i 2 pi f_k tau_e(r, s)),
//     tau_e = sqrt(t0_e^2 + |x_r - x_s|^2 / v_e^2),  f_k = k df,
// on a co-located square grid (flat index iy * n_side + ix, spacing dx).
// The phase in cycles, k * df * tau_e, is reduced in float64 (to frac(k * frac(df * tau_e)),
// or, in the rectangular variant, incremented by frac(df * tau_e) per bin), so the float32
// sine/cosine of the reduced argument leaves only float32 rounding in G.  W(f_k) * scale is
// supplied by the caller as a float64 table.
#include <cuda_runtime.h>
#include <stdint.h>

#define SYNTH_MAX_EVENTS 32
#define SYNTH_MAX_NF 2049

struct SynthParams {
    int nf, n_side, E;
    double dx, df;
    double t0[SYNTH_MAX_EVENTS], vel[SYNTH_MAX_EVENTS], amp[SYNTH_MAX_EVENTS];
};

__constant__ double c_wscale[SYNTH_MAX_NF];

// Frequencies k0 .. k0+P.nf-1 (c_wscale holds their weights from index 0).  The phase of
// bin k is frac(k * frac(df * tau)), evaluated per bin in float64, so a slab is
// bit-identical to the same frequencies of the whole kernel.
__global__ void synth_kernel(float2* __restrict__ G, SynthParams P, int k0) {
    const int64_t n = (int64_t)P.n_side * P.n_side;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int64_t r = idx / n, s = idx - r * n;
    const double ddx = P.dx * (double)((r % P.n_side) - (s % P.n_side));
    const double ddy = P.dx * (double)((r / P.n_side) - (s / P.n_side));
    const double d2 = ddx * ddx + ddy * ddy;
    double step[SYNTH_MAX_EVENTS];
    for (int e = 0; e < P.E; ++e) {
        const double tau = sqrt(P.t0[e] * P.t0[e] + d2 / (P.vel[e] * P.vel[e]));
        const double ph = P.df * tau;
        step[e] = ph - floor(ph);
    }
    for (int k = 0; k < P.nf; ++k) {
        const double kk = (double)(k0 + k);
        double re = 0.0, im = 0.0;
        for (int e = 0; e < P.E; ++e) {
            float sn, cs;
            const double cyc = kk * step[e];
            const double c = cyc - rint(cyc);
            sincospif((float)(2.0 * c), &sn, &cs);
            re += P.amp[e] * (double)cs;
            im -= P.amp[e] * (double)sn;
        }
        const double w = c_wscale[k];
        G[((int64_t)k * n + r) * n + s] = make_float2((float)(w * re), (float)(w * im));
    }
}

// G [nf][n][n] receives frequencies k0 .. k0+nf-1; wscale[nf] their weights.
extern "C" int synth_kernel_slab_c64(void* G, int k0, int nf, int n_side, double dx, double df, int E,
                                     const double* t0, const double* vel, const double* amp,
                                     const double* wscale, void* stream) {
    if (!G || k0 < 0 || nf < 1 || nf > SYNTH_MAX_NF || n_side < 1 || E < 1 || E > SYNTH_MAX_EVENTS) return -1;
    SynthParams P{};
    P.nf = nf; P.n_side = n_side; P.E = E; P.dx = dx; P.df = df;
    for (int e = 0; e < E; ++e) { P.t0[e] = t0[e]; P.vel[e] = vel[e]; P.amp[e] = amp[e]; }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyToSymbolAsync(c_wscale, wscale, sizeof(double) * nf, 0, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return -3;
    const int64_t n = (int64_t)n_side * n_side;
    const int64_t total = n * n;
    const int threads = 256;
    synth_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>((float2*)G, P, k0);
    if (cudaGetLastError() != cudaSuccess) return -3;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -3;
    return 0;
}

extern "C" int synth_kernel_c64(void* G, int nf, int n_side, double dx, double df, int E,
                                const double* t0, const double* vel, const double* amp,
                                const double* wscale, void* stream) {
    return synth_kernel_slab_c64(G, 0, nf, n_side, dx, df, E, t0, vel, amp, wscale, stream);
}

// Rectangular variant: rows and columns are arbitrary point sets (x, y in m), e.g. surface
// receivers by subsurface focusing points for the down-going Green's function of Eq. 8.
__global__ void synth_kernel_rect(float2* __restrict__ G, SynthParams P, int nr, int ns,
                                  const double* __restrict__ xr, const double* __restrict__ xs) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nr * ns) return;
    const int64_t r = idx / ns, s = idx - r * ns;
    const double ddx = xr[2 * r] - xs[2 * s], ddy = xr[2 * r + 1] - xs[2 * s + 1];
    const double d2 = ddx * ddx + ddy * ddy;
    double step[SYNTH_MAX_EVENTS], cur[SYNTH_MAX_EVENTS];
    for (int e = 0; e < P.E; ++e) {
        const double tau = sqrt(P.t0[e] * P.t0[e] + d2 / (P.vel[e] * P.vel[e]));
        const double ph = P.df * tau;
        step[e] = ph - floor(ph);
        cur[e] = 0.0;
    }
    for (int k = 0; k < P.nf; ++k) {
        double re = 0.0, im = 0.0;
        for (int e = 0; e < P.E; ++e) {
            float sn, cs;
            const double c = cur[e] - rint(cur[e]);
            sincospif((float)(2.0 * c), &sn, &cs);
            re += P.amp[e] * (double)cs;
            im -= P.amp[e] * (double)sn;
            double nx = cur[e] + step[e];
            cur[e] = nx >= 1.0 ? nx - 1.0 : nx;
        }
        const double w = c_wscale[k];
        G[((int64_t)k * nr + r) * ns + s] = make_float2((float)(w * re), (float)(w * im));
    }
}

extern "C" int synth_kernel_rect_c64(void* G, int nf, int nr, int ns, const double* xy_rows, const double* xy_cols,
                                     double df, int E, const double* t0, const double* vel, const double* amp,
                                     const double* wscale, void* stream) {
    if (!G || !xy_rows || !xy_cols || nf < 1 || nf > SYNTH_MAX_NF || nr < 1 || ns < 1 || E < 1 ||
        E > SYNTH_MAX_EVENTS)
        return -1;
    SynthParams P{};
    P.nf = nf; P.n_side = 0; P.E = E; P.dx = 0.0; P.df = df;
    for (int e = 0; e < E; ++e) { P.t0[e] = t0[e]; P.vel[e] = vel[e]; P.amp[e] = amp[e]; }
    cudaStream_t s = (cudaStream_t)stream;
    double *xr = nullptr, *xs = nullptr;
    if (cudaMalloc(&xr, sizeof(double) * 2 * nr) != cudaSuccess) return -2;
    if (cudaMalloc(&xs, sizeof(double) * 2 * ns) != cudaSuccess) { cudaFree(xr); return -2; }
    int st = 0;
    if (cudaMemcpyAsync(xr, xy_rows, sizeof(double) * 2 * nr, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(xs, xy_cols, sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_wscale, wscale, sizeof(double) * nf, 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = -3;
    if (st == 0) {
        const int64_t total = (int64_t)nr * ns;
        synth_kernel_rect<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((float2*)G, P, nr, ns, xr, xs);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = -3;
    }
    cudaFree(xr);
    cudaFree(xs);
    return st;
}
