"""Pins for the FP64 MDC oracle (Eq. 1-3): each check is independent of the FFT path.

* brute force: the time-domain circular convolution of Eq. 1, with the kernel's
  time response built from explicit cosine sums over the retained frequencies;
* dot-product test <C x, y> = <x, C^H y>;
* identity kernel with every frequency kept: C = dt*dr*I exactly;
* identity kernel with frequencies dropped: C/(dt*dr) is an orthogonal projector;
* one hyperbolic event, impulse input: closed-form cosine sum;
* conjugate kernel = time reversal around the convolution: R* = P R P;
* linearity.
"""
import math

import numpy as np
import pytest

import synth
from oracle import mdc
from oracle.marchenko import time_reverse

RNG = np.random.default_rng(1234)


def rand_kernel(nf, nr, ns, rng=RNG):
    return rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))


def brute_force_forward(G, x, dt, dr):
    """Eq. 1 discretised: y[t, r] = sum_s sum_tau h[(t - tau) mod nt, r, s] x[tau, s].

    h is the real time response of the band-limited kernel: for each retained
    bin k the positive-frequency bin and its mirror contribute 2 Re(...), the
    DC and Nyquist bins contribute once; written as explicit cosines and sines.
    """
    nf, nr, ns = G.shape
    nt = x.shape[0]
    h = np.zeros((nt, nr, ns))
    for m in range(nt):
        for k in range(nf):
            w = 1.0 if (k == 0 or 2 * k == nt) else 2.0
            ang = 2.0 * math.pi * k * m / nt
            h[m] += w * (G[k].real * math.cos(ang) - G[k].imag * math.sin(ang))
    h *= dt * dr / nt
    y = np.zeros((nt, nr) + x.shape[2:])
    for t in range(nt):
        for tau in range(nt):
            y[t] += np.einsum("rs,s...->r...", h[(t - tau) % nt], x[tau])
    return y


@pytest.mark.parametrize("nt,nr,ns,nf,nv", [
    (16, 3, 5, 9, 1),      # every bin kept, Nyquist included
    (16, 7, 4, 5, 2),      # truncated, nr != ns
    (32, 9, 9, 17, 1),
    (32, 4, 8, 1, 3),      # DC only
    (32, 5, 3, 12, 1),
])
def test_forward_equals_brute_force_convolution(nt, nr, ns, nf, nv):
    G = rand_kernel(nf, nr, ns)
    x = RNG.standard_normal((nt, ns, nv))
    dt, dr = 0.004, 400.0
    y = mdc.forward(G, x, dt, dr)
    yb = brute_force_forward(G, x, dt, dr)
    assert np.linalg.norm(y - yb) <= 1e-12 * np.linalg.norm(yb)


@pytest.mark.parametrize("nt,nr,ns,nf,nv", [(16, 3, 5, 9, 2), (32, 6, 4, 10, 1), (64, 5, 7, 33, 3)])
def test_adjoint_equals_brute_force_correlation(nt, nr, ns, nf, nv):
    """C^H is the correlation with the same real time response (transpose of Eq. 1)."""
    G = rand_kernel(nf, nr, ns)
    y = RNG.standard_normal((nt, nr, nv))
    dt, dr = 0.002, 225.0
    x = mdc.adjoint(G, y, dt, dr)
    # the transposed convolution: time-reverse, convolve with h^T, time-reverse
    GT = np.swapaxes(G, 1, 2)
    xb = time_reverse(brute_force_forward(GT, time_reverse(y), dt, dr))
    assert np.linalg.norm(x - xb) <= 1e-12 * np.linalg.norm(xb)


@pytest.mark.parametrize("nt,nr,ns,nf,nv", [(16, 3, 5, 9, 1), (64, 11, 7, 20, 4), (128, 9, 9, 65, 2)])
def test_dot_product(nt, nr, ns, nf, nv):
    G = rand_kernel(nf, nr, ns)
    x = RNG.standard_normal((nt, ns, nv))
    y = RNG.standard_normal((nt, nr, nv))
    Cx = mdc.forward(G, x, 0.004, 400.0)
    CHy = mdc.adjoint(G, y, 0.004, 400.0)
    lhs, rhs = np.vdot(Cx, y), np.vdot(x, CHy)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Cx) * np.linalg.norm(y)


@pytest.mark.parametrize("nt", [16, 64, 256])
def test_identity_kernel_all_bins(nt):
    n, nv = 5, 2
    nf = nt // 2 + 1
    G = np.broadcast_to(np.eye(n, dtype=np.complex128), (nf, n, n)).copy()
    x = RNG.standard_normal((nt, n, nv))
    y = mdc.forward(G, x, 0.5, 3.0)
    assert np.max(np.abs(y - 1.5 * x)) <= 1e-13 * np.max(np.abs(x))


def test_identity_kernel_truncated_is_projector():
    nt, n, nf = 32, 2, 7
    G = np.broadcast_to(np.eye(n, dtype=np.complex128), (nf, n, n)).copy()
    N = nt * n
    P = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        P[:, j] = mdc.forward(G, e.reshape(nt, n, 1), 1.0, 1.0).ravel()
    assert np.allclose(P, P.T, atol=1e-14)
    assert np.allclose(P @ P, P, atol=1e-13)
    # rank = number of real degrees of freedom kept: DC (1) + 2 per other bin, per trace
    assert np.linalg.matrix_rank(P, tol=1e-9) == n * (1 + 2 * (nf - 1))


def test_single_event_closed_form():
    """One event of unit amplitude, impulse at (t=0, s0): cosine sum at the event's time."""
    cfg = synth.tiny(n_side=3, nt=64, nf=20, n_events=1, nv=1)
    d = synth.draw(cfg)
    d.amp[:] = 1.0
    G = synth.kernel(cfg, d)
    s0 = 4
    x = np.zeros((cfg.nt, cfg.ns, 1))
    x[0, s0, 0] = 1.0
    y = mdc.forward(G, x, cfg.dt, cfg.dr)
    tau = synth.event_times(cfg, d, np.arange(cfg.nr), [s0])[0, :, 0]   # [nr]
    f = cfg.freqs
    W = synth.ricker_spectrum(f)
    w = np.where(np.arange(cfg.nf) == 0, 1.0, 2.0)
    t = np.arange(cfg.nt) * cfg.dt
    expect = (cfg.dt * cfg.dr / cfg.nt) * np.sum(
        w[None, None, :] * W[None, None, :]
        * np.cos(2 * np.pi * f[None, None, :] * (t[:, None, None] - tau[None, :, None])), axis=2)
    assert np.max(np.abs(y[:, :, 0] - expect)) <= 1e-12 * np.max(np.abs(expect))


@pytest.mark.parametrize("nf", [5, 17])
def test_conjugate_kernel_is_time_reversal(nf):
    nt, nr, ns, nv = 32, 4, 6, 2
    G = rand_kernel(nf, nr, ns)
    x = RNG.standard_normal((nt, ns, nv))
    a = mdc.forward_conj_kernel(G, x, 0.004, 400.0)
    b = time_reverse(mdc.forward(G, time_reverse(x), 0.004, 400.0))
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)
    y = RNG.standard_normal((nt, nr, nv))
    a = mdc.adjoint_conj_kernel(G, y, 0.004, 400.0)
    b = time_reverse(mdc.adjoint(G, time_reverse(y), 0.004, 400.0))
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)


def test_linearity():
    nt, nr, ns, nf, nv = 64, 5, 6, 20, 2
    G = rand_kernel(nf, nr, ns)
    x1 = RNG.standard_normal((nt, ns, nv))
    x2 = RNG.standard_normal((nt, ns, nv))
    a, b = 0.7, -2.3
    lhs = mdc.forward(G, a * x1 + b * x2, 0.004, 400.0)
    rhs = a * mdc.forward(G, x1, 0.004, 400.0) + b * mdc.forward(G, x2, 0.004, 400.0)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_row_sampled_forms_match_full():
    cfg = synth.tiny(n_side=4, nt=32, nf=12, n_events=4, nv=2)
    G = synth.kernel(cfg)
    x = synth.random_traces(cfg, 2).astype(np.float64)
    y = mdc.forward(G, x, cfg.dt, cfg.dr)
    rows = [0, 5, 15]
    Gr = synth.kernel(cfg, rows=rows)
    assert np.allclose(mdc.forward_rows(Gr, x, cfg.dt, cfg.dr), y[:, rows], rtol=0, atol=1e-12)
    yy = synth.random_traces(cfg, 2, seed_offset=1).astype(np.float64)
    xa = mdc.adjoint(G, yy, cfg.dt, cfg.dr)
    cols = [1, 2, 14]
    Gc = synth.kernel(cfg, cols=cols)
    assert np.allclose(mdc.adjoint_cols(Gc, yy, cfg.dt, cfg.dr), xa[:, cols], rtol=0, atol=1e-12)
