"""Independent pins for the oracle's data vector (Eq. 5) and Green's functions (Eq. 6).

Neither check calls the oracle's MDC: R is rebuilt as the time-domain circular convolution of
Eq. 1 (the brute force of the MDC pins), R* through the time reversal identity R* = P R P (P
the reversal t -> -t mod nt, written here as an explicit index loop), and Theta as an explicit
loop over signed circular time.  The kernel is random and non-symmetric, so R, R* and R^H all
differ and an exchanged operator shows.

* d = [Theta (h * f_d+) ; 0]                                   (Eq. 5, right-hand side)
* with f- = 0:          g- = h * (f_d+ + f_m+),  g+* = f_d+ + f_m+          (Eq. 6)
* with f+ = 0, f- != 0: g- = -f-,  g+* = -P (h * (P f-))                     (Eq. 6)
* in general g+ is P g+*.
"""
import numpy as np

from oracle import marchenko
from test_oracle_mdc import brute_force_forward

DT, DR = 0.004, 1.0


def reverse_loop(x):
    """(P x)[t] = x[(-t) mod nt], written out index by index."""
    nt = x.shape[0]
    out = np.empty_like(x)
    for t in range(nt):
        out[t] = x[(nt - t) % nt]
    return out


def theta_loop(cut, nt):
    """1 where the signed circular time |tau(t)| lies below the cut-off of (s, v), else 0."""
    ns, nv = cut.shape
    th = np.zeros((nt, ns, nv))
    for t in range(nt):
        tau = t if t < nt // 2 else t - nt
        for s in range(ns):
            for v in range(nv):
                if abs(tau) < cut[s, v]:
                    th[t, s, v] = 1.0
    return th


def case(seed, nt=16, n=4, nf=7, nv=2):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((nf, n, n)) + 1j * rng.standard_normal((nf, n, n))
    cut = rng.integers(1, nt // 2, size=(n, nv)).astype(np.int32)
    fd = rng.standard_normal((nt, n, nv))
    fm = rng.standard_normal((nt, n, nv))
    fp = rng.standard_normal((nt, n, nv))
    return G, cut, fd, fm, fp


def close(a, b, tol=1e-12):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) <= tol * max(np.linalg.norm(b), 1e-300)


def test_data_vector_is_windowed_convolution():
    for seed in (1, 2):
        G, cut, fd, _, _ = case(seed)
        nt = fd.shape[0]
        op = marchenko.Marchenko(G, DT, DR, cut, nt)
        d_minus, d_plus = op.data(fd)
        expect = theta_loop(cut, nt) * brute_force_forward(G, fd, DT, DR)
        assert close(d_minus, expect)
        assert np.count_nonzero(expect) > 0 and np.count_nonzero(expect) < expect.size   # window cuts
        assert np.array_equal(d_plus, np.zeros_like(fd))


def test_greens_with_zero_f_minus():
    """f- = 0: the up-going field is R f+ alone and the down-going one is f+ itself."""
    G, cut, fd, fm, _ = case(3)
    nt = fd.shape[0]
    op = marchenko.Marchenko(G, DT, DR, cut, nt)
    g_minus, g_plus_star, g_plus = op.greens(np.zeros_like(fd), fm, fd)
    f_plus = fd + fm
    assert close(g_minus, brute_force_forward(G, f_plus, DT, DR))
    assert close(g_plus_star, f_plus)
    assert close(g_plus, reverse_loop(f_plus))


def test_greens_with_zero_f_plus():
    """f+ = 0 (f_m+ = -f_d+): g- = -f- and g+* = -R* f- = -P R P f-, a correlation with the
    kernel, not the convolution R f- (the kernel is not symmetric)."""
    G, cut, fd, _, fp = case(4)
    nt = fd.shape[0]
    op = marchenko.Marchenko(G, DT, DR, cut, nt)
    f_minus = fp
    g_minus, g_plus_star, g_plus = op.greens(f_minus, -fd, fd)
    expect = -reverse_loop(brute_force_forward(G, reverse_loop(f_minus), DT, DR))
    assert close(g_minus, -f_minus)
    assert close(g_plus_star, expect)
    assert not close(expect, -brute_force_forward(G, f_minus, DT, DR), 1e-3)   # R* != R here
    assert close(g_plus, reverse_loop(expect))


def test_greens_general_case_is_linear_combination():
    """Both f- and f+ non-zero: g- = R f+ - f- and g+* = f+ - P R P f- (Eq. 6 by superposition)."""
    G, cut, fd, fm, fp = case(5)
    nt = fd.shape[0]
    op = marchenko.Marchenko(G, DT, DR, cut, nt)
    g_minus, g_plus_star, _ = op.greens(fp, fm, fd)
    f_plus = fd + fm
    assert close(g_minus, brute_force_forward(G, f_plus, DT, DR) - fp)
    assert close(g_plus_star, f_plus - reverse_loop(brute_force_forward(G, reverse_loop(fp), DT, DR)))
