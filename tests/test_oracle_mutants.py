"""The oracle's pins catch plausible mistakes: each mutant is planted in the oracle (CPU only)
and at least one pin must fail on it."""
import numpy as np
import pytest

from oracle import marchenko, mdc, solvers

import test_oracle_greens as pins_g
import test_oracle_marchenko_lsqr as pins_m
import test_oracle_mdc as pins


def _adjoint_no_conj(G, y, dt, dr):
    Y = mdc.rfft_truncate(y, G.shape[0])
    return mdc.pad_irfft(np.matmul(np.swapaxes(G, 1, 2) * (dt * dr), Y), y.shape[0])


def _forward_no_weight(G, x, dt, dr):
    X = mdc.rfft_truncate(x, G.shape[0])
    return mdc.pad_irfft(np.matmul(G, X), x.shape[0])


def _pad_off_by_one(Y, nt):
    full = np.zeros((nt // 2 + 1,) + Y.shape[1:], dtype=np.complex128)
    full[1: Y.shape[0]] = Y[:-1]
    return np.fft.irfft(full, n=nt, axis=0)


def _rstar_without_conj(G, x, dt, dr):
    return mdc.forward(G, x, dt, dr)


def _one_sided_window(cutoffs, nt):
    t = np.arange(nt)
    return (t[:, None, None] < np.asarray(cutoffs)[None]).astype(np.float64)


def _rmatvec_wrong_block(self, g):
    a, b = g
    return (a - self.RH(self.theta * b), b - self.RH(self.theta * a))


def _data_without_window(self, fd_plus):
    fd_plus = np.asarray(fd_plus, dtype=np.float64)
    return (self.R(fd_plus), np.zeros_like(fd_plus))


def _greens_r_rstar_swapped(self, f_minus, f_mplus, fd_plus):
    f_plus = np.asarray(fd_plus, dtype=np.float64) + f_mplus
    g_minus = -(f_minus - self.Rstar(f_plus))
    g_plus_star = f_plus - self.R(f_minus)
    return g_minus, g_plus_star, marchenko.time_reverse(g_plus_star)


def _greens_g_minus_sign(self, f_minus, f_mplus, fd_plus):
    f_plus = np.asarray(fd_plus, dtype=np.float64) + f_mplus
    g_minus = f_minus - self.R(f_plus)
    g_plus_star = f_plus - self.Rstar(f_minus)
    return g_minus, g_plus_star, marchenko.time_reverse(g_plus_star)


def _lsqr_wrong_rhobar_sign(matvec, rmatvec, b, niter, tol=0.0, x_like=None):
    # copy of the recurrence with rhobar = +c alpha (sign error)
    import math
    beta = solvers.norm(b)
    u = solvers.scale(1.0 / beta, b)
    v = rmatvec(u)
    alpha = solvers.norm(v)
    v = solvers.scale(1.0 / alpha, v)
    w = v
    x = solvers.zeros_like(v)
    phibar, rhobar = beta, alpha
    for _ in range(niter):
        u = solvers.lincomb(1.0, matvec(v), -alpha, u)
        beta = solvers.norm(u)
        u = solvers.scale(1.0 / beta, u)
        v = solvers.lincomb(1.0, rmatvec(u), -beta, v)
        alpha = solvers.norm(v)
        v = solvers.scale(1.0 / alpha, v)
        rho = math.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = solvers.lincomb(1.0, x, phi / rho, w)
        w = solvers.lincomb(1.0, v, -theta / rho, w)
    return solvers.LSQRResult(x, [phibar], niter, [], [])


MUTANTS = [
    ("adjoint without conjugation", mdc, "adjoint", _adjoint_no_conj,
     lambda: pins.test_dot_product(64, 11, 7, 20, 4)),
    ("integration weight dropped", mdc, "forward", _forward_no_weight,
     lambda: pins.test_identity_kernel_all_bins(64)),
    ("frequency padding off by one bin", mdc, "pad_irfft", _pad_off_by_one,
     lambda: pins.test_forward_equals_brute_force_convolution(16, 7, 4, 5, 2)),
    ("R* without conjugated kernel", mdc, "forward_conj_kernel", _rstar_without_conj,
     lambda: pins.test_conjugate_kernel_is_time_reversal(5)),
    ("one-sided window", marchenko, "window", _one_sided_window,
     pins_m.test_window_is_two_sided_in_signed_time),
    ("M^H uses R^H in both blocks", marchenko.Marchenko, "rmatvec", _rmatvec_wrong_block,
     pins_m.test_dense_adjoint_is_transpose),
    ("LSQR rhobar sign error", solvers, "lsqr", _lsqr_wrong_rhobar_sign,
     pins_m.test_lsqr_n_iterations_equals_dense_lstsq),
    ("data vector without the window", marchenko.Marchenko, "data", _data_without_window,
     pins_g.test_data_vector_is_windowed_convolution),
    ("Green's functions with R and R* exchanged", marchenko.Marchenko, "greens", _greens_r_rstar_swapped,
     pins_g.test_greens_with_zero_f_minus),
    ("Green's functions with R and R* exchanged (f+ = 0)", marchenko.Marchenko, "greens",
     _greens_r_rstar_swapped, pins_g.test_greens_with_zero_f_plus),
    ("g- with the opposite sign", marchenko.Marchenko, "greens", _greens_g_minus_sign,
     pins_g.test_greens_general_case_is_linear_combination),
]


@pytest.mark.parametrize("name,owner,attr,mutant,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(monkeypatch, name, owner, attr, mutant, pin):
    pin()   # passes on the real oracle
    monkeypatch.setattr(owner, attr, mutant)
    with pytest.raises(AssertionError):
        pin()
