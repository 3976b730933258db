"""Pins for the FP64 Marchenko operator (Eq. 5, Eq. 6) and the LSQR/CGLS solvers.

* M and M^H built densely on a tiny problem: M^H is the transpose of M;
* Theta = 0 gives M = I; a full window gives the plain block form of Eq. 5;
* Green's functions with a zero kernel reduce to -f^- and f^+ (Eq. 6);
* LSQR after n iterations equals the dense least-squares solution;
* LSQR and CGLS iterates coincide on a well-conditioned problem;
* the LSQR residual estimate is non-increasing and equals the true residual;
* with ||R|| <= 0.5 the solution equals the Neumann sum of N = I - M.
"""
import numpy as np
import pytest

import synth
from oracle import marchenko, mdc, solvers

RNG = np.random.default_rng(99)


def tiny_problem(nt=16, n_side=2, nf=6, nv=1, norm_R=None, seed=0):
    rng = np.random.default_rng(seed)
    n = n_side * n_side
    G = rng.standard_normal((nf, n, n)) + 1j * rng.standard_normal((nf, n, n))
    dt, dr = 0.004, 1.0
    if norm_R is not None:
        # scale so that the largest per-frequency singular value times dt*dr is norm_R
        smax = max(np.linalg.norm(G[k], 2) for k in range(nf))
        G *= norm_R / (smax * dt * dr)
    cut = rng.integers(1, nt // 2, size=(n, nv)).astype(np.int32)
    return G, dt, dr, cut, n


def flat(t):
    return np.concatenate([np.ravel(a) for a in t])


def unflat(v, shape):
    m = int(np.prod(shape))
    return (v[:m].reshape(shape), v[m:].reshape(shape))


def dense(op, shape):
    m = int(np.prod(shape))
    A = np.zeros((2 * m, 2 * m))
    for j in range(2 * m):
        e = np.zeros(2 * m)
        e[j] = 1.0
        A[:, j] = flat(op(unflat(e, shape)))
    return A


def test_dense_adjoint_is_transpose():
    nt = 16
    G, dt, dr, cut, n = tiny_problem(nt=nt, nv=2)
    op = marchenko.Marchenko(G, dt, dr, cut, nt)
    shape = (nt, n, 2)
    M = dense(op.matvec, shape)
    MH = dense(op.rmatvec, shape)
    assert np.allclose(MH, M.T, atol=1e-13 * np.abs(M).max())


def test_zero_window_is_identity():
    nt = 16
    G, dt, dr, cut, n = tiny_problem(nt=nt)
    op = marchenko.Marchenko(G, dt, dr, np.zeros_like(cut), nt)
    f = (RNG.standard_normal((nt, n, 1)), RNG.standard_normal((nt, n, 1)))
    out = op.matvec(f)
    assert np.array_equal(out[0], f[0]) and np.array_equal(out[1], f[1])


def test_full_window_block_structure():
    nt = 16
    G, dt, dr, cut, n = tiny_problem(nt=nt)
    op = marchenko.Marchenko(G, dt, dr, np.full_like(cut, nt), nt)
    a, b = RNG.standard_normal((nt, n, 1)), RNG.standard_normal((nt, n, 1))
    out = op.matvec((a, b))
    assert np.allclose(out[0], a - mdc.forward(G, b, dt, dr), atol=1e-13)
    assert np.allclose(out[1], b - mdc.forward(np.conj(G), a, dt, dr), atol=1e-13)


def test_window_is_two_sided_in_signed_time():
    cut = np.array([[3]], dtype=np.int32)
    th = marchenko.window(cut, 16)[:, 0, 0]
    assert list(np.nonzero(th)[0]) == [0, 1, 2, 14, 15]


def test_greens_with_zero_kernel():
    nt, n = 16, 4
    op = marchenko.Marchenko(np.zeros((5, n, n), complex), 0.004, 1.0, np.ones((n, 1), np.int32), nt)
    fm = RNG.standard_normal((nt, n, 1))
    fmp = RNG.standard_normal((nt, n, 1))
    fd = RNG.standard_normal((nt, n, 1))
    gm, gps, gp = op.greens(fm, fmp, fd)
    assert np.allclose(gm, -fm) and np.allclose(gps, fd + fmp)
    assert np.allclose(gp, marchenko.time_reverse(fd + fmp))


def test_lsqr_n_iterations_equals_dense_lstsq():
    nt = 16
    G, dt, dr, cut, n = tiny_problem(nt=nt, norm_R=0.9)
    op = marchenko.Marchenko(G, dt, dr, cut, nt)
    shape = (nt, n, 1)
    M = dense(op.matvec, shape)
    fd = RNG.standard_normal(shape)
    d = op.data(fd)
    x_ref = np.linalg.lstsq(M, flat(d), rcond=None)[0]
    res = solvers.lsqr(op.matvec, op.rmatvec, d, niter=M.shape[0])
    assert np.linalg.norm(flat(res.x) - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_lsqr_on_rectangular_dense_matrix():
    A = RNG.standard_normal((60, 25))
    b = RNG.standard_normal(60)
    res = solvers.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, niter=25)
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(res.x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # residual estimates are non-increasing and match the true residual
    r = res.resid
    assert all(r[i + 1] <= r[i] * (1 + 1e-12) for i in range(len(r) - 1))
    assert abs(r[-1] - np.linalg.norm(b - A @ res.x)) <= 1e-9 * np.linalg.norm(b)


def test_lsqr_matches_cgls_iterates():
    nt = 16
    G, dt, dr, cut, n = tiny_problem(nt=nt, nv=2, norm_R=0.6, seed=3)
    op = marchenko.Marchenko(G, dt, dr, cut, nt)
    d = op.data(RNG.standard_normal((nt, n, 2)))
    for k in (1, 3, 6):
        xl = solvers.lsqr(op.matvec, op.rmatvec, d, niter=k).x
        xc, _ = solvers.cgls(op.matvec, op.rmatvec, d, niter=k)
        assert np.linalg.norm(flat(xl) - flat(xc)) <= 1e-10 * np.linalg.norm(flat(xc))


def test_lsqr_identity_operator_one_iteration():
    b = (RNG.standard_normal((8, 3)), RNG.standard_normal((8, 3)))
    res = solvers.lsqr(lambda v: v, lambda u: u, b, niter=5)
    assert res.iters == 1
    assert np.allclose(res.x[0], b[0]) and np.allclose(res.x[1], b[1])


def test_lsqr_residual_estimate_tracks_true_residual():
    nt = 32
    G, dt, dr, cut, n = tiny_problem(nt=nt, n_side=3, nf=12, nv=2, norm_R=0.8, seed=5)
    op = marchenko.Marchenko(G, dt, dr, cut, nt)
    d = op.data(RNG.standard_normal((nt, n, 2)))
    for k in (2, 5, 9):
        res = solvers.lsqr(op.matvec, op.rmatvec, d, niter=k)
        r = solvers.lincomb(1.0, d, -1.0, op.matvec(res.x))
        assert abs(solvers.norm(r) - res.resid[-1]) <= 1e-10 * solvers.norm(d)


def test_lsqr_tolerance_stop():
    nt = 32
    G, dt, dr, cut, n = tiny_problem(nt=nt, n_side=3, nf=12, nv=1, norm_R=0.5, seed=6)
    op = marchenko.Marchenko(G, dt, dr, cut, nt)
    d = op.data(RNG.standard_normal((nt, n, 1)))
    res = solvers.lsqr(op.matvec, op.rmatvec, d, niter=100, tol=1e-3)
    assert res.iters < 100
    assert res.resid[-1] <= 1e-3 * res.resid[0]
    assert res.resid[-2] > 1e-3 * res.resid[0]


def test_converged_lsqr_equals_neumann_sum():
    nt = 32
    G, dt, dr, cut, n = tiny_problem(nt=nt, n_side=3, nf=10, nv=2, norm_R=0.5, seed=11)
    op = marchenko.Marchenko(G, dt, dr, cut, nt)
    d = op.data(RNG.standard_normal((nt, n, 2)))

    def apply_N(f):   # N = I - M
        m = op.matvec(f)
        return (f[0] - m[0], f[1] - m[1])

    xn = solvers.neumann(apply_N, d, 80)
    xl = solvers.lsqr(op.matvec, op.rmatvec, d, niter=200, tol=1e-14).x
    assert np.linalg.norm(flat(xl) - flat(xn)) <= 1e-8 * np.linalg.norm(flat(xn))


def test_synth_inputs_shapes_and_window():
    cfg = synth.tiny(n_side=3, nt=64, nf=20, nv=4, z_point=200.0, point_grid=2)
    cut = synth.window_cutoffs(cfg)
    fd = synth.direct_focusing(cfg)
    assert cut.shape == (cfg.ns, 4) and cut.dtype == np.int32
    assert fd.shape == (cfg.nt, cfg.ns, 4)
    # the direct arrival sits outside the window it defines (|tau| = t_d > cutoff)
    td = synth.direct_times(cfg)
    peak = np.argmax(np.abs(fd), axis=0)
    tau = synth.signed_time_index(cfg.nt)[peak]
    assert np.all(np.abs(tau) >= cut)
    assert np.allclose(-tau * cfg.dt, td, atol=cfg.dt)
