"""Pins of the FP64 MDD oracle (Eq. 8) against closed forms, not against itself.

For a tall kernel whose frequency slices have full column rank, the row space
of the MDC operator is every real signal band-limited to the first nf bins, so
the minimum-norm least-squares solution of G+ r = G+ r_true is the band-limit
projection of r_true (computed with NumPy's FFT, no MDC code).  Dense lstsq of
the operator built column by column must give that projection, and LSQR from
r = 0 must converge to it.
"""
import numpy as np
import pytest

from oracle import mdc, mdd

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def band_limit(r, nf):
    R = np.fft.rfft(r, axis=0)
    R[nf:] = 0.0
    return np.fft.irfft(R, n=r.shape[0], axis=0)


def tall_kernel(nf, nS, nF, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((nf, nS, nF)) + 1j * rng.standard_normal((nf, nS, nF))
    G[:, :nF, :] += 3.0 * np.eye(nF)            # well conditioned, full column rank
    return G


@pytest.mark.parametrize("nt,nf,nS,nF,nv", [(16, 5, 6, 3, 1), (32, 9, 5, 4, 2)])
def test_min_norm_solution_is_band_limit_projection(nt, nf, nS, nF, nv):
    G = tall_kernel(nf, nS, nF, seed=nt + nS)
    op = mdd.MDD(G, 0.004, 400.0)
    rng = np.random.default_rng(7)
    r_true = rng.standard_normal((nt, nF, nv))
    g = op.matvec(r_true)
    n = nt * nF * nv
    A = np.stack([op.matvec(np.eye(n)[:, i].reshape(nt, nF, nv)).ravel() for i in range(n)], axis=1)
    x_ls = np.linalg.lstsq(A, g.ravel(), rcond=1e-10)[0].reshape(nt, nF, nv)
    P = band_limit(r_true, nf)
    assert np.linalg.norm(x_ls - P) <= 1e-9 * np.linalg.norm(P)
    res = op.solve(g, niter=4 * n, tol=1e-12)      # stop once converged (beta -> rounding level)
    assert np.linalg.norm(res.x - P) <= 1e-8 * np.linalg.norm(P)
    assert res.resid[-1] <= 1e-8 * res.resid[0]


def test_adjoint_estimate_is_one_adjoint_mdc():
    nt, nf, nS, nF = 16, 5, 6, 3
    G = tall_kernel(nf, nS, nF, seed=3)
    op = mdd.MDD(G, 0.004, 400.0)
    g = np.random.default_rng(1).standard_normal((nt, nS, 2))
    # <G+ r, g> = <r, G+^H g> for a random r: the correlation estimate is the exact adjoint
    r = np.random.default_rng(2).standard_normal((nt, nF, 2))
    lhs = float(np.sum(op.matvec(r) * g))
    rhs = float(np.sum(r * op.adjoint_estimate(g)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_planted_mistake_in_operator_breaks_the_pin():
    """A transposed kernel (a plausible wiring mistake) no longer reproduces the projection."""
    nt, nf, nS, nF = 16, 5, 4, 4
    G = tall_kernel(nf, nS, nF, seed=11)
    good = mdd.MDD(G, 0.004, 400.0)
    bad = mdd.MDD(np.swapaxes(G, 1, 2), 0.004, 400.0)
    r_true = np.random.default_rng(5).standard_normal((nt, nF, 1))
    g = good.matvec(r_true)
    P = band_limit(r_true, nf)
    x_bad = bad.solve(g, niter=200, tol=1e-12).x
    assert np.linalg.norm(x_bad - P) > 1e-3 * np.linalg.norm(P)
