"""FP64 LSQR and CGLS (test infrastructure).

The paper solves the Marchenko system (Eq. 5) and the MDD system (Eq. 8)
with CGLS for 10 iterations (Applications section and the cost discussion);
the GPU library uses LSQR, which produces the same iterates in exact
arithmetic.  Both are written here from their published definitions:

* LSQR -- Paige and Saunders (1982), bidiagonalisation with Givens updates,
  x0 = 0 and no damping.  Stops after ``niter`` iterations, when the residual
  estimate phibar falls to ``tol * beta_1`` (tol > 0), or on breakdown
  (beta or alpha equal to zero).
* CGLS -- Hestenes and Stiefel conjugate gradients on the normal equations,
  x0 = 0.

Vectors are tuples of arrays (the block vectors of Eq. 5) or single arrays.
"""
from __future__ import annotations

import math

import numpy as np


def _tup(v):
    return v if isinstance(v, tuple) else (v,)


def _untup(v, like):
    return v if isinstance(like, tuple) else v[0]


def dot(a, b) -> float:
    return float(sum(np.vdot(np.asarray(x, np.float64), np.asarray(y, np.float64)).real
                     for x, y in zip(_tup(a), _tup(b))))


def norm(a) -> float:
    return math.sqrt(dot(a, a))


def lincomb(ca, a, cb, b):
    """ca * a + cb * b, block-wise."""
    return _untup(tuple(ca * np.asarray(x, np.float64) + cb * np.asarray(y, np.float64)
                        for x, y in zip(_tup(a), _tup(b))), a)


def scale(c, a):
    return _untup(tuple(c * np.asarray(x, np.float64) for x in _tup(a)), a)


def zeros_like(a):
    return _untup(tuple(np.zeros_like(np.asarray(x, np.float64)) for x in _tup(a)), a)


class LSQRResult:
    def __init__(self, x, resid, iters, alphas, betas):
        self.x = x
        self.resid = resid        # [phibar_1, phibar_2, ...] residual-norm estimates
        self.iters = iters
        self.alphas = alphas
        self.betas = betas


def lsqr(matvec, rmatvec, b, niter: int, tol: float = 0.0, x_like=None) -> LSQRResult:
    """Paige-Saunders LSQR for min ||A x - b||, x0 = 0."""
    beta = norm(b)
    if x_like is None:
        x_like = rmatvec(b)
    x = zeros_like(x_like)
    if beta == 0.0:
        return LSQRResult(x, [0.0], 0, [], [0.0])
    u = scale(1.0 / beta, b)
    v = rmatvec(u)
    alpha = norm(v)
    alphas, betas = [alpha], [beta]
    if alpha == 0.0:
        return LSQRResult(x, [beta], 0, alphas, betas)
    v = scale(1.0 / alpha, v)
    w = v
    phibar, rhobar = beta, alpha
    beta1 = beta
    resid = [beta]
    it = 0
    for it in range(1, niter + 1):
        # bidiagonalisation: beta u = A v - alpha u ; alpha v = A^H u - beta v
        u = lincomb(1.0, matvec(v), -alpha, u)
        beta = norm(u)
        if beta > 0.0:
            u = scale(1.0 / beta, u)
            v = lincomb(1.0, rmatvec(u), -beta, v)
            alpha = norm(v)
            if alpha > 0.0:
                v = scale(1.0 / alpha, v)
        else:
            alpha = 0.0
        alphas.append(alpha)
        betas.append(beta)
        # plane rotation eliminating beta from the lower bidiagonal
        rho = math.hypot(rhobar, beta)
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        # solution and search-direction updates
        x = lincomb(1.0, x, phi / rho, w)
        w = lincomb(1.0, v, -theta / rho, w)
        resid.append(phibar)
        if beta == 0.0 or alpha == 0.0:
            break
        if tol > 0.0 and phibar <= tol * beta1:
            break
    return LSQRResult(x, resid, it, alphas, betas)


def cgls(matvec, rmatvec, b, niter: int, x_like=None):
    """Hestenes-Stiefel CG on A^H A x = A^H b, x0 = 0.  Returns (x, [||r_k||])."""
    r = b
    s = rmatvec(r)
    x = zeros_like(s if x_like is None else x_like)
    p = s
    gamma = dot(s, s)
    resid = [norm(r)]
    for _ in range(niter):
        if gamma == 0.0:
            break
        q = matvec(p)
        qq = dot(q, q)
        if qq == 0.0:
            break
        a = gamma / qq
        x = lincomb(1.0, x, a, p)
        r = lincomb(1.0, r, -a, q)
        s = rmatvec(r)
        gnew = dot(s, s)
        p = lincomb(1.0, s, gnew / gamma, p)
        gamma = gnew
        resid.append(norm(r))
    return x, resid


def neumann(apply_N, d, nterms: int):
    """Partial Neumann sum sum_{j<nterms} N^j d (forward-only Marchenko iteration)."""
    term = d
    acc = d
    for _ in range(1, nterms):
        term = apply_N(term)
        acc = lincomb(1.0, acc, 1.0, term)
    return acc
