"""FP64 multi-dimensional deconvolution (Eq. 8), test infrastructure only.

Eq. 8 models the up-going field at the receivers x_S for a virtual source x_F'
as the MDC of the local reflectivity r(t, x_F, x_F') with the down-going
Green's function G^+(w, x_S, x_F) as kernel (integration over the focusing
points x_F), written compactly as g^- = G^+ r.  It is a Fredholm equation of
the first kind (no Neumann expansion), so r is estimated by an iterative
least-squares solver applied to the MDC operator and its adjoint; the paper
solves it for batches of virtual sources x_F' at a time.

Arrays: kernel ``[nf, n_S, n_F]`` complex, data g^- ``[nt, n_S, nv]`` and
reflectivity ``[nt, n_F, nv]`` real, nv the virtual sources of one batch.
The MDC readings (scaling, circular time) are those of ``oracle.mdc``.
"""
from __future__ import annotations

import numpy as np

from . import mdc, solvers


class MDD:
    """g^- = G^+ r with G^+ the kernel of an MDC operator (Eq. 8)."""

    def __init__(self, Gplus, dt: float, dr: float):
        self.G = np.asarray(Gplus, dtype=np.complex128)
        self.dt, self.dr = dt, dr

    def matvec(self, r):
        return mdc.forward(self.G, r, self.dt, self.dr)

    def rmatvec(self, g):
        return mdc.adjoint(self.G, g, self.dt, self.dr)

    def solve(self, g_minus, niter: int, tol: float = 0.0):
        """LSQR from r = 0 on the MDC operator (the least-squares estimate of r)."""
        return solvers.lsqr(self.matvec, self.rmatvec, np.asarray(g_minus, np.float64), niter=niter, tol=tol)

    def adjoint_estimate(self, g_minus):
        """r ~ G^{+H} g^-: one adjoint MDC, the correlation-type estimate the paper contrasts with
        the inversion (Section "Source-side redatuming via Multi-dimensional deconvolution")."""
        return self.rmatvec(g_minus)
