"""FP64 Marchenko block operator (Eq. 5), its adjoint, and Green's functions (Eq. 6).

Test infrastructure only.  Eq. 5 stacks the unknown focusing functions
[f^-; f_m^+] (each ``[nt, ns, nv]``) and applies

    M = [[ I,        -Theta R ],
         [ -Theta R*,  I      ]],      d = [Theta R f_d^+ ; 0],

where R is the MDC with the reflection response as kernel, R* the MDC with
the complex-conjugated kernel (a correlation), and Theta a 0/1 time-space
window.  Eq. 6 then evaluates the up- and down-going fields from the solved
focusing functions with f^+ = f_d^+ + f_m^+:

    [-g^- ; g^{+*}] = [[ I, -R ], [ -R*, I ]] [f^- ; f^+].

Window reading (design notes): Theta[t, s, v] = 1 when |tau(t)| < c[s, v],
tau the signed circular time sample (t for t < nt/2, t - nt otherwise), with
c the caller's integer cut-offs.
"""
from __future__ import annotations

import numpy as np

from . import mdc


def signed_time(nt: int) -> np.ndarray:
    t = np.arange(nt)
    return np.where(t < nt // 2, t, t - nt)


def window(cutoffs: np.ndarray, nt: int) -> np.ndarray:
    """Theta as a 0/1 float64 array [nt, ns, nv] from integer cut-offs [ns, nv]."""
    tau = np.abs(signed_time(nt))
    return (tau[:, None, None] < np.asarray(cutoffs)[None, :, :]).astype(np.float64)


class Marchenko:
    """Eq. 5 operator on the stacked unknown (f^-, f_m^+), each [nt, ns, nv]."""

    def __init__(self, G, dt, dr, cutoffs, nt):
        self.G = np.asarray(G, dtype=np.complex128)
        if self.G.shape[1] != self.G.shape[2]:
            raise ValueError("the Marchenko operator needs a square kernel (nr == ns)")
        self.dt, self.dr, self.nt = dt, dr, nt
        self.theta = window(cutoffs, nt)

    def R(self, x):
        return mdc.forward(self.G, x, self.dt, self.dr)

    def Rstar(self, x):
        return mdc.forward_conj_kernel(self.G, x, self.dt, self.dr)

    def RH(self, y):
        return mdc.adjoint(self.G, y, self.dt, self.dr)

    def RstarH(self, y):
        return mdc.adjoint_conj_kernel(self.G, y, self.dt, self.dr)

    def matvec(self, f):
        """M [f^-; f_m^+] = [f^- - Theta R f_m^+ ; f_m^+ - Theta R* f^-]."""
        fm, fp = f
        return (fm - self.theta * self.R(fp), fp - self.theta * self.Rstar(fm))

    def rmatvec(self, g):
        """M^H [a; b] = [a - (R*)^H Theta b ; b - R^H Theta a]."""
        a, b = g
        return (a - self.RstarH(self.theta * b), b - self.RH(self.theta * a))

    def data(self, fd_plus):
        """d = [Theta R f_d^+ ; 0] of Eq. 5."""
        fd_plus = np.asarray(fd_plus, dtype=np.float64)
        return (self.theta * self.R(fd_plus), np.zeros_like(fd_plus))

    def greens(self, f_minus, f_mplus, fd_plus):
        """Eq. 6: returns (g^-, g^{+*}, g^+) with g^+ the time reversal of g^{+*}."""
        f_plus = np.asarray(fd_plus, dtype=np.float64) + f_mplus
        g_minus = -(f_minus - self.R(f_plus))
        g_plus_star = f_plus - self.Rstar(f_minus)
        return g_minus, g_plus_star, time_reverse(g_plus_star)


def time_reverse(x):
    """(P x)[t] = x[(-t) mod nt] along axis 0."""
    x = np.asarray(x)
    return np.roll(x[::-1], 1, axis=0)
