"""FP64 multi-dimensional convolution: forward C and adjoint C^H (test infrastructure).

Eq. 2 writes the MDC in the frequency domain: Fourier transform the input
along time, keep the first n_wmax frequencies, integrate the kernel against
it over the receiver axis at every frequency, and transform back.  Eq. 3
writes the same as C = F^H I^H K I F (forward) and C^H = F^H I^H K^H I F
(adjoint), K being the block-diagonal batch of per-frequency dense products
with the kernel already multiplied by the integration weight (Eq. 4 and the
discretisation paragraph of the Theory section).

Readings taken here (listed with the others in the design notes):

* the real FFT is unnormalised forward and carries 1/nt on the inverse; this
  is the same operator as the orthonormal pair the paper describes for F and
  F^H and keeps C^H the exact adjoint of C (the kernel's time response is real);
* the integration weight is the constant dt*dr (time step times the areal
  extent of one receiver); it multiplies the kernel;
* the convolution is circular over nt samples (no zero padding in time).

Arrays: time-domain real ``[nt, n_space, nv]``, frequency-domain complex
``[nf, n_space, nv]``, kernel complex ``[nf, nr, ns]``.
"""
from __future__ import annotations

import numpy as np


def rfft_truncate(x: np.ndarray, nf: int) -> np.ndarray:
    """F then I_wmax of Eq. 3: real FFT along time, keep the first nf bins."""
    X = np.fft.rfft(np.asarray(x, dtype=np.float64), axis=0)
    return X[:nf]


def pad_irfft(Y: np.ndarray, nt: int) -> np.ndarray:
    """I_wmax^H then F^H of Eq. 3: zero-pad to nt/2+1 bins and inverse real FFT."""
    full = np.zeros((nt // 2 + 1,) + Y.shape[1:], dtype=np.complex128)
    full[: Y.shape[0]] = Y
    return np.fft.irfft(full, n=nt, axis=0)


def batch_matmul(G: np.ndarray, X: np.ndarray) -> np.ndarray:
    """K of Eq. 3/4: one dense product per frequency slice, G(w) X(w)."""
    return np.matmul(G, X)


def weighted_kernel(G: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Receiver-dependent integration weights (the areal extent of each point's Voronoi cell for
    an irregular geometry) pre-multiplied into the kernel's columns, the integration axis, before
    the batched products (Theory section, discretisation paragraph)."""
    return np.asarray(G, np.complex128) * np.asarray(w, np.float64)[None, None, :]


def forward(G: np.ndarray, x: np.ndarray, dt: float, dr: float) -> np.ndarray:
    """g = C f (Eq. 3, left): x [nt, ns, nv] -> y [nt, nr, nv]."""
    G = np.asarray(G, dtype=np.complex128)
    nt = x.shape[0]
    X = rfft_truncate(x, G.shape[0])
    Y = batch_matmul(G * (dt * dr), X)
    return pad_irfft(Y, nt)


def adjoint(G: np.ndarray, y: np.ndarray, dt: float, dr: float) -> np.ndarray:
    """f = C^H g (Eq. 3, right): y [nt, nr, nv] -> x [nt, ns, nv], kernel G(w)^H."""
    G = np.asarray(G, dtype=np.complex128)
    nt = y.shape[0]
    Y = rfft_truncate(y, G.shape[0])
    X = batch_matmul(np.conj(np.swapaxes(G, 1, 2)) * (dt * dr), Y)
    return pad_irfft(X, nt)


def forward_conj_kernel(G, x, dt, dr):
    """R* of Eq. 5 and the text after it: the MDC whose kernel is conj(G) (correlation)."""
    return forward(np.conj(G), x, dt, dr)


def adjoint_conj_kernel(G, y, dt, dr):
    """(R*)^H: the adjoint of the conjugate-kernel MDC."""
    return adjoint(np.conj(G), y, dt, dr)


# ------------------------------------------------------------------ row-sampled forms
def forward_rows(G_rows: np.ndarray, x: np.ndarray, dt: float, dr: float) -> np.ndarray:
    """Selected output rows of C x, given the kernel rows G[:, rows, :] (Eq. 3).

    Each output receiver row depends only on its own kernel row, so a sample of
    rows of a kernel too large to hold is evaluated exactly.
    Returns y[:, rows, :] as [nt, len(rows), nv].
    """
    return forward(G_rows, x, dt, dr)


def adjoint_cols(G_cols: np.ndarray, y: np.ndarray, dt: float, dr: float) -> np.ndarray:
    """Selected output columns of C^H y, given the kernel columns G[:, :, cols] (Eq. 3).

    Returns x[:, cols, :] as [nt, len(cols), nv].
    """
    return adjoint(G_cols, y, dt, dr)
