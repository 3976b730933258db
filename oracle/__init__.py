"""FP64 CPU oracle for the multi-dimensional convolution (MDC) operator, the
Marchenko block operator and LSQR/CGLS.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) use it.
It shares no code with the CUDA library; the two meet only through the seeded
inputs of ``synth``.

Every routine is written plainly, in float64/complex128, in the order of the
paper's equations, with NumPy's FFT and matrix product as library primitives:

* ``mdc``       -- Eq. 2 and Eq. 3 (forward C and adjoint C^H), Eq. 7 (the
                   seismic convention: conjugate kernel R*), row-sampled
                   evaluation for kernels too large to hold.
* ``marchenko`` -- Eq. 5 (block operator M, its adjoint, data vector), Eq. 6
                   (Green's functions), the time-space window Theta.
* ``solvers``   -- LSQR (Paige and Saunders, 1982) and CGLS (Hestenes and
                   Stiefel), the solvers used on Eq. 5 and Eq. 8.

Pins (tests under ``tests/test_oracle_*.py``) tie each routine to something
other than itself: brute-force circular convolution, the dot-product test,
identity and projector special cases, a single-event closed form, the
time-reversal identity, dense least squares and Neumann sums.
"""
from . import mdc, marchenko, solvers  # noqa: F401
