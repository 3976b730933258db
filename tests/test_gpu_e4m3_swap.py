"""E4M3 products of few columns with the operands swapped: the kernel's bytes are the wide (N = 256)
operand of kind::f8f6f4 MMAs (K-major forward, MN-major adjoint) and the spectra are split exactly
into three E4M3 terms (h0 + h1/16 + h2/256, about 12 significant bits).

Against the FP64 oracle on the dequantised E4M3 kernel the only error is the spectra's three-term
rounding (relative 2^-12 per element) and float32 accumulation, so the tolerance is 2^-10, tighter
than the 4 u16 of the 16-bit-spectra path.  Shapes: ragged kernel rows across two and three
256-row tiles, ragged reduction (ns not a multiple of 64), 8 / 16 / 21 columns (21 fills 126 of the
128 stacked rows) and 22 columns (back on the widening kernel); the dot-product test ties forward
and adjoint together.
"""
import numpy as np
import pytest

from oracle import mdc as omdc
from test_gpu_precision import dequantised, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2.0 ** -10
U16 = 2.0 ** -11


@pytest.mark.parametrize("nt,nr,ns,nf,nv", [
    (64, 300, 70, 5, 8),        # two kernel-row tiles (256 + 44), short reduction
    (128, 600, 301, 7, 16),     # three tiles, ns ragged against 64
    (64, 257, 129, 3, 21),      # 21 columns: 126 stacked rows; one row past a tile
    (64, 130, 90, 4, 22),       # 22 columns: widening kernel
])
def test_e4m3_swapped_forward_matches_oracle(nt, nr, ns, nf, nv):
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(7 + nr + nv)
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 400.0, storage="ce4m3")
    try:
        yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
        m.mdc_device_status(op.h)
        assert m.mdc_tc_fallback_count(op.h) == 0
    finally:
        op.close()
    Gq = dequantised(G, "ce4m3")
    ef = rel(yg, omdc.forward(Gq, x, 0.004, 400.0))
    ea = rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0))
    print(f"e4m3 nr={nr} ns={ns} nv={nv}: vs dequantised kernel forward {ef:.2e} adjoint {ea:.2e}")
    tol = TOL if nv <= 21 else 4 * U16
    assert ef <= tol and ea <= tol
    lhs = np.vdot(yg.astype(np.float64), y)
    rhs = np.vdot(x.astype(np.float64), xg)
    assert abs(lhs - rhs) <= 8 * U16 * np.linalg.norm(yg) * np.linalg.norm(y)
