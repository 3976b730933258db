"""GPU parity of the tcgen05 tensor-core products (FP16/BF16/E4M3 kernel copies, >= 8 columns).

The tensor-core path also rounds the spectra (B operand) to the 16-bit type, after a
power-of-two column scaling, so its error against the FP64 oracle on the dequantised
kernel is bounded by the B rounding (tolerance 4u) and against the exact kernel by
both roundings (tolerance 8u), u the format's unit roundoff.  It is also checked
against the decoding SIMT path on the same stored kernel, and by the dot-product test.
"""
import numpy as np
import pytest

from oracle import mdc as omdc
from test_gpu_precision import FORMATS, dequantised, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(storage, nt, nr, ns, nf, nv, seed=0):
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(seed + nt + nr + ns + nv)
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 400.0, storage=storage)
    yg = op.forward(torch.from_numpy(x).cuda())
    xg = op.adjoint(torch.from_numpy(y).cuda())
    m.mdc_device_status(op.h)
    op.close()
    return G, x, y, yg.cpu().numpy(), xg.cpu().numpy()


@pytest.mark.parametrize("storage", ["c16f", "cbf16"])
def test_tc_tiny_first(storage):
    """Smallest tensor-core case: one tile in every dimension."""
    G, x, y, yg, xg = run(storage, 64, 100, 60, 2, 8)
    u = FORMATS[storage][0]
    Gq = dequantised(G, storage)
    assert rel(yg, omdc.forward(Gq, x, 0.004, 400.0)) <= 4 * u
    assert rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0)) <= 4 * u


CASES = [
    (64, 130, 70, 5, 8),        # ragged rows and columns, 2 row tiles
    (128, 257, 300, 20, 16),    # adjoint K tail (nr not a multiple of 64)
    (256, 129, 129, 40, 40),    # column tail inside a 128-wide tile
    (64, 64, 64, 9, 64),        # exact tiles
    (128, 200, 190, 12, 150),   # two N tiles (300 real columns)
]


@pytest.mark.parametrize("storage", ["c16f", "cbf16"])
@pytest.mark.parametrize("nt,nr,ns,nf,nv", CASES)
def test_tc_matches_oracle(storage, nt, nr, ns, nf, nv):
    G, x, y, yg, xg = run(storage, nt, nr, ns, nf, nv)
    u = FORMATS[storage][0]
    Gq = dequantised(G, storage)
    ef = rel(yg, omdc.forward(Gq, x, 0.004, 400.0))
    ea = rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0))
    print(f"tc {storage} nr={nr} ns={ns} nv={nv}: vs dequantised kernel fwd {ef:.2e} adj {ea:.2e}")
    assert ef <= 4 * u and ea <= 4 * u
    assert rel(yg, omdc.forward(G, x, 0.004, 400.0)) <= 8 * u
    assert rel(xg, omdc.adjoint(G, y, 0.004, 400.0)) <= 8 * u
    lhs = np.vdot(yg.astype(np.float64), y)
    rhs = np.vdot(x.astype(np.float64), xg)
    assert abs(lhs - rhs) <= 8 * u * np.linalg.norm(yg) * np.linalg.norm(y)


U16 = 2.0 ** -11     # FP16 unit roundoff


@pytest.mark.parametrize("nt,nr,ns,nf,nv", CASES)
def test_tc_e4m3_widened_matches_oracle(nt, nr, ns, nf, nv):
    """E4M3 kernel copy on tensor cores: TMA brings the kernel as bytes; the GEMM widens them to
    FP16 (exactly: E4M3 is a subset of FP16), or, for forward products of at most 21 columns, feeds
    them unwidened to E4M3 MMAs against a three-term E4M3 split of the spectra.  Against the FP64
    oracle on the dequantised E4M3 kernel the only error is the rounding of the spectra (FP16, or
    about 12 bits for the split: tolerance 4 u16 for both), like the FP16 copy's."""
    G, x, y, yg, xg = run("ce4m3", nt, nr, ns, nf, nv)
    Gq = dequantised(G, "ce4m3")
    ef = rel(yg, omdc.forward(Gq, x, 0.004, 400.0))
    ea = rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0))
    print(f"tc ce4m3 nr={nr} ns={ns} nv={nv}: vs dequantised kernel fwd {ef:.2e} adj {ea:.2e}")
    assert ef <= 4 * U16 and ea <= 4 * U16
    lhs = np.vdot(yg.astype(np.float64), y)
    rhs = np.vdot(x.astype(np.float64), xg)
    assert abs(lhs - rhs) <= 8 * U16 * np.linalg.norm(yg) * np.linalg.norm(y)
