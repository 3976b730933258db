"""GPU: the chunked GEMV kernels for long kernel rows and columns.

When the spectrum a GEMV keeps in shared memory (X(w) of ns values in the forward pass, Y(w) of
nr values in the adjoint, per column) would exceed 48 KB, it is staged in 32 KB chunks instead,
so that several CTAs still fit on an SM (the paper's Full geometry has 9801 traces: 78 KB per
column).  Each lane keeps its summation order, so the chunked kernels must give exactly the
bits of the whole-row kernels (compared in two processes, MDC_GEMV_CHUNK=0 turning chunking
off) and match the FP64 oracle like them, in every storage format and for 1 to 4 columns.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import mdc as omdc
from test_gpu_precision import FORMATS, dequantised, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STORAGES = ["c64", "c16f", "cbf16", "ce4m3", "c32s"]


def _run(storage, G, x, y, nt):
    import paper_2011_11120_gb300 as m
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 400.0, storage=storage)
    yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    m.mdc_device_status(op.h)
    op.close()
    return yg, xg


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("nv", [1, 2, 3, 4])
def test_chunked_gemv_matches_oracle(storage, nv):
    """Forward chunked on 6500-value rows (4 chunks of complex64, ragged last chunk); adjoint
    chunked on 6500-value columns; the other direction of each operator is short."""
    nt, nf = 64, 3
    rng = np.random.default_rng(100 + nv)
    for nr, ns in ((29, 6500), (6500, 29)):
        G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(max(nr, ns))
        x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
        y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
        yg, xg = _run(storage, G, x, y, nt)
        Gq = G if storage in ("c64", "c32s") else dequantised(G, storage)
        ef = rel(yg, omdc.forward(Gq, x, 0.004, 400.0))
        ea = rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0))
        print(f"chunked {storage} nv={nv} nr={nr} ns={ns}: fwd {ef:.2e} adj {ea:.2e}")
        assert ef <= 1e-5 and ea <= 1e-5


_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2011_11120_gb300 as m
gen = torch.Generator(device="cuda")
gen.manual_seed(7)
nt, nf, n = 64, 2, 6200          # 49.7 KB per column: chunked by default; whole rows fit up to 4 columns
G = torch.complex(torch.randn((nf, n, n), generator=gen, device="cuda"),
                  torch.randn((nf, n, n), generator=gen, device="cuda")) / 80.0
outs = []
for storage in {storages!r}:
    op = m.MDC(G, nt, 0.004, 400.0, storage=storage)
    for nv in (1, 2, 3, 4):
        x = torch.randn((nt, n, nv), generator=gen, device="cuda")
        outs.append(op.forward(x).cpu().numpy().ravel())
        outs.append(op.adjoint(x).cpu().numpy().ravel())
    m.mdc_device_status(op.h)
    op.close()
np.save({out!r}, np.concatenate(outs))
"""


def test_chunked_and_whole_row_gemv_are_bit_identical(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for chunk in ("1", "0"):
        out = str(tmp_path / f"c{chunk}.npy")
        env = dict(os.environ, MDC_GEMV_CHUNK=chunk)
        code = _SCRIPT.format(root=root, storages=STORAGES, out=out)
        subprocess.run([sys.executable, "-c", code], env=env, check=True, timeout=600)
        res.append(np.load(out))
    assert np.isfinite(res[0]).all()
    assert np.array_equal(res[0], res[1])
