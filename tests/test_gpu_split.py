"""GPU parity of the split FP16 storage (MDC_C32S): each component is kept as an FP16 pair
hi + lo (about 22 significant bits, row-scaled), so every product path -- GEMV, SIMT GEMM
and the three-product tensor-core GEMM (hi*hi + hi*lo + lo*hi) -- must meet the float32
tolerance of the complex64 path: relative L2 <= 1e-5 against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import mdc as omdc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nt,nr,ns,nf,nv", [
    (64, 7, 9, 33, 1),          # GEMV
    (128, 130, 70, 40, 3),      # GEMV
    (64, 40, 90, 20, 6),        # SIMT GEMM
    (64, 100, 60, 12, 8),       # tensor cores, one tile
    (128, 257, 300, 20, 17),    # tensor cores, ragged tiles and adjoint K tail
    (256, 129, 129, 40, 64),    # tensor cores, full column tile
    (128, 200, 190, 12, 150),   # tensor cores, two column tiles
])
def test_split_storage_meets_float32_tolerance(nt, nr, ns, nf, nv):
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(nt + nr + ns + nv)
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 400.0, storage="c32s")
    yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    m.mdc_device_status(op.h)
    op.close()
    ef = rel(yg, omdc.forward(G, x, 0.004, 400.0))
    ea = rel(xg, omdc.adjoint(G, y, 0.004, 400.0))
    print(f"c32s nr={nr} ns={ns} nv={nv}: forward {ef:.2e} adjoint {ea:.2e}")
    assert ef <= TOL and ea <= TOL


def test_split_storage_synthetic_kernel_full_size_config1():
    import paper_2011_11120_gb300 as m
    cfg = synth.config(1)
    d = synth.draw(cfg)
    G = synth.kernel(cfg, d)
    x = synth.random_traces(cfg, 16)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr, storage="c32s")
    yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    op.close()
    assert rel(yg, omdc.forward(G, x, cfg.dt, cfg.dr)) <= TOL
