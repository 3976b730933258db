"""GPU: NaN canaries.  Every output buffer is filled with NaN before the call; the call must overwrite
every element (an element a kernel forgot to write stays NaN), on ragged shapes that leave partial
tiles in every kernel: GEMV (1-4 columns), SIMT GEMM, tensor cores, the chunked GEMV, the FFT column
tails, the Marchenko and MDD solvers.  Inputs are finite, so every correct output is finite.
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def nan_like(shape):
    return torch.full(shape, math.nan, dtype=torch.float32, device="cuda")


def kernel(nf, nr, ns, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.complex(torch.randn((nf, nr, ns), generator=g, device="cuda"),
                         torch.randn((nf, nr, ns), generator=g, device="cuda")) / math.sqrt(ns)


@pytest.mark.parametrize("storage", ["c64", "c16f", "ce4m3", "c32s"])
@pytest.mark.parametrize("nt,nr,ns,nf,nv", [
    (64, 7, 9, 33, 1),          # tiny, every bin
    (128, 130, 70, 40, 3),      # GEMV, ragged rows
    (256, 65, 201, 60, 9),      # tensor cores / SIMT, ragged columns
    (2048, 33, 40, 300, 2),     # half-length transforms
    (64, 29, 6500, 3, 1),       # chunked forward GEMV
])
def test_mdc_outputs_fully_written(storage, nt, nr, ns, nf, nv):
    import paper_2011_11120_gb300 as m
    op = m.MDC(kernel(nf, nr, ns, nt + nr + ns), nt, 0.004, 1.0, storage=storage)
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    x = torch.randn((nt, ns, nv), generator=g, device="cuda")
    y = torch.randn((nt, nr, nv), generator=g, device="cuda")
    for conj in (False, True):
        yo = nan_like((nt, nr, nv))
        op.forward(x, out=yo, conj=conj)
        xo = nan_like((nt, ns, nv))
        op.adjoint(y, out=xo, conj=conj)
        assert bool(torch.isfinite(yo).all()) and bool(torch.isfinite(xo).all())
    m.mdc_device_status(op.h)
    op.close()


@pytest.mark.parametrize("storage", ["c64", "c16f"])
def test_solver_outputs_fully_written(storage):
    import paper_2011_11120_gb300 as m
    cfg = synth.tiny(n_side=5, nt=128, nf=40, n_events=4, nv=9, point_grid=3, z_point=200.0)
    d = synth.draw(cfg)
    G = torch.from_numpy(synth.kernel(cfg, d).astype(np.complex64)).cuda() * 1e-4
    op = m.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=storage)
    cut = torch.from_numpy(synth.window_cutoffs(cfg, d)).cuda()
    fd = torch.from_numpy(synth.direct_focusing(cfg, d)).cuda()
    nv = fd.shape[2]
    outs = [nan_like(fd.shape) for _ in range(4)]
    m.marchenko_lsqr(op.h, cut, fd, nv, 4, 0.0, *outs)
    assert all(bool(torch.isfinite(o).all()) for o in outs)
    outs = [nan_like(fd.shape) for _ in range(4)]
    m.marchenko_neumann(op.h, cut, fd, nv, 3, *outs)
    assert all(bool(torch.isfinite(o).all()) for o in outs)
    r = nan_like((cfg.nt, cfg.ns, nv))
    m.mdd_lsqr(op.h, fd, nv, 3, 0.0, r)
    assert bool(torch.isfinite(r).all())
    m.mdc_device_status(op.h)
    op.close()
