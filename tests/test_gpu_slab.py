"""GPU: kernels loaded frequency slab by frequency slab (mdc_create_empty + mdc_load_slab).

A kernel too large to stage whole beside its library copy (the paper's Full geometry, Table 1:
300 frequencies of a 9801 x 9801 kernel, 230 GB in complex64) is filled one slab of frequencies
at a time.  Loading every frequency once must give the operator mdc_create gives on the whole
kernel, bit for bit in every storage format; the slab generator of the synthetic workload must
reproduce the whole-kernel generator bit for bit; and at the Full size the forward and adjoint
outputs on sampled rows match the FP64 oracle.
"""
import numpy as np
import pytest

import synth
from oracle import mdc as omdc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_slab_generator_matches_whole_kernel():
    from synth import gpu as sgpu
    cfg = synth.tiny(n_side=9, nt=256, nf=70, n_events=6)
    d = synth.draw(cfg)
    whole = sgpu.kernel_on_device(cfg, d)
    parts = [sgpu.kernel_slab_on_device(cfg, k0, nk, d) for k0, nk in ((0, 1), (1, 32), (33, 37))]
    assert torch.equal(torch.cat(parts).view(torch.float32), whole.view(torch.float32))


@pytest.mark.parametrize("storage", ["c64", "c16f", "cbf16", "ce4m3", "c32s"])
def test_slab_loaded_operator_is_bit_identical(storage):
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(11)
    nt, nf, nr, ns, nv = 256, 45, 130, 70, 3          # ragged rows and columns (not tile multiples)
    G = torch.from_numpy((rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns)))
                         .astype(np.complex64)).cuda()
    x = torch.from_numpy(rng.standard_normal((nt, ns, nv)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal((nt, nr, nv)).astype(np.float32)).cuda()
    whole = m.MDC(G, nt, 0.004, 2.5, storage=storage)
    slab = m.MDC.empty(nf, nr, ns, nt, 0.004, 2.5, storage=storage)
    for k0, k1 in ((30, 45), (0, 1), (1, 30)):          # any order, uneven slabs
        slab.load_slab(G[k0:k1].contiguous(), k0)
    for conj in (False, True):
        assert torch.equal(slab.forward(x, conj=conj), whole.forward(x, conj=conj))
        assert torch.equal(slab.adjoint(y, conj=conj), whole.adjoint(y, conj=conj))
    whole.close()
    slab.close()


def test_unloaded_frequencies_are_zero():
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(12)
    nt, nf, nr, ns, nv = 128, 30, 40, 50, 2
    G = torch.from_numpy((rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns)))
                         .astype(np.complex64)).cuda()
    x = torch.from_numpy(rng.standard_normal((nt, ns, nv)).astype(np.float32)).cuda()
    for storage in ("c64", "c16f"):
        part = m.MDC.empty(nf, nr, ns, nt, 0.004, 1.0, storage=storage)
        part.load_slab(G[5:17].contiguous(), 5)
        Gz = torch.zeros_like(G)
        Gz[5:17] = G[5:17]
        ref = m.MDC(Gz, nt, 0.004, 1.0, storage=storage)
        assert torch.equal(part.forward(x), ref.forward(x))
        part.close()
        ref.close()


def test_slab_bad_arguments():
    import paper_2011_11120_gb300 as m
    op = m.MDC.empty(10, 8, 6, 64, 0.004, 1.0)
    G = torch.zeros((4, 8, 6), dtype=torch.complex64, device="cuda")
    for k0 in (-1, 7, 10):                                # outside [0, nfmax - nk]
        with pytest.raises(m.MDCError):
            op.load_slab(G, k0)
    with pytest.raises(m.MDCError):
        m.MDC.empty(40, 8, 6, 64, 0.004, 1.0)             # nfmax > nt/2 + 1
    op.close()


def test_paper_full_size_sampled_rows():
    """Full geometry of Table 1: 99 x 99 = 9801 co-located sources and receivers, 300 frequencies,
    complex64 (about 232 GB on the device), loaded in 20-frequency slabs.  Forward and adjoint at
    one virtual point, two sampled output rows and columns against the FP64 oracle."""
    import paper_2011_11120_gb300 as m
    from synth import gpu as sgpu
    torch.cuda.empty_cache()
    cfg = synth.config(6)
    ldg = -(-cfg.ns // 64) * 64
    need = cfg.nf * cfg.nr * ldg * 8 + 20 * cfg.nr * cfg.ns * 8 + (4 << 30)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB free on the device, {free / 1e9:.0f} GB free")
    d = synth.draw(cfg)
    op = m.MDC.empty(cfg.nf, cfg.nr, cfg.ns, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    buf = torch.empty((20, cfg.nr, cfg.ns), dtype=torch.complex64, device="cuda")
    for k0 in range(0, cfg.nf, 20):
        sgpu.kernel_slab_on_device(cfg, k0, 20, d, out=buf)
        op.load_slab(buf, k0)
    del buf
    torch.cuda.empty_cache()
    x = synth.ricker_traces(cfg, d)                       # [nt, ns, 1]
    rng = np.random.default_rng(5)
    y = rng.standard_normal((cfg.nt, cfg.nr, 1)).astype(np.float32)
    yg = op.forward(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    op.close()
    for r in (123, 7777):
        Grow = synth.kernel(cfg, d, rows=[r])             # FP64 [nf, 1, ns]
        assert rel(yg[:, r:r + 1], omdc.forward(Grow, x, cfg.dt, cfg.dr)) <= 1e-5
        Gcol = synth.kernel(cfg, d, cols=[r])             # [nf, nr, 1]
        assert rel(xg[:, r:r + 1], omdc.adjoint(Gcol, y, cfg.dt, cfg.dr)) <= 1e-5
