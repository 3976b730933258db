"""GPU parity: MDC forward/adjoint (Eq. 3), conjugate kernel (Eq. 5), against the FP64 oracle.

Tolerance: relative L2 <= 1e-5 over the whole output for the float32 path (the
kernel is rounded once to complex64, FFTs and products run in float32 with
float32 accumulation).
"""
import numpy as np
import pytest

import synth
from oracle import mdc as omdc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    import paper_2011_11120_gb300 as m
    return m


def rand_case(nt, nr, ns, nf, nv, seed):
    rng = np.random.default_rng(seed)
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    return G, x, y


CASES = [
    # nt, nr, ns, nf, nv      (ragged sizes, nr != ns, every bin, GEMV and GEMM column counts)
    (64, 7, 9, 33, 1),
    (128, 130, 70, 40, 2),
    (256, 65, 200, 64, 3),
    (64, 33, 33, 17, 4),
    (128, 100, 77, 50, 5),
    (64, 40, 90, 20, 17),
    (512, 150, 129, 100, 64),
    (1024, 61, 67, 200, 1),
    (4096, 9, 5, 2049, 2),
    (2048, 17, 23, 300, 1),
    (128, 45, 133, 40, 11),     # GEMV passes over column groups of 4, 4 and 3
    (2048, 33, 40, 1025, 3),    # every bin of nt = 2048, Nyquist included
    (2048, 9, 14, 1, 6),        # DC only
]


@pytest.mark.parametrize("nt,nr,ns,nf,nv", CASES)
@pytest.mark.parametrize("conj", [False, True])
def test_forward_adjoint_match_oracle(lib, nt, nr, ns, nf, nv, conj):
    G, x, y = rand_case(nt, nr, ns, nf, nv, seed=nt + nr + ns + nv)
    dt, dr = 0.004, 400.0
    op = lib.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, dt, dr)
    yg = op.forward(torch.from_numpy(x).cuda(), conj=conj).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda(), conj=conj).cpu().numpy()
    Gk = np.conj(G) if conj else G
    assert rel(yg, omdc.forward(Gk, x, dt, dr)) <= TOL
    assert rel(xg, omdc.adjoint(Gk, y, dt, dr)) <= TOL
    op.close()


def test_config1_full_size_and_dot_test(lib):
    cfg = synth.config(1)
    d = synth.draw(cfg)
    G = synth.kernel(cfg, d)
    x = synth.ricker_traces(cfg, d)
    yrand = synth.random_traces(cfg, 1, seed_offset=3, nspace=cfg.nr)
    op = lib.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    y = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xa = op.adjoint(torch.from_numpy(yrand).cuda()).cpu().numpy()
    assert rel(y, omdc.forward(G, x, cfg.dt, cfg.dr)) <= TOL
    assert rel(xa, omdc.adjoint(G, yrand, cfg.dt, cfg.dr)) <= TOL
    # dot-product test of the GPU operator pair
    lhs = np.vdot(y.astype(np.float64), yrand)
    rhs = np.vdot(x.astype(np.float64), xa)
    assert abs(lhs - rhs) <= TOL * np.linalg.norm(y) * np.linalg.norm(yrand)
    op.close()


def test_device_generated_kernel_matches_synth(lib):
    from synth import gpu as sgpu
    cfg = synth.config(1)
    d = synth.draw(cfg)
    Gd = sgpu.kernel_on_device(cfg, d).cpu().numpy()
    G = synth.kernel(cfg, d)
    assert rel(Gd, G) <= 3e-7


def test_empty_and_bad_arguments(lib):
    G = torch.zeros((5, 3, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.MDCError):
        lib.MDC(G, 100, 0.004, 1.0)          # nt not a power of two
    with pytest.raises(lib.MDCError):
        lib.MDC(G, 8, 0.004, 1.0)            # nfmax > nt/2 + 1 and nt < 64
    op = lib.MDC(G, 64, 0.004, 1.0)
    x = torch.zeros((64, 4, 1), device="cuda")
    y = torch.empty((64, 3, 1), device="cuda")
    with pytest.raises(lib.MDCError):
        lib.mdc_forward(op.h, x, y, 0)       # nv < 1
    with pytest.raises(lib.MDCError):
        lib.mdc_forward(op.h, x, y, 1, 0x80)  # unknown flag
    # zero kernel gives exactly zero output
    op.forward(torch.randn((64, 4, 2), device="cuda"), out=torch.empty((64, 3, 2), device="cuda"))
    out = op.forward(torch.randn((64, 4, 2), device="cuda"))
    assert float(out.abs().max()) == 0.0
    op.close()


@pytest.mark.parametrize("nv,storage", [(1, "c64"), (64, "c64"), (64, "c32s")])
def test_config2_full_size_sampled_rows(lib, nv, storage):
    """nr = ns = 3721, nt = 1024, nf = 200: the bench workload; oracle on sampled rows/columns.
    The split FP16 storage runs the 64-column products on tensor cores at float32 tolerance."""
    from synth import gpu as sgpu
    cfg = synth.config(2, nv=nv)
    d = synth.draw(cfg)
    Gdev = sgpu.kernel_on_device(cfg, d)
    op = lib.MDC(Gdev, cfg.nt, cfg.dt, cfg.dr, storage=storage)
    del Gdev
    torch.cuda.empty_cache()
    x = synth.ricker_traces(cfg, d)
    y = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    yr = synth.random_traces(cfg, nv, seed_offset=5, nspace=cfg.nr)
    xa = op.adjoint(torch.from_numpy(yr).cuda()).cpu().numpy()
    op.close()
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(cfg.nr, size=6, replace=False))
    rows[0] = cfg.nr - 1          # ragged tail row
    Gr = synth.kernel(cfg, d, rows=rows)
    ef = rel(y[:, rows], omdc.forward_rows(Gr, x, cfg.dt, cfg.dr))
    print(f"config2 {storage} nv={nv}: sampled forward rel L2 {ef:.2e}")
    assert ef <= TOL
    cols = np.sort(rng.choice(cfg.ns, size=6, replace=False))
    cols[-1] = cfg.ns - 1
    Gc = synth.kernel(cfg, d, cols=cols)
    ea = rel(xa[:, cols], omdc.adjoint_cols(Gc, yr, cfg.dt, cfg.dr))
    print(f"config2 {storage} nv={nv}: sampled adjoint rel L2 {ea:.2e}")
    assert ea <= TOL
