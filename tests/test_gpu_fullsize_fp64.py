"""The batched redatuming solve at its real size against the FP64 oracle.

The bench's redatuming workload -- 1681 traces (41 x 41), nt = 512, nfmax = 150, kernel normalised to
||R|| = 0.5, 256 focusing points on a 16 x 16 lattice solved as ONE LSQR system (one set of FP64
scalars coupling all 512 columns of every pass), 20 iterations -- is solved on the GPU exactly as the
bench does (FP16 kernel on tensor cores, one refinement step of 5 iterations against a split-FP16
float32-accurate reference), and plainly in complex64; the FP64 oracle (NumPy, on the host cores)
solves the same 256-point system with 20 LSQR iterations and evaluates the Green's functions.

The oracle needs about 15 minutes of host CPU and 30 GB of host memory, so the test runs only when
MDC_FULL_FP64=1 is set (the measured figures are kept in the design notes).  Tolerances: complex64
<= 1e-5 relative L2 (the float32 path's bound); FP16 with refinement <= 1e-3 (the reduced-precision
target), both on f-, f_m+, g- and g+.  The GPU kernel comes from the device generator, which agrees
with the FP64 formula to about 3e-7; the oracle evaluates the formula in FP64 itself.
"""
import os
import time

import numpy as np
import pytest

import synth
from oracle import marchenko as omar
from oracle import solvers

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("MDC_FULL_FP64") != "1",
                                 reason="full-size FP64 comparison: set MDC_FULL_FP64=1 (about 15 min of host CPU)")]


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_redatuming_256_points_full_size_vs_fp64_oracle():
    import paper_2011_11120_gb300 as m
    from synth import gpu as sgpu
    cfg = synth.config(4)
    d = synth.draw(cfg)
    cut = synth.window_cutoffs(cfg, d)
    fd = synth.direct_focusing(cfg, d)
    niter, nref, nin = cfg.niter, 1, 5

    # ---- GPU: the bench's solve (FP16 + split-FP16 refinement) and the plain complex64 solve
    G = sgpu.kernel_on_device(cfg, d)
    lo = m.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c16f")
    ref = m.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c32s")
    c64 = m.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    del G
    torch.cuda.empty_cache()
    cut_t, fd_t = torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda()
    out16 = lo.marchenko_refined(ref, cut_t, fd_t, niter, nrefine=nref, niter_refine=nin)
    out32 = c64.marchenko(cut_t, fd_t, niter)
    keys = ("f_minus", "f_mplus", "g_minus", "g_plus")
    g16 = {k: out16[k].cpu().numpy() for k in keys}
    g32 = {k: out32[k].cpu().numpy() for k in keys}
    for op in (lo, ref, c64):
        op.close()
    del out16, out32, cut_t, fd_t
    torch.cuda.empty_cache()

    # ---- FP64 oracle: the same 256-point system, 20 LSQR iterations, Eq. 6
    t0 = time.perf_counter()
    Gh = synth.kernel(cfg, d)
    op = omar.Marchenko(Gh, cfg.dt, cfg.dr, cut, cfg.nt)
    res = solvers.lsqr(op.matvec, op.rmatvec, op.data(fd), niter=niter)
    gm, _, gp = op.greens(res.x[0], res.x[1], fd)
    oracle = {"f_minus": res.x[0], "f_mplus": res.x[1], "g_minus": gm, "g_plus": gp}
    t_oracle = time.perf_counter() - t0

    e32 = {k: rel(g32[k], oracle[k]) for k in keys}
    e16 = {k: rel(g16[k], oracle[k]) for k in keys}
    print(f"full-size redatuming vs FP64 oracle ({t_oracle:.0f} s of oracle): complex64 {e32}; "
          f"FP16 + refinement {e16}")
    assert res.iters == niter
    for k in keys:
        assert e32[k] <= 1e-5, (k, e32[k])
        assert e16[k] <= 1e-3, (k, e16[k])
