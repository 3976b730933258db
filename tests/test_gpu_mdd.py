"""GPU parity: multi-dimensional deconvolution (Eq. 8) by LSQR against the FP64 oracle.

The kernel is rectangular (receivers x_S by focusing points x_F) and scaled so that the
MDC operator has 2-norm about 1 with a condition number of a few; float32 vectors with
float64 LSQR scalars then track the oracle to relative L2 <= 1e-5.
"""
import numpy as np
import pytest

from oracle import mdd as omdd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
DT, DR = 0.004, 400.0


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def problem(nt, nf, nS, nF, nv, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((nf, nS, nF)) + 1j * rng.standard_normal((nf, nS, nF))
    k = min(nS, nF)
    G[:, :k, :k] += 2.0 * np.sqrt(max(nS, nF)) * np.eye(k)
    smax = max(np.linalg.norm(G[k], 2) for k in range(nf))
    G *= 1.0 / (DT * DR * smax)
    g = rng.standard_normal((nt, nS, nv)).astype(np.float32)
    return G, g


@pytest.mark.parametrize("nt,nf,nS,nF,nv,niter", [
    (64, 20, 30, 12, 1, 8),         # one virtual source (GEMV products)
    (128, 40, 100, 49, 20, 15),     # a batch of 20 virtual sources, as in the paper's MDD runs
    (256, 60, 70, 130, 3, 10),      # more focusing points than receivers (wide kernel)
    (2048, 200, 40, 25, 4, 6),      # half-length transforms, the next product's spectra fused
])
def test_mdd_lsqr_matches_oracle(nt, nf, nS, nF, nv, niter):
    import paper_2011_11120_gb300 as m
    G, g = problem(nt, nf, nS, nF, nv, seed=nt + nS + nF)
    res = omdd.MDD(G, DT, DR).solve(g, niter)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, DT, DR)
    out = op.mdd(torch.from_numpy(g).cuda(), niter)
    op.close()
    assert out["iters"] == res.iters == niter
    assert rel(out["r"].cpu().numpy(), res.x) <= TOL
    assert np.allclose(out["resid"], res.resid, rtol=TOL, atol=0)


def test_mdd_tolerance_stop_matches_oracle():
    import paper_2011_11120_gb300 as m
    G, _ = problem(128, 40, 60, 30, 4, seed=4)
    o = omdd.MDD(G, DT, DR)
    g = o.matvec(np.random.default_rng(3).standard_normal((128, 30, 4))).astype(np.float32)   # consistent data
    res = o.solve(g, 60, tol=1e-3)
    assert 1 < res.iters < 60
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), 128, DT, DR)
    out = op.mdd(torch.from_numpy(g).cuda(), 60, tol=1e-3)
    op.close()
    assert out["iters"] == res.iters
    assert all(r == -1.0 for r in out["resid"][res.iters + 1:])
    assert rel(out["r"].cpu().numpy(), res.x) <= TOL


def test_mdd_fp16_kernel_on_tensor_cores():
    """FP16 kernel copy, 20 virtual sources: tensor-core products inside LSQR; the stated bound
    is the FP16 operator error amplified by the conditioning of the problem."""
    import paper_2011_11120_gb300 as m
    G, g = problem(128, 40, 100, 49, 20, seed=9)
    res = omdd.MDD(G, DT, DR).solve(g, 12)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), 128, DT, DR, storage="c16f")
    out = op.mdd(torch.from_numpy(g).cuda(), 12)
    op.close()
    e = rel(out["r"].cpu().numpy(), res.x)
    print(f"mdd c16f rel L2 {e:.2e}")
    assert e <= 5e-3


def test_mdd_zero_data_and_bad_arguments():
    import paper_2011_11120_gb300 as m
    G, g = problem(64, 20, 30, 12, 2, seed=1)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), 64, DT, DR)
    out = op.mdd(torch.zeros((64, 30, 2), device="cuda"), 5)
    assert out["iters"] == 0 and float(out["r"].abs().max()) == 0.0
    r = torch.empty((64, 12, 2), device="cuda")
    with pytest.raises(m.MDCError):
        m.mdd_lsqr(op.h, torch.from_numpy(g).cuda(), 2, 0, 0.0, r)
    op.close()
