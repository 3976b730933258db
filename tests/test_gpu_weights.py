"""GPU parity: per-column integration weights (irregular geometry, Voronoi areas).

The kernel's columns are multiplied by the weights before they are stored (complex64) or
quantised (FP16), so forward, adjoint and the Marchenko solve on an irregular half of a
grid match the oracle with the weighted kernel.
"""
import numpy as np
import pytest

import synth
from oracle import marchenko as omar
from oracle import mdc as omdc
from oracle import solvers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("storage,tol", [("c64", 1e-5), ("c16f", 5e-4), ("c32s", 1e-5)])
def test_weighted_forward_adjoint(storage, tol):
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(3)
    nt, nf, nr, ns, nv = 128, 40, 70, 90, 9
    G = rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))
    w = rng.uniform(100.0, 900.0, size=ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 1.0, storage=storage, weights=w)
    yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    op.close()
    Gw = omdc.weighted_kernel(G, w)
    assert rel(yg, omdc.forward(Gw, x, 0.004, 1.0)) <= tol
    assert rel(xg, omdc.adjoint(Gw, y, 0.004, 1.0)) <= tol


def test_marchenko_on_irregular_geometry():
    """Half of an 11 x 11 grid kept at random; each receiver integrates over its Voronoi cell."""
    import paper_2011_11120_gb300 as m
    cfg = synth.Config(96, "irregular", 11, 256, 0.004, 60, 5, 4, 500.0, point_grid=2)  # window keeps part of R f_d+
    d = synth.draw(cfg)
    idx = synth.irregular_subset(cfg.n_side, 0.5, seed=2)
    xy = synth.grid_xy(cfg.n_side)[idx]
    lo, hi = -0.5 * synth.GRID_DX, synth.GRID_DX * (cfg.n_side - 0.5)
    w = synth.voronoi_areas(xy, lo, hi, res=512)
    G = synth.kernel(cfg, d, rows=idx, cols=idx)
    Gw = omdc.weighted_kernel(G, w)
    smax = max(np.linalg.norm(Gw[k], 2) for k in range(cfg.nf))
    G *= 0.5 / (cfg.dt * smax)                   # ||R|| = 0.5 with the weights folded in
    Gw = omdc.weighted_kernel(G, w)
    cut = synth.window_cutoffs(cfg, d)[idx]
    fd = synth.direct_focusing(cfg, d)[:, idx]
    op_o = omar.Marchenko(Gw, cfg.dt, 1.0, cut, cfg.nt)
    res = solvers.lsqr(op_o.matvec, op_o.rmatvec, op_o.data(fd), niter=12)
    gm, _, gp = op_o.greens(res.x[0], res.x[1], fd)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, 1.0, weights=w)
    out = op.marchenko(torch.from_numpy(np.ascontiguousarray(cut)).cuda(),
                       torch.from_numpy(np.ascontiguousarray(fd)).cuda(), 12)
    op.close()
    assert rel(out["f_minus"].cpu().numpy(), res.x[0]) <= 1e-5
    assert rel(out["f_mplus"].cpu().numpy(), res.x[1]) <= 1e-5
    assert rel(out["g_minus"].cpu().numpy(), gm) <= 1e-5
    assert rel(out["g_plus"].cpu().numpy(), gp) <= 1e-5


def test_weights_rejected_when_invalid():
    import paper_2011_11120_gb300 as m
    G = torch.zeros((5, 4, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(m.MDCError):
        m.MDC(G, 64, 0.004, 1.0, weights=[1.0, -1.0, 1.0])
    with pytest.raises(m.MDCError):
        m.MDC(G, 64, 0.004, 1.0, weights=[1.0, float("nan"), 1.0])
