"""GPU parity: Marchenko LSQR (Eq. 5) and Green's functions (Eq. 6) against the FP64 oracle.

The kernel is normalised so that ||R||_2 = 0.5 (the redatuming workload's
reading), which keeps M well conditioned; float32 vectors with float64 LSQR
scalars then track the float64 oracle to relative L2 <= 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import marchenko as omar
from oracle import solvers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def problem(n_side, nt, nf, nv_grid, z, n_events=5, seed_number=95):
    cfg = synth.Config(seed_number, "redatum-test", n_side, nt, 0.004, nf, n_events, nv_grid * nv_grid, z,
                       point_grid=nv_grid)
    d = synth.draw(cfg)
    G = synth.kernel(cfg, d)
    smax = max(np.linalg.norm(G[k], 2) for k in range(cfg.nf))
    G *= 0.5 / (cfg.dt * cfg.dr * smax)
    cut = synth.window_cutoffs(cfg, d)
    fd = synth.direct_focusing(cfg, d)
    return cfg, G, cut, fd


def oracle_solve(cfg, G, cut, fd, niter, tol=0.0):
    op = omar.Marchenko(G, cfg.dt, cfg.dr, cut, cfg.nt)
    d = op.data(fd)
    res = solvers.lsqr(op.matvec, op.rmatvec, d, niter=niter, tol=tol)
    gm, gps, gp = op.greens(res.x[0], res.x[1], fd)
    return res, gm, gp


@pytest.mark.parametrize("n_side,nt,nf,nvg,z,niter", [
    (3, 64, 20, 1, 120.0, 6),       # nv = 1: 2 columns per pass (GEMV)
    (5, 128, 40, 2, 200.0, 10),     # nv = 4: 8 columns per pass (GEMM)
    (21, 512, 150, 2, 800.0, 20),   # redatuming shapes at reduced aperture
    (3, 2048, 300, 1, 600.0, 6),    # nt = 2048 (half-length real transforms), GEMV
    (5, 2048, 301, 2, 600.0, 6),    # nt = 2048, GEMM, odd nf
    (3, 4096, 100, 2, 600.0, 4),    # nt = 4096 (radix-2 kernels: forward transforms as launches of their own)
])
def test_marchenko_lsqr_matches_oracle(n_side, nt, nf, nvg, z, niter):
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(n_side, nt, nf, nvg, z)
    res, gm, gp = oracle_solve(cfg, G, cut, fd, niter)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    out = op.marchenko(torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda(), niter)
    op.close()
    assert out["iters"] == res.iters == niter
    assert rel(out["f_minus"].cpu().numpy(), res.x[0]) <= TOL
    assert rel(out["f_mplus"].cpu().numpy(), res.x[1]) <= TOL
    assert rel(out["g_minus"].cpu().numpy(), gm) <= TOL
    assert rel(out["g_plus"].cpu().numpy(), gp) <= TOL
    assert np.allclose(out["resid"], res.resid, rtol=TOL, atol=0)


def test_marchenko_tolerance_stop_matches_oracle():
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(5, 128, 40, 2, 200.0)
    res, _, _ = oracle_solve(cfg, G, cut, fd, niter=50, tol=1e-4)
    assert 1 < res.iters < 50
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    out = op.marchenko(torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda(), 50, tol=1e-4, greens=False)
    op.close()
    assert out["iters"] == res.iters
    assert all(r == -1.0 for r in out["resid"][res.iters + 1:])
    assert rel(out["f_minus"].cpu().numpy(), res.x[0]) <= TOL


def test_marchenko_zero_window_gives_zero_solution():
    """Theta = 0: d = 0, so x = 0 and Eq. 6 reduces to g- = R f_d+, g+ = P f_d+."""
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(3, 64, 20, 1, 120.0)
    cut0 = np.zeros_like(cut)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    out = op.marchenko(torch.from_numpy(cut0).cuda(), torch.from_numpy(fd).cuda(), 5)
    op.close()
    assert out["iters"] == 0
    assert float(out["f_minus"].abs().max()) == 0.0 and float(out["f_mplus"].abs().max()) == 0.0
    ref = omar.Marchenko(G, cfg.dt, cfg.dr, cut0, cfg.nt)
    _, _, gp = ref.greens(np.zeros_like(fd, np.float64), np.zeros_like(fd, np.float64), fd)
    assert rel(out["g_plus"].cpu().numpy(), gp) <= TOL
    assert rel(out["g_minus"].cpu().numpy(), ref.R(fd)) <= TOL


def test_marchenko_rejects_rectangular_kernel():
    import paper_2011_11120_gb300 as m
    G = torch.zeros((5, 3, 4), dtype=torch.complex64, device="cuda")
    op = m.MDC(G, 64, 0.004, 1.0)
    fd = torch.zeros((64, 4, 1), device="cuda")
    with pytest.raises(m.MDCError):
        op.marchenko(torch.zeros((4, 1), dtype=torch.int32, device="cuda"), fd, 3)
    op.close()


@pytest.mark.parametrize("storage,tol_plain,tol_refined", [("c16f", 5e-3, 1e-4), ("cbf16", 3e-2, 1e-3)])
def test_marchenko_reduced_precision_with_refinement(storage, tol_plain, tol_refined):
    """FP16/BF16 kernel inside LSQR (tensor-core products at 2nv = 8 columns), float32 refinement.

    Stated figures: without refinement the solution carries the operator's rounding amplified
    by the conditioning (kappa <= 3 here); one refinement step brings it to the float32 level.
    """
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(21, 512, 150, 2, 800.0)
    niter = 20
    res, gm, gp = oracle_solve(cfg, G, cut, fd, niter)
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda()
    lo = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage=storage)
    ref = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    cut_t, fd_t = torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda()
    plain = lo.marchenko(cut_t, fd_t, niter, greens=False)
    out = lo.marchenko_refined(ref, cut_t, fd_t, niter, nrefine=1, niter_refine=10)
    lo.close()
    ref.close()
    e_plain = rel(plain["f_minus"].cpu().numpy(), res.x[0])
    e_ref = max(rel(out["f_minus"].cpu().numpy(), res.x[0]), rel(out["f_mplus"].cpu().numpy(), res.x[1]))
    e_g = max(rel(out["g_minus"].cpu().numpy(), gm), rel(out["g_plus"].cpu().numpy(), gp))
    print(f"{storage}: plain {e_plain:.2e} refined {e_ref:.2e} greens {e_g:.2e} "
          f"final residual {out['final_residual']:.2e} iters {out['iters']}")
    assert e_plain <= tol_plain
    assert e_ref <= tol_refined and e_g <= tol_refined
    assert out["iters"] == niter + 10
    assert 0.0 <= out["final_residual"] <= 1e-3


def test_refined_rejects_reduced_reference():
    import paper_2011_11120_gb300 as m
    G = torch.zeros((5, 4, 4), dtype=torch.complex64, device="cuda")
    a = m.MDC(G, 64, 0.004, 1.0, storage="c16f")
    b = m.MDC(G, 64, 0.004, 1.0, storage="c16f")
    fd = torch.zeros((64, 4, 1), device="cuda")
    with pytest.raises(m.MDCError):
        a.marchenko_refined(b, torch.zeros((4, 1), dtype=torch.int32, device="cuda"), fd, 3)
    a.close()
    b.close()


def test_marchenko_graph_replay_matches_direct_solve():
    """MDC_OPT_GRAPHS: the repeated solve is captured once and replayed; results equal the
    direct solve bit for bit, replays read the current contents of the input buffers, and a
    replay issues no host-side kernel launches."""
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(5, 128, 40, 2, 200.0)
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda()
    op = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage="c16f")
    ref = m.MDC(Gt, cfg.nt, cfg.dt, cfg.dr, storage="c32s")
    cut_t, fd_t = torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda()
    nv = fd.shape[2]
    direct = op.marchenko_refined(ref, cut_t, fd_t, 10, nrefine=1, niter_refine=4)
    m.mdc_set_option(op.h, m.MDC_OPT_GRAPHS, 1)
    outs = [torch.empty_like(fd_t) for _ in range(4)]
    for rep in range(3):
        n0 = m.mdc_launch_count(op.h)
        resid, fin, iters = m.marchenko_lsqr_refined(op.h, ref.h, cut_t, fd_t, nv, 10, 1, 4, 0.0, *outs)
        if rep > 0:
            assert m.mdc_launch_count(op.h) == n0      # replay: no host launches
        assert iters == direct["iters"] and fin == direct["final_residual"]
        for o, k in zip(outs, ("f_minus", "f_mplus", "g_minus", "g_plus")):
            assert torch.equal(o, direct[k])
    fd_t.mul_(2.0)
    m.marchenko_lsqr_refined(op.h, ref.h, cut_t, fd_t, nv, 10, 1, 4, 0.0, *outs)
    assert torch.equal(outs[0], 2.0 * direct["f_minus"])
    m.mdc_set_option(op.h, m.MDC_OPT_GRAPHS, 0)
    op.close()
    ref.close()


@pytest.mark.parametrize("niter", [0, 1, 6])
def test_marchenko_neumann_matches_oracle(niter):
    """Neumann series of Eq. 5 against the oracle's partial sum; niter = 0 gives the
    single-scattering Green's functions g0- = R f_d+ (f = 0 in Eq. 6)."""
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(5, 128, 40, 2, 200.0)
    op_o = omar.Marchenko(G, cfg.dt, cfg.dr, cut, cfg.nt)
    d = op_o.data(fd)
    apply_N = lambda x: solvers.lincomb(1.0, x, -1.0, op_o.matvec(x))  # noqa: E731  N = I - M
    if niter == 0:
        x = [np.zeros_like(d[0]), np.zeros_like(d[1])]
    else:
        x = solvers.neumann(apply_N, d, niter)
    gm, _, gp = op_o.greens(x[0], x[1], fd)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    out = op.neumann(torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda(), niter)
    op.close()
    if niter == 0:
        assert float(out["f_minus"].abs().max()) == 0.0 and float(out["f_mplus"].abs().max()) == 0.0
        assert rel(out["g_minus"].cpu().numpy(), op_o.R(fd)) <= TOL
    else:
        assert rel(out["f_minus"].cpu().numpy(), x[0]) <= TOL
        if niter == 1:                  # x = d = [Theta R f_d+; 0]
            assert float(out["f_mplus"].abs().max()) == 0.0
        else:
            assert rel(out["f_mplus"].cpu().numpy(), x[1]) <= TOL
    assert rel(out["g_minus"].cpu().numpy(), gm) <= TOL
    assert rel(out["g_plus"].cpu().numpy(), gp) <= TOL


def test_marchenko_neumann_nt2048_matches_oracle():
    """Neumann series at nt = 2048: the half-length transforms with every fused epilogue term."""
    import paper_2011_11120_gb300 as m
    cfg, G, cut, fd = problem(3, 2048, 300, 2, 600.0)
    op_o = omar.Marchenko(G, cfg.dt, cfg.dr, cut, cfg.nt)
    d = op_o.data(fd)
    apply_N = lambda x: solvers.lincomb(1.0, x, -1.0, op_o.matvec(x))  # noqa: E731  N = I - M
    x = solvers.neumann(apply_N, d, 4)
    gm, _, gp = op_o.greens(x[0], x[1], fd)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    out = op.neumann(torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda(), 4)
    op.close()
    assert rel(out["f_minus"].cpu().numpy(), x[0]) <= TOL
    assert rel(out["f_mplus"].cpu().numpy(), x[1]) <= TOL
    assert rel(out["g_minus"].cpu().numpy(), gm) <= TOL
    assert rel(out["g_plus"].cpu().numpy(), gp) <= TOL


def test_redatuming_workload_full_size_two_points():
    """The bench's redatuming workload at full size (1681 x 1681 kernel, nt = 512, nfmax = 150,
    ||R|| = 0.5), sampled to two of its 256 focusing points: the complex64 LSQR solve and the
    FP16 solve refined against the split-FP16 reference (the bench's configuration) both match the
    FP64 oracle's converged solution."""
    import paper_2011_11120_gb300 as m
    from synth import gpu as sgpu
    cfg = synth.config(4)
    d = synth.draw(cfg)
    pick = [0, 137]
    cut = np.ascontiguousarray(synth.window_cutoffs(cfg, d)[:, pick])
    fd = np.ascontiguousarray(synth.direct_focusing(cfg, d)[:, :, pick])
    Gd = sgpu.kernel_on_device(cfg, d)
    G = Gd.cpu().numpy().astype(np.complex128)            # the workload's kernel, for the oracle
    op_o = omar.Marchenko(G, cfg.dt, cfg.dr, cut, cfg.nt)
    res = solvers.lsqr(op_o.matvec, op_o.rmatvec, op_o.data(fd), niter=30)
    del G, op_o
    cut_t, fd_t = torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda()
    plain = m.MDC(Gd, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    out = plain.marchenko(cut_t, fd_t, 20, greens=False)
    plain.close()
    lo = m.MDC(Gd, cfg.nt, cfg.dt, cfg.dr, storage="c16f")
    ref = m.MDC(Gd, cfg.nt, cfg.dt, cfg.dr, storage="c32s")
    del Gd
    outr = lo.marchenko_refined(ref, cut_t, fd_t, 20, nrefine=1, niter_refine=5, greens=False)
    lo.close()
    ref.close()
    e_plain = max(rel(out["f_minus"].cpu().numpy(), res.x[0]), rel(out["f_mplus"].cpu().numpy(), res.x[1]))
    e_ref = max(rel(outr["f_minus"].cpu().numpy(), res.x[0]), rel(outr["f_mplus"].cpu().numpy(), res.x[1]))
    print(f"full-size redatuming, 2 points: complex64 {e_plain:.2e}, FP16 + refinement {e_ref:.2e}")
    assert e_plain <= TOL
    assert e_ref <= TOL
