"""The Marchenko solve's kernel passes against the paper's cost count (tests/golden/cost_model.json).

The Discussion section counts the MDCs of a Marchenko inversion: 2 per application of the Eq. 5
operator and 2 per application of its adjoint, so 4 per iteration; 1 more for the data vector and 2 for
the Green's functions of Eq. 6, about 43 for 10 iterations.  Here R and R* share one pass over the kernel
(one product launch over 2nv columns = 2 MDCs), as do R^H and (R*)^H, so the per-kernel-class launch
counters must show, for niter iterations: niter + 2 forward products (iterations, data vector with nv
columns, Green's functions) and niter + 1 adjoint products (iterations and the start of LSQR, which the
paper's count leaves out).
"""
import json
import os

import numpy as np
import pytest

from test_gpu_marchenko import problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cost_model.json")


def test_marchenko_product_passes_match_the_papers_count():
    import paper_2011_11120_gb300 as m
    cm = json.load(open(GOLDEN))
    niter = cm["niter"]
    cfg, G, cut, fd = problem(5, 128, 40, 1, 200.0)          # one focusing point: 2 columns per pass
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    try:
        m.mdc_timing(op.h, True)
        out = op.marchenko(torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda(), niter)
        _, nfwd = m.mdc_timing_read(op.h, "product_fwd")
        _, nadj = m.mdc_timing_read(op.h, "product_adj")
        m.mdc_timing(op.h, False)
    finally:
        op.close()
    assert out["iters"] == niter
    assert nfwd == niter + 2 and nadj == niter + 1
    # in MDCs (a launch over 2nv columns counts 2, the data vector's nv-column launch 1)
    mdc_fwd = 2 * niter + cm["mdc_data"] + cm["mdc_greens"]
    mdc_adj = 2 * niter + 2
    assert mdc_fwd + mdc_adj - 2 == cm["mdc_per_iteration"] * niter + cm["mdc_data"] + cm["mdc_greens"]
    assert cm["mdc_per_iteration"] * niter + cm["mdc_data"] + cm["mdc_greens"] == cm["total_quoted"]
