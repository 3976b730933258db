"""Autotuner: every column-count bucket gets a runnable variant, results after tuning still
match the FP64 oracle, and the JSON-lines cache is reused by a second handle."""
import os

import numpy as np
import pytest

from oracle import mdc as omdc
from test_gpu_precision import FORMATS, dequantised, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["c16f", "c32s", "c64"])
def test_autotune_choices_and_parity(tmp_path, storage):
    import paper_2011_11120_gb300 as m
    os.environ["MDC_AUTOTUNE_CACHE"] = str(tmp_path / "tune.jsonl")
    try:
        rng = np.random.default_rng(4)
        nt, nf, nr, ns = 128, 24, 300, 280
        G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
        Gt = torch.from_numpy(G.astype(np.complex64)).cuda()
        op = m.MDC(Gt, nt, 0.004, 400.0, storage=storage)
        m.mdc_autotune(op.h, 40)
        for adj in (False, True):
            for ncol in (1, 3, 5, 8, 17, 40):
                path, bn = m.mdc_autotune_choice(op.h, adj, ncol)
                assert path in ("gemv", "gemv-groups", "simt", "tensor-core")
                if path == "gemv":
                    assert ncol <= 4
                if path == "gemv-groups":
                    assert 4 < ncol <= 64
                if path == "tensor-core":
                    assert storage != "c64" and bn in (32, 64, 128, 256)
        Gq = dequantised(G, storage) if storage == "c16f" else G
        tol = 4 * FORMATS["c16f"][0] if storage == "c16f" else 1e-5
        for nv in (1, 5, 17, 40):
            x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
            y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
            yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
            xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
            assert rel(yg, omdc.forward(Gq, x, 0.004, 400.0)) <= tol
            assert rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0)) <= tol
        first = {(a, n): m.mdc_autotune_choice(op.h, a, n) for a in (False, True) for n in (1, 8, 40)}
        # a second handle of the same shape and storage reads the stored table
        op2 = m.MDC(Gt, nt, 0.004, 400.0, storage=storage)
        m.mdc_autotune(op2.h, 40)
        assert {(a, n): m.mdc_autotune_choice(op2.h, a, n) for a in (False, True) for n in (1, 8, 40)} == first
        lines = open(os.environ["MDC_AUTOTUNE_CACHE"]).read().strip().splitlines()
        assert len(lines) == 1 and '"choices"' in lines[0]
        op.close()
        op2.close()
    finally:
        del os.environ["MDC_AUTOTUNE_CACHE"]
