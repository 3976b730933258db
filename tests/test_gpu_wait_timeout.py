"""Failure detection inside the tensor-core product: a bounded device wait that runs out.

Every wait of the tcgen05 GEMM (TMA stages, MMA completion, accumulator hand-off) is bounded in
wall time by the handle's limit (MDC_OPT_WAIT_LIMIT_US, default 2 s).  Here the limit is set to
1 microsecond on a product whose first output tile alone needs about a thousand pipeline stages
(tens of microseconds), so the epilogue's first wait cannot be met.  Nothing is broken on purpose:
every copy and MMA the kernel issues completes, the kernel drains them before it exits, and only
the short limit makes the waits give up.  The test checks that the handle then reports
MDC_ERR_TIMEOUT, that the flag clears, and that the same handle (limit restored) and a fresh one
compute the product correctly afterwards.  FP16 storage runs the 16-bit GEMM; E4M3 storage at
8 columns runs the swapped-operand E4M3 kernel, whose waits are bounded the same way.
"""
import numpy as np
import pytest

from oracle import mdc as omdc
from test_gpu_precision import FORMATS, dequantised, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MDC_ERR_TIMEOUT = -4


@pytest.mark.parametrize("storage", ["c16f", "ce4m3"])
def test_short_wait_limit_reports_timeout_then_recovers(storage):
    import paper_2011_11120_gb300 as m
    nt, nr, ns, nf, nv = 64, 256, 32768, 2, 8
    rng = np.random.default_rng(77)
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    Gd = torch.from_numpy(G.astype(np.complex64)).cuda()
    xd = torch.from_numpy(x).cuda()
    u = FORMATS["c16f"][0]                 # spectra rounding of both tensor-core paths: within 4 u16
    y_ref = omdc.forward(dequantised(G, storage), x, 0.004, 400.0)

    op = m.MDC(Gd, nt, 0.004, 400.0, storage=storage)
    try:
        m.mdc_reserve(op.h, nv)
        m.mdc_set_option(op.h, m.MDC_OPT_WAIT_LIMIT_US, 1)
        op.forward(xd)
        with pytest.raises(m.MDCError) as exc:
            m.mdc_device_status(op.h)
        assert exc.value.status == MDC_ERR_TIMEOUT
        m.mdc_device_status(op.h)          # the flag was cleared by the first check
        assert m.mdc_tc_fallback_count(op.h) == 0   # the product did run on tensor cores

        # the default limit again: the same handle computes the right product
        m.mdc_set_option(op.h, m.MDC_OPT_WAIT_LIMIT_US, 0)
        y = op.forward(xd)
        m.mdc_device_status(op.h)
        assert rel(y.cpu().numpy(), y_ref) <= 4 * u
    finally:
        op.close()

    op2 = m.MDC(Gd, nt, 0.004, 400.0, storage=storage)
    try:
        y2 = op2.forward(xd)
        m.mdc_device_status(op2.h)
        assert rel(y2.cpu().numpy(), y_ref) <= 4 * u
    finally:
        op2.close()


def test_wait_limit_option_rejects_negative_values():
    import paper_2011_11120_gb300 as m
    G = torch.zeros((2, 8, 8), dtype=torch.complex64, device="cuda")
    op = m.MDC(G, 64, 0.004, 400.0, storage="c16f")
    try:
        with pytest.raises(m.MDCError):
            m.mdc_set_option(op.h, m.MDC_OPT_WAIT_LIMIT_US, -1)
    finally:
        op.close()
