"""mdc_forward_static_scratch: the forward MDC pass that allocates nothing.

Some callers cannot let the library call cudaMalloc while they apply the operator
(their device memory is held by their own pool allocator, or an allocation's implicit
synchronisation is too costly), so this entry point keeps its two frequency-domain
work arrays in a fixed 32 MiB device array compiled into the library.  The test calls
it through the C ABI and checks it against mdc_forward, twice in a row (the fixed
array keeps the previous call's contents), and checks that an oversize request is
refused.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_scratch_forward_matches_mdc_forward_twice():
    import paper_2011_11120_gb300 as m
    L = m.lib()
    cfg = synth.config(1)
    d = synth.draw(cfg)
    G = torch.from_numpy(synth.kernel(cfg, d).astype(np.complex64)).cuda()
    h = m.mdc_create(G, cfg.nt, cfg.dt, cfg.dr)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        inputs = [synth.ricker_traces(cfg, d), synth.random_traces(cfg, 3, seed_offset=9)]
        for x_np in inputs:                       # two calls in a row, different inputs and nv
            nv = x_np.shape[2]
            x = torch.from_numpy(x_np).cuda()
            y_ref = torch.empty((cfg.nt, cfg.nr, nv), device="cuda")
            y_new = torch.full((cfg.nt, cfg.nr, nv), float("nan"), device="cuda")
            assert L.mdc_forward(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y_ref.data_ptr()),
                                 nv, 0, stream) == 0
            assert L.mdc_forward_static_scratch(h, ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(y_new.data_ptr()), nv, 0, stream) == 0
            torch.cuda.synchronize()
            assert rel(y_new.cpu().numpy(), y_ref.cpu().numpy()) <= TOL
        # a request larger than the fixed array is refused before anything is launched
        nv_big = (1 << 21) // (cfg.nf * cfg.nr) + 1
        xb = torch.zeros((cfg.nt, cfg.ns, nv_big), device="cuda")
        yb = torch.zeros((cfg.nt, cfg.nr, nv_big), device="cuda")
        assert L.mdc_forward_static_scratch(h, ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(yb.data_ptr()),
                                            nv_big, 0, stream) == -6
    finally:
        m.mdc_destroy(h)
