"""mdc_forward_static_scratch: the forward MDC pass that allocates nothing.

Some callers cannot let the library call cudaMalloc while they apply the operator
(their device memory is held by their own pool allocator, or an allocation's implicit
synchronisation is too costly), so this entry point keeps its two frequency-domain
work arrays in a fixed 32 MiB device array compiled into the library.  The tests call
it through the C ABI and check it, twice in a row (the fixed array keeps the previous
call's contents), against mdc_forward on the same handle and against the FP64 oracle:
plain and conjugated kernel (R*), complex64 storage on the GEMV path, and FP16 storage
on the tensor-core path after mdc_reserve.  Free device memory must not change across
the calls once the first one has loaded the kernels, and an oversize request is
refused.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import mdc as omdc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5                 # complex64 path vs the FP64 oracle and vs mdc_forward
U16 = 2.0 ** -11           # FP16 unit roundoff: the tensor-core path's tolerance is 4 u16


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("flags", [0, 1], ids=["R", "Rstar"])
def test_static_scratch_forward_matches_mdc_forward_twice(flags):
    import paper_2011_11120_gb300 as m
    L = m.lib()
    cfg = synth.config(1)
    d = synth.draw(cfg)
    G64 = synth.kernel(cfg, d)
    G = torch.from_numpy(G64.astype(np.complex64)).cuda()
    h = m.mdc_create(G, cfg.nt, cfg.dt, cfg.dr)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    oracle = omdc.forward_conj_kernel if flags else omdc.forward
    try:
        inputs = [synth.ricker_traces(cfg, d), synth.random_traces(cfg, 3, seed_offset=9)]
        for x_np in inputs:                       # two calls in a row, different inputs and nv
            nv = x_np.shape[2]
            x = torch.from_numpy(x_np).cuda()
            y_ref = torch.empty((cfg.nt, cfg.nr, nv), device="cuda")
            y_new = torch.full((cfg.nt, cfg.nr, nv), float("nan"), device="cuda")
            assert L.mdc_forward(h, _ptr(x), _ptr(y_ref), nv, flags, stream) == 0
            assert L.mdc_forward_static_scratch(h, _ptr(x), _ptr(y_new), nv, flags, stream) == 0
            torch.cuda.synchronize()
            yn = y_new.cpu().numpy()
            assert rel(yn, y_ref.cpu().numpy()) <= TOL
            assert rel(yn, oracle(G64, x_np, cfg.dt, cfg.dr)) <= TOL
        # a request larger than the fixed array is refused before anything is launched
        nv_big = (1 << 21) // (cfg.nf * cfg.nr) + 1
        xb = torch.zeros((cfg.nt, cfg.ns, nv_big), device="cuda")
        yb = torch.zeros((cfg.nt, cfg.nr, nv_big), device="cuda")
        assert L.mdc_forward_static_scratch(h, _ptr(xb), _ptr(yb), nv_big, 0, stream) == -6
    finally:
        m.mdc_destroy(h)


def test_static_scratch_tensor_core_product_allocates_nothing():
    """FP16 storage at 16 columns: after mdc_reserve (set-up time) the product runs on tensor
    cores; the static calls then leave the device's free memory unchanged and agree with
    mdc_forward bit for bit (same kernels, same operand buffers) and with the oracle on the
    dequantised kernel."""
    import paper_2011_11120_gb300 as m
    from test_gpu_precision import dequantised
    L = m.lib()
    nt, nr, ns, nf, nv = 128, 300, 260, 12, 16
    rng = np.random.default_rng(41)
    G64 = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    op = m.MDC(torch.from_numpy(G64.astype(np.complex64)).cuda(), nt, 0.004, 400.0, storage="c16f")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        m.mdc_reserve(op.h, nv)
        xs = [rng.standard_normal((nt, ns, nv)).astype(np.float32) for _ in range(2)]
        xd = [torch.from_numpy(x).cuda() for x in xs]
        ys = [torch.full((nt, nr, nv), float("nan"), device="cuda") for _ in range(2)]
        yr = [torch.empty((nt, nr, nv), device="cuda") for _ in range(2)]
        # first call: loads the kernels (lazy module loading may take device memory once)
        assert L.mdc_forward_static_scratch(op.h, _ptr(xd[0]), _ptr(ys[0]), nv, 0, stream) == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for i in range(2):
            assert L.mdc_forward_static_scratch(op.h, _ptr(xd[i]), _ptr(ys[i]), nv, 0, stream) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        for i in range(2):
            assert L.mdc_forward(op.h, _ptr(xd[i]), _ptr(yr[i]), nv, 0, stream) == 0
        torch.cuda.synchronize()
        m.mdc_device_status(op.h)
        assert m.mdc_tc_fallback_count(op.h) == 0
        Gq = dequantised(G64, "c16f")
        for i in range(2):
            assert torch.equal(ys[i], yr[i])
            assert rel(ys[i].cpu().numpy(), omdc.forward(Gq, xs[i], 0.004, 400.0)) <= 4 * U16
    finally:
        op.close()
