"""The bounds-checked build (MDC_CHECK_BOUNDS): ragged shapes through every instrumented kernel family.

`python -m paper_2011_11120_gb300.build --debug` compiles the library with device-side index checks:
each instrumented global access of the FFT, GEMV, SIMT-GEMM and tensor-core kernels (and of the
tensor-core operand preparation) compares its index with its buffer's extent; a miss is recorded in
the handle's error flag and the access is skipped, so `mdc_device_status` would raise MDC_ERR_BOUNDS
(-8).  A child process loads that library (MDC_LIB_DEBUG=1) and runs shapes chosen to leave partial
tiles everywhere: odd trace counts and column counts, nr != ns, nt from 64 to 4096 (four-step,
half-length and radix-2 transforms, fused and separate forward transforms), the complex64 GEMV
(whole-row and chunked), the SIMT GEMM (wide and narrow tiles), FP16 tensor cores and the swapped E4M3
kernel, a Marchenko solve and an MDD solve.  Every call must report no miss and match the FP64 oracle.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import paper_2011_11120_gb300 as m
import synth
from oracle import mdc as omdc, marchenko as omar, mdd as omdd, solvers
from test_gpu_precision import dequantised
assert m.LIB_PATH.endswith("libmdc_gb300_debug.so"), m.LIB_PATH

def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))

out = {}
rng = np.random.default_rng(5)
U16 = 2.0 ** -11
# (storage, nt, nr, ns, nf, nv, tolerance vs the oracle on the stored kernel)
cases = [("c64", 64, 37, 29, 20, 1, 1e-5), ("c64", 256, 45, 61, 40, 3, 1e-5),
         ("c64", 512, 33, 27, 100, 20, 1e-5), ("c64", 128, 70, 130, 30, 40, 1e-5),
         ("c64", 2048, 21, 19, 150, 2, 1e-5), ("c64", 4096, 9, 11, 60, 1, 1e-5),
         ("c64", 256, 16, 6200, 4, 1, 1e-5),
         ("c16f", 128, 130, 70, 5, 16, 4 * U16), ("c16f", 64, 257, 129, 3, 40, 4 * U16),
         ("ce4m3", 64, 300, 70, 5, 8, 2.0 ** -10)]
for st, nt, nr, ns, nf, nv, tol in cases:
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 400.0, storage=st)
    if st != "c64":
        m.mdc_reserve(op.h, nv)
    yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    m.mdc_device_status(op.h)
    op.close()
    Gq = G if st == "c64" else dequantised(G, st)
    key = f"{st}-nt{nt}-{nr}x{ns}-nf{nf}-nv{nv}"
    out[key] = [rel(yg, omdc.forward(Gq, x, 0.004, 400.0)), rel(xg, omdc.adjoint(Gq, y, 0.004, 400.0)), tol]

# Marchenko LSQR (fused forward transforms, window, time reversal) at nt = 512 and 2048
for n_side, nt, nf, nvg, z, niter in ((5, 512, 100, 2, 400.0, 5), (3, 2048, 200, 1, 600.0, 3)):
    cfg = synth.Config(95, "redatum-test", n_side, nt, 0.004, nf, 5, nvg * nvg, z, point_grid=nvg)
    d = synth.draw(cfg)
    G = synth.kernel(cfg, d)
    G *= 0.5 / (cfg.dt * cfg.dr * max(np.linalg.norm(G[k], 2) for k in range(cfg.nf)))
    cut = synth.window_cutoffs(cfg, d)
    fd = synth.direct_focusing(cfg, d)
    mo = omar.Marchenko(G, cfg.dt, cfg.dr, cut, cfg.nt)
    res = solvers.lsqr(mo.matvec, mo.rmatvec, mo.data(fd), niter=niter)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), cfg.nt, cfg.dt, cfg.dr)
    r = op.marchenko(torch.from_numpy(cut).cuda(), torch.from_numpy(fd).cuda(), niter)
    m.mdc_device_status(op.h)
    op.close()
    out[f"marchenko-nt{nt}"] = [rel(r["f_minus"].cpu().numpy(), res.x[0]), rel(r["f_mplus"].cpu().numpy(), res.x[1]),
                                1e-5]

# MDD (fused forward transforms on a rectangular kernel, conditioned as in the MDD parity tests)
from test_gpu_mdd import problem as mdd_problem
nt = 128
G, g = mdd_problem(nt, 40, 50, 21, 6, seed=9)
ref = omdd.MDD(G, 0.004, 400.0).solve(g, 8)
op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, 0.004, 400.0)
rr = op.mdd(torch.from_numpy(g).cuda(), 8)
m.mdc_device_status(op.h)
op.close()
out["mdd"] = [rel(rr["r"].cpu().numpy(), ref.x), 0.0, 1e-5]
json.dump(out, open(sys.argv[2], "w"))
"""


def test_bounds_checked_build_reports_no_miss_and_matches_oracle(tmp_path):
    from paper_2011_11120_gb300 import build as b
    b.build_debug()
    f = str(tmp_path / "bounds.json")
    env = dict(os.environ, MDC_LIB_DEBUG="1")
    res = subprocess.run([sys.executable, "-c", _CHILD, ROOT, f], env=env, capture_output=True, text=True,
                         timeout=1200)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    out = json.load(open(f))
    for key, (ef, ea, tol) in out.items():
        print(f"bounds-checked {key}: {ef:.2e} {ea:.2e}")
        assert ef <= tol and ea <= tol, (key, ef, ea, tol)
