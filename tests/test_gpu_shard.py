"""Frequency shards of the MDC operator on the GPU (the paper's partitioning of the kernel along
frequency, Section "Implementing the batch matrix multiplication operator", Fig. 2).

* In one process, shard handles whose bands tile the kernel's frequencies give partial outputs
  (no reduction hook) that sum to the whole operator, for every transform length family
  (four-step nt <= 1024, half-length nt = 2048, radix 2 at nt = 4096), with the Nyquist bin in
  the last band, forward, adjoint and the conjugated kernel; compared with the FP64 oracle.
* Two processes on the one GPU, each holding one band, sum their partial transforms through a
  gloo all-reduce of host copies (the reduction hook): the MDC passes, the Marchenko LSQR solve
  (vectors and LSQR scalars replicated, one sum per pass) and the Green's functions match the
  FP64 oracle on both processes.  The processes' kernels never wait on one another; only their
  host threads meet in the all-reduce.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from oracle import mdc as omdc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-5


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nt,nr,ns,nf,nv,cuts", [
    (64, 9, 7, 33, 2, [0, 1, 20, 33]),          # DC alone, Nyquist in the last band
    (512, 40, 30, 150, 3, [0, 50, 100, 150]),
    (1024, 33, 35, 513, 1, [0, 200, 513]),      # every bin, Nyquist included
    (2048, 20, 17, 301, 2, [0, 7, 301]),        # half-length transforms
    (4096, 6, 5, 2049, 1, [0, 1000, 2049]),     # radix-2 transforms, Nyquist included
])
def test_shards_sum_to_the_operator(nt, nr, ns, nf, nv, cuts):
    import paper_2011_11120_gb300 as m
    rng = np.random.default_rng(nt + nf)
    G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
    x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
    y = rng.standard_normal((nt, nr, nv)).astype(np.float32)
    Gc = G.astype(np.complex64)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    parts = {"fwd": 0.0, "adj": 0.0, "conj": 0.0}
    for k0, k1 in zip(cuts[:-1], cuts[1:]):
        h = m.mdc_create_shard(torch.from_numpy(Gc[k0:k1].copy()).cuda(), k0, k1 - k0, nr, ns, nt, 0.004, 400.0)
        try:
            yo = torch.empty((nt, nr, nv), device="cuda")
            xo = torch.empty((nt, ns, nv), device="cuda")
            yc = torch.empty((nt, nr, nv), device="cuda")
            m.mdc_forward(h, xd, yo, nv)
            m.mdc_adjoint(h, yd, xo, nv)
            m.mdc_forward(h, xd, yc, nv, m.MDC_CONJ_KERNEL)
            torch.cuda.synchronize()
            parts["fwd"] = parts["fwd"] + yo.cpu().numpy().astype(np.float64)
            parts["adj"] = parts["adj"] + xo.cpu().numpy().astype(np.float64)
            parts["conj"] = parts["conj"] + yc.cpu().numpy().astype(np.float64)
        finally:
            m.mdc_destroy(h)
    assert rel(parts["fwd"], omdc.forward(G, x, 0.004, 400.0)) <= TOL
    assert rel(parts["adj"], omdc.adjoint(G, y, 0.004, 400.0)) <= TOL
    assert rel(parts["conj"], omdc.forward_conj_kernel(G, x, 0.004, 400.0)) <= TOL


def test_shard_arguments_are_checked():
    import paper_2011_11120_gb300 as m
    G = torch.zeros((4, 3, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(m.MDCError):
        m.mdc_create_shard(G, 31, 4, 3, 3, 64, 0.004, 1.0)        # bins beyond nt/2 + 1
    h = m.mdc_create_shard(G, 5, 4, 3, 3, 64, 0.004, 1.0)
    try:
        fd = torch.zeros((64, 3, 1), device="cuda")
        out = torch.empty_like(fd)
        with pytest.raises(m.MDCError):                             # a solve needs a reduction hook
            m.marchenko_lsqr(h, torch.ones((3, 1), dtype=torch.int32, device="cuda"), fd, 1, 2, 0.0, out,
                             torch.empty_like(fd))
    finally:
        m.mdc_destroy(h)
    plain = m.mdc_create(G, 64, 0.004, 1.0)
    try:
        with pytest.raises(m.MDCError):                             # hooks belong to shards only
            m.mdc_set_allreduce(plain, m.MDC_ALLREDUCE_FN(lambda *a: 0))
    finally:
        m.mdc_destroy(plain)


_RANK_SCRIPT = r"""
import json, os, sys
import numpy as np, torch, torch.distributed as dist
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import paper_2011_11120_gb300 as m
from test_gpu_marchenko import problem, oracle_solve, rel
from oracle import mdc as omdc
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
torch.cuda.set_device(0)
cfg, G, cut, fd = problem(5, 128, 40, 2, 200.0)
k0, nk = m.shard_bounds(cfg.nf, world, rank)
op = m.ShardedMDC(torch.from_numpy(G[k0:k0 + nk].astype(np.complex64)).cuda(), k0, cfg.nt, cfg.dt, cfg.dr)
x = torch.from_numpy(fd).cuda()
err = {{}}
err["forward"] = rel(op.forward(x).cpu().numpy(), omdc.forward(G, fd, cfg.dt, cfg.dr))
err["adjoint"] = rel(op.adjoint(x).cpu().numpy(), omdc.adjoint(G, fd, cfg.dt, cfg.dr))
err["rstar"] = rel(op.forward(x, conj=True).cpu().numpy(), omdc.forward_conj_kernel(G, fd, cfg.dt, cfg.dr))
niter = 10
res, gm, gp = oracle_solve(cfg, G, cut, fd, niter)
out = op.marchenko(torch.from_numpy(cut).cuda(), x, niter)
err["iters"] = out["iters"]
err["f_minus"] = rel(out["f_minus"].cpu().numpy(), res.x[0])
err["f_mplus"] = rel(out["f_mplus"].cpu().numpy(), res.x[1])
err["g_minus"] = rel(out["g_minus"].cpu().numpy(), gm)
err["g_plus"] = rel(out["g_plus"].cpu().numpy(), gp)
err["resid"] = float(np.max(np.abs(np.asarray(out["resid"]) - np.asarray(res.resid)) / np.asarray(res.resid)))
err["digest"] = float(out["f_minus"].double().sum().item())
op.close()
dist.barrier()
json.dump(err, open({out!r} + str(rank), "w"))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_process_shards_with_gloo_sum_match_oracle(tmp_path):
    out = str(tmp_path / "rank")
    code = _RANK_SCRIPT.format(root=ROOT, out=out)
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env))
    rcs = [p.wait(timeout=600) for p in procs]
    assert rcs == [0, 0]
    errs = [json.load(open(out + str(r))) for r in range(2)]
    for e in errs:
        print("shard rank errors:", e)
        assert e["iters"] == 10
        for key in ("forward", "adjoint", "rstar", "f_minus", "f_mplus", "g_minus", "g_plus", "resid"):
            assert e[key] <= TOL, key
    assert errs[0]["digest"] == errs[1]["digest"]       # every shard holds the same solution
