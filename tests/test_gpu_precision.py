"""GPU parity of the reduced-storage kernels (FP16, BF16, FP8 E4M3 with per-row scales).

Two checks per case:
* against the FP64 oracle applied to the *dequantised* kernel (the quantisation rule
  re-done on the CPU with torch's IEEE conversions): relative L2 <= 1e-5, so decoding,
  row scales and accumulation are exact up to float32 rounding;
* against the FP64 oracle on the exact kernel: relative L2 <= 4u, u the format's unit
  roundoff (2^-11 FP16, 2^-8 BF16, 2^-4 E4M3).  Independent rounding errors of relative
  RMS u/sqrt(3) give an expected error near u/sqrt(3); 4u leaves room for structure.
"""
import numpy as np
import pytest

import synth
from oracle import mdc as omdc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMATS = {"c16f": (2.0 ** -11, 32768.0, torch.float16),
           "cbf16": (2.0 ** -8, 1.0, torch.bfloat16),
           "ce4m3": (2.0 ** -4, 448.0, torch.float8_e4m3fn)}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def dequantised(G64: np.ndarray, storage: str) -> np.ndarray:
    """Per-(frequency, row) scale = rowmax / QMAX in float32, q = RNE(G * (QMAX / rowmax))."""
    _, qmax, dt = FORMATS[storage]
    G = torch.from_numpy(G64.astype(np.complex64))
    re, im = G.real.contiguous(), G.imag.contiguous()
    rowmax = torch.maximum(re.abs().amax(dim=2), im.abs().amax(dim=2))          # float32
    sc = torch.where(rowmax > 0, rowmax / qmax, torch.zeros_like(rowmax))
    inv = torch.where(rowmax > 0, torch.tensor(qmax, dtype=torch.float32) / rowmax, torch.zeros_like(rowmax))
    qr = (re * inv[..., None]).to(dt).to(torch.float64)
    qi = (im * inv[..., None]).to(dt).to(torch.float64)
    s64 = sc.to(torch.float64)[..., None]
    return (qr * s64).numpy() + 1j * (qi * s64).numpy()


CASES = [(256, 441, 441, 64, 1, "synth"), (128, 100, 77, 50, 2, "rand"), (64, 40, 90, 20, 7, "rand"),
         (512, 130, 70, 100, 4, "rand")]


@pytest.mark.parametrize("storage", list(FORMATS))
@pytest.mark.parametrize("nt,nr,ns,nf,nv,kind", CASES)
def test_reduced_storage_matches_oracle(storage, nt, nr, ns, nf, nv, kind):
    import paper_2011_11120_gb300 as m
    u = FORMATS[storage][0]
    if kind == "synth":
        cfg = synth.config(1)
        d = synth.draw(cfg)
        G = synth.kernel(cfg, d)
        x = synth.ricker_traces(cfg, d)
        dt, dr = cfg.dt, cfg.dr
    else:
        rng = np.random.default_rng(nt + nr + ns + nv)
        G = (rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))) / np.sqrt(ns)
        x = rng.standard_normal((nt, ns, nv)).astype(np.float32)
        dt, dr = 0.004, 400.0
    y = np.random.default_rng(5).standard_normal((nt, nr, nv)).astype(np.float32)
    op = m.MDC(torch.from_numpy(G.astype(np.complex64)).cuda(), nt, dt, dr, storage=storage)
    yg = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xg = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    op.close()
    Gq = dequantised(G, storage)
    assert rel(yg, omdc.forward(Gq, x, dt, dr)) <= 1e-5
    assert rel(xg, omdc.adjoint(Gq, y, dt, dr)) <= 1e-5
    ef = rel(yg, omdc.forward(G, x, dt, dr))
    ea = rel(xg, omdc.adjoint(G, y, dt, dr))
    print(f"{storage} {kind} nt={nt} nr={nr} ns={ns} nv={nv}: forward {ef:.2e} adjoint {ea:.2e} (4u = {4*u:.2e})")
    assert ef <= 4 * u and ea <= 4 * u


def test_kernel_bytes_by_storage():
    import paper_2011_11120_gb300 as m
    n64 = m.mdc_kernel_bytes(200, 3721, 3721, "c64")
    assert m.mdc_kernel_bytes(200, 3721, 3721, "c16f") == n64 // 2 + 200 * 3721 * 4
    assert m.mdc_kernel_bytes(200, 3721, 3721, "ce4m3") == n64 // 4 + 200 * 3721 * 4
