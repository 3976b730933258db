"""Compute and store the kernel scale of the redatuming configuration.

The Marchenko workload scales its hyperbolic-event kernel so that the MDC
operator R has 2-norm 0.5; the block operator of Eq. 5 then has singular
values in [0.5, 1.5].  R is block-diagonal over frequency (Eq. 4), so its
2-norm is dt*dr times the largest singular value over the kernel's frequency
slices; each slice's largest singular value is found by power iteration on
G(w)^H G(w) in float64.  The resulting constant is written to
``synth/manifest.json`` and from then on is an input like the drawn event
parameters.

    python synth/normalise_kernel.py [config-number ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synth  # noqa: E402


def sigma_max(Gk: np.ndarray, iters: int = 40, seed: int = 0) -> float:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(Gk.shape[1]) + 1j * rng.standard_normal(Gk.shape[1])
    v /= np.linalg.norm(v)
    s = 0.0
    for _ in range(iters):
        w = Gk.conj().T @ (Gk @ v)
        s = np.linalg.norm(w)
        if s == 0.0:
            return 0.0
        v = w / s
    return float(np.sqrt(s))


def kernel_slice(cfg, d, k, chunk=1024):
    """One frequency slice G[k] in complex128, generated in row chunks to bound memory."""
    out = np.empty((cfg.nr, cfg.ns), dtype=np.complex128)
    for r0 in range(0, cfg.nr, chunk):
        rows = np.arange(r0, min(cfg.nr, r0 + chunk))
        out[rows] = synth.kernel(cfg, d, ks=[k], rows=rows)[0]
    return out


def frequencies(cfg):
    """Frequencies searched for the largest singular value: every one for small kernels; for
    kernels above 4096 traces, every third bin from 0.3 to 1.3 times the Ricker peak."""
    if cfg.nr <= 4096:
        return list(range(cfg.nf))
    kp = synth.RICKER_FP * cfg.nt * cfg.dt
    return list(range(int(0.3 * kp), min(cfg.nf, int(1.3 * kp) + 1), 3))


def main(numbers):
    man = {}
    path = os.path.join(HERE, "manifest.json")
    if os.path.exists(path):
        with open(path) as fh:
            man = json.load(fh)
    for num in numbers:
        cfg = synth.config(num).with_(normalise=False)
        d = synth.draw(cfg)
        t0 = time.time()
        sig = []
        ks = frequencies(cfg)
        for k in ks:
            Gk = kernel_slice(cfg, d, k)
            sig.append(sigma_max(Gk))
            print(f"  k={k} sigma={sig[-1]:.4f} ({time.time() - t0:.0f} s)", flush=True)
        smax = max(sig)
        scale = 0.5 / (cfg.dt * cfg.dr * smax)
        key = synth._scale_key(synth.config(num))
        man[key] = {"scale": scale, "sigma_max_unscaled": smax, "k_at_max": int(ks[int(np.argmax(sig))]),
                    "frequencies_searched": [int(k) for k in ks],
                    "target_norm": 0.5, "seconds": round(time.time() - t0, 1)}
        print(key, man[key], flush=True)
    with open(path, "w") as fh:
        json.dump(man, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [4])
