"""Generate the synthetic hyperbolic-event kernel directly on the GPU.

Large kernels (tens of GB) cannot be evaluated on the host in reasonable time,
so the workload library ``libsynth_gen.so`` evaluates the same formula as
``synth.kernel`` on the device (phase reduced in float64, float32 output).
The event parameters come from ``synth.draw``; the float64 table
``scale * W(f_k)`` is computed here.  This is workload generation only.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

import synth

_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth_gen.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise RuntimeError(f"{_LIB} missing: run `python -m paper_2011_11120_gb300.build`")
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.synth_kernel_c64.restype = ctypes.c_int
        L.synth_kernel_c64.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, ctypes.c_void_p]
        L.synth_kernel_slab_c64.restype = ctypes.c_int
        L.synth_kernel_slab_c64.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp,
                                            ctypes.c_void_p]
        L.synth_kernel_rect_c64.restype = ctypes.c_int
        L.synth_kernel_rect_c64.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                            ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, ctypes.c_void_p]
        _lib = L
    return _lib


def kernel_on_device(cfg: synth.Config, d: synth.Draw = None, device="cuda", out=None) -> torch.Tensor:
    """complex64 G[nf, nr, ns] on the device, same formula and draws as ``synth.kernel``."""
    if d is None:
        d = synth.draw(cfg)
    L = _load()
    if out is None:
        out = torch.empty((cfg.nf, cfg.nr, cfg.ns), dtype=torch.complex64, device=device)
    f = cfg.freqs
    ws = np.ascontiguousarray(synth.ricker_spectrum(f) * d.scale, dtype=np.float64)
    t0 = np.ascontiguousarray(d.t0, np.float64)
    vel = np.ascontiguousarray(d.vel, np.float64)
    amp = np.ascontiguousarray(d.amp, np.float64)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.synth_kernel_c64(ctypes.c_void_p(out.data_ptr()), cfg.nf, cfg.n_side, synth.GRID_DX,
                            1.0 / (cfg.nt * cfg.dt), len(t0), dp(t0), dp(vel), dp(amp), dp(ws), stream)
    if st != 0:
        raise RuntimeError(f"synth_kernel_c64 failed ({st})")
    return out


def kernel_slab_on_device(cfg: synth.Config, k0: int, nk: int, d: synth.Draw = None, device="cuda",
                          out=None) -> torch.Tensor:
    """complex64 G[nk, nr, ns]: frequencies k0 .. k0+nk-1 of ``kernel_on_device(cfg)``, bit for bit,
    for kernels too large to generate whole (the complex64 copy is assembled slab by slab)."""
    if d is None:
        d = synth.draw(cfg)
    if k0 < 0 or nk < 1 or k0 + nk > cfg.nf:
        raise ValueError("slab outside the kernel's frequencies")
    L = _load()
    if out is None:
        out = torch.empty((nk, cfg.nr, cfg.ns), dtype=torch.complex64, device=device)
    ws = np.ascontiguousarray((synth.ricker_spectrum(cfg.freqs) * d.scale)[k0:k0 + nk], dtype=np.float64)
    t0 = np.ascontiguousarray(d.t0, np.float64)
    vel = np.ascontiguousarray(d.vel, np.float64)
    amp = np.ascontiguousarray(d.amp, np.float64)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.synth_kernel_slab_c64(ctypes.c_void_p(out.data_ptr()), k0, nk, cfg.n_side, synth.GRID_DX,
                                 1.0 / (cfg.nt * cfg.dt), len(t0), dp(t0), dp(vel), dp(amp), dp(ws), stream)
    if st != 0:
        raise RuntimeError(f"synth_kernel_slab_c64 failed ({st})")
    return out


def focusing_inputs_on_device(cfg: synth.Config, points: np.ndarray, device="cuda", margin: int = 4):
    """Window cut-offs int32 [ns][nv] and direct focusing function float32 [nt][ns][nv] for the
    given focusing points (z = cfg.z_point), evaluated on the device with the formulas of
    synth.window_cutoffs and synth.direct_focusing (float64 arithmetic, float32 output)."""
    xy = torch.from_numpy(synth.grid_xy(cfg.n_side)).to(device)
    pts = torch.from_numpy(np.asarray(points, np.float64)).to(device)
    dd = ((xy[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    td = torch.sqrt(cfg.z_point * cfg.z_point + dd) / synth.POINT_SPEED            # [ns, nv]
    cut = (torch.round(td / cfg.dt).to(torch.int64) - margin).to(torch.int32)
    tau = torch.from_numpy(synth.signed_time_index(cfg.nt).astype(np.float64) * cfg.dt).to(device)
    fd = torch.empty((cfg.nt, cfg.ns, pts.shape[0]), dtype=torch.float32, device=device)
    a2 = (np.pi * synth.RICKER_FP) ** 2
    for t0 in range(0, cfg.nt, 64):
        arg = tau[t0:t0 + 64, None, None] + td[None]
        q = a2 * arg * arg
        fd[t0:t0 + 64] = ((1.0 - 2.0 * q) * torch.exp(-q)).to(torch.float32)
    return cut, fd


def rect_kernel_on_device(cfg: synth.Config, xy_rows: np.ndarray, xy_cols: np.ndarray, d: synth.Draw = None,
                          device="cuda") -> torch.Tensor:
    """complex64 G[nf, len(xy_rows), len(xy_cols)] on the device: the formula of ``synth.kernel_between``
    (the event draws of cfg) between two point sets."""
    if d is None:
        d = synth.draw(cfg)
    L = _load()
    xr = np.ascontiguousarray(xy_rows, np.float64)
    xs = np.ascontiguousarray(xy_cols, np.float64)
    out = torch.empty((cfg.nf, len(xr), len(xs)), dtype=torch.complex64, device=device)
    ws = np.ascontiguousarray(synth.ricker_spectrum(cfg.freqs) * d.scale, dtype=np.float64)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (d.t0, d.vel, d.amp)]
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.synth_kernel_rect_c64(ctypes.c_void_p(out.data_ptr()), cfg.nf, len(xr), len(xs), dp(xr), dp(xs),
                                 1.0 / (cfg.nt * cfg.dt), len(arrs[0]), dp(arrs[0]), dp(arrs[1]), dp(arrs[2]),
                                 dp(ws), stream)
    if st != 0:
        raise RuntimeError(f"synth_kernel_rect_c64 failed ({st})")
    return out
