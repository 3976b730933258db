"""GB300 multi-dimensional convolution (MDC) and Marchenko-LSQR redatuming.

Thin ctypes binding over the C ABI of ``include/mdc.h`` (``libmdc_gb300.so``).
Functions keep the ABI's names and only marshal arguments: torch CUDA tensors
become device pointers, the current torch stream becomes the ``stream``
argument.  Every operation runs in the library's CUDA kernels; if the library
is missing this module raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# MDC_LIB_DEBUG=1: the bounds-checked build (python -m paper_2011_11120_gb300.build --debug)
LIB_PATH = os.path.join(_HERE, "libmdc_gb300_debug.so" if os.environ.get("MDC_LIB_DEBUG") == "1"
                        else "libmdc_gb300.so")

MDC_OK = 0
MDC_C64, MDC_C16F, MDC_CBF16, MDC_CE4M3, MDC_C32S = 0, 1, 2, 3, 4
STORAGE = {"c64": MDC_C64, "c16f": MDC_C16F, "cbf16": MDC_CBF16, "ce4m3": MDC_CE4M3, "c32s": MDC_C32S}
MDC_CONJ_KERNEL = 0x1
MDC_OPT_GRAPHS, MDC_OPT_WAIT_LIMIT_US = 1, 2
KC_RFFT, KC_PRODUCT_FWD, KC_PRODUCT_ADJ, KC_IRFFT, KC_SOLVER, KC_TC_PREP = range(6)
KERNEL_CLASSES = {"rfft": KC_RFFT, "product_fwd": KC_PRODUCT_FWD, "product_adj": KC_PRODUCT_ADJ,
                  "irfft": KC_IRFFT, "solver": KC_SOLVER, "tc_prep": KC_TC_PREP}

# exported symbol -> (restype, argtypes)
_vp, _i, _d, _u, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_int64
# mdc_allreduce_fn: int (*)(float* buf, int64_t count, void* stream, void* ctx)
MDC_ALLREDUCE_FN = ctypes.CFUNCTYPE(_i, _vp, _i64, _vp, _vp)
SIGNATURES = {
    "mdc_create": (_i, [ctypes.POINTER(_vp), _vp, _i, _i, _i, _i, _d, _d, _i, _vp]),
    "mdc_create_weighted": (_i, [ctypes.POINTER(_vp), _vp, ctypes.POINTER(_d), _i, _i, _i, _i, _d, _d, _i, _vp]),
    "mdc_create_empty": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _d, _d, _i, _vp]),
    "mdc_load_slab": (_i, [_vp, _vp, _i, _i, _vp]),
    "mdc_create_shard": (_i, [ctypes.POINTER(_vp), _vp, _i, _i, _i, _i, _i, _d, _d, _i, _vp]),
    "mdc_set_allreduce": (_i, [_vp, MDC_ALLREDUCE_FN, _vp]),
    "mdc_forward": (_i, [_vp, _vp, _vp, _i, _u, _vp]),
    "mdc_adjoint": (_i, [_vp, _vp, _vp, _i, _u, _vp]),
    "mdc_reserve": (_i, [_vp, _i]),
    "mdc_forward_static_scratch": (_i, [_vp, _vp, _vp, _i, _u, _vp]),
    "marchenko_lsqr": (_i, [_vp, _vp, _vp, _i, _i, _d, _vp, _vp, _vp, _vp,
                            ctypes.POINTER(_d), ctypes.POINTER(_i), _vp]),
    "marchenko_lsqr_refined": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _d, _vp, _vp, _vp, _vp,
                                    ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_i), _vp]),
    "marchenko_neumann": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "mdd_lsqr": (_i, [_vp, _vp, _i, _i, _d, _vp, ctypes.POINTER(_d), ctypes.POINTER(_i), _vp]),
    "mdc_destroy": (_i, [_vp]),
    "mdc_strerror": (ctypes.c_char_p, [_i]),
    "mdc_last_cuda_error": (_i, []),
    "mdc_kernel_bytes": (_i64, [_i, _i, _i, _i]),
    "mdc_timing": (_i, [_vp, _i]),
    "mdc_timing_read": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_i64)]),
    "mdc_launch_count": (_i64, [_vp]),
    "mdc_device_status": (_i, [_vp, _vp]),
    "mdc_set_option": (_i, [_vp, _i, _i]),
    "mdc_tc_fallback_count": (_i64, [_vp]),
    "mdc_autotune": (_i, [_vp, _i, _vp]),
    "mdc_autotune_choice": (_i, [_vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "srv_create": (_i, [ctypes.POINTER(_vp), _vp, _vp, _i64, _i, _i, _i, _vp]),
    "srv_submit": (_i, [_vp, _vp, _vp, _i, _i, _i, _d, _vp, _vp, _vp, _vp, ctypes.POINTER(_i64)]),
    "srv_step": (_i, [_vp, ctypes.POINTER(_i)]),
    "srv_poll": (_i, [_vp, _i64, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_d),
                      ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "srv_result": (_i, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "srv_keep_results": (_i, [_vp, _i]),
    "srv_release": (_i, [_vp, _i64]),
    "srv_stats": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i64), ctypes.POINTER(_i)]),
    "srv_checkpoint": (_i, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "srv_resume": (_i, [_vp, _vp, _i64, ctypes.POINTER(_i64), _i, ctypes.POINTER(_i)]),
    "srv_bind": (_i, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "srv_destroy": (_i, [_vp]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2011_11120_gb300.build` (the MDC path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class MDCError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().mdc_strerror(status).decode()
        if status == -3:
            msg += f" (cudaError {lib().mdc_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{status}]")
        self.status = status


def _check(status: int, where: str) -> None:
    if status != MDC_OK:
        raise MDCError(status, where)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: Optional[torch.Tensor], dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ ABI-named calls
def mdc_create(G: torch.Tensor, nt: int, dt: float, dr: float, storage="c64", stream=None,
               weights=None) -> ctypes.c_void_p:
    """Build an MDC handle from a complex64 CUDA tensor G[nfmax, nr, ns] (copied).  ``weights``
    (length ns, e.g. Voronoi cell areas) multiplies the kernel's columns (mdc_create_weighted)."""
    if G.dtype != torch.complex64 or G.dim() != 3:
        raise ValueError("G must be complex64 [nfmax, nr, ns]")
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    h = ctypes.c_void_p()
    nf, nr, ns = G.shape
    if weights is None:
        _check(lib().mdc_create(ctypes.byref(h), _ptr(G, name="G"), nf, nr, ns, nt, dt, dr, st, _stream(stream)),
               "mdc_create")
    else:
        w = np.ascontiguousarray(np.asarray(weights, np.float64).reshape(-1))
        if w.shape[0] != ns:
            raise ValueError("weights needs one value per kernel column")
        _check(lib().mdc_create_weighted(ctypes.byref(h), _ptr(G, name="G"),
                                         w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nf, nr, ns, nt, dt, dr,
                                         st, _stream(stream)), "mdc_create_weighted")
    return h


def mdc_create_empty(nfmax: int, nr: int, ns: int, nt: int, dt: float, dr: float, storage="c64",
                     stream=None) -> ctypes.c_void_p:
    """An MDC handle whose kernel copy is zero until filled by ``mdc_load_slab``."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    h = ctypes.c_void_p()
    _check(lib().mdc_create_empty(ctypes.byref(h), nfmax, nr, ns, nt, dt, dr, st, _stream(stream)),
           "mdc_create_empty")
    return h


def mdc_load_slab(h, G_slab: torch.Tensor, k0: int, stream=None) -> None:
    """Load kernel frequencies k0 .. k0+nk-1 from a complex64 CUDA tensor G_slab[nk, nr, ns]."""
    if G_slab.dtype != torch.complex64 or G_slab.dim() != 3:
        raise ValueError("G_slab must be complex64 [nk, nr, ns]")
    _check(lib().mdc_load_slab(h, _ptr(G_slab, name="G_slab"), k0, G_slab.shape[0], _stream(stream)),
           "mdc_load_slab")


def mdc_forward(h, x: torch.Tensor, y: torch.Tensor, nv: int, flags: int = 0, stream=None) -> None:
    _check(lib().mdc_forward(h, _ptr(x, torch.float32, "x"), _ptr(y, torch.float32, "y"), nv, flags,
                             _stream(stream)), "mdc_forward")


def mdc_adjoint(h, y: torch.Tensor, x: torch.Tensor, nv: int, flags: int = 0, stream=None) -> None:
    _check(lib().mdc_adjoint(h, _ptr(y, torch.float32, "y"), _ptr(x, torch.float32, "x"), nv, flags,
                             _stream(stream)), "mdc_adjoint")


def mdc_forward_static_scratch(h, x: torch.Tensor, y: torch.Tensor, nv: int, flags: int = 0,
                               stream=None) -> None:
    """mdc_forward without any device allocation (fixed 32 MiB library work array)."""
    _check(lib().mdc_forward_static_scratch(h, _ptr(x, torch.float32, "x"), _ptr(y, torch.float32, "y"), nv,
                                            flags, _stream(stream)), "mdc_forward_static_scratch")


def mdc_reserve(h, nv_max: int) -> None:
    _check(lib().mdc_reserve(h, nv_max), "mdc_reserve")


def marchenko_lsqr(h, window: torch.Tensor, fd_plus: torch.Tensor, nv: int, niter: int, tol: float,
                   f_minus: torch.Tensor, f_mplus: torch.Tensor, g_minus=None, g_plus=None, stream=None):
    """Solve Eq. 5 by LSQR and evaluate Eq. 6; returns (resid list, iterations done)."""
    resid = (ctypes.c_double * (niter + 1))()
    it = ctypes.c_int(0)
    st = lib().marchenko_lsqr(h, _ptr(window, torch.int32, "window"), _ptr(fd_plus, torch.float32, "fd_plus"),
                              nv, niter, tol, _ptr(f_minus, torch.float32, "f_minus"),
                              _ptr(f_mplus, torch.float32, "f_mplus"), _ptr(g_minus, torch.float32, "g_minus"),
                              _ptr(g_plus, torch.float32, "g_plus"), resid, ctypes.byref(it), _stream(stream))
    _check(st, "marchenko_lsqr")
    return [resid[i] for i in range(niter + 1)], it.value


def marchenko_neumann(h, window: torch.Tensor, fd_plus: torch.Tensor, nv: int, niter: int,
                      f_minus: torch.Tensor, f_mplus: torch.Tensor, g_minus=None, g_plus=None, stream=None):
    """Eq. 5 by its Neumann series (niter terms; 0 gives the single-scattering Green's functions)."""
    st = lib().marchenko_neumann(h, _ptr(window, torch.int32, "window"), _ptr(fd_plus, torch.float32, "fd_plus"),
                                 nv, niter, _ptr(f_minus, torch.float32, "f_minus"),
                                 _ptr(f_mplus, torch.float32, "f_mplus"), _ptr(g_minus, torch.float32, "g_minus"),
                                 _ptr(g_plus, torch.float32, "g_plus"), _stream(stream))
    _check(st, "marchenko_neumann")


def mdd_lsqr(h, g_minus: torch.Tensor, nv: int, niter: int, tol: float, r: torch.Tensor, stream=None):
    """Eq. 8 by LSQR: r [nt][ns][nv] from g_minus [nt][nr][nv]; returns (resid list, iterations)."""
    resid = (ctypes.c_double * (niter + 1))()
    it = ctypes.c_int(0)
    st = lib().mdd_lsqr(h, _ptr(g_minus, torch.float32, "g_minus"), nv, niter, tol, _ptr(r, torch.float32, "r"),
                        resid, ctypes.byref(it), _stream(stream))
    _check(st, "mdd_lsqr")
    return [resid[i] for i in range(niter + 1)], it.value


def marchenko_lsqr_refined(h, h_ref, window: torch.Tensor, fd_plus: torch.Tensor, nv: int, niter: int,
                           nrefine: int, niter_refine: int, tol: float, f_minus: torch.Tensor,
                           f_mplus: torch.Tensor, g_minus=None, g_plus=None, stream=None):
    """Reduced-precision LSQR with float32 refinement; returns (resid list, final residual, iterations)."""
    nres = (niter + 1) + nrefine * (niter_refine + 1)
    resid = (ctypes.c_double * nres)()
    fin = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    st = lib().marchenko_lsqr_refined(h, h_ref, _ptr(window, torch.int32, "window"),
                                      _ptr(fd_plus, torch.float32, "fd_plus"), nv, niter, nrefine, niter_refine,
                                      tol, _ptr(f_minus, torch.float32, "f_minus"),
                                      _ptr(f_mplus, torch.float32, "f_mplus"),
                                      _ptr(g_minus, torch.float32, "g_minus"), _ptr(g_plus, torch.float32, "g_plus"),
                                      resid, ctypes.byref(fin), ctypes.byref(it), _stream(stream))
    _check(st, "marchenko_lsqr_refined")
    return [resid[i] for i in range(nres)], fin.value, it.value


def mdc_destroy(h) -> None:
    _check(lib().mdc_destroy(h), "mdc_destroy")


def mdc_kernel_bytes(nfmax: int, nr: int, ns: int, storage="c64") -> int:
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    return int(lib().mdc_kernel_bytes(nfmax, nr, ns, st))


def mdc_timing(h, enable: bool) -> None:
    _check(lib().mdc_timing(h, 1 if enable else 0), "mdc_timing")


def mdc_timing_read(h, kernel_class) -> tuple:
    cls = KERNEL_CLASSES[kernel_class] if isinstance(kernel_class, str) else int(kernel_class)
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(lib().mdc_timing_read(h, cls, ctypes.byref(ms), ctypes.byref(n)), "mdc_timing_read")
    return ms.value, n.value


def mdc_launch_count(h) -> int:
    return int(lib().mdc_launch_count(h))


MDC_OPT_GRAPHS = 1
PATHS = {0: "default", 1: "gemv", 2: "simt", 3: "tensor-core", 4: "gemv-groups"}


def mdc_autotune(h, ncol_max: int, stream=None) -> None:
    _check(lib().mdc_autotune(h, ncol_max, _stream(stream)), "mdc_autotune")


def mdc_autotune_choice(h, adjoint: bool, ncol: int) -> tuple:
    pa, bn = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().mdc_autotune_choice(h, 1 if adjoint else 0, ncol, ctypes.byref(pa), ctypes.byref(bn)),
           "mdc_autotune_choice")
    return PATHS[pa.value], bn.value


def mdc_set_option(h, option: int, value: int) -> None:
    _check(lib().mdc_set_option(h, option, value), "mdc_set_option")


def mdc_tc_fallback_count(h) -> int:
    """Products the tensor-core rule chose that ran on the SIMT/GEMV path (operands not reserved)."""
    return int(lib().mdc_tc_fallback_count(h))


def mdc_device_status(h, stream=None) -> None:
    """Raise MDCError(MDC_ERR_TIMEOUT) if a bounded device wait of this handle gave up (and, in the
    bounds-checked build, MDCError(MDC_ERR_BOUNDS) if a kernel index fell outside its buffer)."""
    _check(lib().mdc_device_status(h, _stream(stream)), "mdc_device_status")


# ------------------------------------------------------------------ convenience wrapper
class MDC:
    """Owning wrapper: ``MDC(G, nt, dt, dr)``, ``.forward(x)``, ``.adjoint(y)``, ``.marchenko(...)``."""

    def __init__(self, G: torch.Tensor, nt: int, dt: float, dr: float, storage="c64", stream=None, weights=None):
        self.nf, self.nr, self.ns = G.shape
        self.nt, self.dt, self.dr = nt, dt, dr
        self.h = mdc_create(G, nt, dt, dr, storage, stream, weights)

    @classmethod
    def empty(cls, nfmax: int, nr: int, ns: int, nt: int, dt: float, dr: float, storage="c64", stream=None):
        """An operator with a zero kernel, to be filled frequency slab by slab with ``load_slab``."""
        op = cls.__new__(cls)
        op.nf, op.nr, op.ns = nfmax, nr, ns
        op.nt, op.dt, op.dr = nt, dt, dr
        op.h = mdc_create_empty(nfmax, nr, ns, nt, dt, dr, storage, stream)
        return op

    def load_slab(self, G_slab: torch.Tensor, k0: int, stream=None) -> None:
        mdc_load_slab(self.h, G_slab, k0, stream)

    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, conj=False, stream=None):
        nv = x.shape[2]
        if out is None:
            out = torch.empty((self.nt, self.nr, nv), dtype=torch.float32, device=x.device)
        mdc_forward(self.h, x, out, nv, MDC_CONJ_KERNEL if conj else 0, stream)
        return out

    def adjoint(self, y: torch.Tensor, out: Optional[torch.Tensor] = None, conj=False, stream=None):
        nv = y.shape[2]
        if out is None:
            out = torch.empty((self.nt, self.ns, nv), dtype=torch.float32, device=y.device)
        mdc_adjoint(self.h, y, out, nv, MDC_CONJ_KERNEL if conj else 0, stream)
        return out

    def marchenko(self, window: torch.Tensor, fd_plus: torch.Tensor, niter: int, tol: float = 0.0,
                  greens: bool = True, stream=None):
        nv = fd_plus.shape[2]
        mk = lambda: torch.empty_like(fd_plus)  # noqa: E731
        fm, fmp = mk(), mk()
        gm, gp = (mk(), mk()) if greens else (None, None)
        resid, iters = marchenko_lsqr(self.h, window, fd_plus, nv, niter, tol, fm, fmp, gm, gp, stream)
        return {"f_minus": fm, "f_mplus": fmp, "g_minus": gm, "g_plus": gp, "resid": resid, "iters": iters}

    def mdd(self, g_minus: torch.Tensor, niter: int, tol: float = 0.0, stream=None):
        """Local reflectivity r solving g- = G+ r (this handle's kernel is G+), Eq. 8."""
        nt, _, nv = g_minus.shape
        r = torch.empty((nt, self.ns, nv), dtype=torch.float32, device=g_minus.device)
        resid, iters = mdd_lsqr(self.h, g_minus, nv, niter, tol, r, stream)
        return {"r": r, "resid": resid, "iters": iters}

    def neumann(self, window: torch.Tensor, fd_plus: torch.Tensor, niter: int, greens: bool = True, stream=None):
        nv = fd_plus.shape[2]
        mk = lambda: torch.empty_like(fd_plus)  # noqa: E731
        fm, fmp = mk(), mk()
        gm, gp = (mk(), mk()) if greens else (None, None)
        marchenko_neumann(self.h, window, fd_plus, nv, niter, fm, fmp, gm, gp, stream)
        return {"f_minus": fm, "f_mplus": fmp, "g_minus": gm, "g_plus": gp}

    def marchenko_refined(self, ref: "MDC", window: torch.Tensor, fd_plus: torch.Tensor, niter: int,
                          nrefine: int = 1, niter_refine: int = 10, tol: float = 0.0, greens: bool = True,
                          stream=None):
        """Solve with this (reduced-precision) handle, refining against ``ref`` (complex64)."""
        nv = fd_plus.shape[2]
        mk = lambda: torch.empty_like(fd_plus)  # noqa: E731
        fm, fmp = mk(), mk()
        gm, gp = (mk(), mk()) if greens else (None, None)
        resid, fin, iters = marchenko_lsqr_refined(self.h, ref.h, window, fd_plus, nv, niter, nrefine,
                                                   niter_refine, tol, fm, fmp, gm, gp, stream)
        return {"f_minus": fm, "f_mplus": fmp, "g_minus": gm, "g_plus": gp, "resid": resid,
                "final_residual": fin, "iters": iters}

    def close(self):
        if self.h is not None:
            mdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ frequency shards
def shard_bounds(nf: int, world: int, rank: int) -> tuple:
    """Bins (k0, nk) of shard ``rank`` when nf kernel frequencies are split into ``world``
    contiguous bands of near-equal size (the first nf % world bands one bin longer)."""
    if world < 1 or not 0 <= rank < world or nf < world:
        raise ValueError("need 0 <= rank < world <= nf")
    base, extra = divmod(nf, world)
    k0 = rank * base + min(rank, extra)
    return k0, base + (1 if rank < extra else 0)


def mdc_create_shard(G_shard: Optional[torch.Tensor], k0: int, nk: int, nr: int, ns: int, nt: int, dt: float,
                     dr: float, storage="c64", stream=None) -> ctypes.c_void_p:
    """A handle for kernel bins k0 .. k0+nk-1 (G_shard complex64 [nk, nr, ns], or None for a zero
    kernel filled with ``mdc_load_slab``)."""
    if G_shard is not None and (G_shard.dtype != torch.complex64 or tuple(G_shard.shape) != (nk, nr, ns)):
        raise ValueError("G_shard must be complex64 [nk, nr, ns]")
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    h = ctypes.c_void_p()
    _check(lib().mdc_create_shard(ctypes.byref(h), _ptr(G_shard, name="G_shard"), k0, nk, nr, ns, nt, dt, dr, st,
                                  _stream(stream)), "mdc_create_shard")
    return h


def mdc_set_allreduce(h, fn, ctx=None) -> None:
    """Register an MDC_ALLREDUCE_FN (keep a reference to it while the handle lives), or None."""
    _check(lib().mdc_set_allreduce(h, fn if fn is not None else MDC_ALLREDUCE_FN(), ctx), "mdc_set_allreduce")


class _DeviceFloats:
    """A float32 device array owned by the library, seen by torch without a copy."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 2,
                                         "strides": None}


class ShardedMDC(MDC):
    """This process's frequency shard of an MDC operator; the partial inverse transforms are
    summed over a ``torch.distributed`` group (NCCL on device buffers, or any CPU backend such as
    gloo through host copies), once per pass.  Every process of the group holds the complete
    results, and solves (``marchenko``, ``neumann``, ``mdd``, ``marchenko_refined``) run in lock
    step on every process with identical arguments.

    ``G_shard`` is the kernel's bins ``k0 .. k0+nk-1`` (complex64 [nk, nr, ns]), or None with
    ``shape=(nk, nr, ns)`` for a zero kernel filled with ``load_slab``."""

    def __init__(self, G_shard: Optional[torch.Tensor], k0: int, nt: int, dt: float, dr: float, storage="c64",
                 group=None, shape=None, stream=None):
        import torch.distributed as dist
        nk, nr, ns = tuple(G_shard.shape) if G_shard is not None else tuple(shape)
        self.nf, self.nr, self.ns, self.k0 = nk, nr, ns, k0
        self.nt, self.dt, self.dr = nt, dt, dr
        self.group = group
        self._dist = dist
        self._nccl = dist.get_backend(group) == "nccl"
        self.h = mdc_create_shard(G_shard, k0, nk, nr, ns, nt, dt, dr, storage, stream)
        self._fn = MDC_ALLREDUCE_FN(self._allreduce)
        mdc_set_allreduce(self.h, self._fn)

    def _allreduce(self, buf, count, stream, ctx):
        try:
            t = torch.as_tensor(_DeviceFloats(int(buf), int(count)), device="cuda")
            st = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                if self._nccl:
                    self._dist.all_reduce(t, group=self.group)
                else:
                    host = t.cpu()                   # ordered after the partial transform
                    self._dist.all_reduce(host, group=self.group)
                    t.copy_(host)
            return MDC_OK
        except Exception:                             # noqa: BLE001 -- no exception crosses the C ABI
            return -7


# ------------------------------------------------------------------ serving
import numpy as np  # noqa: E402

JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


def _hptr(a):
    """Host pointer of a contiguous numpy array (or None)."""
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def srv_create(h, h_ref, hbm_budget_bytes: int, max_cols: int, nrefine: int = 0, niter_refine: int = 0,
               stream=None):
    v = ctypes.c_void_p()
    _check(lib().srv_create(ctypes.byref(v), h, h_ref, int(hbm_budget_bytes), max_cols, nrefine, niter_refine,
                            _stream(stream)), "srv_create")
    return v


def srv_submit(v, window, fd_plus, nv: int, niter: int, tol: float = 0.0, outputs=(None, None, None, None)) -> int:
    """Queue a job from host numpy arrays: int32 window [ns][ld], float32 fd_plus [nt][ns][ld]
    (first nv columns used).  The arrays are read at admission: keep them alive and unchanged
    until the job completes."""
    if window.dtype != np.int32 or fd_plus.dtype != np.float32:
        raise ValueError("window must be int32 and fd_plus float32")
    ld = window.shape[-1]
    if fd_plus.shape[-1] != ld or nv > ld:
        raise ValueError("window and fd_plus need the same last dimension >= nv")
    jid = ctypes.c_int64(0)
    o = [_hptr(a) for a in outputs]
    _check(lib().srv_submit(v, _hptr(window), _hptr(fd_plus), nv, ld, niter, tol, o[0], o[1], o[2], o[3],
                            ctypes.byref(jid)), "srv_submit")
    return jid.value


def srv_step(v) -> int:
    n = ctypes.c_int(0)
    _check(lib().srv_step(v, ctypes.byref(n)), "srv_step")
    return n.value


def srv_poll(v, job_id: int) -> dict:
    st, it = ctypes.c_int(0), ctypes.c_int(0)
    fr, lat, qs = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    rc = lib().srv_poll(v, job_id, ctypes.byref(st), ctypes.byref(it), ctypes.byref(fr), ctypes.byref(lat),
                        ctypes.byref(qs))
    return {"state": st.value, "iters": it.value, "final_residual": fr.value, "latency_s": lat.value,
            "queue_s": qs.value, "status": rc}


def srv_keep_results(v, keep: bool = True) -> None:
    _check(lib().srv_keep_results(v, 1 if keep else 0), "srv_keep_results")


def srv_result(v, job_id: int, outputs=(None, None, None, None)) -> None:
    """Copy a completed job's f-, f_m+, g-, g+ (float32 [nt][ns][nv] numpy arrays, may be None)."""
    o = [_hptr(a) for a in outputs]
    _check(lib().srv_result(v, job_id, o[0], o[1], o[2], o[3]), "srv_result")


def srv_release(v, job_id: int) -> None:
    _check(lib().srv_release(v, job_id), "srv_release")


def srv_stats(v) -> dict:
    q, r, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    b = ctypes.c_int64(0)
    _check(lib().srv_stats(v, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c)), "srv_stats")
    return {"queued": q.value, "running": r.value, "bytes": b.value, "cols": c.value}


def srv_checkpoint(v) -> bytearray:
    """Serialised queued and running jobs (inputs and solver state) as a host byte array."""
    n = ctypes.c_int64(0)
    _check(lib().srv_checkpoint(v, None, 0, ctypes.byref(n)), "srv_checkpoint")
    buf = bytearray(n.value)
    cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
    _check(lib().srv_checkpoint(v, ctypes.addressof(cbuf), len(buf), ctypes.byref(n)), "srv_checkpoint")
    del cbuf
    return buf


def srv_resume(v, data) -> list:
    """Rebuild the jobs of a checkpoint on an idle server; returns their ids in checkpoint order."""
    data = bytes(data)
    n = ctypes.c_int(0)
    # job count: the tenth 32-bit field after the 8-byte tag of the header
    njobs = int(np.frombuffer(data, np.int32, count=1, offset=8 + 4 * 9)[0]) if len(data) >= 48 else 1
    cnt = min(max(1, njobs), max(1, len(data) // 72))    # a job record takes at least 72 bytes
    ids = (ctypes.c_int64 * cnt)()
    _check(lib().srv_resume(v, data, len(data), ids, cnt, ctypes.byref(n)), "srv_resume")
    return [int(ids[i]) for i in range(n.value)]


def srv_bind(v, job_id: int, outputs=(None, None, None, None)) -> None:
    """Host output buffers (f-, f_m+, g-, g+; float32 [nt][ns][nv], may be None) of a resumed job."""
    o = [_hptr(a) for a in outputs]
    _check(lib().srv_bind(v, job_id, o[0], o[1], o[2], o[3]), "srv_bind")


def srv_destroy(v) -> None:
    _check(lib().srv_destroy(v), "srv_destroy")
