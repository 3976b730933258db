"""Benchmark: MDC forward + adjoint on the paper-scale synthetic workload, one JSON line.

Workload (default): nr = ns = 3721 (61 x 61 grid, 20 m), nt = 1024, dt = 4 ms,
nfmax = 200, 20 hyperbolic events, complex64 kernel (22.15 GB), nv = 1 virtual
point.  One step = y = C x followed by x' = C^H y (Eq. 3), i.e. every stage of
the MDC path: rFFT+truncate, per-frequency product (forward and adjoint), zero
pad + irFFT.  The kernel (22 GB) is far larger than L2 (129 MB), so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--nv 1] [--impl ours|reference]

Metric: algorithmic GB/s of a forward+adjoint pair, bytes = 2 x (kernel bytes
nf*nr*ns*8 + input + output trace bytes).  With N GPUs (torchrun) each rank runs
an independent replica of the same workload (the operator needs no exchange
between replicas), value = all ranks' bytes / max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "MDC fwd+adj HBM GB/s vs peak; redatum solves/s and p99 at <=1e-3 vs FP64"
UNIT = "GB/s"


BYTES_PER_COMPLEX = {"c64": 8, "c16f": 4, "cbf16": 4, "ce4m3": 2, "c32s": 8}


def algorithmic_bytes(cfg, nv, storage="c64"):
    kernel = cfg.nf * cfg.nr * cfg.ns * BYTES_PER_COMPLEX[storage]
    traces = cfg.nt * (cfg.nr + cfg.ns) * nv * 4
    return 2 * (kernel + traces), kernel


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tc_peak(sustained=False):
    """Dense bf16 tensor peak (FP16 runs at the same rate) from MEASURED_PEAKS.json: the burst figure
    for a kernel timed alone, the sustained one for a kernel timed inside a long step."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in p else "bf16_tflops"
        return float(p[key]), f"measured ({key})"
    return (1700.0 if sustained else 1900.0), "fallback"


def kernel_source_sha(kernel_file):
    """sha256 of the complex64 GEMV kernels' source text (between their begin/end markers)."""
    src = open(os.path.join(ROOT, "paper_2011_11120_gb300", "csrc", kernel_file)).read()
    a = src.index("// ---- complex64 GEMV kernels (begin)")
    b = src.index("// ---- complex64 GEMV kernels (end)")
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def profile_traffic(kernel_file):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "product_gemv_c64_3721x3721_nf200_nv1.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        prof = json.load(fh)
    if prof.get("source_sha256") != kernel_source_sha(kernel_file):
        return None
    return prof.get("dram_bytes_per_launch")


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, tag=""):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples are kept in MDC_CLOCK_LOG_DIR when it is set, else in a temporary file
        log_dir = os.environ.get("MDC_CLOCK_LOG_DIR")
        if log_dir:
            self.path = os.path.join(log_dir, f"clocks_rank{gpu_index}{tag}.csv")
        else:
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_rank{gpu_index}{tag}_", suffix=".csv")
            os.close(fd)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sms, maxs, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms),
                "power_w_median": statistics.median(pw) if pw else None}


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over the process group (all ranks get it)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(cfg, nv, min_seconds=10.0, rows=32):
    """FP64 oracle (as it stands) on a bounded sample: `rows` output rows of C x and
    `rows` output columns of C^H y, repeated until min_seconds of CPU time."""
    from oracle import mdc as omdc
    d = synth.draw(cfg)
    rng = np.random.default_rng(11)
    r_idx = np.sort(rng.choice(cfg.nr, size=rows, replace=False))
    c_idx = np.sort(rng.choice(cfg.ns, size=rows, replace=False))
    Gr = synth.kernel(cfg, d, rows=r_idx)
    Gc = synth.kernel(cfg, d, cols=c_idx)
    x = synth.ricker_traces(cfg, d)
    y = synth.random_traces(cfg, nv, seed_offset=5, nspace=cfg.nr)
    reps = 0
    t0 = time.perf_counter()
    while True:
        omdc.forward_rows(Gr, x, cfg.dt, cfg.dr)
        omdc.adjoint_cols(Gc, y, cfg.dt, cfg.dr)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    bytes_per_rep = 2 * rows * cfg.nf * cfg.ns * 8
    return {"value": bytes_per_rep * reps / el / 1e9, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{rows} output rows of C x and {rows} output columns of C^H y of the "
                      f"{cfg.nr}x{cfg.ns}x{cfg.nf} nt={cfg.nt} nv={nv} workload (full input FFTs each "
                      f"repetition), {reps} repetitions in {el:.1f} s; bytes = complex64 kernel "
                      f"bytes of the sampled rows/columns",
            "seconds": el}


def paper_style_cpu(cfg, nv, nslices=4, min_seconds=5.0):
    """The paper's CPU formulation on the host cores: NumPy complex64 matmul per frequency slice
    (forward G x and adjoint G^H y) with NumPy real FFTs of the traces, on `nslices` full
    frequency slices of the workload's shape (random complex64 values: the timing does not depend
    on them); context beside the oracle, not a target."""
    rng = np.random.default_rng(12)
    G = (rng.standard_normal((nslices, cfg.nr, cfg.ns), dtype=np.float32)
         + 1j * rng.standard_normal((nslices, cfg.nr, cfg.ns), dtype=np.float32)).astype(np.complex64)
    x = rng.standard_normal((cfg.nt, cfg.ns, nv), dtype=np.float32)
    y = rng.standard_normal((cfg.nt, cfg.nr, nv), dtype=np.float32)
    reps, t0 = 0, time.perf_counter()
    while True:
        X = np.fft.rfft(x, axis=0)[:nslices].astype(np.complex64)
        Y = np.fft.rfft(y, axis=0)[:nslices].astype(np.complex64)
        yo = np.matmul(G, X)
        xo = np.matmul(np.conj(np.swapaxes(G, 1, 2)), Y)
        np.fft.irfft(yo, n=cfg.nt, axis=0)
        np.fft.irfft(xo, n=cfg.nt, axis=0)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    bytes_per_rep = 2 * nslices * cfg.nr * cfg.ns * 8
    return {"value": bytes_per_rep * reps / el / 1e9, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "paper-style NumPy (complex64 matmul per frequency + NumPy FFT)",
            "sample": f"{nslices} of {cfg.nf} frequency slices ({cfg.nr}x{cfg.ns}, nv={nv}), forward and "
                      f"adjoint, {reps} repetitions in {el:.1f} s; bytes = complex64 kernel bytes of the slices"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cfg = synth.config(args.config, nv=args.nv)
    if args.nf:
        cfg = cfg.with_(nf=args.nf, normalise=False)   # profiling case: normalisation not needed
    from oracle import mdc as omdc
    d = synth.draw(cfg)
    rows = 8
    rng = np.random.default_rng(11)
    r_idx = np.sort(rng.choice(cfg.nr, size=rows, replace=False))
    c_idx = np.sort(rng.choice(cfg.ns, size=rows, replace=False))
    Gr = synth.kernel(cfg, d, rows=r_idx)
    Gc = synth.kernel(cfg, d, cols=c_idx)
    x = synth.ricker_traces(cfg, d)
    y = synth.random_traces(cfg, args.nv, seed_offset=5, nspace=cfg.nr)

    def step():
        omdc.forward_rows(Gr, x, cfg.dt, cfg.dr)
        omdc.adjoint_cols(Gc, y, cfg.dt, cfg.dr)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    bytes_step = 2 * rows * cfg.nf * cfg.ns * 8
    val = bytes_step * args.steps / el / 1e9
    sample = (f"{rows} output rows of C x and {rows} output columns of C^H y per step "
              f"(complex64-equivalent kernel bytes of the sample)")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_block(cfg, args.nv),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def config_block(cfg, nv, storage="c64"):
    return {"workload": f"MDC fwd+adj, nr=ns={cfg.nr} ({cfg.n_side}x{cfg.n_side}, 20 m), nt={cfg.nt}, "
                        f"dt={cfg.dt}, nfmax={cfg.nf}, {cfg.n_events} hyperbolic events, {storage} kernel "
                        f"{cfg.nf * cfg.nr * cfg.ns * BYTES_PER_COMPLEX[storage] / 1e9:.2f} GB, nv={nv}",
            "nr": cfg.nr, "ns": cfg.ns, "nt": cfg.nt, "nfmax": cfg.nf, "nv": nv, "storage": storage,
            "l2": "inputs larger than L2 (kernel streamed every pass)"}


def run_redatum(args, dev):
    """Marchenko redatuming (Eq. 5/6) at 1681 x 1681, nt=512, nfmax=150, nv=256 (16 x 16 focusing
    points), kernel normalised to ||R|| = 0.5: FP16 kernel inside LSQR with float32 refinement,
    timed per solve; the plain float32 (complex64) solve of the same job gives the comparison."""
    import torch
    import paper_2011_11120_gb300 as mdc
    from synth import gpu as sgpu
    cfg = synth.config(4)
    d = synth.draw(cfg)
    G = sgpu.kernel_on_device(cfg, d)
    lo = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=args.redatum_storage)
    ref = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=args.redatum_ref_storage)
    plain_op = ref if args.redatum_ref_storage == "c64" else mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    del G
    torch.cuda.empty_cache()
    nvp = args.redatum_nv if 0 < args.redatum_nv < cfg.nv else cfg.nv     # fewer points: profiling cases
    cut = torch.from_numpy(np.ascontiguousarray(synth.window_cutoffs(cfg, d)[:, :nvp])).to(dev)
    fd = torch.from_numpy(np.ascontiguousarray(synth.direct_focusing(cfg, d)[:, :, :nvp])).to(dev)
    niter, nref, nin = cfg.niter, 1, args.redatum_refine_iters

    def solve():
        return lo.marchenko_refined(ref, cut, fd, niter, nrefine=nref, niter_refine=nin)

    out = solve()                                      # warm-up (allocations, tensor maps)
    torch.cuda.synchronize()
    times = []
    sampler = ClockSampler(dev.index if dev.index is not None else 0, "_redatum")
    sampler.start()
    for _ in range(args.redatum_solves):
        t0 = time.perf_counter()
        out = solve()
        times.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    # device time per kernel class in one more solve (CUDA events around every launch)
    breakdown = {}
    for name, h in (("fp16_kernel", lo.h), ("reference_kernel", ref.h)):
        mdc.mdc_timing(h, True)
    solve()
    torch.cuda.synchronize()
    for name, h in (("fp16_kernel", lo.h), ("reference_kernel", ref.h)):
        breakdown[name] = {}
        for cls in ("rfft", "tc_prep", "product_fwd", "product_adj", "irfft", "solver"):
            t, n = mdc.mdc_timing_read(h, cls)
            breakdown[name][cls] = {"ms": t, "launches": n}
        mdc.mdc_timing(h, False)
    t_plain, err, plain = None, None, {"iters": None}
    if not args.redatum_skip_fp32:
        t0 = time.perf_counter()
        plain = plain_op.marchenko(cut, fd, niter)     # complex64 SIMT operator, one job, no refinement
        t_plain = time.perf_counter() - t0
        fm = out["f_minus"].double()
        err = float((fm - plain["f_minus"].double()).norm() / plain["f_minus"].double().norm())
    lo.close()
    ref.close()
    plain_op.close()
    med = statistics.median(times)
    # the tensor-core GEMM of the FP16 kernel on its own (B-operand preparation excluded), against the
    # sustained bf16 peak (it runs inside a long solve); every such product has 2 nv columns
    fb = breakdown["fp16_kernel"]
    gemm_ms = fb["product_fwd"]["ms"] + fb["product_adj"]["ms"]
    gemm_n = fb["product_fwd"]["launches"] + fb["product_adj"]["launches"]
    tc_roof = None
    if gemm_n and gemm_ms > 0:
        flops = 8.0 * cfg.nf * cfg.nr * cfg.ns * 2 * nvp
        achieved = flops / (gemm_ms / gemm_n / 1e3) / 1e12
        pk, kind = tc_peak(sustained=True)
        tc_roof = {"bound": "tensor", "kernel": f"tc_gemm_kernel (FP16, {2 * nvp} columns, forward and adjoint)",
                   "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                   "ms_per_launch": gemm_ms / gemm_n, "peak_kind": kind,
                   "operand_prep_ms_per_launch": fb["tc_prep"]["ms"] / max(fb["tc_prep"]["launches"], 1)}
    return {"workload": f"Marchenko LSQR, nr=ns={cfg.nr} (41x41, 20 m), nt={cfg.nt}, nfmax={cfg.nf}, "
                        f"nv={nvp} (of the 16x16 focusing points, z=800 m), ||R||=0.5, {niter} LSQR iterations "
                        f"on a {args.redatum_storage} kernel + {nref} float32 refinement step of {nin} iterations "
                        f"({args.redatum_ref_storage} reference kernel)",
            "solves_per_s": 1.0 / med, "ms_per_solve": 1e3 * med, "solves_timed": len(times),
            "p50_ms": 1e3 * med, "p99_ms": 1e3 * float(np.percentile(np.asarray(times), 99)),
            "max_ms": 1e3 * max(times),
            "iterations": out["iters"], "final_residual": out["final_residual"],
            "rel_l2_vs_fp32_solve": err,
            "device_ms_per_kernel_class": breakdown,
            "tc_roofline": tc_roof,
            "clocks": clocks,
            "fp32_one_job": ({"solves_per_s": 1.0 / t_plain, "ms_per_solve": 1e3 * t_plain,
                              "iterations": plain["iters"], "storage": "c64"} if t_plain else None)}


def run_mdd(args, dev):
    """Multi-dimensional deconvolution (Eq. 8): a stand-in down-going Green's function G+ between
    the 61 x 61 surface grid and a 29 x 29 lattice of focusing points (nt=1024, nfmax=200), one
    batch of 20 virtual sources per LSQR solve, with complex64 (FP32 SIMT products), split FP16
    (float32-accurate tensor-core products) and FP16 (tensor cores) kernel copies; the tensor-core
    results are compared with the complex64 one."""
    import torch
    import paper_2011_11120_gb300 as mdc
    from synth import gpu as sgpu
    cfg = synth.config(2)
    d = synth.draw(cfg)
    xs = synth.focus_lattice(29, synth.GRID_DX, 0.5 * synth.GRID_DX * (cfg.n_side - 1))
    Gp = sgpu.rect_kernel_on_device(cfg, synth.grid_xy(cfg.n_side), xs, d)
    nv, niter = 20, args.mdd_iters
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg.seed)
    g = torch.randn((cfg.nt, cfg.nr, nv), generator=gen, device=dev, dtype=torch.float32)
    out = {}
    sol = {}
    for storage in ("c64", "c32s", "c16f"):
        op = mdc.MDC(Gp, cfg.nt, cfg.dt, cfg.dr, storage=storage)
        r = op.mdd(g, niter)                               # warm-up
        torch.cuda.synchronize()
        times = []
        for _ in range(3):
            t0 = time.perf_counter()
            r = op.mdd(g, niter)
            times.append(time.perf_counter() - t0)
        op.close()
        med = statistics.median(times)
        sol[storage] = r["r"]
        n_mdc = 2 * niter + 1
        out[storage] = {"solves_per_s": 1.0 / med, "virtual_sources_per_s": nv / med, "ms_per_solve": 1e3 * med,
                        "ms_per_mdc": 1e3 * med / n_mdc, "iterations": r["iters"],
                        "kernel_gb": cfg.nf * cfg.nr * len(xs) * BYTES_PER_COMPLEX[storage] / 1e9,
                        "tflops_products": 8.0 * cfg.nf * cfg.nr * len(xs) * nv * n_mdc / med / 1e12}
    del Gp
    torch.cuda.empty_cache()
    b = sol["c64"].double()
    for storage in ("c32s", "c16f"):
        out[storage]["rel_l2_vs_c64"] = float((sol[storage].double() - b).norm() / b.norm())
    out["workload"] = (f"MDD (Eq. 8) by LSQR, G+ {cfg.nr} receivers (61x61, 20 m) x {len(xs)} focusing points "
                       f"(29x29, 20 m), nt={cfg.nt}, nfmax={cfg.nf}, {cfg.n_events} hyperbolic events, "
                       f"{nv} virtual sources per batch, {niter} iterations")
    return out


def run_precision(args, dev):
    """Precision sweep on the 8281-trace kernel (nfmax=160): forward and adjoint MDC per storage
    format at nv = 1 (GEMV, streaming the kernel), 16 and 128 (tensor cores for the FP16, BF16, split
    FP16 and E4M3 copies),
    with the relative L2 error of 8 sampled output rows (forward) and columns (adjoint) against the
    FP64 oracle at nv = 16."""
    import torch
    import paper_2011_11120_gb300 as mdc
    from oracle import mdc as omdc
    from synth import gpu as sgpu
    cfg = synth.config(3)
    d = synth.draw(cfg)
    G = sgpu.kernel_on_device(cfg, d)
    rng = np.random.default_rng(31)
    rows = np.sort(rng.choice(cfg.nr, size=8, replace=False))
    cols = np.sort(rng.choice(cfg.ns, size=8, replace=False))
    Gr = synth.kernel(cfg, d, rows=rows)
    Gc = synth.kernel(cfg, d, cols=cols)
    x16 = synth.random_traces(cfg, 16, seed_offset=7)
    y16 = synth.random_traces(cfg, 16, seed_offset=8, nspace=cfg.nr)
    ref_f = omdc.forward_rows(Gr, x16, cfg.dt, cfg.dr)
    ref_a = omdc.adjoint_cols(Gc, y16, cfg.dt, cfg.dr)
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg.seed)
    out = {"workload": f"MDC fwd+adj, nr=ns={cfg.nr} (91x91, 20 m), nt={cfg.nt}, nfmax={cfg.nf}, "
                       f"{cfg.n_events} hyperbolic events; rel L2 on 8 sampled rows/columns at nv=16 vs the FP64 oracle"}

    def timed(fn, cls, h):
        """(whole product ms, tensor-core operand preparation ms) per call"""
        fn()
        torch.cuda.synchronize()
        mdc.mdc_timing(h, True)
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ms, n = mdc.mdc_timing_read(h, cls)
        pms, _ = mdc.mdc_timing_read(h, "tc_prep")
        mdc.mdc_timing(h, False)
        return (ms + pms) / max(n, 1), pms / max(n, 1)

    for fmt in ("c64", "c32s", "c16f", "cbf16", "ce4m3"):
        op = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=fmt)
        kb = cfg.nf * cfg.nr * cfg.ns * BYTES_PER_COMPLEX[fmt]     # algorithmic kernel bytes per pass
        res = {"kernel_gb": kb / 1e9}
        for nv in (1, 16, 128):
            x = torch.randn((cfg.nt, cfg.ns, nv), generator=gen, device=dev)
            y = torch.randn((cfg.nt, cfg.nr, nv), generator=gen, device=dev)
            tf, pf = timed(lambda: op.forward(x), "product_fwd", op.h)
            ta, pa = timed(lambda: op.adjoint(y), "product_adj", op.h)
            flops = 8.0 * cfg.nf * cfg.nr * cfg.ns * nv
            res[f"nv{nv}"] = {"product_fwd_ms": tf, "product_adj_ms": ta,
                              "kernel_gbs": kb / (0.5 * (tf + ta)) / 1e6,
                              "tflops": flops / (0.5 * (tf + ta)) / 1e9}
            if pf + pa > 0:          # tensor-core products: the GEMM alone, without its operand preparation
                res[f"nv{nv}"].update({"tc_prep_fwd_ms": pf, "tc_prep_adj_ms": pa,
                                       "tflops_gemm": flops / (0.5 * (tf + ta - pf - pa)) / 1e9})
            del x, y
        yg = op.forward(torch.from_numpy(x16).to(dev)).cpu().numpy()[:, rows]
        xg = op.adjoint(torch.from_numpy(y16).to(dev)).cpu().numpy()[:, cols]
        res["rel_l2_forward"] = float(np.linalg.norm(yg - ref_f) / np.linalg.norm(ref_f))
        res["rel_l2_adjoint"] = float(np.linalg.norm(xg - ref_a) / np.linalg.norm(ref_a))
        op.close()
        torch.cuda.empty_cache()
        out[fmt] = res
    del G
    torch.cuda.empty_cache()
    return out


FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz max SM clock


def run_small(args, dev):
    """The small workload (441 x 441, nt=256, nfmax=64, nv=1; complex64 kernel 99.6 MB, smaller than
    L2): forward+adjoint pairs timed one by one (CUDA events around each pair, median of
    ``--small-reps``), with the kernel left resident in L2 between pairs and with L2 flushed
    (a 512 MB buffer written) before each pair, each as ordinary stream launches and as a replayed
    CUDA graph of the pair.  At this size launch overhead is a large part of a pass."""
    import torch
    import paper_2011_11120_gb300 as mdc
    cfg = synth.config(1)
    d = synth.draw(cfg)
    op = mdc.MDC(torch.from_numpy(synth.kernel(cfg, d).astype(np.complex64)).to(dev), cfg.nt, cfg.dt, cfg.dr)
    mdc.mdc_reserve(op.h, 1)
    x = torch.from_numpy(synth.ricker_traces(cfg, d)).to(dev)
    y = torch.empty((cfg.nt, cfg.nr, 1), device=dev)
    xo = torch.empty((cfg.nt, cfg.ns, 1), device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        op.forward(x, out=y)
        op.adjoint(y, out=xo)

    for _ in range(10):
        step()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    torch.cuda.synchronize()
    bytes_pair, _ = algorithmic_bytes(cfg, 1)
    peak, _ = peaks()
    out = {"workload": f"MDC fwd+adj, nr=ns={cfg.nr} (21x21, 20 m), nt={cfg.nt}, nfmax={cfg.nf}, "
                       f"{cfg.n_events} events, c64 kernel {cfg.nf * cfg.nr * cfg.ns * 8 / 1e6:.1f} MB, nv=1",
           "reps": args.small_reps, "bytes_per_pair": bytes_pair}
    stream = torch.cuda.current_stream()
    for name, use_graph, do_flush in (("l2_resident", False, False), ("l2_flushed", False, True),
                                      ("l2_resident_graph", True, False), ("l2_flushed_graph", True, True)):
        evs = []
        for i in range(args.small_reps):
            if do_flush:
                flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if use_graph:
                graph.replay()
            else:
                step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        us = sorted(1e3 * a.elapsed_time(b) for a, b in evs)
        med = statistics.median(us)
        out[name] = {"median_us": med, "p10_us": us[len(us) // 10], "p90_us": us[(9 * len(us)) // 10],
                     "gbs": bytes_pair / med / 1e3, "frac_of_measured_hbm": bytes_pair / med / 1e3 / peak}
    n0 = mdc.mdc_launch_count(op.h)
    step()
    out["launches_per_pair"] = int(mdc.mdc_launch_count(op.h) - n0)
    del graph
    op.close()
    return out


def run_batched64(args, dev):
    """The paper-scale kernel (3721 x 3721, nt=1024, nfmax=200) with nv = 64 random focusing points:
    every product is a dense GEMM per frequency (1.42 TFLOP).  Split FP16 storage (three FP16
    tensor-core products per GEMM, float32-level accuracy) against complex64 on the FP32 SIMT GEMM;
    sampled rows/columns against the FP64 oracle."""
    import torch
    import paper_2011_11120_gb300 as mdc
    from oracle import mdc as omdc
    from synth import gpu as sgpu
    nv = 64
    cfg = synth.config(2, nv=nv)
    d = synth.draw(cfg)
    G = sgpu.kernel_on_device(cfg, d)
    x_np = synth.ricker_traces(cfg, d)
    rng = np.random.default_rng(32)
    y_np = rng.standard_normal((cfg.nt, cfg.nr, nv)).astype(np.float32)
    rows = np.sort(rng.choice(cfg.nr, size=8, replace=False))
    cols = np.sort(rng.choice(cfg.ns, size=8, replace=False))
    ref_f = omdc.forward_rows(synth.kernel(cfg, d, rows=rows), x_np, cfg.dt, cfg.dr)
    ref_a = omdc.adjoint_cols(synth.kernel(cfg, d, cols=cols), y_np, cfg.dt, cfg.dr)
    x, y = torch.from_numpy(x_np).to(dev), torch.from_numpy(y_np).to(dev)
    flops = 8.0 * cfg.nf * cfg.nr * cfg.ns * nv
    out = {"workload": f"MDC fwd+adj, nr=ns={cfg.nr} (61x61, 20 m), nt={cfg.nt}, nfmax={cfg.nf}, "
                       f"{cfg.n_events} events, nv={nv} random focusing points; {flops / 1e12:.2f} TFLOP per product"}
    for storage in ("c32s", "c64"):
        op = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=storage)
        mdc.mdc_reserve(op.h, nv)
        yo = torch.empty((cfg.nt, cfg.nr, nv), device=dev)
        xo = torch.empty((cfg.nt, cfg.ns, nv), device=dev)
        op.forward(x, out=yo)
        op.adjoint(y, out=xo)
        torch.cuda.synchronize()
        reps = args.batched_reps if storage == "c32s" else max(2, args.batched_reps // 4)
        mdc.mdc_timing(op.h, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            op.forward(x, out=yo)
            op.adjoint(y, out=xo)
        e1.record()
        torch.cuda.synchronize()
        kc = {c: mdc.mdc_timing_read(op.h, c) for c in ("rfft", "tc_prep", "product_fwd", "product_adj", "irfft")}
        mdc.mdc_timing(op.h, False)
        mdc.mdc_device_status(op.h)
        gemm_ms = (kc["product_fwd"][0] + kc["product_adj"][0]) / max(kc["product_fwd"][1] + kc["product_adj"][1], 1)
        pair_ms = e0.elapsed_time(e1) / reps
        res = {"ms_per_pair": pair_ms, "tflops_per_pair": 2 * flops / pair_ms / 1e9,
               "product_ms": gemm_ms, "tflops_product": flops / gemm_ms / 1e9,
               "device_ms_per_kernel_class_per_pair": {c: v[0] / reps for c, v in kc.items()},
               "tc_fallbacks": mdc.mdc_tc_fallback_count(op.h),
               "rel_l2_forward": float(np.linalg.norm(yo.cpu().numpy()[:, rows] - ref_f) / np.linalg.norm(ref_f)),
               "rel_l2_adjoint": float(np.linalg.norm(xo.cpu().numpy()[:, cols] - ref_a) / np.linalg.norm(ref_a))}
        if storage == "c32s":
            pk, kind = tc_peak(sustained=False)
            issued = 3 * flops / gemm_ms / 1e9
            res["roofline"] = {"bound": "tensor", "kernel": "tc_gemm_kernel (split FP16: three FP16 MMAs per product)",
                               "achieved": issued, "peak": pk, "unit": "TFLOP/s", "frac": issued / pk,
                               "peak_kind": kind, "note": "achieved counts the three tensor-core products issued"}
        else:
            res["roofline"] = {"bound": "alu", "kernel": "cgemm_simt (FP32 FMA)", "achieved": flops / gemm_ms / 1e9,
                               "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                               "frac": flops / gemm_ms / 1e9 / FP32_ALU_TFLOPS,
                               "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz"}
        out[storage] = res
        op.close()
        torch.cuda.empty_cache()
    del G
    torch.cuda.empty_cache()
    return out


def sections_summary(result):
    """A compact digest of every section's headline numbers, kept as the line's last key."""
    def g(dct, *path):
        for k in path:
            if not isinstance(dct, dict) or k not in dct:
                return None
            dct = dct[k]
        return float(f"{dct:.4g}") if isinstance(dct, float) else dct
    out = {"headline_gbs": g(result, "value"), "headline_frac": g(result, "roofline", "frac"),
           "e2e_gbs": g(result, "e2e", "value")}
    if "redatum" in result:
        out["redatum"] = {"solves_per_s": g(result, "redatum", "solves_per_s"), "p50_ms": g(result, "redatum", "p50_ms"),
                          "p99_ms": g(result, "redatum", "p99_ms"), "solves": g(result, "redatum", "solves_timed"),
                          "rel_l2_vs_fp32": g(result, "redatum", "rel_l2_vs_fp32_solve"),
                          "gemm_frac": g(result, "redatum", "tc_roofline", "frac"),
                          "fp32_one_job_solves_per_s": g(result, "redatum", "fp32_one_job", "solves_per_s")}
    if "small" in result:
        out["small_us"] = {k: g(result, "small", k, "median_us") for k in
                           ("l2_resident", "l2_flushed", "l2_resident_graph", "l2_flushed_graph")}
    if "batched64" in result:
        out["batched64"] = {k: {"tflops_product": g(result, "batched64", k, "tflops_product"),
                                "frac": g(result, "batched64", k, "roofline", "frac"),
                                "rel_l2_fwd": g(result, "batched64", k, "rel_l2_forward")} for k in ("c32s", "c64")}
    if "mdd" in result:
        out["mdd_batches_per_s"] = {k: g(result, "mdd", k, "solves_per_s") for k in ("c64", "c32s", "c16f")}
    if "precision" in result:
        out["precision_nv128_tflops"] = {k: g(result, "precision", k, "nv128", "tflops")
                                         for k in ("c64", "c32s", "c16f", "cbf16", "ce4m3")}
        out["precision_rel_l2_fwd"] = {k: g(result, "precision", k, "rel_l2_forward")
                                       for k in ("c64", "c32s", "c16f", "cbf16", "ce4m3")}
    if "serving" in result:
        out["serving"] = {"capacity_solves_per_s": g(result, "serving", "offered", "solves_per_s"),
                          "offered_p50_s": g(result, "serving", "offered", "p50_s"),
                          "offered_p99_s": g(result, "serving", "offered", "p99_s"),
                          "at_0.7_p50_s": g(result, "serving", "at_0.7_capacity", "p50_s"),
                          "at_0.7_p99_s": g(result, "serving", "at_0.7_capacity", "p99_s"),
                          "fp32_one_job_solves_per_s": g(result, "serving", "fp32_one_job_at_a_time", "solves_per_s"),
                          "rel_l2_fp16_vs_fp32": g(result, "serving", "rel_l2_fp16_vs_fp32")}
    if "paper_full" in result:
        out["paper_full"] = {"c64_pair_ms": g(result, "paper_full", "c64", "ms_per_mdc_pair"),
                             "c64_frac": g(result, "paper_full", "c64", "frac_of_measured_hbm"),
                             "c64_marchenko_1pt_s": g(result, "paper_full", "c64", "marchenko_nv1", "s_per_solve"),
                             "c16f_marchenko_20pt_s": g(result, "paper_full", "c16f", "marchenko_nv20", "s_per_solve")}
    return out


PAPER_FULL = synth.config(6)


def run_paper_full(args, dev):
    """The paper's Full geometry (Table 1) on one GPU: 99 x 99 = 9801 co-located sources and
    receivers, 300 frequencies (nt = 2048, dt = 4 ms), 20 hyperbolic events.  The complex64 kernel
    (232 GB) and then an FP16 copy (116 GB) are filled slab by slab (20 frequencies at a time,
    generated on the device), then timed: one forward+adjoint MDC at one virtual point, and
    Marchenko LSQR solves of 10 iterations for 1 and 20 focusing points (z = 600 m).  The paper's
    16-node CPU figures for the same geometry are quoted beside them as context."""
    import torch
    import paper_2011_11120_gb300 as mdc
    from synth import gpu as sgpu
    cfg = PAPER_FULL
    d = synth.draw(cfg)
    ldg = -(-cfg.ns // 64) * 64
    slab, niter = 20, 10
    extent = synth.GRID_DX * (cfg.n_side - 1)
    pts20 = np.random.default_rng(cfg.seed).uniform(0.25 * extent, 0.75 * extent, size=(20, 2))
    x = torch.from_numpy(np.ascontiguousarray(synth.ricker_traces(cfg, d), np.float32)).to(dev)
    yo = torch.empty((cfg.nt, cfg.nr, 1), device=dev)
    xo = torch.empty((cfg.nt, cfg.ns, 1), device=dev)
    peak, _ = peaks()
    out = {"workload": f"paper Full geometry: nr=ns={cfg.nr} (99x99, 20 m), nt={cfg.nt}, dt={cfg.dt}, "
                       f"nfmax={cfg.nf}, {cfg.n_events} hyperbolic events; MDC fwd+adj at nv=1; Marchenko LSQR "
                       f"({niter} iterations) for 1 and 20 focusing points at z={cfg.z_point:.0f} m",
           "paper_context": {"hardware": "16 nodes x 2 octa-core Xeon @ 2.90 GHz, 128 GB each (Dask)",
                             "setup_s": 180, "one_point_inversion_s": 260, "twenty_point_inversion_s": 1760,
                             "ms_per_mdc_derived": 6000, "solver": "10 CGLS iterations",
                             "kernel": "300 x 9801 x 9801 complex64, 230 GB"}}
    fm_c64 = None
    for storage in ("c64", "c16f"):
        torch.cuda.empty_cache()
        need = cfg.nf * cfg.nr * ldg * BYTES_PER_COMPLEX[storage] + slab * cfg.nr * cfg.ns * 8 + (8 << 30)
        free, _ = torch.cuda.mem_get_info()
        if free < need:
            out[storage] = {"skipped": f"needs {need / 1e9:.0f} GB free on the device, {free / 1e9:.0f} GB free"}
            continue
        t0 = time.perf_counter()
        op = mdc.MDC.empty(cfg.nf, cfg.nr, cfg.ns, cfg.nt, cfg.dt, cfg.dr, storage=storage)
        buf = torch.empty((slab, cfg.nr, cfg.ns), dtype=torch.complex64, device=dev)
        for k0 in range(0, cfg.nf, slab):
            nk = min(slab, cfg.nf - k0)
            sgpu.kernel_slab_on_device(cfg, k0, nk, d, out=buf[:nk])
            op.load_slab(buf[:nk], k0)
        del buf
        torch.cuda.empty_cache()
        res = {"kernel_gb": cfg.nf * cfg.nr * cfg.ns * BYTES_PER_COMPLEX[storage] / 1e9,
               "setup_s": time.perf_counter() - t0}
        for _ in range(3):
            op.forward(x, out=yo)
            op.adjoint(yo, out=xo)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        for _ in range(5):
            op.forward(x, out=yo)
            op.adjoint(yo, out=xo)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        bytes_pair, _ = algorithmic_bytes(cfg, 1, storage)
        res.update({"ms_per_mdc_pair": ms, "gbs": bytes_pair / ms / 1e6,
                    "frac_of_measured_hbm": bytes_pair / ms / 1e6 / peak})
        for nv, pts in ((1, d.points), (20, pts20)):
            cut, fd = sgpu.focusing_inputs_on_device(cfg, pts, device=dev)
            sol = op.marchenko(cut, fd, niter)                       # warm-up (workspace, tensor maps)
            torch.cuda.synchronize()
            times = []
            for _ in range(2):
                t1 = time.perf_counter()
                sol = op.marchenko(cut, fd, niter)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t1)
            mdc.mdc_timing(op.h, True)                              # device time per kernel class, one more solve
            op.marchenko(cut, fd, niter)
            torch.cuda.synchronize()
            split = {}
            for cls in ("rfft", "tc_prep", "product_fwd", "product_adj", "irfft", "solver"):
                t, n = mdc.mdc_timing_read(op.h, cls)
                split[cls] = {"ms": t, "launches": n}
            mdc.mdc_timing(op.h, False)
            r = {"s_per_solve": min(times), "iterations": sol["iters"],
                 "final_residual": sol["resid"][sol["iters"]], "device_ms_per_kernel_class": split}
            if nv == 1 and storage == "c64":
                fm_c64 = sol["f_minus"].double()
            elif nv == 1 and fm_c64 is not None:
                r["rel_l2_f_minus_vs_c64"] = float((sol["f_minus"].double() - fm_c64).norm() / fm_c64.norm())
            res[f"marchenko_nv{nv}"] = r
            del cut, fd, sol
            if storage == "c64":
                break          # 20 points on complex64 run on the SIMT product (minutes); FP16 only
        op.close()
        out[storage] = res
    del x, yo, xo, fm_c64
    torch.cuda.empty_cache()
    return out


def serve_loop(mdc, srv, arrivals, pool, horizon, drain):
    """Submit arrivals (t, nv, niter, tol, entry) as their time comes, step the server, and
    collect completed jobs; returns (completed records, jobs still queued or running)."""
    t0 = time.perf_counter()
    ia, pending, done = 0, {}, []
    while True:
        now = time.perf_counter() - t0
        while ia < len(arrivals) and arrivals[ia][0] <= now and now < horizon:
            _, nv, niter, tol, e = arrivals[ia]
            cut, fd = pool[e]
            jid = mdc.srv_submit(srv, cut, fd, nv, niter, tol)
            pending[jid] = (nv, niter, tol)
            ia += 1
        if now >= horizon and (not drain or not pending):
            break
        if not pending:
            time.sleep(0.0005)
            continue
        mdc.srv_step(srv)
        for jid in list(pending):
            p = mdc.srv_poll(srv, jid)
            if p["state"] >= mdc.JOB_DONE:
                done.append(dict(p, nv=pending[jid][0], niter=pending[jid][1], tol=pending[jid][2]))
                mdc.srv_release(srv, jid)
                del pending[jid]
    return done, len(pending), time.perf_counter() - t0


def percentile(vals, q):
    return float(np.percentile(np.asarray(vals), q)) if vals else None


def run_serving(args, dev):
    """Continuous batching of redatuming jobs on the resident FP16 kernel (Poisson arrivals,
    nv ~ U{1..128}, niter ~ U{10..30}, half of the jobs with tolerance 1e-3)."""
    import torch
    import paper_2011_11120_gb300 as mdc
    from synth import gpu as sgpu
    cfg = synth.config(args.serving_config)
    d = synth.draw(cfg.with_(nv=1, point_grid=0))
    G = sgpu.kernel_on_device(cfg, d)
    lo = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c16f")
    del G
    torch.cuda.empty_cache()
    rng = np.random.default_rng(synth.SEED_BASE + 5)
    extent = synth.GRID_DX * (cfg.n_side - 1)
    pool = []
    for _ in range(args.serving_pool):
        pts = rng.uniform(0.0, extent, size=(128, 2))
        cut, fd = sgpu.focusing_inputs_on_device(cfg.with_(z_point=800.0), pts, device=dev)
        fd_h = torch.empty(fd.shape, dtype=torch.float32, pin_memory=True)
        fd_h.copy_(fd)
        pool.append((cut.cpu().numpy(), fd_h.numpy()))
        del fd
    torch.cuda.empty_cache()
    per_point = 12 * cfg.nt * cfg.ns * 4 + 4 * cfg.ns * 8 + cfg.ns * 4
    free = torch.cuda.mem_get_info()[0]
    max_cols = int(min(2048, 2 * (0.8 * free) // per_point))
    # scratch of the server: two spectra and the tensor-core operand for max_cols columns
    scratch = 2 * cfg.nf * cfg.ns * max_cols * 8 + cfg.nf * max_cols * 2 * 2 * (cfg.ns + 64) * 2
    budget = int(0.85 * (free - scratch))
    max_cols = int(min(max_cols, 2 * budget // per_point))

    def arrivals(rate, horizon, seed):
        r = np.random.default_rng(seed)
        t, out = 0.0, []
        while True:
            t += r.exponential(1.0 / rate)
            if t >= horizon:
                return out
            nv = int(r.integers(1, 129))
            niter = int(r.integers(10, 31))
            tol = 1e-3 if r.random() < 0.5 else 0.0
            out.append((t, nv, niter, tol, int(r.integers(0, len(pool)))))

    res = {"workload": f"Poisson redatuming jobs on the {cfg.nr}x{cfg.ns}, nt={cfg.nt}, nfmax={cfg.nf} kernel "
                       f"(FP16 copy resident, ||R||=0.5), nv ~ U{{1..128}} at z=800 m, niter ~ U{{10..30}}, "
                       f"half with tol 1e-3; columns of all running jobs share one product per pass",
           "hbm_budget_gb": budget / 1e9, "max_cols": max_cols}
    # (i)+(ii): the offered load, fixed horizon, backlog stated
    srv = mdc.srv_create(lo.h, None, budget, max_cols)
    arr = arrivals(args.serving_rate, args.serving_horizon, 1)
    done, backlog, el = serve_loop(mdc, srv, arr, pool, args.serving_horizon, False)
    mdc.srv_destroy(srv)
    lat = [j["latency_s"] for j in done]
    cap = len(done) / el if el > 0 else 0.0
    res["offered"] = {"rate_per_s": args.serving_rate, "horizon_s": args.serving_horizon, "submitted": len(arr),
                      "completed": len(done), "backlog": backlog,
                      "solves_per_s": cap, "virtual_points_per_s": sum(j["nv"] for j in done) / el,
                      "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
                      "max_final_residual": max([j["final_residual"] for j in done], default=None)}
    # (iii): 0.7 x the measured capacity, drained
    rate3 = max(0.7 * cap, 0.05)
    srv = mdc.srv_create(lo.h, None, budget, max_cols)
    arr = arrivals(rate3, args.serving_horizon, 2)
    done, backlog, el = serve_loop(mdc, srv, arr, pool, args.serving_horizon, True)
    mdc.srv_destroy(srv)
    lat = [j["latency_s"] for j in done]
    res["at_0.7_capacity"] = {"rate_per_s": rate3, "submitted": len(arr), "completed": len(done),
                              "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
                              "wall_s": el}
    # one job alone through the server: the reference for the FP32 comparison below
    nv0, niter0 = 64, 20
    cut0, fd0 = pool[0]
    out16 = [np.zeros((cfg.nt, cfg.ns, nv0), np.float32) for _ in range(4)]
    srv = mdc.srv_create(lo.h, None, budget, max_cols)
    jid = mdc.srv_submit(srv, cut0, fd0, nv0, niter0, 0.0, out16)
    t0 = time.perf_counter()
    while mdc.srv_poll(srv, jid)["state"] < mdc.JOB_DONE:
        mdc.srv_step(srv)
    t_alone = time.perf_counter() - t0
    mdc.srv_destroy(srv)
    lo.close()
    # (iv): the plain float32 one-job-at-a-time solve (complex64 kernel, no batching)
    G = sgpu.kernel_on_device(cfg, d)
    op = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    del G
    torch.cuda.empty_cache()
    cut_t = torch.from_numpy(np.ascontiguousarray(cut0[:, :nv0])).to(dev)
    fd_t = torch.from_numpy(np.ascontiguousarray(fd0[:, :, :nv0])).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out32 = op.marchenko(cut_t, fd_t, niter0)
    t32 = time.perf_counter() - t0
    f32 = out32["f_minus"].double().cpu().numpy()
    err = float(np.linalg.norm(out16[0] - f32) / np.linalg.norm(f32))
    op.close()
    res["one_job_fp16_alone"] = {"nv": nv0, "niter": niter0, "seconds": t_alone}
    res["fp32_one_job_at_a_time"] = {"nv": nv0, "niter": niter0, "seconds": t32, "solves_per_s": 1.0 / t32,
                                     "storage": "c64"}
    res["rel_l2_fp16_vs_fp32"] = err
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2011_11120_gb300 as mdc
    from synth import gpu as sgpu

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    cfg = synth.config(args.config, nv=args.nv)
    if args.nf:
        cfg = cfg.with_(nf=args.nf, normalise=False)   # profiling case: normalisation not needed
    nv = args.nv
    d = synth.draw(cfg)
    shard = args.shard and world > 1
    if shard:
        # this rank's band of frequencies; every pass ends with one NCCL all-reduce of the traces
        k0, nk = mdc.shard_bounds(cfg.nf, world, rank)
        G = sgpu.kernel_slab_on_device(cfg, k0, nk, d)
        op = mdc.ShardedMDC(G, k0, cfg.nt, cfg.dt, cfg.dr, storage=args.storage)
    else:
        k0, nk = 0, cfg.nf
        G = sgpu.kernel_on_device(cfg, d)
        op = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=args.storage)
    del G
    torch.cuda.empty_cache()
    mdc.mdc_reserve(op.h, nv)
    xr = synth.ricker_traces(cfg, d)
    if xr.shape[2] != nv:          # configs with a fixed point lattice: repeat its columns up to nv
        xr = np.ascontiguousarray(np.take(xr, np.arange(nv) % xr.shape[2], axis=2))
    x_host = torch.from_numpy(xr).pin_memory()
    xd = x_host.to(dev)
    yd = torch.empty((cfg.nt, cfg.nr, nv), device=dev)
    xo = torch.empty((cfg.nt, cfg.ns, nv), device=dev)
    out_host = torch.empty((cfg.nt, cfg.ns, nv)).pin_memory()
    stream = torch.cuda.current_stream()

    def step():
        op.forward(xd, out=yd)
        op.adjoint(yd, out=xo)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bytes_step, kernel_bytes = algorithmic_bytes(cfg, nv, args.storage)

    # ---- device-timed region
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    mdc.mdc_timing(op.h, True)
    n0 = mdc.mdc_launch_count(op.h)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = mdc.mdc_launch_count(op.h) - n0
    ms = e0.elapsed_time(e1)
    kern = {}
    for name in ("rfft", "tc_prep", "product_fwd", "product_adj", "irfft"):
        t, n = mdc.mdc_timing_read(op.h, name)
        kern[name] = {"ms_total": t, "launches": n, "ms_avg": t / n if n else None}
    mdc.mdc_timing(op.h, False)
    mdc.mdc_device_status(op.h)

    # ---- end-to-end: pinned host input -> device, fwd+adj, result -> pinned host, every step
    for _ in range(2):
        xd.copy_(x_host, non_blocking=True)
        step()
        out_host.copy_(xo, non_blocking=True)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        xd.copy_(x_host, non_blocking=True)
        step()
        out_host.copy_(xo, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = f0.elapsed_time(f1)

    if world > 1:
        ms, ms_e2e = max_over_ranks([ms, ms_e2e], dev)
    op.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # replicas: every rank runs the whole operator; shards: the ranks together run one operator
    copies = 1 if shard else world
    value = copies * bytes_step * args.steps / (ms / 1e3) / 1e9
    e2e_value = copies * bytes_step * args.steps / (ms_e2e / 1e3) / 1e9
    peak, peak_kind = peaks()
    prod_ms = kern["product_fwd"]["ms_total"] + kern["product_adj"]["ms_total"]
    prod_n = kern["product_fwd"]["launches"] + kern["product_adj"]["launches"]
    kernel_bytes = kernel_bytes * nk // cfg.nf         # this rank's band (the whole kernel unless sharded)
    achieved = kernel_bytes * prod_n / (prod_ms / 1e3) / 1e9 if prod_ms > 0 else None
    # the committed DRAM capture covers the complex64 GEMV pair of the default workload only
    profiled = args.config == 2 and not args.nf and nv == 1 and args.storage == "c64"
    traffic = profile_traffic("product.cu") if profiled else None
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(config_block(cfg, nv, args.storage),
                       parallelism=(f"frequency shards x{world} (one NCCL all-reduce per pass)" if shard
                                    else f"replicas x{world}" if world > 1 else "single GPU")),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "kernel": f"per-frequency product (forward + adjoint, {args.storage}, {nv} column(s))",
                     "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s"},
        "kernels": kern,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x_host.numel() * 4),
                "d2h_bytes_per_step": int(out_host.numel() * 4), "ms_per_step": ms_e2e / args.steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if world == 1 and not args.no_small:
        result["small"] = run_small(args, dev)
    if world == 1 and not args.no_batched64:
        result["batched64"] = run_batched64(args, dev)
    if world == 1 and not args.no_redatum:
        result["redatum"] = run_redatum(args, dev)
    if world == 1 and not args.no_mdd:
        result["mdd"] = run_mdd(args, dev)
    if world == 1 and not args.no_precision:
        result["precision"] = run_precision(args, dev)
    if world == 1 and not args.no_serving:
        result["serving"] = run_serving(args, dev)
    if world == 1 and not args.no_paper_full:
        result["paper_full"] = run_paper_full(args, dev)
    if world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(cfg, nv, min_seconds=args.cpu_seconds)
        result["cpu_baseline"]["paper_style"] = paper_style_cpu(cfg, nv)
    result["sections_summary"] = sections_summary(result)
    print(json.dumps(result), flush=True)
    if args.metrics_jsonl:
        with open(args.metrics_jsonl, "a") as fh:
            fh.write(json.dumps(result) + "\n")
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--nv", type=int, default=1)
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--nf", type=int, default=0, help="override nfmax (smaller profiling case)")
    ap.add_argument("--storage", default="c64", choices=["c64", "c16f", "cbf16", "ce4m3", "c32s"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-redatum", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-mdd", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-paper-full", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-batched64", action="store_true")
    ap.add_argument("--small-reps", type=int, default=200)
    ap.add_argument("--batched-reps", type=int, default=8)
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1 GPUs: split the kernel's frequencies over the ranks (one all-reduce per "
                         "pass, strong scaling) instead of running N replicas")
    ap.add_argument("--metrics-jsonl", default="", help="also append the result line to this file")
    ap.add_argument("--mdd-iters", type=int, default=10)
    ap.add_argument("--serving-config", type=int, default=5)
    ap.add_argument("--serving-rate", type=float, default=50.0)
    ap.add_argument("--serving-horizon", type=float, default=20.0)
    ap.add_argument("--serving-pool", type=int, default=2)
    ap.add_argument("--redatum-solves", type=int, default=10)
    ap.add_argument("--redatum-storage", default="c16f", choices=["c16f", "cbf16"])
    ap.add_argument("--redatum-refine-iters", type=int, default=5)
    ap.add_argument("--redatum-ref-storage", default="c32s", choices=["c64", "c32s"])
    ap.add_argument("--redatum-nv", type=int, default=0, help="first N focusing points only (profiling cases)")
    ap.add_argument("--redatum-skip-fp32", action="store_true", help="skip the float32 one-job comparison solve")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
