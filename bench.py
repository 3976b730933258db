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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "MDC fwd+adj HBM GB/s vs peak; redatum solves/s and p99 at <=1e-3 vs FP64"
UNIT = "GB/s"


BYTES_PER_COMPLEX = {"c64": 8, "c16f": 4, "cbf16": 4, "ce4m3": 2}


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


def profile_traffic(kernel_file):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "product_gemv_c64_3721x3721_nf200_nv1.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        prof = json.load(fh)
    src = open(os.path.join(ROOT, "paper_2011_11120_gb300", "csrc", kernel_file), "rb").read()
    if prof.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return prof.get("dram_bytes_per_launch")


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

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
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms)}


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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cfg = synth.config(args.config, nv=args.nv)
    if args.nf:
        cfg = cfg.with_(nf=args.nf)
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
    ref = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage="c64")
    del G
    torch.cuda.empty_cache()
    cut = torch.from_numpy(synth.window_cutoffs(cfg, d)).to(dev)
    fd = torch.from_numpy(synth.direct_focusing(cfg, d)).to(dev)
    niter, nref, nin = cfg.niter, 1, args.redatum_refine_iters

    def solve():
        return lo.marchenko_refined(ref, cut, fd, niter, nrefine=nref, niter_refine=nin)

    out = solve()                                      # warm-up (allocations, tensor maps)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.redatum_solves):
        t0 = time.perf_counter()
        out = solve()
        times.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    plain = ref.marchenko(cut, fd, niter)              # float32 operator, one job, no refinement
    t_plain = time.perf_counter() - t0
    fm = out["f_minus"].double()
    err = float((fm - plain["f_minus"].double()).norm() / plain["f_minus"].double().norm())
    lo.close()
    ref.close()
    med = statistics.median(times)
    return {"workload": f"Marchenko LSQR, nr=ns={cfg.nr} (41x41, 20 m), nt={cfg.nt}, nfmax={cfg.nf}, "
                        f"nv={cfg.nv} (16x16 focusing points, z=800 m), ||R||=0.5, {niter} LSQR iterations "
                        f"on a {args.redatum_storage} kernel + {nref} float32 refinement step of {nin} iterations",
            "solves_per_s": 1.0 / med, "ms_per_solve": 1e3 * med, "solves_timed": len(times),
            "p50_ms": 1e3 * med, "p99_ms": 1e3 * max(times),
            "iterations": out["iters"], "final_residual": out["final_residual"],
            "rel_l2_vs_fp32_solve": err,
            "fp32_one_job": {"solves_per_s": 1.0 / t_plain, "ms_per_solve": 1e3 * t_plain,
                             "iterations": plain["iters"], "storage": "c64"}}


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
        cfg = cfg.with_(nf=args.nf)
    nv = args.nv
    d = synth.draw(cfg)
    G = sgpu.kernel_on_device(cfg, d)
    op = mdc.MDC(G, cfg.nt, cfg.dt, cfg.dr, storage=args.storage)
    del G
    torch.cuda.empty_cache()
    mdc.mdc_reserve(op.h, nv)
    x_host = torch.from_numpy(synth.ricker_traces(cfg, d)).pin_memory()
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
    for name in ("rfft", "product_fwd", "product_adj", "irfft"):
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
        t = torch.tensor([ms, ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_e2e = float(t[0]), float(t[1])
    op.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    value = world * bytes_step * args.steps / (ms / 1e3) / 1e9
    e2e_value = world * bytes_step * args.steps / (ms_e2e / 1e3) / 1e9
    peak, peak_kind = peaks()
    prod_ms = kern["product_fwd"]["ms_total"] + kern["product_adj"]["ms_total"]
    prod_n = kern["product_fwd"]["launches"] + kern["product_adj"]["launches"]
    achieved = kernel_bytes * prod_n / (prod_ms / 1e3) / 1e9 if prod_ms > 0 else None
    traffic = profile_traffic("product.cu")
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(config_block(cfg, nv, args.storage), parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
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
    if world == 1 and not args.no_redatum:
        result["redatum"] = run_redatum(args, dev)
    if world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(cfg, nv, min_seconds=args.cpu_seconds)
    print(json.dumps(result), flush=True)
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
    ap.add_argument("--storage", default="c64", choices=["c64", "c16f", "cbf16", "ce4m3"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-redatum", action="store_true")
    ap.add_argument("--redatum-solves", type=int, default=3)
    ap.add_argument("--redatum-storage", default="c16f", choices=["c16f", "cbf16"])
    ap.add_argument("--redatum-refine-iters", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
