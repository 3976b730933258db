"""bench.py keeps its output contract: the reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the output contract, and the helpers count algorithmic bytes as stated."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=900, cwd=ROOT, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["impl"] == "reference" and r["steps"] == 1 and r["warmup"] >= 3
    assert r["value"] > 0 and r["unit"] == "GB/s" and r["higher_is_better"] is True
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["cores"] >= 1
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in r["config"]


def test_algorithmic_bytes():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    cfg = synth.config(2)
    step, kernel = bench.algorithmic_bytes(cfg, 1, "c64")
    assert kernel == cfg.nf * cfg.nr * cfg.ns * 8
    assert step == 2 * (kernel + cfg.nt * (cfg.nr + cfg.ns) * 4)
    assert bench.algorithmic_bytes(cfg, 1, "c16f")[1] == kernel // 2
